// Instantiations of the persistent MLMQ kernel for fp32 arc lengths (IEEE bit
// patterns): the extended
// kernel, with the optional paths (pending marks, the in-warp duplicate filter,
// the single-queue baseline, run-time sampling, the debug trace).
#include "kernels_inst.cuh"

namespace sssp {

cudaError_t launch_mlmq_f32x(const KernelKey& k, dim3 grid, dim3 block, size_t smem,
                             cudaStream_t stream, const KParams& p) {
    return MlmqInstances<1, true>::launch(k, grid, block, smem, stream, p);
}

cudaError_t occupancy_mlmq_f32x(const KernelKey& k, int threads, size_t smem, int* blocks) {
    return MlmqInstances<1, true>::occupancy(k, threads, smem, blocks);
}

}  // namespace sssp
