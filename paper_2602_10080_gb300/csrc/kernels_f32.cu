// Instantiations of the persistent MLMQ kernel for fp32 arc lengths (IEEE bit
// patterns): the lean
// kernel, without the optional paths.
#include "kernels_inst.cuh"

namespace sssp {

cudaError_t launch_mlmq_f32(const KernelKey& k, dim3 grid, dim3 block, size_t smem,
                            cudaStream_t stream, const KParams& p) {
    return MlmqInstances<1, false>::launch(k, grid, block, smem, stream, p);
}

cudaError_t occupancy_mlmq_f32(const KernelKey& k, int threads, size_t smem, int* blocks) {
    return MlmqInstances<1, false>::occupancy(k, threads, smem, blocks);
}

}  // namespace sssp
