// Instantiations of the persistent MLMQ kernel for fp32 arc lengths (IEEE
// bit patterns).  fp32 predecessors always use the strict-improvement rule:
// one rounded add can absorb a tiny weight (fl(d + w) == d), so the
// smallest-index tight rule could close a cycle of equal labels.
#include "internal.h"

namespace sssp {

namespace {
template <int PRED, bool MQ>
cudaError_t launch_one(dim3 grid, dim3 block, size_t smem, cudaStream_t stream, const KParams& p) {
    auto fn = mlmq_kernel<1, PRED, MQ, kL0Rows>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fn<<<grid, block, smem, stream>>>(p);
    return cudaGetLastError();
}
template <int PRED, bool MQ>
cudaError_t occ_one(int threads, size_t smem, int* blocks) {
    auto fn = mlmq_kernel<1, PRED, MQ, kL0Rows>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, fn, threads, smem);
}
}  // namespace

cudaError_t launch_mlmq_f32(const KernelKey& k, dim3 grid, dim3 block, size_t smem,
                            cudaStream_t stream, const KParams& p) {
    if (k.pred == 0) return k.mq ? launch_one<0, true>(grid, block, smem, stream, p)
                                 : launch_one<0, false>(grid, block, smem, stream, p);
    if (k.pred == 2) return k.mq ? launch_one<2, true>(grid, block, smem, stream, p)
                                 : launch_one<2, false>(grid, block, smem, stream, p);
    return cudaErrorInvalidValue;
}

cudaError_t occupancy_mlmq_f32(const KernelKey& k, int threads, size_t smem, int* blocks) {
    if (k.pred == 0) return k.mq ? occ_one<0, true>(threads, smem, blocks)
                                 : occ_one<0, false>(threads, smem, blocks);
    if (k.pred == 2) return k.mq ? occ_one<2, true>(threads, smem, blocks)
                                 : occ_one<2, false>(threads, smem, blocks);
    return cudaErrorInvalidValue;
}

}  // namespace sssp
