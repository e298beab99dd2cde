// Instantiations of the persistent MLMQ kernel for uint32 arc lengths.
#include "internal.h"

namespace sssp {

namespace {
template <int PRED, bool MQ>
cudaError_t launch_one(dim3 grid, dim3 block, size_t smem, cudaStream_t stream, const KParams& p) {
    auto fn = mlmq_kernel<0, PRED, MQ, kL0Rows>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fn<<<grid, block, smem, stream>>>(p);
    return cudaGetLastError();
}
template <int PRED, bool MQ>
cudaError_t occ_one(int threads, size_t smem, int* blocks) {
    auto fn = mlmq_kernel<0, PRED, MQ, kL0Rows>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, fn, threads, smem);
}
}  // namespace

cudaError_t launch_mlmq_u32(const KernelKey& k, dim3 grid, dim3 block, size_t smem,
                            cudaStream_t stream, const KParams& p) {
    switch (k.pred * 2 + (k.mq ? 1 : 0)) {
        case 0: return launch_one<0, false>(grid, block, smem, stream, p);
        case 1: return launch_one<0, true>(grid, block, smem, stream, p);
        case 2: return launch_one<1, false>(grid, block, smem, stream, p);
        case 3: return launch_one<1, true>(grid, block, smem, stream, p);
        case 4: return launch_one<2, false>(grid, block, smem, stream, p);
        case 5: return launch_one<2, true>(grid, block, smem, stream, p);
    }
    return cudaErrorInvalidValue;
}

cudaError_t occupancy_mlmq_u32(const KernelKey& k, int threads, size_t smem, int* blocks) {
    switch (k.pred * 2 + (k.mq ? 1 : 0)) {
        case 0: return occ_one<0, false>(threads, smem, blocks);
        case 1: return occ_one<0, true>(threads, smem, blocks);
        case 2: return occ_one<1, false>(threads, smem, blocks);
        case 3: return occ_one<1, true>(threads, smem, blocks);
        case 4: return occ_one<2, false>(threads, smem, blocks);
        case 5: return occ_one<2, true>(threads, smem, blocks);
    }
    return cudaErrorInvalidValue;
}

}  // namespace sssp
