// kernels_inst.cuh -- launch and occupancy dispatch for the instantiations of
// mlmq_kernel of one weight type (WT) and one variant (X: the extended kernel
// with the optional paths, or the lean one without them).  Each of
// kernels_{u32,f32}{,x}.cu instantiates one (WT, X) pair, so the four compile
// in parallel.
#pragma once

#include "internal.h"

namespace sssp {

template <int WT, bool X>
struct MlmqInstances {
    template <int PRED, bool MQ>
    static cudaError_t launch_one(dim3 grid, dim3 block, size_t smem, cudaStream_t stream, const KParams& p) {
        auto fn = mlmq_kernel<WT, PRED, MQ, kL0Rows, X>;
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        fn<<<grid, block, smem, stream>>>(p);
        return cudaGetLastError();
    }
    template <int PRED, bool MQ>
    static cudaError_t occ_one(int threads, size_t smem, int* blocks) {
        auto fn = mlmq_kernel<WT, PRED, MQ, kL0Rows, X>;
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, fn, threads, smem);
    }
    // fp32 predecessors always use the strict-improvement rule (PRED 2): one
    // rounded add can absorb a tiny weight (fl(d + w) == d), so the
    // smallest-index tight rule could close a cycle of equal labels.
    static bool has(int pred) { return pred == 0 || pred == 2 || (WT == 0 && pred == 1); }

    static cudaError_t launch(const KernelKey& k, dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                              const KParams& p) {
        if (!has(k.pred)) return cudaErrorInvalidValue;
        switch (k.pred * 2 + (k.mq ? 1 : 0)) {
            case 0: return launch_one<0, false>(grid, block, smem, stream, p);
            case 1: return launch_one<0, true>(grid, block, smem, stream, p);
            case 2: return launch_one<WT == 0 ? 1 : 2, false>(grid, block, smem, stream, p);
            case 3: return launch_one<WT == 0 ? 1 : 2, true>(grid, block, smem, stream, p);
            case 4: return launch_one<2, false>(grid, block, smem, stream, p);
            case 5: return launch_one<2, true>(grid, block, smem, stream, p);
        }
        return cudaErrorInvalidValue;
    }
    static cudaError_t occupancy(const KernelKey& k, int threads, size_t smem, int* blocks) {
        if (!has(k.pred)) return cudaErrorInvalidValue;
        switch (k.pred * 2 + (k.mq ? 1 : 0)) {
            case 0: return occ_one<0, false>(threads, smem, blocks);
            case 1: return occ_one<0, true>(threads, smem, blocks);
            case 2: return occ_one<WT == 0 ? 1 : 2, false>(threads, smem, blocks);
            case 3: return occ_one<WT == 0 ? 1 : 2, true>(threads, smem, blocks);
            case 4: return occ_one<2, false>(threads, smem, blocks);
            case 5: return occ_one<2, true>(threads, smem, blocks);
        }
        return cudaErrorInvalidValue;
    }
};

}  // namespace sssp
