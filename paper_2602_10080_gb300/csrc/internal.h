// internal.h -- host-side declarations shared by the libsssp translation
// units (not part of the public C ABI).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "mlmq.cuh"

namespace sssp {

// One instantiation of the persistent relaxation kernel.
struct KernelKey {
    int wt;    // 0 = u32, 1 = f32
    int pred;  // 0 = none, 1 = smallest-index tight predecessor, 2 = strict-improvement predecessor
    int mq;    // 0 = one query, 1 = several queries share the worklist
};

// Launches mlmq_kernel for `key` (defined per weight type in kernels_u32.cu /
// kernels_f32.cu).  Returns the launch error.
cudaError_t launch_mlmq_u32(const KernelKey& key, dim3 grid, dim3 block, size_t smem,
                            cudaStream_t stream, const KParams& p);
cudaError_t launch_mlmq_f32(const KernelKey& key, dim3 grid, dim3 block, size_t smem,
                            cudaStream_t stream, const KParams& p);
// Resident blocks per SM for the instantiation at the given shape.
cudaError_t occupancy_mlmq_u32(const KernelKey& key, int threads, size_t smem, int* blocks);
cudaError_t occupancy_mlmq_f32(const KernelKey& key, int threads, size_t smem, int* blocks);

inline cudaError_t launch_mlmq(const KernelKey& key, dim3 grid, dim3 block, size_t smem,
                               cudaStream_t stream, const KParams& p) {
    return key.wt == 0 ? launch_mlmq_u32(key, grid, block, smem, stream, p)
                       : launch_mlmq_f32(key, grid, block, smem, stream, p);
}
inline cudaError_t occupancy_mlmq(const KernelKey& key, int threads, size_t smem, int* blocks) {
    return key.wt == 0 ? occupancy_mlmq_u32(key, threads, smem, blocks)
                       : occupancy_mlmq_f32(key, threads, smem, blocks);
}

constexpr int kL0Rows = 2;  // L0 ring rows per warp compiled into the kernels

}  // namespace sssp
