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

// Launches mlmq_kernel for `key` (defined per weight type and variant in
// kernels_{u32,f32}{,x}.cu).  Returns the launch error.
#define SSSP_DECLARE_INSTANCES(name)                                                                  \
    cudaError_t launch_mlmq_##name(const KernelKey& key, dim3 grid, dim3 block, size_t smem,          \
                                   cudaStream_t stream, const KParams& p);                            \
    cudaError_t occupancy_mlmq_##name(const KernelKey& key, int threads, size_t smem, int* blocks);
SSSP_DECLARE_INSTANCES(u32)
SSSP_DECLARE_INSTANCES(u32x)
SSSP_DECLARE_INSTANCES(f32)
SSSP_DECLARE_INSTANCES(f32x)
#undef SSSP_DECLARE_INSTANCES

// The extended kernel runs a launch that uses one of the optional paths (or
// an L1 policy with a block lock: near-far, SLF); the lean one, compiled
// without them, runs every other launch.
inline bool needs_extended(const KParams& p) {
    return p.pend != nullptr || p.dedup != 0 || p.l2_only != 0 || p.timeline != nullptr || p.trace != nullptr ||
           p.l1_type == 1 /* near-far */ || p.l1_type == 3 /* SLF */;
}

inline cudaError_t launch_mlmq(const KernelKey& key, dim3 grid, dim3 block, size_t smem,
                               cudaStream_t stream, const KParams& p) {
    const bool x = needs_extended(p);
    if (key.wt == 0) return x ? launch_mlmq_u32x(key, grid, block, smem, stream, p)
                              : launch_mlmq_u32(key, grid, block, smem, stream, p);
    return x ? launch_mlmq_f32x(key, grid, block, smem, stream, p)
             : launch_mlmq_f32(key, grid, block, smem, stream, p);
}
// Resident blocks per SM at the given shape, for the extended kernel: the
// lean one uses no more registers or shared memory, so a grid sized by it
// is resident with either.
inline cudaError_t occupancy_mlmq(const KernelKey& key, int threads, size_t smem, int* blocks) {
    return key.wt == 0 ? occupancy_mlmq_u32x(key, threads, smem, blocks)
                       : occupancy_mlmq_f32x(key, threads, smem, blocks);
}

constexpr int kL0Rows = 2;  // L0 ring rows per warp compiled into the kernels

}  // namespace sssp
