// sssp_api.cu -- the C ABI of libsssp.so (include/sssp.h): graph upload,
// validation and device layout, per-graph workspace, single-source and
// batched solves, statistics.  Autotuning lives in sssp_autotune.cu, serving
// in sssp_serve.cu.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/sssp.h"
#include "api_internal.h"

using namespace sssp;

// ===================================================================== misc

extern "C" const char* sssp_strerror(int status) {
    switch (status) {
        case SSSP_OK: return "ok";
        case SSSP_E_INVAL: return "invalid argument";
        case SSSP_E_NOMEM: return "out of memory or queue capacity exhausted";
        case SSSP_E_CUDA: return "CUDA runtime error";
        case SSSP_E_TIMEOUT: return "device wait timed out";
        case SSSP_E_BADGRAPH: return "invalid CSR graph";
        case SSSP_E_BUSY: return "server busy";
        case SSSP_E_NODEV: return "no CUDA device";
        case SSSP_E_NOTFOUND: return "unknown ticket";
        case SSSP_E_CANCELLED: return "query cancelled";
        default: return "unknown status";
    }
}

extern "C" int sssp_version(void) { return 2 * 10000 + 0 * 100 + 0; }

namespace sssp {

static int debug_level() {
    const char* e = std::getenv("SSSP_DEBUG");
    return e ? std::atoi(e) : 0;
}

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return SSSP_OK;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return SSSP_E_NOMEM;
    }
    if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) return SSSP_E_NODEV;
    return SSSP_E_CUDA;
}

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static uint32_t next_pow2(uint64_t v) {
    uint64_t p = 1;
    while (p < v && p < (1ull << 31)) p <<= 1;
    return (uint32_t)p;
}

static int grid_for(size_t count, int sms) {
    size_t b = (count + 255) / 256;
    size_t cap = (size_t)sms * 8;
    return (int)std::max<size_t>(1, std::min(b, cap));
}

// ------------------------------------------------------------ small kernels

__global__ void fill_u32_kernel(uint32_t* p, size_t count, uint32_t value) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t stride = (size_t)gridDim.x * blockDim.x;
    for (; i < count; i += stride) p[i] = value;
}

__global__ void fill_u64_kernel(unsigned long long* p, size_t count, unsigned long long value) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t stride = (size_t)gridDim.x * blockDim.x;
    for (; i < count; i += stride) p[i] = value;
}

// Queue metadata to the empty state: seq[r][s] = s ("free for ticket s").
__global__ void ring_reset_kernel(Rings r, uint32_t nrings, Ctrl* ctrl) {
    size_t total = (size_t)nrings * r.nch;
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t k = i; k < total; k += stride) {
        r.seq[k] = (uint32_t)(k & (r.nch - 1u));
        r.cnt[k] = 0;
    }
    for (size_t k = i; k < (size_t)nrings * 32; k += stride) {
        r.rt[k] = 0;
        r.wt[k] = 0;
    }
    if (i == 0) {
        ctrl->reserve = 0;
        ctrl->done = 0;
        ctrl->window = 0;
        ctrl->finished = 0;
        ctrl->error = 0;
    }
}

// Resets the control block and puts the sources straight into the current
// L2 bucket, as the start-up of Section 4.1 does; reserve = number of
// queries.  One warp.
__global__ void seed_kernel(KParams P, const int32_t* srcs, int32_t src0, int32_t nq, int packed) {
    Ctrl* C = P.ctrl;
    const uint32_t lane = threadIdx.x & 31u;
    __shared__ uint32_t cur_s;
    if (lane == 0) {
        C->reserve = (unsigned long long)nq;
        C->processed = 0;
        C->done = 0;
        C->finished = 0;
        C->error = 0;
        C->err_where = 0;
        C->err_info = 0;
        for (int i = 0; i < kStCount; i++) C->stats[i] = 0;
        C->window = 0;  // sources sit in absolute bucket 0
        cur_s = 0;
    }
    __syncwarp();
    const uint32_t ring = cur_s * (uint32_t)P.shards;  // bucket 0, shard 0
    uint32_t* wtp = P.l2.wt + (size_t)ring * 32;
    for (int32_t base = 0; base < nq; base += 32) {
        int32_t q = base + (int32_t)lane;
        bool valid = q < nq;
        uint32_t t = 0;
        int ok = 1;
        if (lane == 0) {
            t = *wtp;
            *wtp = t + 1u;
            if (P.l2.seq[(size_t)ring * P.l2.nch + (t & (P.l2.nch - 1u))] != t) ok = 0;
        }
        ok = __shfl_sync(kFull, ok, 0);
        if (!ok) {
            if (lane == 0) C->error = kErrState;
            return;
        }
        t = __shfl_sync(kFull, t, 0);
        const size_t slot = (size_t)ring * P.l2.nch + (t & (P.l2.nch - 1u));
        if (valid) {
            int32_t s = srcs ? srcs[q] : src0;
            uint32_t key = P.vbits ? (((uint32_t)q << P.vbits) | (uint32_t)s) : (uint32_t)s;
            P.l2.data[slot * kChunk + lane] = make_uint2(key, 0u);
            size_t di = (size_t)q * (size_t)P.nv + (size_t)s;
            if (P.pend) P.pend[di] = 0u;   // queued at bucket 0
            if (packed)
                reinterpret_cast<unsigned long long*>(P.dist)[di] = (unsigned long long)(uint32_t)s;
            else
                reinterpret_cast<uint32_t*>(P.dist)[di] = 0u;
        }
        __syncwarp();
        if (lane == 0) {
            int32_t c = nq - base < 32 ? nq - base : 32;
            P.l2.cnt[slot] = (uint32_t)c;
            __threadfence();
            P.l2.seq[slot] = t + 1u;
        }
        __syncwarp();
    }
    __threadfence();
}

// Work slices [nq][nv] -> outputs [nq][n]: (dist << 32 | pred) words split
// into dist / pred (packed), or plain distance words copied (!packed).
__global__ void unpack_kernel(const void* work, int packed, int32_t nq, int32_t n, int32_t nv,
                              uint32_t* dist, int32_t* pred, int f32) {
    const size_t count = (size_t)nq * (size_t)n;
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t stride = (size_t)gridDim.x * blockDim.x;
    for (; i < count; i += stride) {
        size_t q = i / (size_t)n, v = i - q * (size_t)n;
        size_t src = q * (size_t)nv + v;
        if (packed) {
            unsigned long long x = reinterpret_cast<const unsigned long long*>(work)[src];
            uint32_t d = (uint32_t)(x >> 32);
            if (f32 && d == kInfU32) d = kInfF32;
            dist[i] = d;
            if (pred) pred[i] = (int32_t)(uint32_t)x;
        } else {
            dist[i] = reinterpret_cast<const uint32_t*>(work)[src];
        }
    }
}

// CSR validation: flags bit 0 = row_ptr, bit 1 = col range, bit 2 = bad f32 weight.
__global__ void validate_rows_kernel(const int32_t* row_ptr, int32_t n, int64_t m, int* flags) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; i <= n; i += stride) {
        int32_t r = row_ptr[i];
        bool bad = (i == 0 && r != 0) || (i == n && (int64_t)r != m) || r < 0 || (int64_t)r > m ||
                   (i < n && row_ptr[i + 1] < r);
        if (bad) atomicOr(flags, 1);
    }
}

// Packs (col, weight) pairs, normalising -0.0 to +0.0 and validating.
__global__ void pack_kernel(const int32_t* col, const uint32_t* w, int64_t m, int32_t n, int f32,
                            uint2* adj, int* flags) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; i < m; i += stride) {
        int32_t c = col[i];
        uint32_t wb = w[i];
        if (c < 0 || c >= n) atomicOr(flags, 2);
        if (f32) {
            if (wb == 0x80000000u) wb = 0u;                      // -0.0 -> +0.0
            if ((wb & 0x80000000u) || (wb & 0x7f800000u) == 0x7f800000u) atomicOr(flags, 4);
        }
        adj[i] = make_uint2((uint32_t)c, wb);
    }
}

// Shadow layout: vertex v with sfirst[v] >= 0 gets arcs to its shadows
// sfirst[v] .. sfirst[v] + k - 1 (weight 0), and shadow j owns the arc slice
// [j * split, (j + 1) * split) of v.  One warp per vertex.
__global__ void relayout_kernel(const int32_t* rp0, const uint2* adj0, int32_t n, const int32_t* rp1,
                                const int32_t* sfirst, int32_t split, uint2* adj1) {
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t lane = threadIdx.x & 31u;
    for (int64_t v = wid; v < n; v += nw) {
        const int32_t b0 = rp0[v], e0 = rp0[v + 1];
        const int32_t s0 = sfirst[v];
        if (s0 < 0) {
            const int32_t b1 = rp1[v];
            for (int32_t e = b0 + (int32_t)lane; e < e0; e += 32) adj1[b1 + (e - b0)] = adj0[e];
        } else {
            const int32_t k = (e0 - b0 + split - 1) / split;
            const int32_t b1 = rp1[v];
            for (int32_t j = (int32_t)lane; j < k; j += 32) adj1[b1 + j] = make_uint2((uint32_t)(s0 + j), 0u);
            for (int32_t j = 0; j < k; j++) {
                const int32_t lo = b0 + j * split, hi = min(e0, lo + split);
                const int32_t d1 = rp1[s0 + j];
                for (int32_t e = lo + (int32_t)lane; e < hi; e += 32) adj1[d1 + (e - lo)] = adj0[e];
            }
        }
    }
}

// Table 2 features: sums for degree and weight moments.
struct FeatAcc {
    double sdeg, sdeg2, sw, sw2;
    unsigned int maxdeg;
    unsigned int maxw_bits;   // u32 value or f32 bits (non-negative floats order like ints)
    unsigned int minw_bits;
    unsigned int zero_w;
};

__global__ void features_kernel(const int32_t* row_ptr, int32_t n, const uint2* adj, int64_t m,
                                int f32, FeatAcc* acc) {
    double sd = 0, sd2 = 0, sw = 0, sw2 = 0;
    unsigned int md = 0, mw = 0, mnw = 0xffffffffu, zw = 0;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = i; v < n; v += stride) {
        double d = (double)(row_ptr[v + 1] - row_ptr[v]);
        sd += d;
        sd2 += d * d;
        md = max(md, (unsigned int)d);
    }
    for (int64_t e = i; e < m; e += stride) {
        uint32_t wb = adj[e].y;
        double x = f32 ? (double)__uint_as_float(wb) : (double)wb;
        sw += x;
        sw2 += x * x;
        mw = max(mw, wb);
        mnw = min(mnw, wb);
        zw |= (wb == 0u);
    }
    for (int o = 16; o > 0; o >>= 1) {
        sd += __shfl_down_sync(kFull, sd, o);
        sd2 += __shfl_down_sync(kFull, sd2, o);
        sw += __shfl_down_sync(kFull, sw, o);
        sw2 += __shfl_down_sync(kFull, sw2, o);
        md = max(md, __shfl_down_sync(kFull, md, o));
        mw = max(mw, __shfl_down_sync(kFull, mw, o));
        mnw = min(mnw, __shfl_down_sync(kFull, mnw, o));
        zw |= __shfl_down_sync(kFull, zw, o);
    }
    if ((threadIdx.x & 31u) == 0) {
        atomicAdd(&acc->sdeg, sd);
        atomicAdd(&acc->sdeg2, sd2);
        atomicAdd(&acc->sw, sw);
        atomicAdd(&acc->sw2, sw2);
        atomicMax(&acc->maxdeg, md);
        atomicMax(&acc->maxw_bits, mw);
        atomicMin(&acc->minw_bits, mnw);
        atomicOr(&acc->zero_w, zw);
    }
}

// ================================================================ workspace

void Workspace::release() {
    cudaFree(ring_mem);
    cudaFree(ctrl);
    cudaFree(d64);
    cudaFree(d32);
    cudaFree(out_d);
    cudaFree(out_p);
    cudaFree(srcs);
    cudaFree(pend);
    cudaFree(tl);
    if (host_ctrl) cudaFreeHost(host_ctrl);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    if (ev2) cudaEventDestroy(ev2);
    *this = Workspace();
}

template <typename T>
static int grow(T** p, size_t* have, size_t want) {
    if (*have >= want && *p) return SSSP_OK;
    cudaFree(*p);
    *p = nullptr;
    *have = 0;
    cudaError_t e = cudaMalloc((void**)p, std::max<size_t>(want, 1) * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return SSSP_E_NOMEM;
    }
    *have = want;
    return SSSP_OK;
}

int Workspace::ensure_queue(uint32_t nr, uint32_t nch_want, uint32_t margin, cudaStream_t s, int sms) {
    if (!ev0) {
        if (cudaEventCreate(&ev0) != cudaSuccess || cudaEventCreate(&ev1) != cudaSuccess ||
            cudaEventCreate(&ev2) != cudaSuccess)
            return SSSP_E_CUDA;
    }
    if (!host_ctrl) {
        if (cudaMallocHost((void**)&host_ctrl, sizeof(Ctrl)) != cudaSuccess) return SSSP_E_NOMEM;
    }
    if (!ctrl) {
        if (cudaMalloc((void**)&ctrl, sizeof(Ctrl)) != cudaSuccess) return SSSP_E_NOMEM;
        cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), s);
    }
    const bool realloc = !ring_mem || nr != nrings || nch_want > rings.nch;
    if (realloc) {
        const uint32_t nch = std::max(nch_want, nr == nrings ? rings.nch : 0u);
        cudaFree(ring_mem);
        ring_mem = nullptr;
        const size_t tickets = (size_t)nr * 32 * sizeof(uint32_t);
        const size_t meta = (size_t)nr * nch * sizeof(uint32_t);
        const size_t data = (size_t)nr * nch * kChunk * sizeof(uint2);
        const size_t bytes = 2 * tickets + 2 * meta + data + 256;
        if (cudaMalloc((void**)&ring_mem, bytes) != cudaSuccess) {
            cudaGetLastError();
            ring_mem = nullptr;
            nrings = 0;
            return SSSP_E_NOMEM;
        }
        char* p = ring_mem;
        rings.data = reinterpret_cast<uint2*>(p);
        p += data;
        rings.rt = reinterpret_cast<uint32_t*>(p);
        p += tickets;
        rings.wt = reinterpret_cast<uint32_t*>(p);
        p += tickets;
        rings.seq = reinterpret_cast<uint32_t*>(p);
        p += meta;
        rings.cnt = reinterpret_cast<uint32_t*>(p);
        rings.nch = nch;
        nrings = nr;
        ring_bytes = bytes;
        dirty = true;
    }
    rings.margin = margin;
    if (dirty) {
        ring_reset_kernel<<<grid_for((size_t)nrings * rings.nch, sms), 256, 0, s>>>(rings, nrings, ctrl);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_status(e);
        dirty = false;
    }
    return SSSP_OK;
}

// ================================================================= configs

static void config_defaults(sssp_config* c) {
    std::memset(c, 0, sizeof(*c));
    c->l1_type = SSSP_L1_FILTER;
    c->l2_type = SSSP_L2_BUCKET;
    c->l0_rows = kL0Rows;
    c->l1_cap = 2048;
    c->wb = 0;
    c->delta_u32 = 0;     // 0 = derive from the graph's weights
    c->delta_f32 = 0.0f;
    c->bnum = 4;
    c->bmax = 32;
    c->filter_deltas = 1.0f;
    c->near_deltas = 1.0f;
    c->max_arcs = 4096;
    c->claim = 4;
    c->refillers = 8;
    c->stage = 1;
    c->shards = 8;
    c->block_threads = 512;
    c->blocks_per_sm = 0;
    c->timeout_ms = 0;
    c->split_arcs = 0;
    c->hub_bnum = 0;
    c->dedup = 0;
    c->pending_marks = 0;
    c->direct_buckets = 2;
}

// Fills auto fields from the graph features (the prior of Section 3.5).
void resolve_auto(const Graph* g, sssp_config* c) {
    const sssp_features& f = g->feat;
    double avgdeg = std::max(1.0, f.avg_deg);
    if (g->wtype == SSSP_W_U32 && c->delta_u32 == 0) {
        // delta-stepping width: about the average weight over the average
        // degree (Meyer & Sanders use ~ w_max / degree), at least 1
        double d = std::max(1.0, f.avg_w * 4.0 / avgdeg);
        c->delta_u32 = (uint32_t)std::min(d, 4.0e9);
    }
    if (g->wtype == SSSP_W_F32 && !(c->delta_f32 > 0.0f)) {
        double d = std::max(1e-6, f.avg_w * 4.0 / avgdeg);
        c->delta_f32 = (float)d;
    }
    if (c->l2_type == SSSP_L2_VECTOR) {
        c->bmax = 1;
        c->bnum = 1;
    }
}

// A multi-query launch draws its parallelism from its queries, not from
// wide buckets: narrower buckets (delta / div) cut the out-of-order work
// that the shared window admits.  On GB300, 256 R-MAT-20 sources run 1.6x
// (u32) to 2.4x (f32) faster with delta / 8 than with the single-source delta.
// The width starts from the general weight-based delta (not a per-family
// single-source tuning of it).
void batch_delta(const Graph* g, sssp_config* c, int div) {
    c->delta_u32 = 0;
    c->delta_f32 = 0.0f;
    resolve_auto(g, c);
    if (div <= 1) return;
    if (g->wtype == SSSP_W_F32) c->delta_f32 = c->delta_f32 / (float)div;
    else c->delta_u32 = std::max<uint32_t>(1u, c->delta_u32 / (uint32_t)div);
}

int32_t nq_class(int32_t nq) {
    int32_t c = 1;
    while (c <= nq / 2) c *= 2;
    return c;
}

const sssp_config* batch_tuned_for(const Graph* g, int32_t nq) {
    const int32_t k = nq_class(nq);
    for (const Graph::BatchTuned& b : g->batch_tuned)
        if (b.nq_class == k) return &b.cfg;
    return nullptr;
}

const sssp_config* batch_tuned_largest(const Graph* g) {
    const Graph::BatchTuned* best = nullptr;
    for (const Graph::BatchTuned& b : g->batch_tuned)
        if (!best || b.nq_class > best->nq_class) best = &b;
    return best ? &best->cfg : nullptr;
}

int validate_config(const sssp_config* c) {
    auto pow2 = [](int v) { return v > 0 && (v & (v - 1)) == 0; };
    if (c->l1_type < 0 || c->l1_type > 3) return SSSP_E_INVAL;
    if (c->l2_type < 0 || c->l2_type > 1) return SSSP_E_INVAL;
    if (c->l0_rows != kL0Rows) return SSSP_E_INVAL;
    if (!pow2(c->l1_cap) || c->l1_cap < 256 || c->l1_cap > 16384) return SSSP_E_INVAL;
    if (c->wb < 0) return SSSP_E_INVAL;
    if (c->bmax < 1 || c->bmax > 32 || c->bnum < 1 || c->bnum > 32) return SSSP_E_INVAL;
    if (!(c->filter_deltas >= 0.0f) || !(c->near_deltas >= 0.0f)) return SSSP_E_INVAL;
    if (c->max_arcs < 32) return SSSP_E_INVAL;
    if (c->claim < 1 || c->claim > kMaxClaim) return SSSP_E_INVAL;
    if (c->refillers < 1 || c->refillers > 32) return SSSP_E_INVAL;
    if (!pow2(c->shards) || c->shards > 32) return SSSP_E_INVAL;
    if (c->block_threads != 256 && c->block_threads != 512 && c->block_threads != 1024) return SSSP_E_INVAL;
    if (c->blocks_per_sm < 0 || c->blocks_per_sm > 8 || c->timeout_ms < 0) return SSSP_E_INVAL;
    if (c->stage < 0 || c->stage > 1) return SSSP_E_INVAL;
    if (c->l2_only < 0 || c->l2_only > 1) return SSSP_E_INVAL;
    if (c->split_arcs != 0 && (c->split_arcs < 32 || c->split_arcs > (1 << 30))) return SSSP_E_INVAL;
    if (c->hub_bnum < 0 || c->hub_bnum > 32 || c->dedup < 0 || c->dedup > 1) return SSSP_E_INVAL;
    if (c->pending_marks < 0 || c->pending_marks > 1) return SSSP_E_INVAL;
    if (c->direct_buckets < 0 || c->direct_buckets > 32) return SSSP_E_INVAL;
    return SSSP_OK;
}

// ================================================================== launch plan

int pred_mode_for(const Graph* g) {
    // the packed atomicMin keeps the smallest-index tight predecessor when
    // every weight is >= 1; otherwise strict improvements decide (CAS)
    return (g->wtype == SSSP_W_U32 && g->feat.min_w >= 1.0) ? 1 : 2;
}

int plan_launch(const Graph* g, const sssp_config& cfg, int pred_mode, bool mq, LaunchPlan* out, bool unit) {
    LaunchPlan& L = *out;
    const bool f32 = g->wtype == SSSP_W_F32 && !unit;
    L.key = KernelKey{f32 ? 1 : 0, pred_mode, mq ? 1 : 0};
    // shared-memory layout of one block
    L.threads = cfg.block_threads;
    const int warps_per_block = L.threads / 32;
    const size_t scratch_off = (sizeof(BlockShared) + 15) & ~size_t(15);
    const size_t far_off = scratch_off + (size_t)warps_per_block * 32 * sizeof(uint2);
    const size_t stat_off = far_off + (size_t)warps_per_block * kFarCap * sizeof(uint2);
    const size_t stage_off = stat_off + (size_t)warps_per_block * kStCount * sizeof(unsigned long long);
    const size_t l1_off = stage_off + (cfg.stage ? (size_t)cfg.bmax * kStageCap * sizeof(uint2) : 0);
    L.smem = l1_off + (size_t)cfg.l1_cap * sizeof(uint2);
    int occ = 0;
    cudaError_t ce = occupancy_mlmq(L.key, L.threads, L.smem, &occ);
    if (ce != cudaSuccess) return cuda_status(ce);
    if (occ < 1) return SSSP_E_INVAL;
    L.bps = cfg.blocks_per_sm > 0 ? std::min(cfg.blocks_per_sm, occ) : occ;
    L.grid = g->sms * L.bps;

    KParams& P = L.P;
    std::memset(&P, 0, sizeof(P));
    P.row_ptr = g->row_ptr;
    P.adj = g->adj;
    P.owner = g->owner;
    P.n = g->n;
    P.nv = g->nv;
    P.nq = 1;
    P.vmask = 0xffffffffu;
    P.shards = cfg.shards;
    P.delta = f32 ? __float_as_uint_host(cfg.delta_f32) : cfg.delta_u32;
    P.unit_w = unit ? 1 : 0;
    // breadth-first search reads claimed chunks through L1: with descriptors,
    // 5 of 16 R-MAT-22 sources took 1.4-2.3x longer (far more idle warps)
    P.desc = unit ? 0 : 1;
    // hub rings need two shard halves and a bucketed L2
    P.hub_bnum = (cfg.shards >= 2 && cfg.bmax > 1 && !cfg.l2_only) ? cfg.hub_bnum : 0;
    P.dedup = cfg.dedup;
    P.direct = (uint32_t)cfg.direct_buckets;
    P.bnum = std::min(cfg.bnum, cfg.bmax);
    P.bmax = cfg.bmax;
    P.l1_type = cfg.l1_type;
    P.l1_cap = cfg.l1_cap;
    P.wb = cfg.l1_type == SSSP_L1_VECTOR ? cfg.wb : 0;
    P.filter_deltas = cfg.filter_deltas;
    if (cfg.near_deltas > 0.0f) {
        if (f32)
            P.near_w = __float_as_uint_host(cfg.delta_f32 * cfg.near_deltas);
        else
            P.near_w = (uint32_t)std::min(4294967295.0, (double)cfg.delta_u32 * cfg.near_deltas);
    } else {
        P.near_w = kInfU32;   // every write enters L0, as in Listing 1
    }
    P.max_arcs = cfg.max_arcs;
    P.claim = cfg.claim;
    P.refillers = cfg.refillers;
    P.scratch_off = (int32_t)scratch_off;
    P.far_off = (int32_t)far_off;
    P.stat_off = (int32_t)stat_off;
    P.stage_off = (int32_t)stage_off;
    P.l2_only = cfg.l2_only ? 1 : 0;
    P.stage = cfg.stage && !cfg.l2_only ? 1 : 0;
    if (cfg.l2_only) P.claim = 1;
    P.l1_off = (int32_t)l1_off;
    const int tmo = cfg.timeout_ms > 0 ? cfg.timeout_ms : 20000;
    P.timeout_ns = (unsigned long long)tmo * 1000000ull;
    return SSSP_OK;
}

// ================================================================== solve

int run_queries(Graph* g, const int32_t* srcs_host, const int32_t* srcs_dev, int32_t src0, int32_t nq,
                void* dist_out, int32_t* pred_out, const sssp_config* cfg_in, cudaStream_t stream,
                sssp_stats* st_out, bool unit, const Sampling* samp) {
    // a multi-query launch with the library's configuration uses the
    // batch-tuned one of its size class when sssp_autotune_batch made one
    if (!cfg_in && nq > 1 && !unit) cfg_in = batch_tuned_for(g, nq);
    sssp_config cfg = cfg_in ? *cfg_in : (g->tuned_valid ? g->tuned : g->defaults);
    // breadth-first: one bucket per level unless the caller chose a delta
    if (unit && (!cfg_in || cfg.delta_u32 == 0)) cfg.delta_u32 = 1;
    const bool lib_delta = !cfg_in || (g->wtype == SSSP_W_F32 ? !(cfg_in->delta_f32 > 0.0f) : cfg_in->delta_u32 == 0);
    resolve_auto(g, &cfg);
    if (nq > 1 && !unit && lib_delta) batch_config(g, &cfg, nq);
    int rc = validate_config(&cfg);
    if (rc) return rc;
    if (cudaSetDevice(g->device) != cudaSuccess) return SSSP_E_CUDA;
    rc = ensure_layout(g, cfg.split_arcs ? cfg.split_arcs : kDefaultSplit, stream);
    if (rc) return rc;
    const int32_t n = g->n, nv = g->nv;
    const bool mq = nq > 1;
    int vbits = 0;
    if (mq) {
        while (vbits < 31 && (1ll << vbits) <= (long long)nv) vbits++;  // 2^vbits > nv: no key is all ones
        if (vbits == 0) vbits = 1;
        if ((unsigned long long)nq << vbits > (1ull << 32)) return SSSP_E_INVAL;
    }
    // unit weights are >= 1: the packed minimum gives the smallest-index parent
    const int pred_mode = pred_out ? (unit ? 1 : pred_mode_for(g)) : 0;
    const bool f32 = g->wtype == SSSP_W_F32 && !unit;
    LaunchPlan plan;
    rc = plan_launch(g, cfg, pred_mode, mq, &plan, unit);
    if (rc) return rc;
    const KernelKey key = plan.key;
    const int shards = cfg.shards;
    const int threads = plan.threads;
    const int grid = plan.grid;
    const size_t smem = plan.smem;
    const uint32_t warps = (uint32_t)(grid * (threads / 32));
    cudaError_t ce = cudaSuccess;

    Workspace& ws = g->ws;
    const size_t cells = (size_t)nq * (size_t)nv;       // work slices
    const size_t ocells = (size_t)nq * (size_t)n;       // outputs
    const bool dist_dev = is_device_ptr(dist_out);
    const bool pred_dev = pred_out && is_device_ptr(pred_out);
    const int dbg = debug_level();
    int attempts = 0;
    for (;;) {
        attempts++;
        // L2 capacity: ~ cells / 8 chunks over all rings, at least 2x the
        // writer margin per ring; doubled after an overflow.
        const uint32_t nr = (uint32_t)(cfg.bmax * shards);
        const uint64_t total_chunks = (std::max<uint64_t>(cells / 8, 4096)) << ws.grow_shift;
        const uint32_t nch = next_pow2(std::max<uint64_t>(total_chunks / nr + warps,
                                                          2ull * warps + (uint64_t)(nq / 32 + 2)));
        rc = ws.ensure_queue(nr, nch, warps, stream, g->sms);
        if (rc) return rc;
        // distance work buffer
        void* work = nullptr;
        if (pred_mode) {
            rc = grow(&ws.d64, &ws.d64_n, cells);
            if (rc) return rc;
            work = ws.d64;
        } else if (dist_dev && nv == n) {
            work = dist_out;
        } else {
            rc = grow(&ws.d32, &ws.d32_n, cells);
            if (rc) return rc;
            work = ws.d32;
        }
        const int32_t* srcs_d = nullptr;
        if (nq > 1) {
            rc = grow(&ws.srcs, &ws.srcs_n, (size_t)nq);
            if (rc) return rc;
            if (srcs_dev)
                cudaMemcpyAsync(ws.srcs, srcs_dev, sizeof(int32_t) * nq, cudaMemcpyDeviceToDevice, stream);
            else
                cudaMemcpyAsync(ws.srcs, srcs_host, sizeof(int32_t) * nq, cudaMemcpyHostToDevice, stream);
            srcs_d = ws.srcs;
        }

        uint32_t* pend = nullptr;
        if (cfg.pending_marks) {
            rc = grow(&ws.pend, &ws.pend_n, cells);
            if (rc) return rc;
            pend = ws.pend;
        }
        KParams P = plan.P;
        P.nq = nq;
        P.dist = work;
        P.pend = pend;
        P.vbits = mq ? vbits : 0;
        P.vmask = mq ? ((1u << vbits) - 1u) : 0xffffffffu;
        P.l2 = ws.rings;
        P.ctrl = ws.ctrl;
        const int tmo = cfg.timeout_ms > 0 ? cfg.timeout_ms : 20000;

        cudaEventRecord(ws.ev0, stream);
        if (pred_mode)
            fill_u64_kernel<<<grid_for(cells, g->sms), 256, 0, stream>>>(ws.d64, cells, ~0ull);
        else
            fill_u32_kernel<<<grid_for(cells, g->sms), 256, 0, stream>>>(
                (uint32_t*)work, cells, f32 ? kInfF32 : kInfU32);
        if (pend) fill_u32_kernel<<<grid_for(cells, g->sms), 256, 0, stream>>>(pend, cells, kInfU32);
        seed_kernel<<<1, 32, 0, stream>>>(P, srcs_d, src0, nq, pred_mode ? 1 : 0);
        cudaEventRecord(ws.ev1, stream);
        // run-time sampling (sssp_solve_sampled, or SSSP_DEBUG >= 4: printed)
        const bool sampling = samp != nullptr || dbg > 3;
        const int tl_cap = samp ? samp->cap : 4096;
        if (sampling) {
            rc = grow(&ws.tl, &ws.tl_n, (size_t)tl_cap * kTimelineFields);
            if (rc) return rc;
            cudaMemsetAsync(ws.tl, 0xff, (size_t)tl_cap * kTimelineFields * 8, stream);
            P.timeline = ws.tl;
            P.timeline_cap = tl_cap;
            P.timeline_ns = (uint32_t)(samp ? samp->period_us : 20) * 1000u;
        }
        unsigned long long* trace_h = nullptr;
        const size_t nthreads_total = (size_t)grid * threads;
        if (dbg > 2 && cudaHostAlloc((void**)&trace_h, nthreads_total * 8, cudaHostAllocMapped) == cudaSuccess) {
            std::memset(trace_h, 0, nthreads_total * 8);
            cudaHostGetDevicePointer((void**)&P.trace, trace_h, 0);
        }
        if (dbg > 2)
            std::fprintf(stderr, "[sssp] launch wt=%d pred=%d mq=%d nq=%d n=%d nv=%d grid=%d threads=%d smem=%zu "
                                 "bmax=%d shards=%d l1=%d nch=%u\n", key.wt, key.pred, key.mq, nq, n, nv, grid,
                         threads, smem, P.bmax, P.shards, P.l1_type, P.l2.nch);
        ce = launch_mlmq(key, dim3(grid), dim3(threads), smem, stream, P);
        if (ce != cudaSuccess) {
            if (dbg) std::fprintf(stderr, "[sssp] launch failed: %s (grid=%d threads=%d smem=%zu)\n",
                                  cudaGetErrorString(ce), grid, threads, smem);
            if (trace_h) cudaFreeHost(trace_h);
            return cuda_status(ce);
        }
        cudaEventRecord(ws.ev2, stream);
        // outputs
        const bool copy_needed = pred_mode || work != dist_out;
        if (copy_needed) {
            uint32_t* dd = (uint32_t*)dist_out;
            int32_t* pp = pred_out;
            if (!dist_dev) {
                rc = grow(&ws.out_d, &ws.out_d_n, ocells);
                if (rc) return rc;
                dd = ws.out_d;
            }
            if (pred_out && !pred_dev) {
                rc = grow(&ws.out_p, &ws.out_p_n, ocells);
                if (rc) return rc;
                pp = ws.out_p;
            }
            unpack_kernel<<<grid_for(ocells, g->sms), 256, 0, stream>>>(work, pred_mode ? 1 : 0, nq, n, nv, dd,
                                                                        pred_mode ? pp : nullptr, f32);
            if (!dist_dev) cudaMemcpyAsync(dist_out, dd, ocells * 4, cudaMemcpyDeviceToHost, stream);
            if (pred_out && !pred_dev) cudaMemcpyAsync(pred_out, pp, ocells * 4, cudaMemcpyDeviceToHost, stream);
        }
        cudaMemcpyAsync(ws.host_ctrl, ws.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, stream);
        if (trace_h) {
            // debug: poll instead of blocking; report where lanes sit if the solve overruns
            auto t0 = std::chrono::steady_clock::now();
            bool reported = false;
            while (cudaStreamQuery(stream) == cudaErrorNotReady) {
                double el = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
                if (!reported && el > (double)tmo + 3000.0) {
                    unsigned long long hist[64] = {0};
                    for (size_t i = 0; i < nthreads_total; i++) hist[(trace_h[i] >> 48) & 63]++;
                    std::fprintf(stderr, "[sssp] OVERRUN %.0f ms; lanes by location:", el);
                    for (int c = 0; c < 64; c++)
                        if (hist[c]) std::fprintf(stderr, " %d:%llu", c, hist[c]);
                    std::fprintf(stderr, "\n");
                    for (size_t wv = 0; wv < nthreads_total / 32; wv++) {
                        bool live = false;
                        for (int l = 0; l < 32; l++)
                            if ((unsigned)(trace_h[wv * 32 + l] >> 48) != 13) live = true;
                        if (!live) continue;
                        std::fprintf(stderr, "[sssp]  warp %zu (block %zu):", wv, wv / (threads / 32));
                        for (int l = 0; l < 32; l++)
                            std::fprintf(stderr, " %u/%llu", (unsigned)(trace_h[wv * 32 + l] >> 48),
                                         trace_h[wv * 32 + l] & 0xffffffffffffull);
                        std::fprintf(stderr, "\n");
                    }
                    reported = true;
                }
                std::this_thread::sleep_for(std::chrono::milliseconds(1));
            }
            cudaFreeHost(trace_h);
        }
        ce = cudaStreamSynchronize(stream);
        if (ce != cudaSuccess) {
            if (dbg) std::fprintf(stderr, "[sssp] stream error: %s\n", cudaGetErrorString(ce));
            return cuda_status(ce);
        }
        if (sampling) {
            std::vector<unsigned long long> tl((size_t)tl_cap * kTimelineFields);
            if (cudaMemcpy(tl.data(), ws.tl, tl.size() * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
                return SSSP_E_CUDA;
            int ns = 0;
            while (ns < tl_cap && tl[(size_t)ns * kTimelineFields] != ~0ull) ns++;
            if (samp) {
                std::memcpy(samp->out, tl.data(), (size_t)ns * kTimelineFields * 8);
                *samp->n_out = ns;
            }
            if (dbg > 3) {
                std::fprintf(stderr, "[sssp] timeline (us, L2 written, L2 done, processed, window, busy warps of "
                                     "block 0):\n");
                for (int i = 0; i < ns; i++) {
                    const unsigned long long* o = tl.data() + (size_t)i * kTimelineFields;
                    std::fprintf(stderr, "[sssp]   %8.1f %12llu %12llu %12llu %8llu %3llu\n", o[0] / 1000.0, o[1],
                                 o[2], o[3], o[4], o[5]);
                }
            }
        }
        const Ctrl& hc = *ws.host_ctrl;
        float ms_kernel = 0, ms_total = 0;
        cudaEventElapsedTime(&ms_kernel, ws.ev1, ws.ev2);
        cudaEventElapsedTime(&ms_total, ws.ev0, ws.ev2);
        sssp_stats st;
        std::memset(&st, 0, sizeof(st));
        st.kernel_ms = ms_kernel;
        st.total_ms = ms_total;
        st.reached = -1;
        st.reached_arcs = -1;
        st.pops_l0 = (int64_t)hc.stats[kStPopL0];
        st.pops_l1 = (int64_t)hc.stats[kStPopL1];
        st.pops_l2 = (int64_t)hc.stats[kStPopL2];
        st.refills = (int64_t)hc.stats[kStRefill];
        st.relax_arcs = (int64_t)hc.stats[kStRelax];
        st.improved = (int64_t)hc.stats[kStImproved];
        st.stale = (int64_t)hc.stats[kStStale];
        st.l2_chunks_written = (int64_t)hc.stats[kStChunks];
        st.l1_flushes = (int64_t)hc.stats[kStFlush];
        st.far_pushes = (int64_t)hc.stats[kStFar];
        st.cas_fail = (int64_t)hc.stats[kStCasFail];
        st.deferred = (int64_t)hc.stats[kStDeferred];
        st.relax_shadow = (int64_t)hc.stats[kStRelaxShadow];
        for (int k = 0; k < 6; k++) st.cycles[k] = (int64_t)hc.stats[kCyRelax + k];
        st.grid_blocks = grid;
        st.block_threads = threads;
        st.attempts = attempts;
        st.dup_targets = (int64_t)hc.stats[kStDup];
        st.rounds = (int64_t)hc.stats[kStRounds];
        st.refill_tries = (int64_t)hc.stats[kStRefillTry];
        st.wait_spins = (int64_t)hc.stats[kStWaitSpin];
        st.idle_iters = (int64_t)hc.stats[kStIdleIter];
        st.window_pull_backs = (int64_t)hc.stats[kStPullBack];
        st.window_advances = (int64_t)hc.stats[kStAdvance];
        st.lock_spins = (int64_t)hc.stats[kStLockSpin];
        st.cycles_fine[0] = (int64_t)hc.stats[kCyRound];
        st.cycles_fine[1] = (int64_t)hc.stats[kCyPush];
        st.cycles_fine[2] = (int64_t)hc.stats[kCyBatch];
        st.cycles_fine[3] = (int64_t)hc.stats[kCyFarFlush];
        st.cycles_fine[4] = (int64_t)hc.stats[kCyLock];
        st.cycles_fine[5] = (int64_t)hc.stats[kCyClaim];
        st.cycles_fine[6] = (int64_t)hc.stats[kCyChunks];
        st.cycles_fine[7] = (int64_t)hc.stats[kCyStage];
        st.not_queued = (int64_t)hc.stats[kStMarked];
        g->last = st;
        if (st_out) *st_out = st;
        if (dbg > 1)
            std::fprintf(stderr, "[sssp] nq=%d n=%d kernel %.3f ms pops l0/l1/l2 %lld/%lld/%lld refills %lld relax %lld "
                                 "improved %lld far %lld stale %lld chunks %lld casfail %lld err %d fin %d\n",
                         nq, n, ms_kernel, (long long)st.pops_l0, (long long)st.pops_l1, (long long)st.pops_l2,
                         (long long)st.refills, (long long)st.relax_arcs, (long long)st.improved,
                         (long long)st.far_pushes, (long long)st.stale, (long long)st.l2_chunks_written,
                         (long long)st.cas_fail, hc.error, hc.finished);
        if (dbg > 1)
            std::fprintf(stderr, "[sssp]   iter %llu rounds %llu idle %llu refill_try %llu refills %llu lock_spin %llu "
                                 "wait_spin %llu cycles relax/l1/l2w/gread/idle/l0 %llu/%llu/%llu/%llu/%llu/%llu\n",
                         hc.stats[kStIter], hc.stats[kStRounds], hc.stats[kStIdleIter], hc.stats[kStRefillTry],
                         hc.stats[kStRefill], hc.stats[kStLockSpin], hc.stats[kStWaitSpin], hc.stats[kCyRelax],
                         hc.stats[kCyL1], hc.stats[kCyL2Write], hc.stats[kCyGlobalRead], hc.stats[kCyIdle],
                         hc.stats[kCyL0]);
        if (dbg > 1)
            std::fprintf(stderr, "[sssp]   window pull-backs %llu advances %llu elements written to buckets 0-1 %llu "
                                 "chunks read through descriptors %llu\n",
                         hc.stats[kStPullBack], hc.stats[kStAdvance], hc.stats[kStLowWrite], hc.stats[kStPopL2Desc]);
        if (hc.error == kErrNone && hc.finished) return SSSP_OK;
        if (dbg)
            std::fprintf(stderr, "[sssp] solve failed: error=%d where=%d info=%d finished=%d reserve=%llu done=%llu "
                                 "window=%llx grid=%d threads=%d smem=%zu\n",
                         hc.error, hc.err_where, hc.err_info, hc.finished, hc.reserve, hc.done, hc.window, grid,
                         threads, smem);
        // failure: the queue metadata is no longer consistent
        ws.dirty = true;
        if (hc.error == kErrOverflow && attempts < 4) {
            ws.grow_shift++;
            continue;
        }
        rc = ws.ensure_queue(nr, ws.rings.nch, warps, stream, g->sms);
        cudaStreamSynchronize(stream);
        if (hc.error == kErrOverflow) return SSSP_E_NOMEM;
        if (hc.error == kErrTimeout) return SSSP_E_TIMEOUT;
        return SSSP_E_CUDA;
    }
}

// Builds the device layout with shadow vertices for vertices above `split`
// arcs.  rp0/adj0 are the validated original arrays (device); on success
// g->row_ptr / g->adj / g->owner describe the layout (rp0/adj0 are freed
// when new arrays replaced them).
static int build_layout(Graph* g, int32_t* rp0, uint2* adj0, int32_t split, cudaStream_t s) {
    const int32_t n = g->n;
    std::vector<int32_t> h(n + 1);
    if (cudaMemcpyAsync(h.data(), rp0, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return SSSP_E_CUDA;
    int64_t ns = 0;
    for (int32_t v = 0; v < n; v++) {
        int64_t d = h[v + 1] - h[v];
        if (split > 0 && d > split) ns += (d + split - 1) / split;
    }
    if (ns == 0 || (int64_t)n + ns > 2147483647LL || g->m + ns > 2147483647LL) {
        g->row_ptr = rp0;
        g->adj = adj0;
        g->owner = nullptr;
        g->nv = n;
        g->mv = g->m;
        g->split = 0;
        return SSSP_OK;
    }
    const int32_t nv = (int32_t)(n + ns);
    std::vector<int32_t> rp1((size_t)nv + 1), sfirst(n, -1), owner((size_t)ns);
    // real vertices first, then the shadows in vertex order
    int64_t pos = 0;
    int32_t next_shadow = n;
    std::vector<int32_t> sdeg;
    sdeg.reserve((size_t)ns);
    for (int32_t v = 0; v < n; v++) {
        rp1[v] = (int32_t)pos;
        int64_t d = h[v + 1] - h[v];
        if (split > 0 && d > split) {
            int32_t k = (int32_t)((d + split - 1) / split);
            sfirst[v] = next_shadow;
            for (int32_t j = 0; j < k; j++) {
                owner[(size_t)(next_shadow - n) + j] = v;
                sdeg.push_back((int32_t)std::min<int64_t>(split, d - (int64_t)j * split));
            }
            next_shadow += k;
            pos += k;
        } else {
            pos += d;
        }
    }
    for (int64_t i = 0; i < ns; i++) {
        rp1[(size_t)n + i] = (int32_t)pos;
        pos += sdeg[(size_t)i];
    }
    rp1[nv] = (int32_t)pos;
    const int64_t mv = pos;
    int32_t *d_rp1 = nullptr, *d_sfirst = nullptr, *d_owner = nullptr;
    uint2* d_adj1 = nullptr;
    int rc = SSSP_OK;
    if (cudaMalloc(&d_rp1, sizeof(int32_t) * ((size_t)nv + 1)) != cudaSuccess ||
        cudaMalloc(&d_sfirst, sizeof(int32_t) * (size_t)n) != cudaSuccess ||
        cudaMalloc(&d_owner, sizeof(int32_t) * (size_t)ns) != cudaSuccess ||
        cudaMalloc(&d_adj1, sizeof(uint2) * (size_t)mv) != cudaSuccess) {
        cudaGetLastError();
        rc = SSSP_E_NOMEM;
    }
    if (rc == SSSP_OK) {
        cudaMemcpyAsync(d_rp1, rp1.data(), sizeof(int32_t) * ((size_t)nv + 1), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(d_sfirst, sfirst.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(d_owner, owner.data(), sizeof(int32_t) * (size_t)ns, cudaMemcpyHostToDevice, s);
        relayout_kernel<<<g->sms * 8, 256, 0, s>>>(rp0, adj0, n, d_rp1, d_sfirst, split, d_adj1);
        if (cudaStreamSynchronize(s) != cudaSuccess) rc = SSSP_E_CUDA;
    }
    cudaFree(d_sfirst);
    if (rc != SSSP_OK) {
        cudaFree(d_rp1);
        cudaFree(d_owner);
        cudaFree(d_adj1);
        return rc;
    }
    cudaFree(rp0);
    cudaFree(adj0);
    g->row_ptr = d_rp1;
    g->adj = d_adj1;
    g->owner = d_owner;
    g->nv = nv;
    g->mv = mv;
    g->split = split;
    return SSSP_OK;
}

// Original arc order from a shadow layout: the arcs of vertex v are its own
// row, or (a split hub) the rows of its shadows, which are consecutive.  One
// warp per vertex copies them to their place in the original CSR.
__global__ void unsplit_kernel(const uint2* adj1, const int32_t* src_start, const int32_t* rp0, int32_t n,
                               uint2* adj0) {
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t lane = threadIdx.x & 31u;
    for (int64_t v = wid; v < n; v += nw) {
        const int32_t b = rp0[v], e = rp0[v + 1], src = src_start[v];
        for (int32_t i = (int32_t)lane; i < e - b; i += 32) adj0[b + i] = adj1[src + i];
    }
}

int lane_refs(uint64_t uid, int delta) {
    static std::mutex mu;
    static std::vector<std::pair<uint64_t, int>> refs;
    std::lock_guard<std::mutex> lk(mu);
    for (size_t i = 0; i < refs.size(); i++) {
        if (refs[i].first != uid) continue;
        refs[i].second += delta;
        const int c = refs[i].second;
        if (c <= 0) refs.erase(refs.begin() + (long)i);
        return c;
    }
    if (delta > 0) refs.emplace_back(uid, delta);
    return delta > 0 ? delta : 0;
}

int ensure_layout(Graph* g, int32_t split, cudaStream_t s) {
    if (split == g->layout_req) return SSSP_OK;
    // no vertex is split under either threshold: the layout is the same
    if (g->split == 0 && g->feat.max_deg <= (double)split) {
        g->layout_req = split;
        return SSSP_OK;
    }
    if (lane_refs(g->uid, 0) > 0) return SSSP_E_BUSY;
    const int32_t n = g->n;
    int32_t* rp0 = nullptr;
    uint2* adj0 = nullptr;
    int32_t* old_rp = g->row_ptr;
    uint2* old_adj = g->adj;
    int32_t* old_owner = g->owner;
    if (g->split == 0) {
        // the current layout is the original CSR: hand it over
        rp0 = g->row_ptr;
        adj0 = g->adj;
    } else {
        const int32_t nv = g->nv;
        std::vector<int32_t> rp1((size_t)nv + 1), owner((size_t)(nv - n));
        if (cudaMemcpyAsync(rp1.data(), g->row_ptr, sizeof(int32_t) * ((size_t)nv + 1), cudaMemcpyDeviceToHost,
                            s) != cudaSuccess ||
            cudaMemcpyAsync(owner.data(), g->owner, sizeof(int32_t) * (size_t)(nv - n), cudaMemcpyDeviceToHost,
                            s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return SSSP_E_CUDA;
        std::vector<int32_t> first(n, -1), count(n, 0);
        for (int32_t i = 0; i < nv - n; i++) {
            const int32_t v = owner[(size_t)i];
            if (first[v] < 0) first[v] = n + i;
            count[v]++;
        }
        std::vector<int32_t> h0((size_t)n + 1), src((size_t)n);
        int64_t pos = 0;
        for (int32_t v = 0; v < n; v++) {
            h0[v] = (int32_t)pos;
            if (first[v] >= 0) {
                src[v] = rp1[first[v]];
                pos += rp1[first[v] + count[v]] - rp1[first[v]];
            } else {
                src[v] = rp1[v];
                pos += rp1[v + 1] - rp1[v];
            }
        }
        h0[n] = (int32_t)pos;
        if (pos != g->m) return SSSP_E_BADGRAPH;
        int32_t* d_src = nullptr;
        if (cudaMalloc(&rp0, sizeof(int32_t) * ((size_t)n + 1)) != cudaSuccess ||
            cudaMalloc(&adj0, sizeof(uint2) * std::max<size_t>((size_t)g->m, 1)) != cudaSuccess ||
            cudaMalloc(&d_src, sizeof(int32_t) * (size_t)n) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(rp0);
            cudaFree(adj0);
            cudaFree(d_src);
            return SSSP_E_NOMEM;
        }
        cudaMemcpyAsync(rp0, h0.data(), sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(d_src, src.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, s);
        unsplit_kernel<<<g->sms * 8, 256, 0, s>>>(g->adj, d_src, rp0, n, adj0);
        const cudaError_t e = cudaStreamSynchronize(s);
        cudaFree(d_src);
        if (e != cudaSuccess) {
            cudaFree(rp0);
            cudaFree(adj0);
            return cuda_status(e);
        }
    }
    // build_layout frees rp0/adj0 when it makes new arrays and keeps them
    // as the layout otherwise; it leaves the graph untouched on failure
    const bool handed = rp0 == old_rp;
    const int rc = build_layout(g, rp0, adj0, split, s);
    if (rc != SSSP_OK) {
        if (!handed) {
            cudaFree(rp0);
            cudaFree(adj0);
        }
        return rc;
    }
    if (!handed) {
        // the previous layout was split: its arrays are no longer used
        cudaFree(old_rp);
        cudaFree(old_adj);
        cudaFree(old_owner);
    }
    g->layout_req = split;
    g->feat.shadows = g->nv - g->n;
    g->ws.dirty = true;
    return SSSP_OK;
}

}  // namespace sssp

// ==================================================================== C ABI

extern "C" int sssp_config_default(sssp_config* cfg) {
    if (!cfg) return SSSP_E_INVAL;
    config_defaults(cfg);
    return SSSP_OK;
}

extern "C" int sssp_graph_create(const int32_t* row_ptr, const int32_t* col_idx, const void* weights,
                                 int32_t n, int64_t m, int32_t wtype, sssp_graph** out) {
    if (!out) return SSSP_E_INVAL;
    *out = nullptr;
    if (!row_ptr || n < 1 || m < 0 || m > 2147483647LL || (m > 0 && (!col_idx || !weights)))
        return SSSP_E_INVAL;
    if (wtype != SSSP_W_U32 && wtype != SSSP_W_F32) return SSSP_E_INVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        cudaGetLastError();
        return SSSP_E_NODEV;
    }
    static std::atomic<uint64_t> next_uid{1};
    Graph* g = new (std::nothrow) Graph();
    if (!g) return SSSP_E_NOMEM;
    g->uid = next_uid.fetch_add(1);
    cudaGetDevice(&g->device);
    cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, g->device);
    g->n = n;
    g->m = m;
    g->wtype = wtype;
    config_defaults(&g->defaults);
    cudaStream_t s = nullptr;
    int rc = SSSP_OK;
    int32_t* col_tmp = nullptr;
    uint32_t* w_tmp = nullptr;
    int32_t* rp0 = nullptr;
    uint2* adj0 = nullptr;
    int* flags = nullptr;
    FeatAcc* facc = nullptr;
    FeatAcc hacc;
    int hflags = 0;
    cudaError_t e;
    do {
        if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) { rc = cuda_status(e); break; }
        if ((e = cudaMalloc(&rp0, sizeof(int32_t) * ((size_t)n + 1))) != cudaSuccess) { rc = cuda_status(e); break; }
        if ((e = cudaMalloc(&adj0, sizeof(uint2) * std::max<size_t>((size_t)m, 1))) != cudaSuccess) { rc = cuda_status(e); break; }
        if ((e = cudaMalloc(&flags, sizeof(int))) != cudaSuccess) { rc = cuda_status(e); break; }
        if ((e = cudaMalloc(&facc, sizeof(FeatAcc))) != cudaSuccess) { rc = cuda_status(e); break; }
        cudaMemsetAsync(flags, 0, sizeof(int), s);
        cudaMemcpyAsync(rp0, row_ptr, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyDefault, s);
        const int32_t* col_d = col_idx;
        const uint32_t* w_d = (const uint32_t*)weights;
        if (m > 0) {
            if (!is_device_ptr(col_idx)) {
                if ((e = cudaMalloc(&col_tmp, sizeof(int32_t) * (size_t)m)) != cudaSuccess) { rc = cuda_status(e); break; }
                cudaMemcpyAsync(col_tmp, col_idx, sizeof(int32_t) * (size_t)m, cudaMemcpyHostToDevice, s);
                col_d = col_tmp;
            }
            if (!is_device_ptr(weights)) {
                if ((e = cudaMalloc(&w_tmp, sizeof(uint32_t) * (size_t)m)) != cudaSuccess) { rc = cuda_status(e); break; }
                cudaMemcpyAsync(w_tmp, weights, sizeof(uint32_t) * (size_t)m, cudaMemcpyHostToDevice, s);
                w_d = w_tmp;
            }
        }
        validate_rows_kernel<<<grid_for((size_t)n + 1, g->sms), 256, 0, s>>>(rp0, n, m, flags);
        if (m > 0)
            pack_kernel<<<grid_for((size_t)m, g->sms), 256, 0, s>>>(col_d, w_d, m, n, wtype == SSSP_W_F32,
                                                                  adj0, flags);
        cudaMemcpyAsync(&hflags, flags, sizeof(int), cudaMemcpyDeviceToHost, s);
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) { rc = cuda_status(e); break; }
        cudaFree(col_tmp);
        cudaFree(w_tmp);
        col_tmp = nullptr;
        w_tmp = nullptr;
        if (hflags) { rc = SSSP_E_BADGRAPH; break; }
        FeatAcc init;
        std::memset(&init, 0, sizeof(init));
        init.minw_bits = 0xffffffffu;
        cudaMemcpyAsync(facc, &init, sizeof(init), cudaMemcpyHostToDevice, s);
        features_kernel<<<grid_for((size_t)std::max<int64_t>(n, m), g->sms), 256, 0, s>>>(
            rp0, n, adj0, m, wtype == SSSP_W_F32, facc);
        cudaMemcpyAsync(&hacc, facc, sizeof(FeatAcc), cudaMemcpyDeviceToHost, s);
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) { rc = cuda_status(e); break; }
        sssp_features& f = g->feat;
        f.n = n;
        f.m = m;
        f.avg_deg = hacc.sdeg / n;
        f.max_deg = hacc.maxdeg;
        f.std_deg = std::sqrt(std::max(0.0, hacc.sdeg2 / n - f.avg_deg * f.avg_deg));
        auto wval = [&](uint32_t b) {
            if (wtype == SSSP_W_F32) {
                float x;
                std::memcpy(&x, &b, 4);
                return (double)x;
            }
            return (double)b;
        };
        if (m > 0) {
            f.avg_w = hacc.sw / (double)m;
            f.std_w = std::sqrt(std::max(0.0, hacc.sw2 / (double)m - f.avg_w * f.avg_w));
            f.max_w = wval(hacc.maxw_bits);
            f.min_w = wval(hacc.minw_bits);
        } else {
            f.avg_w = f.std_w = f.max_w = f.min_w = 1.0;
        }
        f.symmetric = -1;
        f.has_zero_w = hacc.zero_w ? 1 : 0;
        // the graph's default configuration: the feature prior (Section 3.5); its hub
        // split threshold gives the initial layout
        g->defaults = prior_config(g);
        const int32_t split0 = g->defaults.split_arcs ? g->defaults.split_arcs : kDefaultSplit;
        rc = build_layout(g, rp0, adj0, split0, s);
        g->layout_req = split0;
        f.shadows = g->nv - g->n;
        if (rc == SSSP_OK) {
            rp0 = nullptr;  // owned by the graph now (or freed by the relayout)
            adj0 = nullptr;
        }
    } while (0);
    cudaFree(col_tmp);
    cudaFree(w_tmp);
    cudaFree(flags);
    cudaFree(facc);
    if (s) cudaStreamDestroy(s);
    if (rc != SSSP_OK) {
        cudaFree(rp0);
        cudaFree(adj0);
        delete g;
        return rc;
    }
    *out = reinterpret_cast<sssp_graph*>(g);
    return SSSP_OK;
}

extern "C" int sssp_graph_destroy(sssp_graph* gh) {
    if (!gh) return SSSP_OK;
    Graph* g = reinterpret_cast<Graph*>(gh);
    {
        std::lock_guard<std::mutex> lk(g->mu);
        cudaSetDevice(g->device);
        g->ws.release();
        cudaFree(g->row_ptr);
        cudaFree(g->adj);
        cudaFree(g->owner);
    }
    delete g;
    return SSSP_OK;
}

extern "C" int sssp_graph_features(const sssp_graph* gh, sssp_features* out) {
    if (!gh || !out) return SSSP_E_INVAL;
    *out = reinterpret_cast<const Graph*>(gh)->feat;
    return SSSP_OK;
}

extern "C" int sssp_solve(sssp_graph* gh, int32_t src, void* dist_out, int32_t* pred_out,
                          const sssp_config* cfg, void* stream) {
    if (!gh || !dist_out) return SSSP_E_INVAL;
    Graph* g = reinterpret_cast<Graph*>(gh);
    if (src < 0 || src >= g->n) return SSSP_E_INVAL;
    std::lock_guard<std::mutex> lk(g->mu);
    try {
        return run_queries(g, nullptr, nullptr, src, 1, dist_out, pred_out, cfg, (cudaStream_t)stream, nullptr);
    } catch (...) {
        return SSSP_E_NOMEM;
    }
}

extern "C" int sssp_bfs(sssp_graph* gh, int32_t src, uint32_t* level_out, int32_t* pred_out,
                        const sssp_config* cfg, void* stream) {
    if (!gh || !level_out) return SSSP_E_INVAL;
    Graph* g = reinterpret_cast<Graph*>(gh);
    if (src < 0 || src >= g->n) return SSSP_E_INVAL;
    std::lock_guard<std::mutex> lk(g->mu);
    try {
        return run_queries(g, nullptr, nullptr, src, 1, level_out, pred_out, cfg, (cudaStream_t)stream, nullptr,
                           true);
    } catch (...) {
        return SSSP_E_NOMEM;
    }
}

extern "C" int sssp_solve_sampled(sssp_graph* gh, int32_t src, void* dist_out, int32_t* pred_out,
                                  const sssp_config* cfg, uint64_t* samples_out, int32_t cap, int32_t period_us,
                                  int32_t* n_out) {
    if (!gh || !dist_out || !samples_out || !n_out || cap < 1 || cap > (1 << 24) || period_us < 1)
        return SSSP_E_INVAL;
    if (is_device_ptr(samples_out)) return SSSP_E_INVAL;
    Graph* g = reinterpret_cast<Graph*>(gh);
    if (src < 0 || src >= g->n) return SSSP_E_INVAL;
    *n_out = 0;
    Sampling samp{reinterpret_cast<unsigned long long*>(samples_out), cap, period_us, n_out};
    std::lock_guard<std::mutex> lk(g->mu);
    try {
        return run_queries(g, nullptr, nullptr, src, 1, dist_out, pred_out, cfg, nullptr, nullptr, false, &samp);
    } catch (...) {
        return SSSP_E_NOMEM;
    }
}

extern "C" int sssp_solve_batch(sssp_graph* gh, const int32_t* srcs, int32_t nq, void* dist_out,
                                int32_t* pred_out, const sssp_config* cfg, void* stream) {
    if (!gh || !dist_out || !srcs || nq < 1) return SSSP_E_INVAL;
    Graph* g = reinterpret_cast<Graph*>(gh);
    std::lock_guard<std::mutex> lk(g->mu);
    try {
        std::vector<int32_t> hs;
        const int32_t* host = nullptr;
        const int32_t* dev = nullptr;
        if (is_device_ptr(srcs)) {
            hs.resize(nq);
            if (cudaMemcpy(hs.data(), srcs, sizeof(int32_t) * nq, cudaMemcpyDeviceToHost) != cudaSuccess)
                return SSSP_E_CUDA;
            dev = srcs;
        } else {
            hs.assign(srcs, srcs + nq);
            host = srcs;
        }
        for (int32_t i = 0; i < nq; i++)
            if (hs[i] < 0 || hs[i] >= g->n) return SSSP_E_INVAL;
        if (nq == 1)
            return run_queries(g, nullptr, nullptr, hs[0], 1, dist_out, pred_out, cfg, (cudaStream_t)stream, nullptr);
        return run_queries(g, host, dev, 0, nq, dist_out, pred_out, cfg, (cudaStream_t)stream, nullptr);
    } catch (...) {
        return SSSP_E_NOMEM;
    }
}

extern "C" int sssp_last_stats(const sssp_graph* gh, sssp_stats* out) {
    if (!gh || !out) return SSSP_E_INVAL;
    const Graph* g = reinterpret_cast<const Graph*>(gh);
    *out = g->last;
    return SSSP_OK;
}
