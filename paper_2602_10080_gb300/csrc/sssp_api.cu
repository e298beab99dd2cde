// sssp_api.cu -- the C ABI of libsssp.so (include/sssp.h): graph upload and
// validation, per-graph device workspace, single-source and batched solves,
// statistics.  Autotuning lives in sssp_autotune.cu, serving in
// sssp_serve.cu.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <thread>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
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
        default: return "unknown status";
    }
}

extern "C" int sssp_version(void) { return 1 * 10000 + 0 * 100 + 0; }

namespace sssp {

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

// Queue metadata to the empty state: seq[b][s] = s ("free for ticket s").
__global__ void ring_reset_kernel(Rings r, uint32_t nbuckets, TaskRing hv, Ctrl* ctrl) {
    size_t total = (size_t)nbuckets * r.nch;
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t k = i; k < total; k += stride) {
        r.seq[k] = (uint32_t)(k & (r.nch - 1u));
        r.cnt[k] = 0;
    }
    for (size_t k = i; k < hv.nslot; k += stride) hv.seq[k] = (uint32_t)k;
    for (size_t k = i; k < (size_t)nbuckets * 32; k += stride) {
        r.rt[k] = 0;
        r.wt[k] = 0;
    }
    if (i < 32) {
        hv.rt[i] = 0;
        hv.wt[i] = 0;
    }
    if (i == 0) {
        ctrl->reserve = 0;
        ctrl->done = 0;
        ctrl->window = 0;
        ctrl->finished = 0;
        ctrl->error = 0;
    }
}

// Resets the control block and writes the sources through to the current
// L2 bucket (Section 4.1: "the source vertex is first written through to
// the L2 queue"), reserve = number of queries.  One warp.
__global__ void seed_kernel(KParams P, const int32_t* srcs, int32_t src0, int32_t nq, int packed) {
    Ctrl* C = P.ctrl;
    const uint32_t lane = threadIdx.x & 31u;
    __shared__ uint32_t cur_s;
    if (lane == 0) {
        C->reserve = (unsigned long long)nq;
        C->done = 0;
        C->finished = 0;
        C->error = 0;
        C->err_where = 0;
        C->err_info = 0;
        for (int i = 0; i < 16; i++) C->stats[i] = 0;
        uint32_t cur = (uint32_t)(C->window >> 32) % (uint32_t)P.bmax;
        C->window = (unsigned long long)cur << 32;  // base distance 0
        cur_s = cur;
    }
    __syncwarp();
    const uint32_t cur = cur_s;
    uint32_t* wtp = P.l2.wt + (size_t)cur * 32;
    for (int32_t base = 0; base < nq; base += 32) {
        int32_t q = base + (int32_t)lane;
        bool valid = q < nq;
        uint32_t t = 0;
        int ok = 1;
        if (lane == 0) {
            t = *wtp;
            *wtp = t + 1u;
            if (P.l2.seq[(size_t)cur * P.l2.nch + (t & (P.l2.nch - 1u))] != t) ok = 0;
        }
        ok = __shfl_sync(kFull, ok, 0);
        if (!ok) {
            if (lane == 0) C->error = kErrState;
            return;
        }
        t = __shfl_sync(kFull, t, 0);
        const size_t slot = (size_t)cur * P.l2.nch + (t & (P.l2.nch - 1u));
        if (valid) {
            int32_t s = srcs ? srcs[q] : src0;
            uint32_t key = P.vbits ? (((uint32_t)q << P.vbits) | (uint32_t)s) : (uint32_t)s;
            P.l2.data[slot * kChunk + lane] = make_uint2(key, 0u);
            size_t di = (size_t)q * (size_t)P.n + (size_t)s;
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

// (dist << 32 | pred) words -> separate dist / pred arrays.
__global__ void unpack_kernel(const unsigned long long* w, size_t count, uint32_t* dist,
                              int32_t* pred, int f32) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t stride = (size_t)gridDim.x * blockDim.x;
    for (; i < count; i += stride) {
        unsigned long long x = w[i];
        uint32_t d = (uint32_t)(x >> 32);
        if (f32 && d == kInfU32) d = kInfF32;
        dist[i] = d;
        if (pred) pred[i] = (int32_t)(uint32_t)x;
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

static int grid_for(size_t count, int sms) {
    size_t b = (count + 255) / 256;
    size_t cap = (size_t)sms * 8;
    return (int)std::max<size_t>(1, std::min(b, cap));
}

// ================================================================ workspace

void Workspace::release() {
    cudaFree(ring_mem);
    cudaFree(task_mem);
    cudaFree(ctrl);
    cudaFree(d64);
    cudaFree(d32);
    cudaFree(out_d);
    cudaFree(out_p);
    cudaFree(srcs);
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

int Workspace::ensure_queue(uint32_t nbuckets, uint32_t nch_want, uint32_t margin,
                            uint32_t nslot_want, cudaStream_t s, int sms) {
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
    bool realloc = !ring_mem || nbuckets != bmax || nch_want > rings.nch || nslot_want > hv.nslot;
    if (realloc) {
        cudaFree(ring_mem);
        cudaFree(task_mem);
        ring_mem = nullptr;
        task_mem = nullptr;
        uint32_t nch = std::max(nch_want, rings.nch && nbuckets == bmax ? rings.nch : 0u);
        uint32_t nslot = std::max(nslot_want, hv.nslot);
        size_t tickets = (size_t)nbuckets * 32 * sizeof(uint32_t);
        size_t meta = (size_t)nbuckets * nch * sizeof(uint32_t);
        size_t data = (size_t)nbuckets * nch * kChunk * sizeof(uint2);
        size_t bytes = 2 * tickets + 2 * meta + data + 256;
        if (cudaMalloc((void**)&ring_mem, bytes) != cudaSuccess) {
            cudaGetLastError();
            ring_mem = nullptr;
            return SSSP_E_NOMEM;
        }
        size_t tbytes = 2 * 32 * sizeof(uint32_t) + (size_t)nslot * (sizeof(uint32_t) + sizeof(uint4)) + 256;
        if (cudaMalloc((void**)&task_mem, tbytes) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(ring_mem);
            ring_mem = nullptr;
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
        char* q = task_mem;
        hv.data = reinterpret_cast<uint4*>(q);
        q += (size_t)nslot * sizeof(uint4);
        hv.rt = reinterpret_cast<uint32_t*>(q);
        q += 32 * sizeof(uint32_t);
        hv.wt = reinterpret_cast<uint32_t*>(q);
        q += 32 * sizeof(uint32_t);
        hv.seq = reinterpret_cast<uint32_t*>(q);
        hv.nslot = nslot;
        bmax = nbuckets;
        ring_bytes = bytes + tbytes;
        dirty = true;
    }
    rings.margin = margin;
    hv.margin = margin;
    if (dirty) {
        size_t total = std::max<size_t>((size_t)bmax * rings.nch, hv.nslot);
        ring_reset_kernel<<<grid_for(total, sms), 256, 0, s>>>(rings, bmax, hv, ctrl);
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
    c->l1_cap = 4096;
    c->wb = 0;
    c->delta_u32 = 0;     // 0 = derive from the graph's weights
    c->delta_f32 = 0.0f;
    c->bnum = 4;
    c->bmax = 32;
    c->filter_deltas = 2.0f;
    c->th_heavy = 2048;
    c->split = 1024;
    c->block_threads = 512;
    c->blocks_per_sm = 0;
    c->timeout_ms = 0;
}

// Fills auto fields from the graph features (the prior of Section 3.5).
void resolve_auto(const Graph* g, sssp_config* c) {
    const sssp_features& f = g->feat;
    double avgdeg = std::max(1.0, f.avg_deg);
    if (g->wtype == SSSP_W_U32 && c->delta_u32 == 0) {
        // delta-stepping width: about one average weight scaled by 8/degree,
        // at least 1 (Meyer & Sanders use ~ w_max / degree).
        double d = std::max(1.0, f.avg_w * 8.0 / avgdeg);
        c->delta_u32 = (uint32_t)std::min(d, 4.0e9);
    }
    if (g->wtype == SSSP_W_F32 && !(c->delta_f32 > 0.0f)) {
        double d = std::max(1e-6, f.avg_w * 8.0 / avgdeg);
        c->delta_f32 = (float)d;
    }
    if (c->l2_type == SSSP_L2_VECTOR) {
        c->bmax = 1;
        c->bnum = 1;
    }
}

int validate_config(const sssp_config* c) {
    auto pow2 = [](int v) { return v > 0 && (v & (v - 1)) == 0; };
    if (c->l1_type < 0 || c->l1_type > 3) return SSSP_E_INVAL;
    if (c->l2_type < 0 || c->l2_type > 1) return SSSP_E_INVAL;
    if (c->l0_rows != kL0Rows) return SSSP_E_INVAL;
    if (!pow2(c->l1_cap) || c->l1_cap < 256 || c->l1_cap > 16384) return SSSP_E_INVAL;
    if (c->wb < 0) return SSSP_E_INVAL;
    if (c->bmax < 1 || c->bmax > 32 || c->bnum < 1 || c->bnum > 32) return SSSP_E_INVAL;
    if (!(c->filter_deltas >= 0.0f)) return SSSP_E_INVAL;
    if (c->th_heavy < 32 || c->split < 32 || (c->split & 31)) return SSSP_E_INVAL;
    if (c->block_threads != 256 && c->block_threads != 512 && c->block_threads != 1024) return SSSP_E_INVAL;
    if (c->blocks_per_sm < 0 || c->blocks_per_sm > 8 || c->timeout_ms < 0) return SSSP_E_INVAL;
    for (int i = 0; i < 7; i++)
        if (c->reserved[i] != 0) return SSSP_E_INVAL;
    return SSSP_OK;
}

// ================================================================== solve

int run_queries(Graph* g, const int32_t* srcs_host, const int32_t* srcs_dev, int32_t src0, int32_t nq,
                void* dist_out, int32_t* pred_out, const sssp_config* cfg_in, cudaStream_t stream,
                sssp_stats* st_out) {
    sssp_config cfg = cfg_in ? *cfg_in : (g->tuned_valid ? g->tuned : g->defaults);
    resolve_auto(g, &cfg);
    int rc = validate_config(&cfg);
    if (rc) return rc;
    if (cudaSetDevice(g->device) != cudaSuccess) return SSSP_E_CUDA;
    const int32_t n = g->n;
    const bool mq = nq > 1;
    int vbits = 0;
    if (mq) {
        while (vbits < 31 && (1ll << vbits) < (long long)n) vbits++;
        if (vbits == 0) vbits = 1;
        if ((unsigned long long)nq << vbits > (1ull << 32)) return SSSP_E_INVAL;
    }
    const int pred_mode = pred_out ? ((g->wtype == SSSP_W_U32 && g->feat.min_w >= 1.0) ? 1 : 2) : 0;
    const KernelKey key{g->wtype == SSSP_W_F32 ? 1 : 0, pred_mode, mq ? 1 : 0};

    // launch shape
    const int threads = cfg.block_threads;
    const int warps_per_block = threads / 32;
    const size_t scratch = (size_t)warps_per_block * 32 * sizeof(uint2);
    const size_t l1_off = (sizeof(BlockShared) + scratch + 15) & ~size_t(15);
    const size_t smem = l1_off + (size_t)cfg.l1_cap * sizeof(uint2);
    int occ = 0;
    cudaError_t ce = occupancy_mlmq(key, threads, smem, &occ);
    if (ce != cudaSuccess) return cuda_status(ce);
    if (occ < 1) return SSSP_E_INVAL;
    int bps = cfg.blocks_per_sm > 0 ? std::min(cfg.blocks_per_sm, occ) : occ;
    const int grid = g->sms * bps;
    const uint32_t warps = (uint32_t)(grid * warps_per_block);

    Workspace& ws = g->ws;
    const size_t cells = (size_t)nq * (size_t)n;
    // L2 capacity: ~ cells / 8 chunks in total over the buckets, at least
    // 4x the writer margin per bucket; doubled after an overflow.
    int attempts = 0;
    for (;;) {
        attempts++;
        uint64_t total_chunks = std::max<uint64_t>(cells / 8 + 1024, 1024) << ws.grow_shift;
        uint32_t nch = next_pow2(std::max<uint64_t>(total_chunks / (uint64_t)cfg.bmax + warps,
                                                    4ull * warps + (uint64_t)(nq / 32 + 2)));
        uint32_t nslot = next_pow2(std::max<uint64_t>(65536, 16ull * warps));
        rc = ws.ensure_queue((uint32_t)cfg.bmax, nch, warps, nslot, stream, g->sms);
        if (rc) return rc;
        // distance work buffer
        const bool dist_dev = is_device_ptr(dist_out);
        const bool pred_dev = pred_out && is_device_ptr(pred_out);
        void* work = nullptr;
        if (pred_mode) {
            rc = grow(&ws.d64, &ws.d64_n, cells);
            if (rc) return rc;
            work = ws.d64;
        } else if (dist_dev) {
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

        KParams P;
        std::memset(&P, 0, sizeof(P));
        P.row_ptr = g->row_ptr;
        P.adj = g->adj;
        P.n = n;
        P.dist = work;
        P.nq = nq;
        P.vbits = mq ? vbits : 0;
        P.vmask = mq ? ((1u << vbits) - 1u) : 0xffffffffu;
        P.l2 = ws.rings;
        P.hv = ws.hv;
        P.ctrl = ws.ctrl;
        P.delta = g->wtype == SSSP_W_F32 ? __float_as_uint_host(cfg.delta_f32) : cfg.delta_u32;
        P.bnum = std::min(cfg.bnum, cfg.bmax);
        P.bmax = cfg.bmax;
        P.l1_type = cfg.l1_type;
        P.l1_cap = cfg.l1_cap;
        P.wb = cfg.l1_type == SSSP_L1_VECTOR ? cfg.wb : 0;
        P.filter_deltas = cfg.filter_deltas;
        P.th_heavy = cfg.th_heavy;
        P.split = cfg.split;
        P.l1_off = (int32_t)l1_off;
        int tmo = cfg.timeout_ms > 0 ? cfg.timeout_ms : 20000;
        P.timeout_ns = (unsigned long long)tmo * 1000000ull;

        cudaEventRecord(ws.ev0, stream);
        if (pred_mode)
            fill_u64_kernel<<<grid_for(cells, g->sms), 256, 0, stream>>>(ws.d64, cells, ~0ull);
        else
            fill_u32_kernel<<<grid_for(cells, g->sms), 256, 0, stream>>>(
                (uint32_t*)work, cells, g->wtype == SSSP_W_F32 ? kInfF32 : kInfU32);
        seed_kernel<<<1, 32, 0, stream>>>(P, srcs_d, src0, nq, pred_mode ? 1 : 0);
        cudaEventRecord(ws.ev1, stream);
        if (std::getenv("SSSP_DEBUG") && std::atoi(std::getenv("SSSP_DEBUG")) > 2)
            std::fprintf(stderr, "[sssp] launch wt=%d pred=%d mq=%d nq=%d n=%d grid=%d threads=%d smem=%zu "
                                 "bmax=%d bnum=%d l1=%d nch=%u\n", key.wt, key.pred, key.mq, nq, n, grid, threads,
                         smem, P.bmax, P.bnum, P.l1_type, P.l2.nch);
        const int dbg = std::getenv("SSSP_DEBUG") ? std::atoi(std::getenv("SSSP_DEBUG")) : 0;
        unsigned long long* trace_h = nullptr;
        const size_t nwarps_total = (size_t)grid * threads;  // per-thread records
        if (dbg > 2 && cudaHostAlloc((void**)&trace_h, nwarps_total * 8, cudaHostAllocMapped) == cudaSuccess) {
            std::memset(trace_h, 0, nwarps_total * 8);
            cudaHostGetDevicePointer((void**)&P.trace, trace_h, 0);
        }
        ce = launch_mlmq(key, dim3(grid), dim3(threads), smem, stream, P);
        if (ce != cudaSuccess) {
            if (std::getenv("SSSP_DEBUG"))
                std::fprintf(stderr, "[sssp] launch failed: %s (grid=%d threads=%d smem=%zu)\n",
                             cudaGetErrorString(ce), grid, threads, smem);
            return cuda_status(ce);
        }
        cudaEventRecord(ws.ev2, stream);
        // outputs
        if (pred_mode) {
            uint32_t* dd = (uint32_t*)dist_out;
            int32_t* pp = pred_out;
            if (!dist_dev) {
                rc = grow(&ws.out_d, &ws.out_d_n, cells);
                if (rc) return rc;
                dd = ws.out_d;
            }
            if (!pred_dev) {
                rc = grow(&ws.out_p, &ws.out_p_n, cells);
                if (rc) return rc;
                pp = ws.out_p;
            }
            unpack_kernel<<<grid_for(cells, g->sms), 256, 0, stream>>>(ws.d64, cells, dd, pp,
                                                                       g->wtype == SSSP_W_F32);
            if (!dist_dev)
                cudaMemcpyAsync(dist_out, dd, cells * 4, cudaMemcpyDeviceToHost, stream);
            if (!pred_dev) cudaMemcpyAsync(pred_out, pp, cells * 4, cudaMemcpyDeviceToHost, stream);
        } else if (!dist_dev) {
            cudaMemcpyAsync(dist_out, work, cells * 4, cudaMemcpyDeviceToHost, stream);
        }
        cudaMemcpyAsync(ws.host_ctrl, ws.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, stream);
        if (trace_h) {
            // debug: poll instead of blocking; report where warps sit if the solve overruns
            auto t0 = std::chrono::steady_clock::now();
            bool reported = false;
            while (cudaStreamQuery(stream) == cudaErrorNotReady) {
                double el = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
                if (!reported && el > (double)tmo + 3000.0) {
                    unsigned long long hist[64] = {0};
                    for (size_t i = 0; i < nwarps_total; i++) hist[(trace_h[i] >> 48) & 63]++;
                    std::fprintf(stderr, "[sssp] OVERRUN %.0f ms; warps by location:", el);
                    for (int c = 0; c < 64; c++)
                        if (hist[c]) std::fprintf(stderr, " %d:%llu", c, hist[c]);
                    std::fprintf(stderr, "\n");
                    for (size_t wv = 0; wv < nwarps_total / 32; wv++) {
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
            if (std::getenv("SSSP_DEBUG"))
                std::fprintf(stderr, "[sssp] stream error: %s\n", cudaGetErrorString(ce));
            return cuda_status(ce);
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
        st.pops_heavy = (int64_t)hc.stats[kStPopHeavy];
        st.relax_arcs = (int64_t)hc.stats[kStRelax];
        st.improved = (int64_t)hc.stats[kStImproved];
        st.stale = (int64_t)hc.stats[kStStale];
        st.l2_chunks_written = (int64_t)hc.stats[kStChunks];
        st.l1_flushes = (int64_t)hc.stats[kStFlush];
        st.heavy_tasks = (int64_t)hc.stats[kStTasks];
        st.grid_blocks = grid;
        st.block_threads = threads;
        st.attempts = attempts;
        g->last = st;
        if (st_out) *st_out = st;
        if (std::getenv("SSSP_DEBUG") && std::atoi(std::getenv("SSSP_DEBUG")) > 1)
            std::fprintf(stderr, "[sssp] nq=%d n=%d kernel %.3f ms pops l0/l1/l2/heavy %lld/%lld/%lld/%lld relax %lld "
                                 "improved %lld stale %lld chunks %lld tasks %lld err %d fin %d\n",
                         nq, n, ms_kernel, (long long)st.pops_l0, (long long)st.pops_l1, (long long)st.pops_l2,
                         (long long)st.pops_heavy, (long long)st.relax_arcs, (long long)st.improved,
                         (long long)st.stale, (long long)st.l2_chunks_written, (long long)st.heavy_tasks,
                         hc.error, hc.finished);
        if (hc.error == kErrNone && hc.finished) return SSSP_OK;
        if (std::getenv("SSSP_DEBUG"))
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
        rc = ws.ensure_queue((uint32_t)cfg.bmax, ws.rings.nch, warps, ws.hv.nslot, stream, g->sms);
        cudaStreamSynchronize(stream);
        if (hc.error == kErrOverflow) return SSSP_E_NOMEM;
        if (hc.error == kErrTimeout) return SSSP_E_TIMEOUT;
        return SSSP_E_CUDA;
    }
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
    Graph* g = new (std::nothrow) Graph();
    if (!g) return SSSP_E_NOMEM;
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
    int* flags = nullptr;
    FeatAcc* facc = nullptr;
    FeatAcc hacc;
    int hflags = 0;
    cudaError_t e;
    do {
        if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) { rc = cuda_status(e); break; }
        if ((e = cudaMalloc(&g->row_ptr, sizeof(int32_t) * ((size_t)n + 1))) != cudaSuccess) { rc = cuda_status(e); break; }
        if ((e = cudaMalloc(&g->adj, sizeof(uint2) * std::max<size_t>((size_t)m, 1))) != cudaSuccess) { rc = cuda_status(e); break; }
        if ((e = cudaMalloc(&flags, sizeof(int))) != cudaSuccess) { rc = cuda_status(e); break; }
        if ((e = cudaMalloc(&facc, sizeof(FeatAcc))) != cudaSuccess) { rc = cuda_status(e); break; }
        cudaMemsetAsync(flags, 0, sizeof(int), s);
        cudaMemcpyAsync(g->row_ptr, row_ptr, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyDefault, s);
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
        validate_rows_kernel<<<grid_for((size_t)n + 1, g->sms), 256, 0, s>>>(g->row_ptr, n, m, flags);
        if (m > 0)
            pack_kernel<<<grid_for((size_t)m, g->sms), 256, 0, s>>>(col_d, w_d, m, n, wtype == SSSP_W_F32,
                                                                  g->adj, flags);
        cudaMemcpyAsync(&hflags, flags, sizeof(int), cudaMemcpyDeviceToHost, s);
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) { rc = cuda_status(e); break; }
        if (hflags) { rc = SSSP_E_BADGRAPH; break; }
        FeatAcc init;
        std::memset(&init, 0, sizeof(init));
        init.minw_bits = 0xffffffffu;
        cudaMemcpyAsync(facc, &init, sizeof(init), cudaMemcpyHostToDevice, s);
        features_kernel<<<grid_for((size_t)std::max<int64_t>(n, m), g->sms), 256, 0, s>>>(
            g->row_ptr, n, g->adj, m, wtype == SSSP_W_F32, facc);
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
    } while (0);
    cudaFree(col_tmp);
    cudaFree(w_tmp);
    cudaFree(flags);
    cudaFree(facc);
    if (s) cudaStreamDestroy(s);
    if (rc != SSSP_OK) {
        cudaFree(g->row_ptr);
        cudaFree(g->adj);
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
