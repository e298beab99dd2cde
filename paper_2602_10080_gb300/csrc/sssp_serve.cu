// sssp_serve.cu -- serving with continuous batching.
//
// An extension beyond the paper, which runs one source per launch (Section
// 4.1).  Queries on the same graph (and predecessor mode) share one "lane":
// a multi-query worklist in which an element carries (query slot, vertex),
// per-slot distance slices, and the lane's own L2 rings and control block.
// A worker thread runs the lanes in time slices.  Each slice is one launch
// of the persistent MLMQ kernel that stops after slice_us and drains its
// L0/L1/staging queues into L2 (so the whole queue state lives in L2
// between launches).  Between slices the host
//   1. reads every slot's count of elements left in the L2 rings (the kernel
//      keeps the counts: an L2 write adds, an L2 read subtracts);
//      a slot with none is finished: its distances are final (Eq. 1 holds
//      for every arc once no improved vertex is left to relax);
//   2. copies finished results to the callers' buffers and frees the slots;
//   3. admits queued queries into free slots: fills the slot's distances
//      with infinity and writes the source through to L2 (Section 4.1) in
//      the bucket of the lane's current window W, remembering W as the
//      query's bucket offset, so the new query's work is ordered with the
//      work already in flight (bucket = floor(d / delta) + offset);
//   4. grows the rings (migrating the live chunks) when one is half full.
// Lanes of different graphs run concurrently on their own streams and
// share the SMs in proportion to their queries in flight.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "api_internal.h"

namespace sssp {
namespace {

using Clock = std::chrono::steady_clock;

// ------------------------------------------------------------- kernels --

// Distance slices of the admitted slots to infinity.  adm[i] = (slot, src).
__global__ void serve_fill_kernel(void* work, int packed, const int2* adm, int32_t nadm, int32_t nv,
                                  uint32_t inf) {
    const size_t count = (size_t)nadm * (size_t)nv;
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (; i < count; i += stride) {
        const size_t a = i / (size_t)nv, v = i - a * (size_t)nv;
        const size_t idx = (size_t)adm[a].x * (size_t)nv + v;
        if (packed)
            reinterpret_cast<unsigned long long*>(work)[idx] = ~0ull;
        else
            reinterpret_cast<uint32_t*>(work)[idx] = inf;
    }
}

// Start of a slice (one warp): clears the finished flag and the slice end,
// then writes the admitted sources through to L2 in the bucket of the
// current window W (shard 0) and records W as their bucket offset.
__global__ void serve_seed_kernel(KParams P, const int2* adm, int32_t nadm, uint32_t* qoff, int packed) {
    Ctrl* C = P.ctrl;
    const uint32_t lane = threadIdx.x & 31u;
    if (lane == 0) {
        C->finished = 0;
        C->slice_end = 0ull;
    }
    if (nadm == 0) return;
    const uint32_t W = (uint32_t)C->window;
    const uint32_t ring = (W % (uint32_t)P.bmax) * (uint32_t)P.shards;
    uint32_t* wtp = P.l2.wt + (size_t)ring * 32;
    const uint32_t* rtp = P.l2.rt + (size_t)ring * 32;
    for (int32_t base = 0; base < nadm; base += 32) {
        const int32_t a = base + (int32_t)lane;
        const bool valid = a < nadm;
        uint32_t t = 0;
        int ok = 1;
        if (lane == 0) {
            t = *wtp;
            const uint32_t r = *rtp;
            const size_t s = (size_t)ring * P.l2.nch + (t & (P.l2.nch - 1u));
            if (t - r + 1u > P.l2.nch || P.l2.seq[s] != t) ok = 0;
            else *wtp = t + 1u;
        }
        ok = __shfl_sync(kFull, ok, 0);
        if (!ok) {
            if (lane == 0) C->error = kErrOverflow;
            return;
        }
        t = __shfl_sync(kFull, t, 0);
        const size_t slot = (size_t)ring * P.l2.nch + (t & (P.l2.nch - 1u));
        if (valid) {
            const int2 q = adm[a];
            const uint32_t key = ((uint32_t)q.x << P.vbits) | (uint32_t)q.y;
            P.l2.data[slot * kChunk + lane] = make_uint2(key, 0u);
            const size_t di = (size_t)q.x * (size_t)P.nv + (size_t)q.y;
            if (packed)
                reinterpret_cast<unsigned long long*>(P.dist)[di] = (unsigned long long)(uint32_t)q.y;
            else
                reinterpret_cast<uint32_t*>(P.dist)[di] = 0u;
            qoff[q.x] = W;
            if (P.qlive) P.qlive[q.x] = 1;   // the source, in L2
        }
        __syncwarp();
        if (lane == 0) {
            P.l2.cnt[slot] = (uint32_t)min(nadm - base, 32);
            __threadfence();
            P.l2.seq[slot] = t + 1u;
        }
        __syncwarp();
    }
    if (lane == 0) C->reserve += (unsigned long long)nadm;
    __threadfence();
}

// The fullest ring's chunk count (occ[0]) and all rings' (occ[1]), between
// slices.  One block.
__global__ void serve_occ_kernel(Rings R, uint32_t nrings, uint32_t* occ) {
    uint32_t mx = 0, sum = 0;
    for (uint32_t k = threadIdx.x; k < nrings; k += blockDim.x) {
        const uint32_t c = R.wt[(size_t)k * 32] - R.rt[(size_t)k * 32];
        mx = max(mx, c);
        sum += c;
    }
    for (int o = 16; o > 0; o >>= 1) {
        mx = max(mx, __shfl_xor_sync(kFull, mx, o));
        sum += __shfl_xor_sync(kFull, sum, o);
    }
    if ((threadIdx.x & 31u) == 0) {
        atomicMax(occ, mx);
        atomicAdd(occ + 1, sum);
    }
}

// Copies every ring's live chunks [rt, wt) to the front of the matching
// ring of `to` (larger), which starts at rt = 0; the rest of `to` is free.
__global__ void serve_migrate_kernel(Rings from, Rings to, uint32_t nrings) {
    const size_t total = (size_t)nrings * to.nch;
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (; i < total; i += stride) {
        const uint32_t ring = (uint32_t)(i / to.nch), j = (uint32_t)(i % to.nch);
        const uint32_t r = from.rt[(size_t)ring * 32], w = from.wt[(size_t)ring * 32];
        const uint32_t count = w - r;
        const size_t dst = (size_t)ring * to.nch + j;
        if (j < count) {
            const size_t src = (size_t)ring * from.nch + ((r + j) & (from.nch - 1u));
            const uint32_t c = from.cnt[src];
            for (uint32_t k = 0; k < c; k++) to.data[dst * kChunk + k] = from.data[src * kChunk + k];
            to.cnt[dst] = c;
            to.seq[dst] = j + 1u;   // full, ticket j
        } else {
            to.cnt[dst] = 0;
            to.seq[dst] = j;        // free for ticket j
        }
        if (j == 0) {
            to.rt[(size_t)ring * 32] = 0;
            to.wt[(size_t)ring * 32] = count;
        }
    }
}

// A slot's work slice -> one caller's outputs ([n] distances, predecessors).
__global__ void serve_unpack_kernel(const unsigned long long* work, int32_t n, uint32_t* dist, int32_t* pred,
                                    int f32) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const int32_t stride = gridDim.x * blockDim.x;
    for (; i < n; i += stride) {
        const unsigned long long x = work[i];
        uint32_t d = (uint32_t)(x >> 32);
        if (f32 && d == kInfU32) d = kInfF32;
        dist[i] = d;
        if (pred) pred[i] = (int32_t)(uint32_t)x;
    }
}

__global__ void serve_reset_kernel(Rings r, uint32_t nrings, Ctrl* ctrl) {
    const size_t total = (size_t)nrings * r.nch;
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
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
        ctrl->err_where = 0;
        ctrl->err_info = 0;
        ctrl->slice_end = 0;
        for (int s = 0; s < kStCount; s++) ctrl->stats[s] = 0;
    }
}

int blocks_for(size_t count, int sms) {
    size_t b = (count + 255) / 256;
    return (int)std::max<size_t>(1, std::min<size_t>(b, (size_t)sms * 8));
}

uint32_t pow2_at_least(uint64_t v) {
    uint32_t p = 1;
    while (p < v && p < (1u << 31)) p <<= 1;
    return p;
}

// ------------------------------------------------------------ host side --

struct Query {
    uint64_t ticket = 0;
    Graph* g = nullptr;
    int32_t src = 0;
    void* dist_out = nullptr;
    int32_t* pred_out = nullptr;
    int state = SSSP_Q_QUEUED;
    int status = SSSP_OK;
    bool cancel = false;        // set by sssp_serve_cancel
    bool delivering = false;    // results are being copied out
    Clock::time_point t_submit, t_admit, t_done;
};

struct Lane {
    Graph* g = nullptr;
    uint64_t uid = 0;
    bool counted = false;       // registered in lane_refs (the graph's layout is pinned)
    int pred_mode = 0;
    LaunchPlan plan;
    int vbits = 1;
    uint32_t cap_limit = 0;     // slots this lane may grow to
    uint32_t cap = 0;           // slots allocated
    size_t cell = 4;            // bytes per distance word
    void* work = nullptr;       // [cap][nv]
    uint32_t* qoff = nullptr;   // [cap]
    uint32_t* live = nullptr;   // [cap + 1]: per-slot counts, then the ring occupancy
    uint32_t* live_h = nullptr; // pinned mirror
    int2* adm = nullptr;        // [cap] admissions of this slice
    int2* adm_h = nullptr;      // pinned
    uint32_t* out_d = nullptr;  // [n] staging for host outputs (packed mode)
    int32_t* out_p = nullptr;
    char* ring_mem = nullptr;
    size_t ring_bytes = 0;
    Rings rings{};
    uint32_t nrings = 0;
    Ctrl* ctrl = nullptr;
    Ctrl* ctrl_h = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t k0 = nullptr, k1 = nullptr, k2 = nullptr;
    size_t bytes = 0;           // device bytes charged to the budget
    std::vector<Query*> slot_q; // [cap]: query in the slot (nullptr = free or draining)
    std::vector<uint8_t> drain; // [cap]: slot holds a cancelled query's leftover elements
    std::vector<uint32_t> free_slots;
    int running = 0;            // slots holding a live query
    int prev_running = 0;       // running when the current admission round began
    bool injected = false;      // a test flag's injected failure has been applied
    bool injected_neg = false;  // SSSP_SERVE_INJECT_NEGATIVE has been applied
    int draining = 0;
    int nadm = 0;               // admissions staged for the next slice
    bool inflight = false;      // a slice is queued or running on the stream
    cudaEvent_t done_ev = nullptr;
    Clock::time_point t_launch;
    double dbg_wall_ms = 0, dbg_kernel_ms = 0, dbg_host_ms = 0, dbg_scan_ms = 0, dbg_chunks = 0, dbg_elems = 0;
    int dbg_slices = 0;
    Clock::time_point idle_since;
};

}  // namespace
}  // namespace sssp

struct sssp_server {
    sssp_serve_options opt{};
    int device = 0;
    int sms = 1;
    size_t budget = 0;
    size_t used = 0;            // bytes held by lanes (worker thread only)
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<sssp::Query*> pending;                       // submitted, not yet seen by the worker
    std::unordered_map<uint64_t, sssp::Query*> tickets;
    std::vector<sssp::Query*> released;                     // cancelled and released; freed with the server
    uint64_t next_ticket = 1;
    bool stop = false;
    int fatal = SSSP_OK;        // sticky CUDA failure
    int debug = 0;              // SSSP_DEBUG level
    sssp_serve_stats stats{};
    std::thread worker;
    // worker-thread state
    std::deque<sssp::Query*> backlog;                       // waiting for a slot
    std::vector<sssp::Lane*> lanes;
};

namespace sssp {
namespace {

void lane_free_buffers(sssp_server* s, Lane* L) {
    if (L->stream) cudaStreamSynchronize(L->stream);
    cudaFree(L->work);
    cudaFree(L->qoff);
    cudaFree(L->live);
    cudaFree(L->adm);
    cudaFree(L->out_d);
    cudaFree(L->out_p);
    cudaFree(L->ring_mem);
    cudaFree(L->ctrl);
    if (L->live_h) cudaFreeHost(L->live_h);
    if (L->adm_h) cudaFreeHost(L->adm_h);
    if (L->ctrl_h) cudaFreeHost(L->ctrl_h);
    s->used -= L->bytes;
    L->bytes = 0;
    L->work = nullptr;
    L->qoff = nullptr;
    L->live = nullptr;
    L->adm = nullptr;
    L->out_d = nullptr;
    L->out_p = nullptr;
    L->ring_mem = nullptr;
    L->ctrl = nullptr;
    L->live_h = nullptr;
    L->adm_h = nullptr;
    L->ctrl_h = nullptr;
    L->cap = 0;
    L->nrings = 0;
}

void lane_destroy(sssp_server* s, Lane* L) {
    lane_free_buffers(s, L);
    if (L->counted) lane_refs(L->uid, -1);
    if (L->k0) cudaEventDestroy(L->k0);
    if (L->k1) cudaEventDestroy(L->k1);
    if (L->k2) cudaEventDestroy(L->k2);
    if (L->done_ev) cudaEventDestroy(L->done_ev);
    if (L->stream) cudaStreamDestroy(L->stream);
    delete L;
}

template <typename T>
int dev_alloc(T** p, size_t count) {
    *p = nullptr;
    if (cudaMalloc((void**)p, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return SSSP_E_NOMEM;
    }
    return SSSP_OK;
}

size_t ring_bytes_for(uint32_t nrings, uint32_t nch) {
    return 2 * (size_t)nrings * 32 * 4 + 2 * (size_t)nrings * nch * 4 + (size_t)nrings * nch * kChunk * 8 + 256;
}

void ring_carve(char* p, uint32_t nrings, uint32_t nch, uint32_t margin, Rings* r) {
    r->data = reinterpret_cast<uint2*>(p);
    p += (size_t)nrings * nch * kChunk * sizeof(uint2);
    r->rt = reinterpret_cast<uint32_t*>(p);
    p += (size_t)nrings * 32 * 4;
    r->wt = reinterpret_cast<uint32_t*>(p);
    p += (size_t)nrings * 32 * 4;
    r->seq = reinterpret_cast<uint32_t*>(p);
    p += (size_t)nrings * nch * 4;
    r->cnt = reinterpret_cast<uint32_t*>(p);
    r->nch = nch;
    r->margin = margin;
}

uint32_t lane_margin(const Lane* L) { return (uint32_t)(L->plan.grid * (L->plan.threads / 32)); }

// Fresh empty rings of nch chunks (old rings and their contents dropped).
int lane_rings_fresh(sssp_server* s, Lane* L, uint32_t nch) {
    const uint32_t nrings = (uint32_t)(L->plan.P.bmax * L->plan.P.shards);
    const size_t want = ring_bytes_for(nrings, nch);
    if (L->ring_mem) {
        cudaStreamSynchronize(L->stream);
        cudaFree(L->ring_mem);
        L->ring_mem = nullptr;
        s->used -= L->ring_bytes;
        L->bytes -= L->ring_bytes;
        L->ring_bytes = 0;
    }
    if (s->used + want > s->budget) return SSSP_E_NOMEM;
    if (dev_alloc(&L->ring_mem, want)) return SSSP_E_NOMEM;
    s->used += want;
    L->bytes += want;
    L->ring_bytes = want;
    L->nrings = nrings;
    ring_carve(L->ring_mem, nrings, nch, lane_margin(L), &L->rings);
    serve_reset_kernel<<<blocks_for((size_t)nrings * nch, s->sms), 256, 0, L->stream>>>(L->rings, nrings,
                                                                                     L->ctrl);
    if (L->live) cudaMemsetAsync(L->live, 0, ((size_t)L->cap + 2) * 4, L->stream);  // the rings are empty
    return cuda_status(cudaGetLastError());
}

// Larger rings with the live chunks moved over (between slices).
int lane_rings_grow(sssp_server* s, Lane* L, uint32_t nch) {
    const size_t want = ring_bytes_for(L->nrings, nch);
    if (s->used + want > s->budget) return SSSP_E_NOMEM;
    char* mem = nullptr;
    if (dev_alloc(&mem, want)) return SSSP_E_NOMEM;
    Rings nr{};
    ring_carve(mem, L->nrings, nch, lane_margin(L), &nr);
    serve_migrate_kernel<<<blocks_for((size_t)L->nrings * nch, s->sms), 256, 0, L->stream>>>(L->rings, nr,
                                                                                           L->nrings);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        cudaFree(mem);
        return cuda_status(e);
    }
    cudaStreamSynchronize(L->stream);
    cudaFree(L->ring_mem);
    s->used -= L->ring_bytes;
    L->bytes -= L->ring_bytes;
    L->ring_mem = mem;
    L->ring_bytes = want;
    s->used += want;
    L->bytes += want;
    L->rings = nr;
    return SSSP_OK;
}

uint32_t lane_initial_nch(const sssp_server* s, const Lane* L, uint32_t slots) {
    const uint32_t nrings = (uint32_t)(L->plan.P.bmax * L->plan.P.shards);
    const uint64_t cells = (uint64_t)slots * (uint64_t)L->g->nv;
    const uint64_t chunks = std::max<uint64_t>(cells >> s->opt.ring_shift, 4096);
    const uint64_t margin = lane_margin(L);
    return pow2_at_least(std::max<uint64_t>(chunks / nrings + margin, 2 * margin + 64));
}

// Grows the lane to `want` slots (power of two), keeping the running
// slots' distances and offsets.  Between slices only.
int lane_grow_slots(sssp_server* s, Lane* L, uint32_t want) {
    uint32_t ncap = std::max<uint32_t>(8, pow2_at_least(want));
    ncap = std::min(ncap, L->cap_limit);
    if (ncap <= L->cap) return SSSP_E_BUSY;
    const size_t nv = (size_t)L->g->nv;
    const size_t work_b = (size_t)ncap * nv * L->cell;
    const size_t side_b = (size_t)ncap * (4 + 8) + (size_t)(ncap + 2) * 4;
    const size_t old_b = L->cap ? (size_t)L->cap * nv * L->cell + (size_t)L->cap * (4 + 8) + (size_t)(L->cap + 2) * 4 : 0;
    if (s->used - old_b + work_b + side_b > s->budget) return SSSP_E_NOMEM;
    void* work = nullptr;
    uint32_t *qoff = nullptr, *live = nullptr;
    int2* adm = nullptr;
    if (dev_alloc((char**)&work, work_b) || dev_alloc(&qoff, ncap) || dev_alloc(&live, (size_t)ncap + 2) ||
        dev_alloc(&adm, ncap)) {
        cudaFree(work);
        cudaFree(qoff);
        cudaFree(live);
        cudaFree(adm);
        return SSSP_E_NOMEM;
    }
    uint32_t* live_h = nullptr;
    int2* adm_h = nullptr;
    if (cudaMallocHost((void**)&live_h, ((size_t)ncap + 2) * 4) != cudaSuccess ||
        cudaMallocHost((void**)&adm_h, (size_t)ncap * sizeof(int2)) != cudaSuccess) {
        cudaGetLastError();
        if (live_h) cudaFreeHost(live_h);
        cudaFree(work);
        cudaFree(qoff);
        cudaFree(live);
        cudaFree(adm);
        return SSSP_E_NOMEM;
    }
    cudaMemsetAsync(live, 0, ((size_t)ncap + 2) * 4, L->stream);
    if (L->cap) {
        cudaMemcpyAsync(live, L->live, (size_t)L->cap * 4, cudaMemcpyDeviceToDevice, L->stream);
        cudaMemcpyAsync(work, L->work, (size_t)L->cap * nv * L->cell, cudaMemcpyDeviceToDevice, L->stream);
        cudaMemcpyAsync(qoff, L->qoff, (size_t)L->cap * 4, cudaMemcpyDeviceToDevice, L->stream);
        // admissions already staged for the coming slice
        std::memcpy(adm_h, L->adm_h, (size_t)L->nadm * sizeof(int2));
    }
    cudaStreamSynchronize(L->stream);
    cudaFree(L->work);
    cudaFree(L->qoff);
    cudaFree(L->live);
    cudaFree(L->adm);
    if (L->live_h) cudaFreeHost(L->live_h);
    if (L->adm_h) cudaFreeHost(L->adm_h);
    L->work = work;
    L->qoff = qoff;
    L->live = live;
    L->adm = adm;
    L->live_h = live_h;
    L->adm_h = adm_h;
    s->used = s->used - old_b + work_b + side_b;
    L->bytes = L->bytes - old_b + work_b + side_b;
    for (uint32_t k = ncap; k-- > L->cap;) L->free_slots.push_back(k);
    std::sort(L->free_slots.begin(), L->free_slots.end(), std::greater<uint32_t>());
    L->slot_q.resize(ncap, nullptr);
    L->drain.resize(ncap, 0);
    L->cap = ncap;
    return SSSP_OK;
}

Lane* lane_create(sssp_server* s, Graph* g, int pred_mode, int* rc) {
    Lane* L = new (std::nothrow) Lane();
    if (!L) {
        *rc = SSSP_E_NOMEM;
        return nullptr;
    }
    L->g = g;
    L->uid = g->uid;
    L->pred_mode = pred_mode;
    sssp_config cfg;
    {
        // the lane uses the graph's layout as it is now; registering the lane
        // under the graph's lock keeps a solve from relaying it out meanwhile
        std::lock_guard<std::mutex> lk(g->mu);
        if (const sssp_config* bt = batch_tuned_largest(g)) {
            // a lane holds many queries at load: the multi-query configuration
            // of sssp_autotune_batch (its largest size class)
            cfg = *bt;
            resolve_auto(g, &cfg);
        } else {
            cfg = g->tuned_valid ? g->tuned : g->defaults;
            resolve_auto(g, &cfg);
            batch_delta(g, &cfg, 4);   // without one: narrower buckets
            cfg.bnum = std::min(cfg.bnum, 4);
            // lanes were measured with 512-thread blocks (several lanes share the SMs)
            cfg.block_threads = 512;
        }
        *rc = validate_config(&cfg);
        if (!*rc) *rc = plan_launch(g, cfg, pred_mode, true, &L->plan);
        if (!*rc) {
            lane_refs(g->uid, 1);
            L->counted = true;
        }
    }
    if (*rc) {
        delete L;
        return nullptr;
    }
    while (L->vbits < 31 && (1ll << L->vbits) <= (long long)g->nv) L->vbits++;  // 2^vbits > nv
    L->cap_limit = (uint32_t)std::min<uint64_t>((uint64_t)s->opt.max_slots, 1ull << (32 - L->vbits));
    L->cell = pred_mode ? 8 : 4;
    L->idle_since = Clock::now();
    if (cudaStreamCreateWithFlags(&L->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&L->k0) != cudaSuccess || cudaEventCreate(&L->k1) != cudaSuccess ||
        cudaEventCreate(&L->k2) != cudaSuccess ||
        cudaEventCreateWithFlags(&L->done_ev, cudaEventDisableTiming) != cudaSuccess ||
        dev_alloc(&L->ctrl, 1) || cudaMallocHost((void**)&L->ctrl_h, sizeof(Ctrl)) != cudaSuccess) {
        cudaGetLastError();
        *rc = SSSP_E_NOMEM;
        lane_destroy(s, L);
        return nullptr;
    }
    if (pred_mode) {
        if (dev_alloc(&L->out_d, (size_t)g->n) || dev_alloc(&L->out_p, (size_t)g->n)) {
            *rc = SSSP_E_NOMEM;
            lane_destroy(s, L);
            return nullptr;
        }
        L->bytes += (size_t)g->n * 8;
        s->used += (size_t)g->n * 8;
    }
    *rc = SSSP_OK;
    return L;
}

// Puts every running query of the lane back at the front of the backlog
// (after an overflow inside a slice lost queue elements), drops draining
// slots, and starts the lane over on rings twice as large.
int lane_restart(sssp_server* s, Lane* L) {
    std::vector<Query*> back;
    for (uint32_t k = 0; k < L->cap; k++) {
        if (L->slot_q[k]) back.push_back(L->slot_q[k]);
        L->slot_q[k] = nullptr;
        L->drain[k] = 0;
    }
    L->free_slots.clear();
    for (uint32_t k = L->cap; k-- > 0;) L->free_slots.push_back(k);
    L->running = 0;
    L->draining = 0;
    L->nadm = 0;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (auto it = back.rbegin(); it != back.rend(); ++it) {
            (*it)->state = SSSP_Q_QUEUED;
            s->backlog.push_front(*it);
        }
        s->stats.restarts++;
    }
    return lane_rings_fresh(s, L, std::min<uint32_t>(L->rings.nch * 2u, 1u << 30));
}

void finish_query(sssp_server* s, Query* q, int status) {
    // caller holds s->mu
    q->t_done = Clock::now();
    if (status == SSSP_OK) {
        q->state = SSSP_Q_DONE;
        s->stats.completed++;
    } else {
        q->state = SSSP_Q_ERROR;
        q->status = status;
        s->stats.failed++;
    }
    q->delivering = false;
}

Lane* find_lane(sssp_server* s, Graph* g, int pred_mode) {
    for (Lane* L : s->lanes)
        if (L->uid == g->uid && L->pred_mode == pred_mode) return L;
    return nullptr;
}

// Moves backlog queries into free slots (FIFO per lane).  Worker thread.
void admit(sssp_server* s) {
    std::vector<Lane*> blocked;
    std::deque<Query*> keep;
    std::deque<Query*> work;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        while (!s->pending.empty()) {
            s->backlog.push_back(s->pending.front());
            s->pending.pop_front();
        }
        work.swap(s->backlog);
    }
    for (Lane* L : s->lanes) L->prev_running = L->running;
    for (Query* q : work) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (q->cancel) continue;   // already ERROR/CANCELLED
        }
        const int pm = q->pred_out ? pred_mode_for(q->g) : 0;
        Lane* L = find_lane(s, q->g, pm);
        if (L && (L->inflight || std::find(blocked.begin(), blocked.end(), L) != blocked.end())) {
            keep.push_back(q);
            continue;
        }
        int rc = SSSP_OK;
        if (!L) {
            L = lane_create(s, q->g, pm, &rc);
            if (L) s->lanes.push_back(L);
        }
        if (L && L->free_slots.empty()) {
            const uint32_t want = L->cap ? L->cap * 2u : 8u;
            rc = lane_grow_slots(s, L, want);
            if (rc == SSSP_E_NOMEM && L->cap == 0) {
                // free idle lanes and try once more
                for (size_t i = 0; i < s->lanes.size();) {
                    Lane* o = s->lanes[i];
                    if (o != L && !o->inflight && o->running == 0 && o->draining == 0 && o->nadm == 0) {
                        lane_destroy(s, o);
                        s->lanes.erase(s->lanes.begin() + (long)i);
                    } else {
                        i++;
                    }
                }
                rc = lane_grow_slots(s, L, want);
            }
        }
        if (L && !L->ring_mem && !L->free_slots.empty()) {
            rc = lane_rings_fresh(s, L, lane_initial_nch(s, L, L->cap));
            if (rc) {
                // not even the rings fit: give the slots back to the budget later
                L->free_slots.clear();
                for (uint32_t k = L->cap; k-- > 0;) L->free_slots.push_back(k);
            }
        }
        if (!L || L->free_slots.empty() || !L->ring_mem) {
            bool lane_busy = L && (L->running + L->draining + L->nadm) > 0;
            bool others_busy = false;
            for (Lane* o : s->lanes)
                if (o != L && (o->running + o->draining + o->nadm) > 0) others_busy = true;
            if (L && (lane_busy || others_busy) && rc != SSSP_E_CUDA) {
                // wait for slots or memory to come free
                blocked.push_back(L);
                keep.push_back(q);
            } else {
                std::lock_guard<std::mutex> lk(s->mu);
                finish_query(s, q, rc ? rc : SSSP_E_NOMEM);
                s->cv_done.notify_all();
            }
            continue;
        }
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (q->cancel) continue;   // cancelled meanwhile
            q->state = SSSP_Q_RUNNING;
            q->t_admit = Clock::now();
            if (L->prev_running > 0) s->stats.joined_running++;
        }
        const uint32_t slot = L->free_slots.back();
        L->free_slots.pop_back();
        L->slot_q[slot] = q;
        L->adm_h[L->nadm++] = make_int2((int)slot, q->src);
        L->running++;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto it = keep.rbegin(); it != keep.rend(); ++it) s->backlog.push_front(*it);
}

// Launches one slice on every lane that has work and no slice in flight.
int launch_ready(sssp_server* s) {
    // the SMs are shared in proportion to each lane's queries in flight
    int total = 0;
    for (Lane* L : s->lanes) total += L->running + L->draining;
    for (Lane* L : s->lanes) {
        if (L->inflight || L->running + L->draining == 0) continue;
        KParams P = L->plan.P;
        P.nq = (int32_t)L->cap;
        P.dist = L->work;
        P.vbits = L->vbits;
        P.vmask = (1u << L->vbits) - 1u;
        P.l2 = L->rings;
        P.ctrl = L->ctrl;
        // a busy lane runs longer slices (fewer drains and restarts); with
        // many queries in flight, one of them finishes every few ms anyway
        const int scale = std::min(8, std::max(1, (L->running + L->draining) / 4));
        P.slice_ns = (unsigned long long)s->opt.slice_us * 1000ull * (unsigned long long)scale;
        P.qoff = L->qoff;
        P.qlive = reinterpret_cast<int*>(L->live);
        // a warp's batch stays short, so a slice ends close to its deadline
        P.max_arcs = std::min(P.max_arcs, 1024);
        const bool packed = L->pred_mode != 0;
        if (L->nadm) {
            cudaMemcpyAsync(L->adm, L->adm_h, (size_t)L->nadm * sizeof(int2), cudaMemcpyHostToDevice, L->stream);
            serve_fill_kernel<<<blocks_for((size_t)L->nadm * L->g->nv, s->sms), 256, 0, L->stream>>>(
                L->work, packed, L->adm, L->nadm, L->g->nv, L->g->wtype == SSSP_W_F32 ? kInfF32 : kInfU32);
        }
        serve_seed_kernel<<<1, 32, 0, L->stream>>>(P, L->adm, L->nadm, L->qoff, packed);
        L->nadm = 0;
        const int share = (int)((long long)L->plan.grid * (L->running + L->draining) / std::max(1, total));
        const int grid = std::max(std::max(8, s->sms / 8), std::min(L->plan.grid, share));
        cudaEventRecord(L->k0, L->stream);
        cudaError_t e = launch_mlmq(L->plan.key, dim3(grid), dim3(L->plan.threads), L->plan.smem, L->stream, P);
        if (e != cudaSuccess) return cuda_status(e);
        cudaEventRecord(L->k1, L->stream);
        // per-slot L2 counts are kept by the kernel; [cap], [cap + 1]: ring occupancy
        cudaMemsetAsync(L->live + L->cap, 0, 2 * 4, L->stream);
        serve_occ_kernel<<<1, 256, 0, L->stream>>>(L->rings, L->nrings, L->live + L->cap);
        cudaMemcpyAsync(L->live_h, L->live, ((size_t)L->cap + 2) * 4, cudaMemcpyDeviceToHost, L->stream);
        cudaEventRecord(L->k2, L->stream);
        cudaMemcpyAsync(L->ctrl_h, L->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, L->stream);
        cudaEventRecord(L->done_ev, L->stream);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_status(e);
        L->inflight = true;
        L->t_launch = Clock::now();
        std::lock_guard<std::mutex> lk(s->mu);
        s->stats.slices++;
    }
    return SSSP_OK;
}

// Copies a finished slot's results to the query's buffers (async on the lane stream).
int deliver(Lane* L, uint32_t slot, Query* q) {
    const Graph* g = L->g;
    const size_t n = (size_t)g->n;
    const size_t off = (size_t)slot * (size_t)g->nv;
    if (!L->pred_mode) {
        const uint32_t* src = reinterpret_cast<const uint32_t*>(L->work) + off;
        cudaMemcpyAsync(q->dist_out, src, n * 4, cudaMemcpyDefault, L->stream);
    } else {
        const unsigned long long* src = reinterpret_cast<const unsigned long long*>(L->work) + off;
        const bool dd = is_device_ptr(q->dist_out), pd = q->pred_out && is_device_ptr(q->pred_out);
        uint32_t* dptr = dd ? reinterpret_cast<uint32_t*>(q->dist_out) : L->out_d;
        int32_t* pptr = q->pred_out ? (pd ? q->pred_out : L->out_p) : nullptr;
        serve_unpack_kernel<<<blocks_for(n, g->sms), 256, 0, L->stream>>>(src, (int32_t)n, dptr, pptr,
                                                                        g->wtype == SSSP_W_F32);
        if (!dd) cudaMemcpyAsync(q->dist_out, dptr, n * 4, cudaMemcpyDeviceToHost, L->stream);
        if (q->pred_out && !pd) cudaMemcpyAsync(q->pred_out, pptr, n * 4, cudaMemcpyDeviceToHost, L->stream);
    }
    return cuda_status(cudaGetLastError());
}

void fail_all(sssp_server* s, int status) {
    // every query anywhere ends with `status` (a sticky CUDA failure)
    std::lock_guard<std::mutex> lk(s->mu);
    s->fatal = status;
    for (Lane* L : s->lanes) {
        for (uint32_t k = 0; k < L->cap; k++)
            if (L->slot_q[k]) {
                if (!L->slot_q[k]->cancel) finish_query(s, L->slot_q[k], status);
                L->slot_q[k] = nullptr;
            }
        L->running = 0;
        L->draining = 0;
    }
    for (Query* q : s->backlog)
        if (!q->cancel) finish_query(s, q, status);
    s->backlog.clear();
    for (Query* q : s->pending)
        if (!q->cancel) finish_query(s, q, status);
    s->pending.clear();
    s->cv_done.notify_all();
}

// After a lane's slice: completions, errors, ring growth.
int collect_lane(sssp_server* s, Lane* L) {
    L->inflight = false;
    {
        cudaError_t e = cudaStreamSynchronize(L->stream);
        if (e != cudaSuccess) return cuda_status(e);
        float ms = 0;
        if (cudaEventElapsedTime(&ms, L->k0, L->k1) == cudaSuccess) {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stats.kernel_ms += ms;
            L->dbg_kernel_ms += ms;
        }
        if (s->debug > 1) {
            float sm = 0;
            if (cudaEventElapsedTime(&sm, L->k1, L->k2) == cudaSuccess) L->dbg_scan_ms += sm;
            L->dbg_chunks += L->live_h[L->cap + 1];
            for (uint32_t k = 0; k < L->cap; k++) L->dbg_elems += (int32_t)L->live_h[k];
        }
    }
    const Clock::time_point now = Clock::now();
    L->dbg_wall_ms += std::chrono::duration<double, std::milli>(now - L->t_launch).count();
    L->dbg_slices++;
    {
        Ctrl& hc = *L->ctrl_h;
        if (!L->injected && (s->opt.flags & (SSSP_SERVE_INJECT_OVERFLOW | SSSP_SERVE_INJECT_TIMEOUT))) {
            L->injected = true;
            if (hc.error == kErrNone)
                hc.error = (s->opt.flags & SSSP_SERVE_INJECT_OVERFLOW) ? kErrOverflow : kErrTimeout;
        }
        if (hc.error != kErrNone) {
            if (s->debug)
                std::fprintf(stderr, "[sssp serve] slice error %d at %d (info %d), lane n=%d pred=%d cap=%u\n",
                             hc.error, hc.err_where, hc.err_info, L->g->n, L->pred_mode, L->cap);
            if (hc.error == kErrOverflow) {
                int rc = lane_restart(s, L);
                if (rc == SSSP_E_CUDA) return rc;
                if (rc) {
                    // larger rings do not fit: the lane's queries fail
                    std::lock_guard<std::mutex> lk(s->mu);
                    std::deque<Query*> keep;
                    for (Query* q : s->backlog) {
                        if (find_lane(s, q->g, q->pred_out ? pred_mode_for(q->g) : 0) == L &&
                            q->state == SSSP_Q_QUEUED)
                            finish_query(s, q, SSSP_E_NOMEM);
                        else
                            keep.push_back(q);
                    }
                    s->backlog.swap(keep);
                    s->cv_done.notify_all();
                }
                return SSSP_OK;
            }
            // a bounded wait ran out: the lane's queries fail, the lane starts over
            {
                std::lock_guard<std::mutex> lk(s->mu);
                for (uint32_t k = 0; k < L->cap; k++) {
                    if (L->slot_q[k] && !L->slot_q[k]->cancel) finish_query(s, L->slot_q[k], SSSP_E_TIMEOUT);
                    L->slot_q[k] = nullptr;
                    L->drain[k] = 0;
                }
                s->cv_done.notify_all();
            }
            L->free_slots.clear();
            for (uint32_t k = L->cap; k-- > 0;) L->free_slots.push_back(k);
            L->running = L->draining = 0;
            int rc = lane_rings_fresh(s, L, L->rings.nch);
            if (rc == SSSP_E_CUDA) return rc;
            return SSSP_OK;
        }
        // completions
        std::vector<std::pair<uint32_t, Query*>> done;
        for (uint32_t k = 0; k < L->cap; k++) {
            const bool occupied = L->slot_q[k] || L->drain[k];
            if (!occupied) continue;
            Query* q = L->slot_q[k];
            if (!L->injected_neg && (s->opt.flags & SSSP_SERVE_INJECT_NEGATIVE)) {
                // test flag: the lane's first scanned slot reads as a negative count
                L->injected_neg = true;
                L->live_h[k] = 0xffffffffu;
            }
            if ((int32_t)L->live_h[k] < 0) {
                // an impossible count (more L2 reads than writes): the lane's
                // accounting is broken; its queries fail and it starts over
                if (s->debug) std::fprintf(stderr, "[sssp serve] negative L2 count %d in slot %u\n",
                                           (int32_t)L->live_h[k], k);
                {
                    std::lock_guard<std::mutex> lk(s->mu);
                    for (uint32_t j = 0; j < L->cap; j++) {
                        if (L->slot_q[j] && !L->slot_q[j]->cancel) finish_query(s, L->slot_q[j], SSSP_E_CUDA);
                        L->slot_q[j] = nullptr;
                        L->drain[j] = 0;
                    }
                    s->cv_done.notify_all();
                }
                L->free_slots.clear();
                for (uint32_t j = L->cap; j-- > 0;) L->free_slots.push_back(j);
                L->running = L->draining = 0;
                return lane_rings_fresh(s, L, L->rings.nch) == SSSP_E_CUDA ? SSSP_E_CUDA : SSSP_OK;
            }
            bool timed_out = false;
            if (q && s->opt.query_timeout_ms > 0 &&
                std::chrono::duration<double, std::milli>(now - q->t_admit).count() > s->opt.query_timeout_ms)
                timed_out = true;
            if (L->live_h[k] != 0 && !timed_out) {
                if (q) {
                    std::lock_guard<std::mutex> lk(s->mu);
                    if (q->cancel) {
                        // cancelled while running: its leftovers drain, nothing is copied
                        L->slot_q[k] = nullptr;
                        L->drain[k] = 1;
                        L->running--;
                        L->draining++;
                    }
                }
                continue;
            }
            if (L->live_h[k] != 0 && timed_out) {
                std::lock_guard<std::mutex> lk(s->mu);
                if (!q->cancel) finish_query(s, q, SSSP_E_TIMEOUT);
                s->cv_done.notify_all();
                L->slot_q[k] = nullptr;
                L->drain[k] = 1;
                L->running--;
                L->draining++;
                continue;
            }
            // no element left: finished
            if (L->drain[k]) {
                L->drain[k] = 0;
                L->draining--;
                L->free_slots.push_back(k);
                continue;
            }
            bool copy = false;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                if (!q->cancel) {
                    q->delivering = true;
                    copy = true;
                }
            }
            if (copy) {
                int rc = deliver(L, k, q);
                if (rc) return rc;
                done.push_back({k, q});
            }
            L->slot_q[k] = nullptr;
            L->running--;
            L->free_slots.push_back(k);
        }
        if (!done.empty()) {
            cudaError_t e = cudaStreamSynchronize(L->stream);
            if (e != cudaSuccess) return cuda_status(e);
            std::lock_guard<std::mutex> lk(s->mu);
            for (auto& d : done) finish_query(s, d.second, SSSP_OK);
            s->cv_done.notify_all();
        }
        // keep the free-slot stack ordered (lowest slot reused first)
        std::sort(L->free_slots.begin(), L->free_slots.end(), std::greater<uint32_t>());
        // rings more than half full: move to rings twice as large
        const uint32_t occ = L->live_h[L->cap];   // fullest ring (chunks); [cap + 1] = all rings
        const bool every = (s->opt.flags & SSSP_SERVE_MIGRATE_EACH_SLICE) != 0;
        if (L->running + L->draining > 0 && (every || (uint64_t)occ + lane_margin(L) > L->rings.nch / 2)) {
            const uint32_t nch = (uint64_t)occ + lane_margin(L) > L->rings.nch / 2 ? L->rings.nch * 2u : L->rings.nch;
            if (lane_rings_grow(s, L, nch) == SSSP_OK) {
                std::lock_guard<std::mutex> lk(s->mu);
                s->stats.ring_growths++;
            }
        }
        // an idle lane starts its window from zero again
        if (L->running + L->draining == 0) {
            serve_reset_kernel<<<blocks_for((size_t)L->nrings * L->rings.nch, s->sms), 256, 0, L->stream>>>(
                L->rings, L->nrings, L->ctrl);
            L->idle_since = Clock::now();
        }
    }
    L->dbg_host_ms += std::chrono::duration<double, std::milli>(Clock::now() - now).count();
    if (s->debug > 1 && L->dbg_slices == 100) {
        std::fprintf(stderr, "[sssp serve] lane n=%d pred=%d cap=%u: 100 slices, kernel %.3f ms, scan %.3f ms, "
                             "launch-to-seen %.3f ms, collect %.3f ms per slice; live chunks %.0f elements %.0f; "
                             "running %d draining %d nch %u\n",
                     L->g->n, L->pred_mode, L->cap, L->dbg_kernel_ms / 100, L->dbg_scan_ms / 100,
                     L->dbg_wall_ms / 100, L->dbg_host_ms / 100, L->dbg_chunks / 100, L->dbg_elems / 100, L->running,
                     L->draining, L->rings.nch);
        L->dbg_slices = 0;
        L->dbg_kernel_ms = L->dbg_wall_ms = L->dbg_host_ms = L->dbg_scan_ms = L->dbg_chunks = L->dbg_elems = 0;
    }
    return SSSP_OK;
}

void worker_main(sssp_server* s) {
    cudaSetDevice(s->device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(s->mu);
            for (;;) {
                bool busy = !s->pending.empty() || !s->backlog.empty();
                for (Lane* L : s->lanes)
                    if (L->inflight || L->running + L->draining > 0) busy = true;
                if (busy || s->stop) break;
                s->cv_work.wait_for(lk, std::chrono::milliseconds(200));
                // lanes idle for a while give their memory back
                const Clock::time_point now = Clock::now();
                for (size_t i = 0; i < s->lanes.size();) {
                    Lane* L = s->lanes[i];
                    if (!L->inflight && L->running + L->draining + L->nadm == 0 &&
                        std::chrono::duration<double>(now - L->idle_since).count() > 5.0) {
                        lk.unlock();
                        lane_destroy(s, L);
                        lk.lock();
                        s->lanes.erase(s->lanes.begin() + (long)i);
                    } else {
                        i++;
                    }
                }
            }
            bool busy = !s->pending.empty() || !s->backlog.empty();
            for (Lane* L : s->lanes)
                if (L->inflight || L->running + L->draining > 0) busy = true;
            if (s->stop && !busy) break;
            if (s->fatal) {
                for (Query* q : s->pending) finish_query(s, q, s->fatal);
                s->pending.clear();
                s->cv_done.notify_all();
                continue;
            }
        }
        admit(s);
        {
            int resident = 0;
            for (Lane* L : s->lanes) resident += L->running;
            std::lock_guard<std::mutex> lk(s->mu);
            s->stats.max_resident = std::max<int64_t>(s->stats.max_resident, resident);
        }
        int rc = launch_ready(s);
        // wait for any lane's slice (lanes run on their own streams); come
        // back now and then for new submissions to idle lanes
        const Clock::time_point t0 = Clock::now();
        bool any = false, inflight = false;
        while (!rc) {
            inflight = false;
            for (Lane* L : s->lanes) {
                if (!L->inflight) continue;
                cudaError_t q = cudaEventQuery(L->done_ev);
                if (q == cudaErrorNotReady) {
                    inflight = true;
                    continue;
                }
                if (q != cudaSuccess) {
                    rc = cuda_status(q);
                    break;
                }
                rc = collect_lane(s, L);
                any = true;
                if (rc) break;
            }
            if (rc || any || !inflight) break;
            if (std::chrono::duration<double, std::micro>(Clock::now() - t0).count() > 250.0) {
                std::lock_guard<std::mutex> lk(s->mu);
                if (!s->pending.empty()) break;
            }
            std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
        if (rc) fail_all(s, rc);
    }
}

}  // namespace
}  // namespace sssp

using sssp::Query;

extern "C" int sssp_serve_options_default(sssp_serve_options* opt) {
    if (!opt) return SSSP_E_INVAL;
    std::memset(opt, 0, sizeof(*opt));
    opt->mem_budget_bytes = 0;
    opt->max_slots = 128;
    opt->slice_us = 1000;
    opt->max_queued = 65536;
    opt->ring_shift = 4;
    opt->query_timeout_ms = 0;
    return SSSP_OK;
}

extern "C" int sssp_serve_create(const sssp_serve_options* opt_in, sssp_server** out) {
    if (!out) return SSSP_E_INVAL;
    *out = nullptr;
    sssp_serve_options opt;
    if (opt_in) opt = *opt_in;
    else sssp_serve_options_default(&opt);
    if (opt.max_slots < 1 || opt.max_slots > 4096 || opt.slice_us < 50 || opt.slice_us > 100000 ||
        opt.max_queued < 1 || opt.ring_shift < 0 || opt.ring_shift > 16 || opt.query_timeout_ms < 0)
        return SSSP_E_INVAL;
    if (opt.flags & ~(SSSP_SERVE_MIGRATE_EACH_SLICE | SSSP_SERVE_INJECT_OVERFLOW | SSSP_SERVE_INJECT_TIMEOUT |
                      SSSP_SERVE_INJECT_NEGATIVE))
        return SSSP_E_INVAL;
    for (int i = 0; i < 2; i++)
        if (opt.reserved[i] != 0) return SSSP_E_INVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        cudaGetLastError();
        return SSSP_E_NODEV;
    }
    sssp_server* s = new (std::nothrow) sssp_server();
    if (!s) return SSSP_E_NOMEM;
    s->opt = opt;
    if (const char* d = std::getenv("SSSP_DEBUG")) s->debug = std::atoi(d);
    cudaGetDevice(&s->device);
    cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device);
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return SSSP_E_CUDA;
    }
    s->budget = opt.mem_budget_bytes ? opt.mem_budget_bytes : fr / 4;
    try {
        s->worker = std::thread(sssp::worker_main, s);
    } catch (...) {
        delete s;
        return SSSP_E_NOMEM;
    }
    *out = s;
    return SSSP_OK;
}

extern "C" int sssp_serve_submit(sssp_server* s, sssp_graph* gh, int32_t src, void* dist_out, int32_t* pred_out,
                                 uint64_t* ticket_out) {
    if (!s || !gh || !dist_out || !ticket_out) return SSSP_E_INVAL;
    sssp::Graph* g = reinterpret_cast<sssp::Graph*>(gh);
    if (src < 0 || src >= g->n || g->device != s->device) return SSSP_E_INVAL;
    Query* q = new (std::nothrow) Query();
    if (!q) return SSSP_E_NOMEM;
    q->g = g;
    q->src = src;
    q->dist_out = dist_out;
    q->pred_out = pred_out;
    q->t_submit = sssp::Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->fatal) {
            delete q;
            return s->fatal;
        }
        if (s->stop) {
            delete q;
            return SSSP_E_INVAL;
        }
        if ((int64_t)(s->pending.size() + s->backlog.size()) >= s->opt.max_queued) {
            delete q;
            return SSSP_E_BUSY;
        }
        q->ticket = s->next_ticket++;
        s->tickets[q->ticket] = q;
        s->pending.push_back(q);
        s->stats.submitted++;
        *ticket_out = q->ticket;
    }
    s->cv_work.notify_one();
    return SSSP_OK;
}

extern "C" int sssp_serve_poll(sssp_server* s, uint64_t ticket, int32_t* state_out, int32_t* status_out) {
    if (!s || !state_out) return SSSP_E_INVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return SSSP_E_NOTFOUND;
    *state_out = it->second->state;
    if (status_out) *status_out = it->second->status;
    return SSSP_OK;
}

extern "C" int sssp_serve_wait(sssp_server* s, uint64_t ticket, int32_t timeout_ms, int32_t* state_out,
                               int32_t* status_out) {
    if (!s) return SSSP_E_INVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return SSSP_E_NOTFOUND;
    Query* q = it->second;
    auto finished = [q] { return q->state == SSSP_Q_DONE || q->state == SSSP_Q_ERROR; };
    if (timeout_ms < 0) s->cv_done.wait(lk, finished);
    else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), finished)) {
        if (state_out) *state_out = q->state;
        return SSSP_E_TIMEOUT;
    }
    if (state_out) *state_out = q->state;
    if (status_out) *status_out = q->status;
    return SSSP_OK;
}

extern "C" int sssp_serve_latency_us(sssp_server* s, uint64_t ticket, double* us_out) {
    if (!s || !us_out) return SSSP_E_INVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return SSSP_E_NOTFOUND;
    if (it->second->state != SSSP_Q_DONE) return SSSP_E_BUSY;
    *us_out = std::chrono::duration<double, std::micro>(it->second->t_done - it->second->t_submit).count();
    return SSSP_OK;
}

extern "C" int sssp_serve_cancel(sssp_server* s, uint64_t ticket) {
    if (!s) return SSSP_E_INVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return SSSP_E_NOTFOUND;
    Query* q = it->second;
    if (q->state == SSSP_Q_DONE || q->state == SSSP_Q_ERROR) return SSSP_E_INVAL;
    if (q->delivering) return SSSP_E_BUSY;
    q->cancel = true;
    q->state = SSSP_Q_ERROR;
    q->status = SSSP_E_CANCELLED;
    q->t_done = sssp::Clock::now();
    s->stats.cancelled++;
    s->stats.failed++;
    s->cv_done.notify_all();
    return SSSP_OK;
}

extern "C" int sssp_serve_release(sssp_server* s, uint64_t ticket) {
    if (!s) return SSSP_E_INVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return SSSP_E_NOTFOUND;
    Query* q = it->second;
    if (q->state != SSSP_Q_DONE && q->state != SSSP_Q_ERROR) return SSSP_E_BUSY;
    // a cancelled query may still sit in a queue or slot of the worker; it
    // is forgotten by ticket but freed with the server
    if (q->cancel) s->released.push_back(q);
    else delete q;
    s->tickets.erase(it);
    return SSSP_OK;
}

extern "C" int sssp_serve_get_stats(sssp_server* s, sssp_serve_stats* out) {
    if (!s || !out) return SSSP_E_INVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    return SSSP_OK;
}

extern "C" int sssp_serve_destroy(sssp_server* s) {
    if (!s) return SSSP_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (sssp::Lane* L : s->lanes) sssp::lane_destroy(s, L);
    s->lanes.clear();
    for (auto& kv : s->tickets) delete kv.second;
    s->tickets.clear();
    for (Query* q : s->released) delete q;
    s->released.clear();
    delete s;
    return SSSP_OK;
}
