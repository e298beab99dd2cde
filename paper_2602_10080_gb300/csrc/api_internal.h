// api_internal.h -- host-side state behind the opaque C handles.
#pragma once

#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/sssp.h"
#include "internal.h"

namespace sssp {

// Device buffers reused across solves on one graph.
struct Workspace {
    char* ring_mem = nullptr;     // L2 rings (data, tickets, seq, cnt)
    size_t ring_bytes = 0;
    Rings rings{};
    uint32_t nrings = 0;          // bmax * shards
    bool dirty = true;            // metadata must be reset before the next solve
    int grow_shift = 0;           // capacity doublings after overflows
    Ctrl* ctrl = nullptr;
    Ctrl* host_ctrl = nullptr;    // pinned mirror
    unsigned long long* d64 = nullptr;
    size_t d64_n = 0;
    uint32_t* d32 = nullptr;
    size_t d32_n = 0;
    uint32_t* out_d = nullptr;
    size_t out_d_n = 0;
    int32_t* out_p = nullptr;
    size_t out_p_n = 0;
    int32_t* srcs = nullptr;
    size_t srcs_n = 0;
    uint32_t* pend = nullptr;     // pending marks, one per distance slot
    size_t pend_n = 0;
    unsigned long long* tl = nullptr;   // run-time sampling buffer
    size_t tl_n = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr;

    int ensure_queue(uint32_t nrings, uint32_t nch, uint32_t margin, cudaStream_t s, int sms);
    void release();
};

struct Graph {
    uint64_t uid = 0;             // unique per created graph (a handle's address may be reused)
    int device = 0;
    int sms = 1;
    int32_t n = 0;                // real vertices
    int64_t m = 0;                // real arcs
    int32_t nv = 0;               // vertices of the device layout (real + shadow)
    int64_t mv = 0;               // arcs of the device layout
    int32_t split = 0;            // arcs per shadow vertex (0 = none split)
    int32_t layout_req = 0;       // split threshold the current layout was built for
    int32_t wtype = 0;
    int32_t* row_ptr = nullptr;   // [nv + 1]
    uint2* adj = nullptr;         // [mv] (col, weight bits)
    int32_t* owner = nullptr;     // [nv - n]
    sssp_features feat{};
    sssp_config defaults{};
    sssp_config tuned{};
    bool tuned_valid = false;
    // multi-query configurations from sssp_autotune_batch, per size class
    // (the number of queries rounded down to a power of two)
    struct BatchTuned {
        int32_t nq_class;
        sssp_config cfg;
    };
    std::vector<BatchTuned> batch_tuned;
    sssp_stats last{};
    Workspace ws;
    std::mutex mu;
};

// Launch shape, shared-memory layout and the graph/config part of the
// kernel parameters for one instantiation; the caller fills nq, dist,
// vbits/vmask, l2 and ctrl.
struct LaunchPlan {
    KernelKey key;
    int threads = 0;
    int bps = 0;       // blocks per SM
    int grid = 0;      // sms * bps
    size_t smem = 0;
    KParams P;
};

constexpr int32_t kDefaultSplit = 1024;   // default hub split threshold (sssp_config.split_arcs = 0)

int cuda_status(cudaError_t e);
// Serving lanes per graph uid: adds delta and returns the new count.  A
// graph whose layout is in use by a lane is not relaid out.
int lane_refs(uint64_t uid, int delta);
// Makes the graph's layout the one for hub split threshold `split` (caller
// holds g->mu); SSSP_E_BUSY while a serving lane uses the graph.
int ensure_layout(Graph* g, int32_t split, cudaStream_t s);
sssp_config prior_config(const Graph* g);   // the feature prior (sssp_autotune.cu)
int pred_mode_for(const Graph* g);
int plan_launch(const Graph* g, const sssp_config& cfg, int pred_mode, bool mq, LaunchPlan* out,
                bool unit = false);
bool is_device_ptr(const void* p);
void resolve_auto(const Graph* g, sssp_config* c);
void batch_delta(const Graph* g, sssp_config* c, int div);   // delta / div for multi-query launches
// The library's configuration of a multi-query launch of nq queries (the
// caller's config otherwise untouched): narrower buckets, fewer active ones
// (sssp_autotune.cu).
void batch_config(const Graph* g, sssp_config* c, int32_t nq);
// Size class of a multi-query launch (nq rounded down to a power of two).
int32_t nq_class(int32_t nq);
// The batch-tuned configuration for nq queries (same size class), or null.
const sssp_config* batch_tuned_for(const Graph* g, int32_t nq);
// The batch-tuned configuration of the largest size class, or null (serving lanes).
const sssp_config* batch_tuned_largest(const Graph* g);
int validate_config(const sssp_config* c);
// Run-time sampling request (sssp_solve_sampled): host output of cap
// samples of kTimelineFields words, the period, and the count taken.
struct Sampling {
    unsigned long long* out;
    int32_t cap;
    int32_t period_us;
    int32_t* n_out;
};

// `unit`: breadth-first search (every arc counts 1; u32 levels out).
int run_queries(Graph* g, const int32_t* srcs_host, const int32_t* srcs_dev, int32_t src0, int32_t nq,
                void* dist_out, int32_t* pred_out, const sssp_config* cfg, cudaStream_t stream,
                sssp_stats* st_out, bool unit = false, const Sampling* samp = nullptr);

inline uint32_t __float_as_uint_host(float f) {
    uint32_t b;
    std::memcpy(&b, &f, 4);
    return b;
}

}  // namespace sssp
