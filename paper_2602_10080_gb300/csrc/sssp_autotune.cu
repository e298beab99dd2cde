// sssp_autotune.cu -- input-adaptive configuration (Section 3.5).
//
// The paper ranks candidate queue configurations with a RandomForest trained
// on 680 SuiteSparse matrices, from the Table 2 features.  Neither the corpus
// nor the trained model is available, so this replaces it with
//   (1) a prior from the Table 2 features and the per-family findings of
//       Section 5.4 (road: L1V/L1NF over a FIFO L2 when small, L1V over the
//       bucket queue when large; meshes: L1FQ-L2V; power-law: priority-aware
//       L1 over the bucket queue), and
//   (2) a short timed coordinate search around the prior on sample sources:
//       L1 policy, delta, near window, bnum, shards, claim size, batch size,
//       block size, L1 depth, refill concurrency, hub split threshold and hub
//       rings, each candidate timed by the CUDA-event duration of the
//       relaxation kernel.
// The winner is cached on the graph and used by solves given cfg == NULL.
//
// sssp_autotune_batch does the same for multi-query launches of a given size:
// it times whole batch launches over the bucket-width divisor, bnum, L1
// depth, claim size, refill concurrency and hub rings, and caches the winner
// per size class for sssp_solve_batch and the serving lanes.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/sssp.h"
#include "api_internal.h"

namespace sssp {

// Graph family from Table 2 features.
enum Family { kRoad = 0, kMesh = 1, kPowerLaw = 2 };

static Family family_of(const sssp_features& f) {
    double cv = f.avg_deg > 0 ? f.std_deg / f.avg_deg : 0.0;
    if (f.max_deg > 16.0 * std::max(1.0, f.avg_deg) || cv > 1.5) return kPowerLaw;
    if (f.avg_deg < 4.5) return kRoad;
    return kMesh;
}

void batch_config(const Graph* g, sssp_config* c, int32_t nq) {
    int div = std::min(16, std::max(1, nq / 32));
    int bnum = 4;   // the batch width was measured with 4 active buckets
    if (family_of(g->feat) == kPowerLaw && g->wtype == SSSP_W_U32) {
        // integer weights on a power-law graph: half the narrowing, 8 active buckets.  256
        // R-MAT-20 sources on GB300 (1024-thread blocks): 141 ms against 145 ms with
        // delta / 8 and 4 buckets; fp32 weights were slower with wider buckets (229 ms
        // against 199 ms), so they keep delta / 8
        div = std::max(1, div / 2);
        bnum = 8;
    }
    batch_delta(g, c, div);
    c->bnum = std::min(c->bnum, bnum);
}

sssp_config prior_config(const Graph* g) {
    sssp_config c;
    sssp_config_default(&c);
    const sssp_features& f = g->feat;
    switch (family_of(f)) {
        case kPowerLaw:
            // priority matters most (Section 5.4): filtered L1 over the bucket queue
            c.l1_type = SSSP_L1_FILTER;
            c.l2_type = SSSP_L2_BUCKET;
            c.filter_deltas = 1.0f;
            c.near_deltas = 1.0f;
            c.bnum = 16;
            // many small buckets of work: fewer, larger L2 reads (16 chunks, of which the
            // refilling warp reads one and other warps the rest: R-MAT-22 on GB300 3.16 ms
            // against 3.53 with 8 and 3.28 with 32)
            c.claim = 16;
            // hub slices of 512 arcs: with each slice relaxed from its hub's current
            // distance, R-MAT-22 took 6.8 ms against 8.0 ms with 1024 (relaxations
            // 237M -> 178M; 384: 7.0, 768: 6.9, 256: 8.3 ms) on GB300
            c.split_arcs = 512;
            // every write is staged until its bucket fills a chunk: on R-MAT-22 on GB300
            // 6.2 ms against 6.7 ms with the first two buckets written directly, and the
            // 256-query batch on R-MAT-20 289 ms against 297 ms
            c.direct_buckets = 0;
            // 16 rings per bucket: fewer refills contend for one ring's read ticket
            // (R-MAT-22 on GB300: 4.70 ms against 4.93 with 8; 32: 5.31 ms)
            c.shards = 16;
            // one block of 1024 threads per SM: R-MAT-22 3.06 ms against 3.17 with two of
            // 512, and 256 R-MAT-20 sources in one launch 145 ms against 152
            c.block_threads = 1024;
            break;
        case kMesh:
            c.l1_type = SSSP_L1_FILTER;
            c.l2_type = SSSP_L2_BUCKET;
            c.filter_deltas = 2.0f;
            c.near_deltas = 2.0f;
            c.bnum = 4;
            break;
        case kRoad:
            // high diameter: wide near window, vector L1, bucket L2 for large graphs;
            // 8 active buckets of 4x the general width (see below)
            c.l1_type = SSSP_L1_VECTOR;
            c.wb = 0;
            c.l2_type = SSSP_L2_BUCKET;
            c.near_deltas = 4.0f;
            c.bnum = f.n > (1 << 22) ? 8 : 4;
            break;
    }
    c.bmax = 32;
    c.delta_u32 = 0;
    c.delta_f32 = 0.0f;
    resolve_auto(g, &c);
    if (family_of(f) == kRoad && f.n > (1 << 22)) {
        // a large road-shaped graph advances as a thin wavefront whose reads are bound by L2
        // claims: wider buckets give each claim more work, and fewer warps contend for the
        // claims.  On the 4096^2 road graph on GB300, 4x the general width with 8 active
        // buckets took 33 ms against 44 ms (2x: 39, 8x: 58 ms); one block per SM with 16 shards
        // per bucket and 4 refilling warps per block then took 21 ms.  On grids of 256^2 and
        // 1024^2 vertices the wider buckets were 15% and 3% slower, hence the size gate
        if (g->wtype == SSSP_W_F32) c.delta_f32 *= 4.0f;
        else c.delta_u32 = (uint32_t)std::min<uint64_t>(4000000000ull, (uint64_t)c.delta_u32 * 4u);
        c.blocks_per_sm = 1;
        c.shards = 16;
        c.refillers = 4;
        c.claim = 8;  // 15.4-15.7 ms against 16.0 with 4
    }
    if (family_of(f) == kPowerLaw) {
        // a quarter of the general width with 16 active buckets (the same
        // active distance range, finer buckets): the hubs supply the
        // parallelism; fastest in a GB300 sweep on R-MAT-22
        if (g->wtype == SSSP_W_F32) c.delta_f32 *= 0.25f;
        else c.delta_u32 = std::max<uint32_t>(1u, c.delta_u32 / 4u);
    }
    return c;
}

}  // namespace sssp

using namespace sssp;

extern "C" int sssp_autotune(sssp_graph* gh, const int32_t* srcs, int32_t nsrc, int32_t budget_ms,
                             sssp_config* out) {
    if (!gh) return SSSP_E_INVAL;
    Graph* g = reinterpret_cast<Graph*>(gh);
    std::lock_guard<std::mutex> lk(g->mu);
    sssp_config best = prior_config(g);
    if (budget_ms <= 0 || nsrc <= 0 || !srcs) {
        g->tuned = best;
        g->tuned_valid = true;
        if (out) *out = best;
        return SSSP_OK;
    }
    std::vector<int32_t> hs(nsrc);
    if (is_device_ptr(srcs)) {
        if (cudaMemcpy(hs.data(), srcs, sizeof(int32_t) * nsrc, cudaMemcpyDeviceToHost) != cudaSuccess)
            return SSSP_E_CUDA;
    } else {
        hs.assign(srcs, srcs + nsrc);
    }
    for (int32_t s : hs)
        if (s < 0 || s >= g->n) return SSSP_E_INVAL;
    hs.resize(std::min<int32_t>(nsrc, 4));

    void* dbuf = nullptr;
    if (cudaMalloc(&dbuf, sizeof(uint32_t) * (size_t)g->n) != cudaSuccess) {
        cudaGetLastError();
        return SSSP_E_NOMEM;
    }
    const auto t0 = std::chrono::steady_clock::now();
    auto elapsed_ms = [&]() {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    };
    // time = median kernel time over the sample sources; failures = +inf
    auto measure = [&](const sssp_config& c) -> double {
        std::vector<double> ts;
        for (int32_t s : hs) {
            sssp_stats st;
            int rc = run_queries(g, nullptr, nullptr, s, 1, dbuf, nullptr, &c, nullptr, &st);
            if (rc != SSSP_OK) return INFINITY;
            ts.push_back(st.kernel_ms);
        }
        std::sort(ts.begin(), ts.end());
        return ts[ts.size() / 2];
    };
    // warm-up (allocations, first launch)
    measure(best);
    double best_t = measure(best);
    const bool f32 = g->wtype == SSSP_W_F32;
    const double d0 = f32 ? best.delta_f32 : (double)best.delta_u32;

    for (int pass = 0; pass < 2 && elapsed_ms() < budget_ms; pass++) {
        std::vector<sssp_config> cands;
        // L1 policy (Table 1), with the L1V flush period
        for (int l1 = 0; l1 < 4; l1++) {
            for (int wb : {0, 16}) {
                if (l1 != SSSP_L1_VECTOR && wb) continue;
                sssp_config c = best;
                c.l1_type = l1;
                c.wb = l1 == SSSP_L1_VECTOR ? wb : 0;
                cands.push_back(c);
            }
        }
        // delta (bucket width) and the L2 policy
        for (double mult : {0.25, 0.5, 2.0, 4.0}) {
            sssp_config c = best;
            if (f32) c.delta_f32 = (float)(d0 * mult);
            else c.delta_u32 = (uint32_t)std::max(1.0, std::round(d0 * mult));
            cands.push_back(c);
        }
        {
            sssp_config c = best;
            c.l2_type = SSSP_L2_VECTOR;
            cands.push_back(c);
        }
        for (float nd : {0.0f, 0.5f, 2.0f, 8.0f}) {
            sssp_config c = best;
            c.near_deltas = nd;
            cands.push_back(c);
        }
        for (int bn : {1, 4, 8}) {
            sssp_config c = best;
            c.bnum = bn;
            cands.push_back(c);
        }
        for (float fd : {0.5f, 2.0f, 4.0f}) {
            sssp_config c = best;
            if (c.l1_type != SSSP_L1_FILTER) continue;
            c.filter_deltas = fd;
            cands.push_back(c);
        }
        for (int sh : {2, 16}) {
            sssp_config c = best;
            c.shards = sh;
            cands.push_back(c);
        }
        for (int cl : {4, 8, 16, 32}) {
            sssp_config c = best;
            if (c.claim == cl) continue;
            c.claim = cl;
            cands.push_back(c);
        }
        for (int ma : {512, 8192}) {
            sssp_config c = best;
            c.max_arcs = ma;
            cands.push_back(c);
        }
        for (int bt : {256, 512, 1024}) {
            sssp_config c = best;
            if (c.block_threads == bt) continue;
            c.block_threads = bt;
            cands.push_back(c);
        }
        // queue depth of L1, refill concurrency, and the hub handling: the
        // split threshold ("threads per vertex" above which a vertex's arcs
        // are spread over warps) and the hub rings
        for (int l1 : {1024, 4096}) {
            sssp_config c = best;
            c.l1_cap = l1;
            cands.push_back(c);
        }
        for (int rf : {4, 16}) {
            sssp_config c = best;
            c.refillers = rf;
            cands.push_back(c);
        }
        for (int hb : {0, 1, 2}) {
            sssp_config c = best;
            if (c.hub_bnum == hb) continue;
            c.hub_bnum = hb;
            cands.push_back(c);
        }
        for (int db : {0, 2}) {
            sssp_config c = best;
            if (c.direct_buckets == db || !c.stage) continue;
            c.direct_buckets = db;
            cands.push_back(c);
        }
        if (g->feat.max_deg > 256.0) {
            for (int sp : {256, 4096}) {
                sssp_config c = best;
                c.split_arcs = sp;
                cands.push_back(c);
            }
        }
        for (const sssp_config& c : cands) {
            if (elapsed_ms() > budget_ms) break;
            if (validate_config(&c) != SSSP_OK) continue;
            double t = measure(c);
            if (t < best_t * 0.97) {
                best_t = t;
                best = c;
            }
        }
    }
    cudaFree(dbuf);
    g->tuned = best;
    g->tuned_valid = true;
    if (out) *out = best;
    return SSSP_OK;
}

extern "C" int sssp_autotune_batch(sssp_graph* gh, const int32_t* srcs, int32_t nq, int32_t budget_ms,
                                   sssp_config* out) {
    if (!gh || !srcs || nq < 2 || budget_ms < 0) return SSSP_E_INVAL;
    Graph* g = reinterpret_cast<Graph*>(gh);
    std::lock_guard<std::mutex> lk(g->mu);
    std::vector<int32_t> hs(nq);
    if (is_device_ptr(srcs)) {
        if (cudaMemcpy(hs.data(), srcs, sizeof(int32_t) * nq, cudaMemcpyDeviceToHost) != cudaSuccess)
            return SSSP_E_CUDA;
    } else {
        hs.assign(srcs, srcs + nq);
    }
    for (int32_t s : hs)
        if (s < 0 || s >= g->n) return SSSP_E_INVAL;
    // the starting point: the graph's configuration with the library's
    // multi-query bucket width (the heuristic sssp_solve_batch uses untuned)
    sssp_config base = g->tuned_valid ? g->tuned : g->defaults;
    base.delta_u32 = 0;
    base.delta_f32 = 0.0f;
    resolve_auto(g, &base);
    batch_config(g, &base, nq);
    sssp_config best = base;
    if (budget_ms > 0) {
        void* dbuf = nullptr;
        if (cudaMalloc(&dbuf, sizeof(uint32_t) * (size_t)g->n * (size_t)nq) != cudaSuccess) {
            cudaGetLastError();
            return SSSP_E_NOMEM;
        }
        const auto t0 = std::chrono::steady_clock::now();
        auto elapsed_ms = [&]() {
            return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        };
        auto measure = [&](const sssp_config& c) -> double {
            sssp_stats st;
            int rc = run_queries(g, hs.data(), nullptr, 0, nq, dbuf, nullptr, &c, nullptr, &st);
            return rc == SSSP_OK ? st.kernel_ms : INFINITY;
        };
        measure(best);   // warm-up (allocations, first launch)
        double best_t = measure(best);
        const bool f32 = g->wtype == SSSP_W_F32;
        sssp_config general = base;
        batch_delta(g, &general, 1);
        const double d1 = f32 ? general.delta_f32 : (double)general.delta_u32;
        for (int pass = 0; pass < 2 && elapsed_ms() < budget_ms; pass++) {
            std::vector<sssp_config> cands;
            for (int div : {2, 4, 8, 16, 32}) {
                sssp_config c = best;
                if (f32) c.delta_f32 = (float)(d1 / div);
                else c.delta_u32 = (uint32_t)std::max(1.0, std::floor(d1 / div));
                cands.push_back(c);
            }
            for (int bn : {1, 2, 4, 8, 16}) {
                sssp_config c = best;
                c.bnum = bn;
                cands.push_back(c);
            }
            // bucket width and active buckets together (a wider bucket wants more of them)
            for (int div : {2, 4}) {
                sssp_config c = best;
                if (f32) c.delta_f32 = (float)(d1 / div);
                else c.delta_u32 = (uint32_t)std::max(1.0, std::floor(d1 / div));
                c.bnum = 16;
                cands.push_back(c);
            }
            for (int bt : {512, 1024}) {
                sssp_config c = best;
                if (c.block_threads == bt) continue;
                c.block_threads = bt;
                cands.push_back(c);
            }
            for (int l1 : {1024, 2048, 4096}) {
                sssp_config c = best;
                c.l1_cap = l1;
                cands.push_back(c);
            }
            for (int cl : {4, 8, 16, 32}) {
                sssp_config c = best;
                c.claim = cl;
                cands.push_back(c);
            }
            for (int rf : {4, 8, 16}) {
                sssp_config c = best;
                c.refillers = rf;
                cands.push_back(c);
            }
            for (int hb : {0, 1, 2}) {
                sssp_config c = best;
                c.hub_bnum = hb;
                cands.push_back(c);
            }
            for (const sssp_config& c : cands) {
                if (elapsed_ms() > budget_ms) break;
                if (std::memcmp(&c, &best, sizeof(c)) == 0 || validate_config(&c) != SSSP_OK) continue;
                const double t = measure(c);
                if (t < best_t * 0.97) {
                    best_t = t;
                    best = c;
                }
            }
        }
        cudaFree(dbuf);
    }
    const int32_t k = nq_class(nq);
    bool found = false;
    for (Graph::BatchTuned& b : g->batch_tuned)
        if (b.nq_class == k) {
            b.cfg = best;
            found = true;
        }
    if (!found) g->batch_tuned.push_back(Graph::BatchTuned{k, best});
    if (out) *out = best;
    return SSSP_OK;
}
