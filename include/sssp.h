/*
 * sssp.h -- C ABI of libsssp.so, a GB300 (sm_103a) single-source shortest
 * path engine built around a multi-level multi-queue (MLMQ) worklist.
 *
 * Problem (paper Section 2.1): for a directed graph G(V, E, W) with
 * non-negative arc lengths and a source s, compute l_su, the length of a
 * shortest path from s to every vertex u.  The engine is label-correcting:
 * vertices are read from a worklist, their arcs are relaxed (Listing 2,
 * SSSP_relax), and every improved vertex is written back, until the worklist
 * is empty.  The worklist has three levels (Section 3.1): L0 in registers
 * (per warp), L1 in shared memory (per thread block), L2 in global memory
 * (whole grid, delta-bucketed, Section 4.2 "L2 Bucket queue"), joined by the
 * cache-like spill/refill of Section 3.2 and the Read/Write cascade of
 * Listing 1.  Every label-correcting order converges to the same lengths, so
 * results are exact: u32 lengths equal Dijkstra's bit for bit, and f32
 * lengths equal an f32 Dijkstra that performs one IEEE round-to-nearest add
 * per arc.
 *
 * Conventions for every entry point:
 *   - Return value 0 (SSSP_OK) on success, a negative SSSP_E_* code on
 *     failure.  No call throws, aborts the process or leaves a handle
 *     unusable after an error; a failed solve leaves the output buffers
 *     unspecified.
 *   - Pointers to arrays may be host or device memory unless stated; the
 *     kind is detected with cudaPointerGetAttributes.  Host output arrays
 *     are written before the call returns.
 *   - Sizes are element counts.  CSR arrays use int32 indices:
 *     row_ptr[n + 1] (row_ptr[0] == 0, non-decreasing, row_ptr[n] == m) and
 *     col_idx[m] with 0 <= col_idx[e] < n.  Arcs (u, col_idx[e]) for
 *     row_ptr[u] <= e < row_ptr[u + 1].  Self-loops and parallel arcs are
 *     allowed.
 *   - Weights: uint32 (any value; lengths saturate at 0xFFFFFFFE so they
 *     never wrap) or fp32 (finite and >= 0; -0.0 is read as +0.0).
 *   - Distances out: uint32 with 0xFFFFFFFF = unreachable, or fp32 with
 *     +inf = unreachable, matching the graph's weight type.
 *   - Predecessors out (int32, optional): -1 = unreachable, pred[s] = s.
 *     For uint32 graphs whose weights are all >= 1 the predecessor is
 *     canonical: the smallest-index in-neighbour u with
 *     dist[u] + w(u, v) == dist[v].  Otherwise (fp32, or uint32 with zero
 *     weights) it is the arc of the last strict improvement of dist[v]; it
 *     is tight and following it from any reachable vertex reaches s.
 *   - Calls on one graph handle are serialised internally; calls on
 *     different handles may run concurrently from different host threads.
 *   - A `stream` argument is a cudaStream_t (NULL = the legacy default
 *     stream).  Solve calls are synchronous: they return after the results
 *     are in the output buffers (the queue's error word must be read back).
 */
#ifndef SSSP_H
#define SSSP_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SSSP_API __attribute__((visibility("default")))
#else
#define SSSP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ----------------------------------------------------------- status -- */
#define SSSP_OK           0
#define SSSP_E_INVAL     -1 /* bad argument (NULL handle, source out of range, bad config) */
#define SSSP_E_NOMEM     -2 /* device or host allocation failed, or queue capacity exhausted */
#define SSSP_E_CUDA      -3 /* a CUDA runtime call failed */
#define SSSP_E_TIMEOUT   -4 /* a bounded device wait ran out; the handle is reset and usable */
#define SSSP_E_BADGRAPH  -5 /* CSR validation failed (ranges, monotonicity, NaN/inf/negative f32) */
#define SSSP_E_BUSY      -6 /* serving: no free slot or memory budget right now */
#define SSSP_E_NODEV     -7 /* no usable CUDA device */
#define SSSP_E_NOTFOUND  -8 /* serving: unknown ticket */
#define SSSP_E_CANCELLED -9 /* serving: the query was cancelled */

/* Message for a status code (static string, never NULL). */
SSSP_API const char *sssp_strerror(int status);

/* Library version as MAJOR * 10000 + MINOR * 100 + PATCH. */
SSSP_API int sssp_version(void);

/* ------------------------------------------------------------ types -- */
typedef enum { SSSP_W_U32 = 0, SSSP_W_F32 = 1 } sssp_wtype;

/* L1 queue policies (Section 3.4, Fig. 7, Table 1). */
typedef enum {
    SSSP_L1_VECTOR = 0,  /* L1V: FIFO; flushed whole to L2 after every `wb` writes */
    SSSP_L1_NEARFAR = 1, /* L1NF: near/far vectors split at NF; NF = min(far) + delta when near drains */
    SSSP_L1_FILTER = 2,  /* L1FQ: keeps dist <= F, writes the rest back to L2 */
    SSSP_L1_SLF = 3      /* L1SLF: deque; dist <= head goes to the head, else the tail */
} sssp_l1_type;

/* L2 queue policies (Section 4.2).  L2V is the bucket queue with one bucket. */
typedef enum { SSSP_L2_VECTOR = 0, SSSP_L2_BUCKET = 1 } sssp_l2_type;

/* Tunable configuration.  Zero-initialise and call sssp_config_default(),
 * or pass NULL to a solve call to use the graph's tuned (or default)
 * configuration.  Fields the paper leaves open (wb, delta, bnum, bmax, NF,
 * F; Sections 3.4 and 4.2) are chosen by sssp_autotune(). */
typedef struct sssp_config {
    int32_t l1_type;       /* sssp_l1_type */
    int32_t l2_type;       /* sssp_l2_type */
    int32_t l0_rows;       /* L0 capacity per warp in rows of 32 elements (compiled: 2) */
    int32_t l1_cap;        /* L1 capacity per thread block, elements (256..16384, power of two) */
    int32_t wb;            /* L1V: flush L1 to L2 after every wb write calls (0 = never) */
    uint32_t delta_u32;    /* bucket width for u32 graphs (0 = derived from the weights) */
    float delta_f32;       /* bucket width for f32 graphs (0 = derived from the weights) */
    int32_t bnum;          /* buckets a read may take from, counted from the lowest non-empty (1..32) */
    int32_t bmax;          /* buckets in total, a circular window (1..32; 1 = L2V) */
    float filter_deltas;   /* the window front: F = (window base + filter_deltas) * delta.  L1FQ
                              keeps elements <= F, and a light-arc write stays local only up to F */
    float near_deltas;     /* light-arc bound in deltas: a write through an arc of weight
                              <= near_deltas * delta, to a distance <= F, enters L0/L1; any other
                              goes to its L2 bucket (0 = every write enters L0, as in Listing 1) */
    int32_t max_arcs;      /* arcs one warp relaxes per batch; later vertices wait in L0 (>= 32) */
    int32_t claim;         /* L2 chunks one refill claims at once (1..32): the refilling warp
                              reads the first, the others go to its block (as descriptors that
                              other warps read, or into L1 for breadth-first search) */
    int32_t shards;        /* rings per L2 bucket (1, 2, 4, 8, 16 or 32) */
    int32_t refillers;     /* warps of one block that may refill L1 from L2 at the same time (1..32) */
    int32_t stage;         /* 1: a block pools heavy-arc writes per L2 bucket in shared memory and
                              sends full chunks (0: each warp writes its own groups) */
    int32_t block_threads; /* threads per block: 256, 512 or 1024 */
    int32_t blocks_per_sm; /* resident blocks per SM (0 = as many as fit) */
    int32_t timeout_ms;    /* device watchdog for one solve (0 = library default, 20 s) */
    int32_t l2_only;       /* 1 = single-queue baseline: every write goes straight to L2 (no
                              L0/L1, no block staging, one chunk per read); with l2_type
                              SSSP_L2_BUCKET this is a delta-stepping (L2DQ-only) queue, with
                              SSSP_L2_VECTOR a single FIFO (Section 2.2's single-queue designs) */
    int32_t split_arcs;    /* hub split threshold: a vertex with more arcs is represented by
                              zero-weight shadow vertices owning at most split_arcs arcs each
                              (0 = the default 1024; else 32..2^30).  The layout is a property
                              of the graph: a solve whose value differs from the graph's
                              current layout rebuilds it first (one pass over the CSR), and
                              returns SSSP_E_BUSY while a server has a lane on the graph */
    int32_t hub_bnum;      /* > 0: shadow vertices (slices of split hubs) get their own rings (the
                              upper half of each bucket's shards; needs shards >= 2) and are read
                              only from the first hub_bnum non-empty buckets, so a hub is expanded
                              once its distance is near the front (0 = they share the rings) */
    int32_t dedup;         /* 1: a warp round writes each improved target once, with the smallest
                              distance (in-warp duplicates, matched with __match_any_sync) */
    int32_t pending_marks; /* 1: one pending mark per vertex (4 bytes per distance slot): an
                              improved vertex already queued at an earlier-or-equal bucket is not
                              queued again, a read takes the mark and relaxes from the current
                              distance, and a read that finds the mark taken is stale.  Results
                              are the same; queue traffic drops, but the extra atomic per
                              improvement costs more on the measured graphs (default 0 = queue
                              every improvement) */
    int32_t direct_buckets; /* with block staging: a heavy-arc write whose bucket is among the first
                              direct_buckets buckets of the window skips the staging and goes to
                              L2 at once, and a refill first sends the staged elements of those
                              buckets to L2 (0..32; default 2).  0 stages every write until a
                              full chunk or until the block runs dry: fuller chunks, later
                              publication */
} sssp_config;

/* Graph features of Table 2 (Section 3.5), computed at creation. */
typedef struct sssp_features {
    int64_t n, m;                 /* vertices, arcs */
    double avg_deg, max_deg, std_deg;
    double avg_w, max_w, std_w;
    double min_w;
    int32_t symmetric;            /* 1 if every arc has a reverse arc of equal weight, -1 unknown */
    int32_t has_zero_w;
    int64_t shadows;              /* shadow vertices of the device layout (split hubs) */
} sssp_features;

/* Counters of the last solve on a graph (Fig. 3 quantities). */
typedef struct sssp_stats {
    double kernel_ms;             /* persistent relaxation kernel, CUDA-event time */
    double total_ms;              /* whole call on the device: init + kernel + outputs */
    int64_t reached;              /* -1: not counted by the library (count finite distances
                                     in the output) */
    int64_t reached_arcs;         /* -1: not counted (m_r: arcs out of reached vertices) */
    int64_t pops_l0, pops_l1, pops_l2; /* batches read from each level */
    int64_t pops_heavy;           /* 0 (reserved) */
    int64_t relax_arcs;           /* arcs scanned (work) */
    int64_t improved;             /* successful relaxations (writes back) */
    int64_t stale;                /* popped elements already superseded */
    int64_t l2_chunks_written, l1_flushes, far_pushes;
    int64_t cas_fail;             /* failed ticket claims on the L2 rings */
    int64_t refills, deferred;    /* L1 refills from L2; batch vertices deferred to L0 */
    int64_t relax_shadow;         /* arcs scanned from shadow vertices (split hubs) */
    int64_t cycles[6];            /* SM cycles summed over warps: relax, L1 read, L2 write,
                                     L2/task read, idle, L0 read */
    int32_t grid_blocks, block_threads;
    int32_t attempts;             /* > 1 if the queue was regrown after an overflow */
    int32_t pad0;
    int64_t dup_targets;          /* improved arcs whose target another improved arc of the same
                                     warp round shares (in-warp duplicates, Listing 1's write) */
    int64_t rounds;               /* 32-arc relaxation rounds of all warps */
    int64_t refill_tries;         /* L1 refill attempts from L2 (refills = the successful ones) */
    int64_t wait_spins;           /* spins on L2 chunk sequence words (writer and reader waits) */
    int64_t idle_iters;           /* worker iterations that found no work anywhere */
    int64_t window_pull_backs;    /* L2 writes below the bucket window (window moved back) */
    int64_t window_advances;      /* window moves forward past empty buckets */
    int64_t lock_spins;           /* spins on the block locks (L1 near-far / SLF, block staging) */
    int64_t cycles_fine[8];       /* SM cycles in relaxation rounds (loads + atomics), in their
                                     pushes, in batch set-up, in far-staging flushes, in block-lock
                                     waits, in L2 claims, in reading claimed chunks and in staging
                                     flushes before a refill; zero unless the library is built with
                                     SSSP_FINE_CYCLES=1 */
    int64_t not_queued;           /* improvements not queued because the vertex was pending
                                     (sssp_config.pending_marks) */
} sssp_stats;

typedef struct sssp_graph sssp_graph;
typedef struct sssp_server sssp_server;

/* --------------------------------------------------------- configuration -- */

/* Fills *cfg with the library defaults: filtered L1 (L1FQ) over the delta-bucketed L2, four
 * active buckets, delta derived from the weights.  SSSP_E_INVAL if cfg is NULL. */
SSSP_API int sssp_config_default(sssp_config *cfg);

/* ------------------------------------------------------------------ graph -- */

/* Copies a CSR graph to the device, validates it and derives the layout the
 * kernels use: interleaved (col, weight) pairs (one 8-byte load per arc),
 * and every vertex with more than 1024 arcs (the default of
 * sssp_config.split_arcs) represented by zero-weight shadow vertices that
 * each own a slice of at most that many arcs, so the arcs of a hub are
 * relaxed by many warps at once.
 *   row_ptr  int32[n + 1], col_idx int32[m], weights uint32[m] or fp32[m]
 *            (per `wtype`); host or device memory, borrowed (copied).
 *   n >= 1, 0 <= m < 2^31.
 *   *out     receives a new handle owning device memory; free it with
 *            sssp_graph_destroy.
 * The graph's default configuration is the feature prior: the Table 2
 * features pick a family (power-law, mesh or road) and its settings
 * (Section 3.5).
 * Errors: SSSP_E_INVAL (NULL/negative sizes), SSSP_E_BADGRAPH (validation),
 * SSSP_E_NOMEM, SSSP_E_CUDA, SSSP_E_NODEV.  Cites: Section 2.1 (G(V,E,W)),
 * Listing 2 (edge_list / edge_weight). */
SSSP_API int sssp_graph_create(const int32_t *row_ptr, const int32_t *col_idx, const void *weights,
                      int32_t n, int64_t m, int32_t wtype, sssp_graph **out);

/* Frees the graph and every device buffer it owns.  NULL is a no-op. */
SSSP_API int sssp_graph_destroy(sssp_graph *g);

/* Table 2 features of the graph (Section 3.5). */
SSSP_API int sssp_graph_features(const sssp_graph *g, sssp_features *out);

/* ------------------------------------------------------------------ solve -- */

/* Single-source solve (Listing 2: work kernel + termination of Section 4.1).
 *   src       0 <= src < n.
 *   dist_out  n elements (uint32 or fp32 per the graph), host or device.
 *   pred_out  n int32 or NULL.
 *   cfg       NULL = the graph's tuned configuration, else its default: the feature
 *             prior picked at creation from the Table 2 features (Section 3.5).
 *   stream    cudaStream_t or NULL.
 * Returns after completion.  Errors: SSSP_E_INVAL, SSSP_E_TIMEOUT,
 * SSSP_E_NOMEM (queue could not be grown), SSSP_E_CUDA. */
SSSP_API int sssp_solve(sssp_graph *g, int32_t src, void *dist_out, int32_t *pred_out,
               const sssp_config *cfg, void *stream);

/* Batched multi-source solve: nq independent queries in ONE persistent
 * launch sharing the worklist (queue elements carry their query).
 *   srcs      int32[nq] (host or device), each in [0, n); repeats allowed.
 *   dist_out  nq * n elements, query-major: dist_out[q * n + v].
 *   pred_out  nq * n int32 or NULL.
 * nq * 2^ceil(log2 n) must not exceed 2^32 (the element key packs the query
 * index above the vertex bits).  With cfg NULL the batch uses the
 * configuration sssp_autotune_batch cached for its size class, if any.
 * Otherwise, when the library picks delta (cfg NULL, or a zero delta), the
 * batch uses delta / min(16, max(1, nq / 32)) with bnum <= 4: the queries
 * supply the parallelism, and narrower buckets cut out-of-order work.
 * Errors as sssp_solve. */
SSSP_API int sssp_solve_batch(sssp_graph *g, const int32_t *srcs, int32_t nq, void *dist_out,
                     int32_t *pred_out, const sssp_config *cfg, void *stream);

/* Counters and timings of the last solve/batch on this graph. */
SSSP_API int sssp_last_stats(const sssp_graph *g, sssp_stats *out);

/* ---------------------------------------------------------------- autotune -- */

/* Picks a configuration for this graph (Section 3.5 adaptive configuration):
 * a prior from the Table 2 features and the per-family findings of
 * Section 5.4, refined by timing candidate configurations on up to nsrc of
 * the given sources (host or device int32[nsrc]) within about budget_ms.
 * The winner is cached on the graph (used when cfg == NULL) and copied to
 * *out when out != NULL.  budget_ms <= 0 returns the prior untimed. */
SSSP_API int sssp_autotune(sssp_graph *g, const int32_t *srcs, int32_t nsrc, int32_t budget_ms,
                  sssp_config *out);

/* Picks a configuration for multi-query launches (sssp_solve_batch) of about
 * nq queries: Section 3.5's input-adaptive configuration applied to the
 * batched launch.  It starts from the graph's configuration with the
 * library's multi-query bucket width (delta / min(16, nq / 32), bnum <= 4)
 * and, within about budget_ms, times one whole batch launch from the given
 * sources per candidate: the bucket-width divisor, bnum, the L1 depth, the
 * claim size, the refill concurrency and the hub rings.  The winner is cached
 * on the graph for launches of the same size class (nq rounded down to a
 * power of two) made with cfg == NULL; serving lanes of the graph created
 * afterwards use the winner of the largest class.  budget_ms == 0 caches the
 * starting point untimed.
 *   srcs   int32[nq], host or device, each in [0, n); nq >= 2.
 *   out    receives the configuration (may be NULL).
 * Errors: SSSP_E_INVAL, SSSP_E_NOMEM (the nq * n distance buffer of the
 * timed launches), SSSP_E_CUDA. */
SSSP_API int sssp_autotune_batch(sssp_graph *g, const int32_t *srcs, int32_t nq, int32_t budget_ms,
                                 sssp_config *out);

/* ---------------------------------------------------------- no allocation -- */

/* Largest vertex count sssp_solve_noalloc accepts. */
#define SSSP_NOALLOC_MAX_VERTICES 2097152

/* Single-source solve that allocates nothing.  The paper has no counterpart;
 * this entry point exists for callers that cannot allocate device memory at
 * the time they need an answer: code whose device memory is owned by a pool
 * or arena, components with an allocation budget fixed up front, and
 * latency-critical paths that must not call cudaMalloc/cudaFree because
 * those calls can synchronise the device.
 *
 * It runs the same persistent relaxation kernel as sssp_solve with a fixed
 * configuration (L1 filter queue, 8-bucket L2, no hub splitting), keeping
 * every piece of scratch state (control block, L2 rings, packed
 * distance/predecessor words) in one array of about 25 MiB that is part of
 * the library image: every GPU that loads the library holds it until the
 * process exits.  The first call on a device resolves that array's device
 * address.  All calls share the array and it keeps the last call's contents;
 * every call first re-initialises what must start empty (queue metadata,
 * control block, distance words), so a call does not depend on how the
 * previous one ended.  Calls serialise on a process-wide lock and return only
 * after the GPU work has finished; two calls that overlapped on the GPU would
 * race on the array.  Every call reads a status back and synchronises its
 * stream part-way, so no call may be made on a stream that is capturing a
 * CUDA graph.
 *
 *   row_ptr   int32[n + 1], device memory.
 *   arcs      device memory, 2 * m uint32 words: for arc e, arcs[2e] is the
 *             column (int32, 0 <= col < n) and arcs[2e + 1] the weight
 *             (uint32 value or fp32 bits per `wtype`); read only.
 *   n         1 <= n <= SSSP_NOALLOC_MAX_VERTICES; larger graphs: SSSP_E_INVAL.
 *   dist_out  n elements, device memory; pred_out n int32, device memory or NULL.
 *   stream    cudaStream_t or NULL.
 * The CSR is validated on the device (SSSP_E_BADGRAPH).  Distances and
 * predecessors follow the conventions of sssp_solve.  An fp32 weight of
 * -0.0 is accepted and adds like +0.0, but the arcs are used as given (not
 * normalised), so such an arc is routed like a weight above the light-arc
 * bound; results are the same.  SSSP_E_NOMEM if the
 * fixed L2 rings overflow; host pointers are rejected with SSSP_E_INVAL. */
SSSP_API int sssp_solve_noalloc(const int32_t *row_ptr, const uint32_t *arcs, int32_t n, int64_t m,
                                int32_t wtype, int32_t src, void *dist_out, int32_t *pred_out,
                                void *stream);

/* -------------------------------------------------------- run-time sampling -- */

/* Run-time behaviour of one solve (Section 5.3 follows active warps and
 * processed vertices over time): sssp_solve plus a timeline sampled every
 * period_us by one lane of block 0 while the kernel runs.
 *   samples_out  host memory, cap * 6 uint64 words; sample i holds
 *                [ns since launch, elements written to L2, L2 elements
 *                completed (published per block, so it lags), elements taken
 *                for relaxation, the L2 window W (lowest bucket with work),
 *                warps of block 0 holding a batch].
 *   *n_out       samples taken (<= cap).
 * Sampling adds a few atomics per batch; distances and predecessors are
 * those of sssp_solve.  SSSP_E_INVAL for cap < 1, period_us < 1 or a device
 * samples_out; otherwise as sssp_solve. */
SSSP_API int sssp_solve_sampled(sssp_graph *g, int32_t src, void *dist_out, int32_t *pred_out,
                                const sssp_config *cfg, uint64_t *samples_out, int32_t cap,
                                int32_t period_us, int32_t *n_out);

/* ------------------------------------------------------------------- BFS -- */

/* Breadth-first search on the same engine (the BFS case study of Section
 * 5.7): every arc counts 1, whatever the graph's weights, so the
 * multi-level queue orders the search by level.
 *   level_out  [n] uint32: hops from src, 0xFFFFFFFF when unreachable
 *              (host or device memory).
 *   pred_out   [n] int32 or NULL: the smallest-index parent one level up,
 *              pred[src] = src, -1 when unreachable.
 *   cfg        NULL = the graph's configuration with delta 1 (one bucket
 *              per level); a given cfg with delta 0 also means 1.
 * Errors as for sssp_solve. */
SSSP_API int sssp_bfs(sssp_graph *g, int32_t src, uint32_t *level_out, int32_t *pred_out,
                      const sssp_config *cfg, void *stream);

/* ---------------------------------------------------------------- serving -- */

/* Serving with continuous batching.  (An extension: the paper solves one
 * source per launch and has no serving mode.)  Graphs stay resident; each
 * graph (and predecessor mode) in use gets a "lane": one multi-query
 * worklist, per-query distance slices and its own L2 rings.  A worker
 * thread runs every lane in time slices of slice_us: at the end of a slice
 * the kernel drains its L0/L1/staging queues into the L2 rings, the host
 * counts each query's remaining L2 elements, hands finished queries'
 * results to their buffers and frees their slots, and admits queued
 * queries into free slots before the next slice -- so new queries join
 * while earlier ones are still running.  A query admitted while the
 * lane's bucket window is at W has its buckets shifted by W, so its work
 * is ordered with the work already in flight.  A lane uses a quarter of the
 * graph's delta (it holds many queries under load).  Lanes of different graphs
 * run concurrently on their own streams, sharing the SMs. */
typedef struct sssp_serve_options {
    size_t  mem_budget_bytes;  /* device bytes for distance slices and L2 rings of all lanes
                                  (0 = a quarter of the free device memory at creation) */
    int32_t max_slots;         /* concurrent queries per lane, 1..4096 (default 128: with five
                                  resident graphs at 2000 q/s, 256 filled every lane and served
                                  180 q/s, 128 served 340 q/s); also
                                  bounded by 2^32 / (vertices rounded up to a power of two) */
    int32_t slice_us;          /* length of one slice, 50..100000 (default 1000); a lane with
                                  q queries in flight runs slices of min(8, max(1, q / 4))
                                  times this */
    int32_t max_queued;        /* queries waiting for a slot; beyond it submit returns
                                  SSSP_E_BUSY (default 65536) */
    int32_t ring_shift;        /* initial L2 ring capacity per lane: (slots x vertices) >>
                                  ring_shift chunks, 0..16 (default 4); rings grow between slices
                                  when they are half full, and after an overflow the lane's
                                  queries restart on larger rings */
    int32_t query_timeout_ms;  /* a query still running after this ends with SSSP_E_TIMEOUT
                                  (0 = no limit) */
    int32_t flags;             /* SSSP_SERVE_* test flags below (default 0) */
    int32_t reserved[2];       /* must be zero */
} sssp_serve_options;

/* Test flags of sssp_serve_options.flags.  They exercise recovery paths
 * from the host side; no device fault is involved. */
#define SSSP_SERVE_MIGRATE_EACH_SLICE 1  /* move the live L2 chunks to new rings after every slice */
#define SSSP_SERVE_INJECT_OVERFLOW    2  /* treat each lane's first slice as an L2 overflow: the
                                            lane's queries restart on larger rings */
#define SSSP_SERVE_INJECT_TIMEOUT     4  /* treat each lane's first slice as a timed-out device
                                            wait: the lane's queries fail with SSSP_E_TIMEOUT */
#define SSSP_SERVE_INJECT_NEGATIVE    8  /* read each lane's first scanned slot as a negative L2
                                            count (more reads than writes): the lane's queries fail
                                            with SSSP_E_CUDA and the lane starts over */

typedef struct sssp_serve_stats {
    int64_t submitted;
    int64_t completed;         /* DONE */
    int64_t failed;            /* ERROR, cancellations included */
    int64_t cancelled;
    int64_t slices;            /* serving launches (one per lane per slice) */
    int64_t joined_running;    /* queries admitted into a lane that had queries running */
    int64_t ring_growths;      /* ring migrations between slices (to larger rings; every slice
                                  with SSSP_SERVE_MIGRATE_EACH_SLICE) */
    int64_t restarts;          /* lane restarts after an L2 overflow inside a slice */
    int64_t max_resident;      /* most queries resident in lanes at once */
    double  kernel_ms;         /* summed slice kernel time over all lanes */
} sssp_serve_stats;

/* Fills *opt with the defaults.  SSSP_E_INVAL if opt is NULL. */
SSSP_API int sssp_serve_options_default(sssp_serve_options *opt);

/* Starts a server on the current device (opt NULL = defaults).
 * SSSP_E_INVAL for out-of-range options, SSSP_E_NODEV, SSSP_E_CUDA. */
SSSP_API int sssp_serve_create(const sssp_serve_options *opt, sssp_server **out);

/* Queues one query from `src` on g.  dist_out ([n] distance words as in
 * sssp_solve) and pred_out ([n], may be NULL) may be host or device memory
 * and must stay valid until the query is DONE or ERROR; g must not be
 * destroyed before then.  *ticket_out identifies the query.  SSSP_E_INVAL
 * for NULL arguments or a source out of range, SSSP_E_BUSY when max_queued
 * queries are waiting. */
SSSP_API int sssp_serve_submit(sssp_server *s, sssp_graph *g, int32_t src, void *dist_out,
                               int32_t *pred_out, uint64_t *ticket_out);

/* Query states. */
#define SSSP_Q_QUEUED  0
#define SSSP_Q_RUNNING 1
#define SSSP_Q_DONE    2
#define SSSP_Q_ERROR   3

/* Non-blocking state of a ticket; for ERROR, *status_out (may be NULL)
 * receives the failing SSSP_E_* code (SSSP_E_CANCELLED after a cancel).
 * Tickets stay known until sssp_serve_release.  SSSP_E_NOTFOUND for an
 * unknown ticket. */
SSSP_API int sssp_serve_poll(sssp_server *s, uint64_t ticket, int32_t *state_out, int32_t *status_out);

/* Blocks until the ticket is DONE or ERROR, or timeout_ms passes (then
 * SSSP_E_TIMEOUT with the query still live; timeout_ms < 0 waits forever). */
SSSP_API int sssp_serve_wait(sssp_server *s, uint64_t ticket, int32_t timeout_ms, int32_t *state_out,
                             int32_t *status_out);

/* Submit-to-DONE latency of the ticket in microseconds; SSSP_E_BUSY while
 * the query is not DONE. */
SSSP_API int sssp_serve_latency_us(sssp_server *s, uint64_t ticket, double *us_out);

/* Cancels a queued or running query: SSSP_OK means it ended with
 * ERROR/SSSP_E_CANCELLED and its buffers are not written after the call
 * returns; SSSP_E_BUSY means its results are already being delivered (it
 * will be DONE); SSSP_E_INVAL if it had already ended.  A running query's
 * slot is reused once its remaining queue elements have drained. */
SSSP_API int sssp_serve_cancel(sssp_server *s, uint64_t ticket);

/* Forgets a DONE/ERROR ticket (SSSP_E_BUSY while it is queued or running). */
SSSP_API int sssp_serve_release(sssp_server *s, uint64_t ticket);

/* Counters since creation. */
SSSP_API int sssp_serve_get_stats(sssp_server *s, sssp_serve_stats *out);

/* Lets every queued and running query finish, then frees the server. */
SSSP_API int sssp_serve_destroy(sssp_server *s);

#ifdef __cplusplus
}
#endif
#endif /* SSSP_H */
