/*
 * CPU ORACLE for single-source shortest paths -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load this file's library.  The GPU product path never calls it and
 * shares no code with it.
 *
 * What it computes (Section 2.1 of the paper): for a graph G(V, E, W) with
 * non-negative weights and a source s, the length l_su of a shortest path
 * from s to every u.  Relaxing edge (u, v) tests whether l_su + |e_uv| is
 * shorter than the current l_sv.  The GPU method is label-correcting and
 * converges to exactly this value, so the oracle is the plain definition:
 *
 *   - Dijkstra with a binary heap and lazy deletion (the strict-priority
 *     end point named in Section 2.1), for three arithmetics:
 *       u32: path lengths accumulate in 64 bits and saturate at 2^32 - 2;
 *            0xFFFFFFFF marks "unreachable".
 *       f32: every addition is one IEEE single-precision add (round to
 *            nearest).  fl(a + w) is monotone in a and >= a for w >= 0, so
 *            Dijkstra's argument holds and the result is the minimum over
 *            paths of the left-to-right rounded sum.  +inf = unreachable.
 *       f64: the same in double precision (tolerance reference for f32).
 *   - Bellman-Ford (the high-parallelism end point in Section 2.1): rounds of
 *     relaxing every arc until nothing changes; a second, independent
 *     algorithm for tiny graphs.
 *   - The canonical predecessor for u32 distances: the smallest-index
 *     in-neighbour u with sat(dist[u] + w(u, v)) == dist[v]; pred[s] = s,
 *     -1 when unreachable.
 *   - An invariant checker for a claimed (dist, pred) pair.
 *
 * Compile with -ffp-contract=off -fexcess-precision=standard and without
 * fast-math so that each f32 addition is exactly one rounded operation.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define U32_INF 0xFFFFFFFFu
#define U32_SAT 0xFFFFFFFEu

/* ---------------------------------------------------- binary min-heap -- */
/* Keys are doubles: u32 and f32 distances are represented exactly. */

typedef struct { double key; int32_t v; } heap_item;
typedef struct { heap_item *a; int64_t size, cap; } heap;

static int heap_push(heap *h, double key, int32_t v) {
    if (h->size == h->cap) {
        int64_t nc = h->cap ? 2 * h->cap : 1024;
        heap_item *na = (heap_item *)realloc(h->a, sizeof(heap_item) * (size_t)nc);
        if (!na) return -1;
        h->a = na;
        h->cap = nc;
    }
    int64_t i = h->size++;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (h->a[p].key <= key) break;
        h->a[i] = h->a[p];
        i = p;
    }
    h->a[i].key = key;
    h->a[i].v = v;
    return 0;
}

static heap_item heap_pop(heap *h) {
    heap_item top = h->a[0];
    heap_item last = h->a[--h->size];
    int64_t i = 0;
    for (;;) {
        int64_t c = 2 * i + 1;
        if (c >= h->size) break;
        if (c + 1 < h->size && h->a[c + 1].key < h->a[c].key) c++;
        if (h->a[c].key >= last.key) break;
        h->a[i] = h->a[c];
        i = c;
    }
    if (h->size > 0) h->a[i] = last;
    return top;
}

static int check_args(int32_t n, const int32_t *row_ptr, int32_t src) {
    if (n < 1 || !row_ptr || src < 0 || src >= n) return -1;
    return 0;
}

/* ----------------------------------------------------------- Dijkstra -- */

static inline uint32_t add_u32_sat(uint32_t d, uint32_t w) {
    uint64_t s = (uint64_t)d + (uint64_t)w;
    return s > U32_SAT ? U32_SAT : (uint32_t)s;
}

/* dist[v] = shortest u32 path length from src (0xFFFFFFFF if unreachable).
 * Returns the number of settled (reachable) vertices, or -1 on error. */
int64_t oracle_dijkstra_u32(int32_t n, const int32_t *row_ptr, const int32_t *col,
                            const uint32_t *w, int32_t src, uint32_t *dist) {
    if (check_args(n, row_ptr, src)) return -1;
    for (int32_t v = 0; v < n; v++) dist[v] = U32_INF;
    heap h = {0};
    int64_t settled = 0;
    dist[src] = 0;
    if (heap_push(&h, 0.0, src)) return -1;
    while (h.size > 0) {
        heap_item it = heap_pop(&h);
        int32_t u = it.v;
        if (it.key > (double)dist[u]) continue; /* stale entry */
        if (it.key < (double)dist[u]) { free(h.a); return -1; } /* impossible */
        settled++;
        for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; e++) {
            int32_t v = col[e];
            uint32_t nd = add_u32_sat(dist[u], w[e]);
            if (nd < dist[v]) {
                dist[v] = nd;
                if (heap_push(&h, (double)nd, v)) { free(h.a); return -1; }
            }
        }
    }
    free(h.a);
    return settled;
}

/* f32 arithmetic: nd = fl32(dist[u] + w).  dist[v] = +inf if unreachable. */
int64_t oracle_dijkstra_f32(int32_t n, const int32_t *row_ptr, const int32_t *col,
                            const float *w, int32_t src, float *dist) {
    if (check_args(n, row_ptr, src)) return -1;
    for (int32_t v = 0; v < n; v++) dist[v] = INFINITY;
    heap h = {0};
    int64_t settled = 0;
    dist[src] = 0.0f;
    if (heap_push(&h, 0.0, src)) return -1;
    while (h.size > 0) {
        heap_item it = heap_pop(&h);
        int32_t u = it.v;
        if (it.key > (double)dist[u]) continue;
        settled++;
        for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; e++) {
            int32_t v = col[e];
            volatile float nd = dist[u] + w[e]; /* one rounded f32 add */
            if (nd < dist[v]) {
                dist[v] = nd;
                if (heap_push(&h, (double)nd, v)) { free(h.a); return -1; }
            }
        }
    }
    free(h.a);
    return settled;
}

/* f64 arithmetic over the same (f32) weights, widened exactly. */
int64_t oracle_dijkstra_f64(int32_t n, const int32_t *row_ptr, const int32_t *col,
                            const float *w, int32_t src, double *dist) {
    if (check_args(n, row_ptr, src)) return -1;
    for (int32_t v = 0; v < n; v++) dist[v] = INFINITY;
    heap h = {0};
    int64_t settled = 0;
    dist[src] = 0.0;
    if (heap_push(&h, 0.0, src)) return -1;
    while (h.size > 0) {
        heap_item it = heap_pop(&h);
        int32_t u = it.v;
        if (it.key > dist[u]) continue;
        settled++;
        for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; e++) {
            int32_t v = col[e];
            double nd = dist[u] + (double)w[e];
            if (nd < dist[v]) {
                dist[v] = nd;
                if (heap_push(&h, nd, v)) { free(h.a); return -1; }
            }
        }
    }
    free(h.a);
    return settled;
}

/* ------------------------------------------------------- Bellman-Ford -- */
/* Textbook: repeat full passes relaxing every arc until a pass changes
 * nothing (at most n passes for non-negative weights).  Returns passes. */

int32_t oracle_bellman_ford_u32(int32_t n, const int32_t *row_ptr, const int32_t *col,
                                const uint32_t *w, int32_t src, uint32_t *dist) {
    if (check_args(n, row_ptr, src)) return -1;
    for (int32_t v = 0; v < n; v++) dist[v] = U32_INF;
    dist[src] = 0;
    for (int32_t pass = 1; pass <= n + 1; pass++) {
        int changed = 0;
        for (int32_t u = 0; u < n; u++) {
            if (dist[u] == U32_INF) continue;
            for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; e++) {
                uint32_t nd = add_u32_sat(dist[u], w[e]);
                if (nd < dist[col[e]]) { dist[col[e]] = nd; changed = 1; }
            }
        }
        if (!changed) return pass;
    }
    return -1;
}

int32_t oracle_bellman_ford_f32(int32_t n, const int32_t *row_ptr, const int32_t *col,
                                const float *w, int32_t src, float *dist) {
    if (check_args(n, row_ptr, src)) return -1;
    for (int32_t v = 0; v < n; v++) dist[v] = INFINITY;
    dist[src] = 0.0f;
    for (int32_t pass = 1; pass <= n + 1; pass++) {
        int changed = 0;
        for (int32_t u = 0; u < n; u++) {
            if (isinf(dist[u])) continue;
            for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; e++) {
                volatile float nd = dist[u] + w[e];
                if (nd < dist[col[e]]) { dist[col[e]] = nd; changed = 1; }
            }
        }
        if (!changed) return pass;
    }
    return -1;
}

/* -------------------------------------------------------- predecessor -- */

/* Canonical u32 predecessor: smallest-index tight in-neighbour.  Scans every
 * arc (u -> v) once, so it needs no transpose.  pred[src] = src. */
int oracle_pred_canonical_u32(int32_t n, const int32_t *row_ptr, const int32_t *col,
                              const uint32_t *w, int32_t src, const uint32_t *dist,
                              int32_t *pred) {
    if (check_args(n, row_ptr, src)) return -1;
    for (int32_t v = 0; v < n; v++) pred[v] = -1;
    for (int32_t u = 0; u < n; u++) {
        if (dist[u] == U32_INF) continue;
        for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; e++) {
            int32_t v = col[e];
            if (v == src) continue;
            if (add_u32_sat(dist[u], w[e]) == dist[v] && (pred[v] < 0 || u < pred[v])) pred[v] = u;
        }
    }
    pred[src] = src;
    return 0;
}

/* ---------------------------------------------------------- invariants -- */

enum {
    CHK_OK = 0,
    CHK_SRC = 1,          /* dist[src] != 0 or pred[src] != src */
    CHK_EDGE = 2,         /* dist[v] > dist[u] (+) w on some arc */
    CHK_NO_TIGHT = 3,     /* reachable v != src without a tight in-arc */
    CHK_PRED_RANGE = 4,   /* pred out of range / inconsistent with reachability */
    CHK_PRED_EDGE = 5,    /* no tight arc pred[v] -> v */
    CHK_PRED_CYCLE = 6,   /* pred chain does not reach src */
    CHK_BAD = 7,          /* bad arguments / allocation */
};

/* Checks a claimed result.  `kind`: 0 = u32 (dist as uint32), 1 = f32
 * (dist as float, weights as float).  pred may be NULL.  Returns one of the
 * CHK_* codes; *bad_vertex receives the first failing vertex (or -1).
 *
 * dist[src] = 0, dist[v] <= dist[u] (+) w(u,v) on every arc, and a tight
 * in-arc into every reachable v != src (from a reachable vertex) together
 * with pred chains that reach src characterise the shortest-path lengths. */
int oracle_check(int kind, int32_t n, const int32_t *row_ptr, const int32_t *col,
                 const void *wv, int32_t src, const void *distv, const int32_t *pred,
                 int32_t *bad_vertex) {
    const uint32_t *wu = (const uint32_t *)wv, *du = (const uint32_t *)distv;
    const float *wf = (const float *)wv, *df = (const float *)distv;
    int32_t dummy;
    if (!bad_vertex) bad_vertex = &dummy;
    *bad_vertex = -1;
    if (check_args(n, row_ptr, src)) return CHK_BAD;
#define REACH(x) (kind == 0 ? du[x] != U32_INF : !isinf(df[x]))
    if (kind == 0 ? du[src] != 0 : df[src] != 0.0f) { *bad_vertex = src; return CHK_SRC; }
    if (kind == 1) {
        for (int32_t v = 0; v < n; v++)
            if (isnan(df[v]) || df[v] < 0.0f || (isinf(df[v]) && df[v] < 0)) { *bad_vertex = v; return CHK_EDGE; }
    }
    uint8_t *tight = (uint8_t *)calloc((size_t)n, 1);
    uint8_t *pred_ok = (uint8_t *)calloc((size_t)n, 1);
    if (!tight || !pred_ok) { free(tight); free(pred_ok); return CHK_BAD; }
    int rc = CHK_OK;
    for (int32_t u = 0; u < n && rc == CHK_OK; u++) {
        if (!REACH(u)) continue;
        for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; e++) {
            int32_t v = col[e];
            int is_tight, violates;
            if (kind == 0) {
                uint32_t nd = add_u32_sat(du[u], wu[e]);
                violates = du[v] > nd;
                is_tight = du[v] == nd;
            } else {
                volatile float nd = df[u] + wf[e];
                violates = df[v] > nd;
                is_tight = df[v] == nd;
            }
            if (violates) { *bad_vertex = v; rc = CHK_EDGE; break; }
            if (is_tight && v != src) {
                tight[v] = 1;
                if (pred && pred[v] == u) pred_ok[v] = 1;
            }
        }
    }
    for (int32_t v = 0; v < n && rc == CHK_OK; v++) {
        if (v == src || !REACH(v)) continue;
        if (!tight[v]) { *bad_vertex = v; rc = CHK_NO_TIGHT; }
    }
    if (rc == CHK_OK && pred) {
        if (pred[src] != src) { *bad_vertex = src; rc = CHK_SRC; }
        for (int32_t v = 0; v < n && rc == CHK_OK; v++) {
            if (v == src) continue;
            if (!REACH(v)) {
                if (pred[v] != -1) { *bad_vertex = v; rc = CHK_PRED_RANGE; }
            } else if (pred[v] < 0 || pred[v] >= n) {
                *bad_vertex = v; rc = CHK_PRED_RANGE;
            } else if (!pred_ok[v]) {
                *bad_vertex = v; rc = CHK_PRED_EDGE;
            }
        }
        /* every chain reaches src: colour vertices 0 = unknown, 1 = on the
         * current walk, 2 = known to reach src. */
        if (rc == CHK_OK) {
            uint8_t *state = tight; /* reuse the buffer */
            memset(state, 0, (size_t)n);
            state[src] = 2;
            for (int32_t v = 0; v < n && rc == CHK_OK; v++) {
                if (!REACH(v) || state[v] == 2) continue;
                int32_t x = v;
                while (state[x] == 0) { state[x] = 1; x = pred[x]; }
                if (state[x] == 1) { *bad_vertex = v; rc = CHK_PRED_CYCLE; break; }
                x = v;
                while (state[x] == 1) { state[x] = 2; x = pred[x]; }
            }
        }
    }
#undef REACH
    free(tight);
    free(pred_ok);
    return rc;
}

/* Number of arcs whose source is reachable (m_r, the traversed-edge count
 * used for GTEPS) and number of reachable vertices (n_r). */
int oracle_reached_counts(int kind, int32_t n, const int32_t *row_ptr, const void *distv,
                          int64_t *m_r, int64_t *n_r) {
    const uint32_t *du = (const uint32_t *)distv;
    const float *df = (const float *)distv;
    int64_t me = 0, nv = 0;
    for (int32_t v = 0; v < n; v++) {
        int reach = kind == 0 ? du[v] != U32_INF : !isinf(df[v]);
        if (reach) { nv++; me += row_ptr[v + 1] - row_ptr[v]; }
    }
    *m_r = me;
    *n_r = nv;
    return 0;
}
