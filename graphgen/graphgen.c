/*
 * Seeded synthetic graph generators shared by the CUDA path and the oracle.
 *
 * This module builds inputs only: CSR adjacency (int32 row_ptr / col) plus
 * per-edge weights.  It contains no shortest-path arithmetic.  Every random
 * draw is a pure function of (seed, stream, counter) through SplitMix64
 * (Steele, Lea & Flood, "Fast splittable pseudorandom number generators",
 * OOPSLA 2014), so results are identical for any thread count and on any
 * host architecture.
 *
 * Workload shapes (the paper's Table 4 graph families, synthesised):
 *   grid   W x H 4-neighbour mesh, both directions stored
 *   road   grid with each undirected edge dropped with probability p and a
 *          fraction of extra long-range edges (weight = mult * Manhattan
 *          length), a high-diameter road-network stand-in
 *   rmat   R-MAT power-law graph (a, b, c, d), symmetrised, self-loops and
 *          duplicate edges removed, vertex ids permuted by a seeded shuffle
 *   er     Erdos-Renyi G(n, m): exactly m distinct undirected pairs
 *
 * Weights are drawn once per undirected edge and shared by both directions.
 * Integer weights are uniform in [lo, hi]; "f32" weights are (k+1) / 2^24
 * with k uniform in [0, 2^24): exactly representable, denormal-free, in (0,1].
 *
 * Build: gcc -O2 -fPIC -shared [-fopenmp] graphgen.c -o libgraphgen.so
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- RNG -- */

static inline uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* i-th output (i >= 0) of the SplitMix64 sequence whose state starts at key. */
static inline uint64_t sm64_at(uint64_t key, uint64_t i) {
    return sm64_mix(key + (i + 1) * 0x9e3779b97f4a7c15ULL);
}

/* Independent stream key for one purpose (edges, weights, drops, ...). */
static inline uint64_t stream_key(uint64_t seed, uint64_t stream) {
    return sm64_at(sm64_mix(seed), stream);
}

enum { ST_EDGES = 1, ST_WEIGHTS = 2, ST_PERM = 3, ST_DROP = 4, ST_LONG = 5, ST_SOURCES = 6, ST_ER = 7 };

/* Uniform integer in [lo, hi] from the top 32 bits (multiply-shift). */
static inline uint32_t uniform_u32(uint64_t r, uint32_t lo, uint32_t hi) {
    uint64_t range = (uint64_t)hi - (uint64_t)lo + 1ULL;
    return lo + (uint32_t)(((r >> 32) * range) >> 32);
}

/* Uniform double in [0, 1) with 53 random bits. */
static inline double uniform_f64(uint64_t r) {
    return (double)(r >> 11) * (1.0 / 9007199254740992.0);
}

/* f32 weight (k+1)/2^24, k uniform in [0, 2^24); returned as IEEE bits. */
static inline uint32_t f32_weight_bits(uint64_t r) {
    uint32_t k = (uint32_t)(r >> 40); /* 24 bits */
    float f = (float)(k + 1u) * (1.0f / 16777216.0f);
    uint32_t b;
    memcpy(&b, &f, 4);
    return b;
}

static inline uint32_t draw_weight(uint64_t key, uint64_t idx, uint32_t lo, uint32_t hi, int wf32) {
    uint64_t r = sm64_at(key, idx);
    return wf32 ? f32_weight_bits(r) : uniform_u32(r, lo, hi);
}

/* -------------------------------------------------------------- graph -- */

typedef struct gg_graph {
    int32_t n;
    int64_t m;
    int32_t *row_ptr; /* n + 1 */
    int32_t *col;     /* m */
    uint32_t *w;      /* m, u32 value or f32 bits */
} gg_graph;

void gg_free(gg_graph *g) {
    if (!g) return;
    free(g->row_ptr);
    free(g->col);
    free(g->w);
    free(g);
}

int32_t gg_n(const gg_graph *g) { return g ? g->n : -1; }
int64_t gg_m(const gg_graph *g) { return g ? g->m : -1; }

int gg_copy_out(const gg_graph *g, int32_t *row_ptr, int32_t *col, uint32_t *w) {
    if (!g) return -1;
    memcpy(row_ptr, g->row_ptr, sizeof(int32_t) * ((size_t)g->n + 1));
    if (g->m) {
        memcpy(col, g->col, sizeof(int32_t) * (size_t)g->m);
        memcpy(w, g->w, sizeof(uint32_t) * (size_t)g->m);
    }
    return 0;
}

/* LSD radix sort of 64-bit keys (16-bit digits) with an optional u32 payload.
 * Only the low `bits` bits of each key are significant. */
static int radix_sort_u64(uint64_t *key, uint32_t *pay, size_t n, int bits) {
    if (n < 2) return 0;
    uint64_t *k2 = (uint64_t *)malloc(sizeof(uint64_t) * n);
    uint32_t *p2 = pay ? (uint32_t *)malloc(sizeof(uint32_t) * n) : NULL;
    size_t *cnt = (size_t *)malloc(sizeof(size_t) * 65536);
    if (!k2 || (pay && !p2) || !cnt) {
        free(k2); free(p2); free(cnt);
        return -1;
    }
    for (int shift = 0; shift < bits; shift += 16) {
        memset(cnt, 0, sizeof(size_t) * 65536);
        for (size_t i = 0; i < n; i++) cnt[(key[i] >> shift) & 0xffff]++;
        size_t s = 0;
        for (int d = 0; d < 65536; d++) { size_t c = cnt[d]; cnt[d] = s; s += c; }
        for (size_t i = 0; i < n; i++) {
            size_t o = cnt[(key[i] >> shift) & 0xffff]++;
            k2[o] = key[i];
            if (pay) p2[o] = pay[i];
        }
        uint64_t *tk = key; key = k2; k2 = tk;
        if (pay) { uint32_t *tp = pay; pay = p2; p2 = tp; }
        /* after an odd number of passes the sorted data lives in the
         * scratch buffers; fix up at the end */
    }
    int passes = (bits + 15) / 16;
    if (passes & 1) {
        /* key currently points at the scratch allocation, k2 at the caller's */
        memcpy(k2, key, sizeof(uint64_t) * n);
        if (pay) memcpy(p2, pay, sizeof(uint32_t) * n);
        free(key);
        if (pay) free(pay);
    } else {
        free(k2);
        if (p2) free(p2);
    }
    free(cnt);
    return 0;
}

static int bits_for(uint64_t v) { int b = 1; while (b < 64 && (v >> b)) b++; return b; }

/* Undirected edge list (canonical key = min<<32 | max, no self-loops) ->
 * symmetric CSR.  Keys are sorted; duplicates keep the minimum weight when
 * `weights` is given, otherwise weights are drawn per unique edge ordinal
 * from (wkey, lo, hi, wf32).  Consumes (frees) keys and weights. */
static gg_graph *undirected_to_csr(int32_t n, uint64_t *keys, uint32_t *weights, size_t ne,
                                   uint64_t wkey, uint32_t lo, uint32_t hi, int wf32) {
    int kbits = 32 + bits_for((uint64_t)(n > 0 ? n - 1 : 0));
    if (radix_sort_u64(keys, weights, ne, kbits) != 0) { free(keys); free(weights); return NULL; }
    /* dedup */
    size_t u = 0;
    for (size_t i = 0; i < ne; i++) {
        if (u > 0 && keys[u - 1] == keys[i]) {
            if (weights && weights[i] < weights[u - 1]) weights[u - 1] = weights[i];
            continue;
        }
        keys[u] = keys[i];
        if (weights) weights[u] = weights[i];
        u++;
    }
    ne = u;
    if (!weights) {
        weights = (uint32_t *)malloc(sizeof(uint32_t) * (ne ? ne : 1));
        if (!weights) { free(keys); return NULL; }
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < (int64_t)ne; i++) weights[i] = draw_weight(wkey, (uint64_t)i, lo, hi, wf32);
    }
    gg_graph *g = (gg_graph *)calloc(1, sizeof(gg_graph));
    if (!g) { free(keys); free(weights); return NULL; }
    g->n = n;
    g->m = (int64_t)(2 * ne);
    g->row_ptr = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    g->col = (int32_t *)malloc(sizeof(int32_t) * (g->m ? g->m : 1));
    g->w = (uint32_t *)malloc(sizeof(uint32_t) * (g->m ? g->m : 1));
    int64_t *fill = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!g->row_ptr || !g->col || !g->w || !fill) {
        free(fill); free(keys); free(weights); gg_free(g); return NULL;
    }
    if (g->m > 2147483647LL) { free(fill); free(keys); free(weights); gg_free(g); return NULL; }
    for (size_t i = 0; i < ne; i++) {
        uint32_t a = (uint32_t)(keys[i] >> 32), b = (uint32_t)keys[i];
        fill[a + 1]++;
        fill[b + 1]++;
    }
    for (int32_t v = 0; v < n; v++) fill[v + 1] += fill[v];
    for (int32_t v = 0; v <= n; v++) g->row_ptr[v] = (int32_t)fill[v];
    /* Pass A: row b receives a (a < b), ascending in a.
     * Pass B: row a receives b (b > a), ascending in b.
     * Each row ends up sorted: smaller neighbours first, then larger. */
    for (size_t i = 0; i < ne; i++) {
        uint32_t a = (uint32_t)(keys[i] >> 32), b = (uint32_t)keys[i];
        int64_t o = fill[b]++;
        g->col[o] = (int32_t)a;
        g->w[o] = weights[i];
    }
    for (size_t i = 0; i < ne; i++) {
        uint32_t a = (uint32_t)(keys[i] >> 32), b = (uint32_t)keys[i];
        int64_t o = fill[a]++;
        g->col[o] = (int32_t)b;
        g->w[o] = weights[i];
    }
    free(fill);
    free(keys);
    free(weights);
    return g;
}

static inline uint64_t ukey(uint32_t a, uint32_t b) {
    return a < b ? ((uint64_t)a << 32) | b : ((uint64_t)b << 32) | a;
}

/* ---------------------------------------------------------------- grid -- */

/* Undirected grid edge ordinals: horizontal (x,y)-(x+1,y) -> y*(W-1)+x,
 * vertical (x,y)-(x,y+1) -> H*(W-1) + y*W + x.  Vertex id = y*W + x. */
gg_graph *gg_grid(int32_t W, int32_t H, uint32_t lo, uint32_t hi, uint64_t seed, int wf32) {
    if (W < 1 || H < 1 || (int64_t)W * H > 2147483647LL) return NULL;
    int64_t nh = (int64_t)(W - 1) * H, nv = (int64_t)W * (H - 1);
    size_t ne = (size_t)(nh + nv);
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (ne ? ne : 1));
    uint32_t *wt = (uint32_t *)malloc(sizeof(uint32_t) * (ne ? ne : 1));
    if (!keys || !wt) { free(keys); free(wt); return NULL; }
    uint64_t wk = stream_key(seed, ST_WEIGHTS);
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < nh + nv; e++) {
        uint32_t a, b;
        if (e < nh) {
            int64_t y = e / (W - 1), x = e % (W - 1);
            a = (uint32_t)(y * W + x); b = a + 1;
        } else {
            int64_t f = e - nh, y = f / W, x = f % W;
            a = (uint32_t)(y * W + x); b = a + (uint32_t)W;
        }
        keys[e] = ukey(a, b);
        wt[e] = draw_weight(wk, (uint64_t)e, lo, hi, wf32);
    }
    return undirected_to_csr(W * H, keys, wt, ne, 0, 0, 0, 0);
}

/* ---------------------------------------------------------------- road -- */

/* Grid with each undirected edge kept with probability 1 - pdrop, plus
 * L = floor(plong * kept) long-range edges: endpoint u uniform, offset
 * (dx, dy) uniform in [-maxlen, maxlen]^2 conditioned on 2 <= |dx|+|dy| <=
 * maxlen and staying inside the grid (rejection, at most 64 tries each);
 * weight = longmul * (|dx|+|dy|). */
gg_graph *gg_road(int32_t W, int32_t H, double pdrop, double plong, int32_t maxlen,
                  uint32_t lo, uint32_t hi, uint32_t longmul, uint64_t seed) {
    if (W < 1 || H < 1 || (int64_t)W * H > 2147483647LL || maxlen < 2) return NULL;
    int64_t nh = (int64_t)(W - 1) * H, nv = (int64_t)W * (H - 1), ng = nh + nv;
    uint64_t dk = stream_key(seed, ST_DROP), wk = stream_key(seed, ST_WEIGHTS), lk = stream_key(seed, ST_LONG);
    uint8_t *keep = (uint8_t *)malloc((size_t)(ng ? ng : 1));
    if (!keep) return NULL;
    int64_t kept = 0;
#pragma omp parallel for schedule(static) reduction(+ : kept)
    for (int64_t e = 0; e < ng; e++) {
        keep[e] = uniform_f64(sm64_at(dk, (uint64_t)e)) >= pdrop;
        kept += keep[e];
    }
    int64_t nl = (int64_t)(plong * (double)kept);
    size_t ne = (size_t)(kept + nl);
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (ne ? ne : 1));
    uint32_t *wt = (uint32_t *)malloc(sizeof(uint32_t) * (ne ? ne : 1));
    if (!keys || !wt) { free(keep); free(keys); free(wt); return NULL; }
    size_t o = 0;
    for (int64_t e = 0; e < ng; e++) {
        if (!keep[e]) continue;
        uint32_t a, b;
        if (e < nh) {
            int64_t y = e / (W - 1), x = e % (W - 1);
            a = (uint32_t)(y * W + x); b = a + 1;
        } else {
            int64_t f = e - nh, y = f / W, x = f % W;
            a = (uint32_t)(y * W + x); b = a + (uint32_t)W;
        }
        keys[o] = ukey(a, b);
        wt[o] = draw_weight(wk, (uint64_t)e, lo, hi, 0);
        o++;
    }
    free(keep);
    int64_t span = 2 * (int64_t)maxlen + 1;
    for (int64_t j = 0; j < nl; j++) {
        for (int t = 0; t < 64; t++) {
            uint64_t r0 = sm64_at(lk, (uint64_t)j * 128 + 2 * t);
            uint64_t r1 = sm64_at(lk, (uint64_t)j * 128 + 2 * t + 1);
            int64_t u = (int64_t)((r0 >> 32) * (uint64_t)((int64_t)W * H) >> 32);
            int64_t dx = (int64_t)(((r1 >> 32) * (uint64_t)span) >> 32) - maxlen;
            int64_t dy = (int64_t)(((r1 & 0xffffffffULL) * (uint64_t)span) >> 32) - maxlen;
            int64_t len = (dx < 0 ? -dx : dx) + (dy < 0 ? -dy : dy);
            if (len < 2 || len > maxlen) continue;
            int64_t ux = u % W, uy = u / W, vx = ux + dx, vy = uy + dy;
            if (vx < 0 || vx >= W || vy < 0 || vy >= H) continue;
            keys[o] = ukey((uint32_t)u, (uint32_t)(vy * W + vx));
            wt[o] = (uint32_t)(longmul * (uint32_t)len);
            o++;
            break;
        }
    }
    return undirected_to_csr(W * H, keys, wt, o, 0, 0, 0, 0);
}

/* ---------------------------------------------------------------- rmat -- */

/* R-MAT (Chakrabarti, Zhan & Faloutsos, SDM 2004) without noise: each of
 * ef * 2^scale edges descends `scale` levels, choosing quadrant
 * (0,0),(0,1),(1,0),(1,1) with probabilities a, b, c, 1-a-b-c from one
 * 32-bit uniform per level.  Vertex ids are then relabelled by a seeded
 * Fisher-Yates permutation; the result is symmetrised with self-loops and
 * duplicates removed. */
gg_graph *gg_rmat(int32_t scale, int32_t ef, double a, double b, double c,
                  uint32_t lo, uint32_t hi, uint64_t seed, int wf32) {
    if (scale < 1 || scale > 30 || ef < 1) return NULL;
    int32_t n = (int32_t)1 << scale;
    int64_t ne0 = (int64_t)ef << scale;
    uint64_t ek = stream_key(seed, ST_EDGES), pk = stream_key(seed, ST_PERM), wk = stream_key(seed, ST_WEIGHTS);
    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)ne0);
    if (!perm || !keys) { free(perm); free(keys); return NULL; }
    for (int32_t i = 0; i < n; i++) perm[i] = i;
    for (int32_t i = n - 1; i > 0; i--) {
        uint64_t r = sm64_at(pk, (uint64_t)i);
        int32_t j = (int32_t)(((r >> 32) * (uint64_t)(i + 1)) >> 32);
        int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
    const double ab = a + b, abc = a + b + c;
    const int per = (scale + 1) / 2; /* 64-bit draws per edge, two levels each */
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < ne0; e++) {
        uint32_t s = 0, d = 0;
        for (int l = 0; l < scale; l++) {
            uint64_t r = sm64_at(ek, (uint64_t)e * (uint64_t)per + (uint64_t)(l >> 1));
            uint32_t bits = (l & 1) ? (uint32_t)r : (uint32_t)(r >> 32);
            double p = (double)bits * (1.0 / 4294967296.0);
            uint32_t bit = 1u << (scale - 1 - l);
            if (p < a) {
            } else if (p < ab) {
                d |= bit;
            } else if (p < abc) {
                s |= bit;
            } else {
                s |= bit; d |= bit;
            }
        }
        uint32_t ps = (uint32_t)perm[s], pd = (uint32_t)perm[d];
        keys[e] = (ps == pd) ? UINT64_MAX : ukey(ps, pd);
    }
    free(perm);
    /* drop self-loops (marked UINT64_MAX) */
    size_t o = 0;
    for (int64_t e = 0; e < ne0; e++) if (keys[e] != UINT64_MAX) keys[o++] = keys[e];
    return undirected_to_csr(n, keys, NULL, o, wk, lo, hi, wf32);
}

/* ------------------------------------------------------------------ er -- */

/* Erdos-Renyi G(n, m): uniform pairs u != v are drawn until exactly m
 * distinct undirected pairs exist (extra rounds draw only the shortfall). */
gg_graph *gg_er(int32_t n, int64_t m, uint32_t lo, uint32_t hi, uint64_t seed, int wf32) {
    if (n < 2 || m < 0 || (double)m > (double)n * (double)(n - 1) / 2.0) return NULL;
    uint64_t rk = stream_key(seed, ST_ER), wk = stream_key(seed, ST_WEIGHTS);
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(m ? m : 1));
    if (!keys) return NULL;
    size_t have = 0;
    uint64_t ctr = 0;
    int kbits = 32 + bits_for((uint64_t)(n - 1));
    for (int round = 0; round < 64 && have < (size_t)m; round++) {
        size_t need = (size_t)m - have;
        size_t start = have;
        for (size_t i = 0; i < need; i++) {
            uint64_t u, v;
            do {
                uint64_t r = sm64_at(rk, ctr++);
                u = ((r >> 32) * (uint64_t)n) >> 32;
                v = ((r & 0xffffffffULL) * (uint64_t)n) >> 32;
            } while (u == v);
            keys[start + i] = ukey((uint32_t)u, (uint32_t)v);
        }
        have = (size_t)m;
        if (radix_sort_u64(keys, NULL, have, kbits) != 0) { free(keys); return NULL; }
        size_t u = 0;
        for (size_t i = 0; i < have; i++) if (u == 0 || keys[u - 1] != keys[i]) keys[u++] = keys[i];
        have = u;
    }
    return undirected_to_csr(n, keys, NULL, have, wk, lo, hi, wf32);
}

/* ------------------------------------------------------- random directed -- */

/* Small random DIRECTED multigraph for tests: m arcs (u, v) uniform, self
 * loops and parallel arcs allowed; weights per arc. */
gg_graph *gg_random_directed(int32_t n, int64_t m, uint32_t lo, uint32_t hi, uint64_t seed, int wf32) {
    if (n < 1 || m < 0 || m > 2147483647LL) return NULL;
    uint64_t rk = stream_key(seed, ST_EDGES), wk = stream_key(seed, ST_WEIGHTS);
    gg_graph *g = (gg_graph *)calloc(1, sizeof(gg_graph));
    if (!g) return NULL;
    g->n = n; g->m = m;
    g->row_ptr = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    g->col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m ? m : 1));
    g->w = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(m ? m : 1));
    uint32_t *su = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(m ? m : 1));
    uint32_t *sv = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(m ? m : 1));
    if (!g->row_ptr || !g->col || !g->w || !su || !sv) { free(su); free(sv); gg_free(g); return NULL; }
    for (int64_t e = 0; e < m; e++) {
        uint64_t r = sm64_at(rk, (uint64_t)e);
        su[e] = (uint32_t)(((r >> 32) * (uint64_t)n) >> 32);
        sv[e] = (uint32_t)(((r & 0xffffffffULL) * (uint64_t)n) >> 32);
        g->row_ptr[su[e] + 1]++;
    }
    for (int32_t v = 0; v < n; v++) g->row_ptr[v + 1] += g->row_ptr[v];
    int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    if (!fill) { free(su); free(sv); gg_free(g); return NULL; }
    memcpy(fill, g->row_ptr, sizeof(int32_t) * (size_t)(n + 1));
    for (int64_t e = 0; e < m; e++) {
        int32_t o = fill[su[e]]++;
        g->col[o] = (int32_t)sv[e];
        g->w[o] = draw_weight(wk, (uint64_t)e, lo, hi, wf32);
    }
    free(fill); free(su); free(sv);
    return g;
}

/* ------------------------------------------------------------- sources -- */

static int32_t uf_find(int32_t *p, int32_t x) {
    while (p[x] != x) { p[x] = p[p[x]]; x = p[x]; }
    return x;
}

/* Size of the largest weakly connected component (ties: the one holding
 * the smallest vertex id), written to *giant_size; `k` distinct sources
 * drawn uniformly (seeded) from it are written to out.  Returns the number
 * of sources written (min(k, giant size)), or -1 on error. */
int32_t gg_giant_sources(const int32_t *row_ptr, const int32_t *col, int32_t n, int32_t k,
                         uint64_t seed, int32_t *out, int32_t *giant_size) {
    if (n < 1 || k < 0) return -1;
    int32_t *p = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *sz = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    uint8_t *used = (uint8_t *)calloc((size_t)n, 1);
    if (!p || !sz || !used) { free(p); free(sz); free(used); return -1; }
    for (int32_t v = 0; v < n; v++) p[v] = v;
    for (int32_t u = 0; u < n; u++)
        for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; e++) {
            int32_t a = uf_find(p, u), b = uf_find(p, col[e]);
            if (a != b) { if (a < b) p[b] = a; else p[a] = b; }
        }
    int32_t best = 0, bestsz = 0;
    for (int32_t v = 0; v < n; v++) sz[uf_find(p, v)]++;
    for (int32_t v = 0; v < n; v++) if (sz[v] > bestsz) { bestsz = sz[v]; best = v; }
    if (giant_size) *giant_size = bestsz;
    int32_t want = k < bestsz ? k : bestsz, got = 0;
    uint64_t sk = stream_key(seed, ST_SOURCES);
    for (uint64_t i = 0; got < want; i++) {
        uint64_t r = sm64_at(sk, i);
        int32_t v = (int32_t)(((r >> 32) * (uint64_t)n) >> 32);
        if (uf_find(p, v) == best && !used[v]) { used[v] = 1; out[got++] = v; }
    }
    free(p); free(sz); free(used);
    return got;
}

/* Seeded uniform stream helpers exposed for other input recipes (e.g.
 * Poisson arrival times), so all synthetic inputs share one generator. */
uint64_t gg_sm64_at(uint64_t seed, uint64_t stream, uint64_t i) {
    return sm64_at(stream_key(seed, stream), i);
}

int gg_uniform_f64(uint64_t seed, uint64_t stream, uint64_t start, int64_t count, double *out) {
    uint64_t k = stream_key(seed, stream);
    for (int64_t i = 0; i < count; i++) out[i] = uniform_f64(sm64_at(k, start + (uint64_t)i));
    return 0;
}
