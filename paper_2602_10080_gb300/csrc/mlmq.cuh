// mlmq.cuh -- device side of the multi-level multi-queue (MLMQ) SSSP engine
// for sm_103a.
//
// One persistent kernel runs the label-correcting loop of Listing 2: every
// warp repeatedly Reads a batch of vertices from the worklist, relaxes their
// arcs, and Writes improved vertices back (Listing 1), until the worklist is
// empty everywhere.  The worklist has the three levels of Section 3.1:
//
//   L0  per warp, in registers: a ring of R rows x 32 lanes (position p lives
//       in lane p % 32, row (p / 32) % R), FIFO (Section 3.4, "L0 queue").
//   L1  per thread block, in shared memory: Vector / Near-far / Filter / SLF
//       policies (Section 3.4, Fig. 7).  Vector and Filter are a lock-free
//       ring (CAS reservations on head and tail, an empty key per slot);
//       Near-far and SLF take a warp-granular lock.
//   L2  whole grid, in global memory: bmax circular delta-buckets
//       (Section 4.2, "L2 Bucket queue"); every bucket is S rings (shards)
//       of 32-element chunks moved with one ticket per claim (Section 4.2,
//       "L2 FIFO queue", Listing 3).
//
// Spill and refill follow the cache-like collaboration of Section 3.2: the
// worker touches L0; an empty level refills from the next one down, a full
// level writes back to it.  On this GPU the refill of L1 from L2 is done by
// at most `refillers` warps of a block at a time (the others keep working),
// which bounds the agents contending for the L2 tickets, and a claim takes
// several chunks at once.  Vertices improved through a heavy arc (weight
// above near_deltas * delta), or to a distance beyond the window front
// (W + F) * delta, skip the local levels and go to their L2 bucket; only
// light-arc improvements inside the front are processed locally at once --
// the light/heavy arc split of delta-stepping, which keeps local processing
// from running ahead of the bucket order (the redundant-wavefront concern of
// Section 2.3).
//
// High-degree vertices are split when the graph is created into zero-weight
// "shadow" vertices that own slices of the arcs, so their arcs are spread
// over warps and blocks through the same queues (load balancing of
// Section 4.1 widened beyond one warp).
//
// Termination (Section 4.1, delayed counting): every element written to L2
// first adds to ctrl.reserve; elements read from L2 are counted in the
// block's `acct` word, whose high half counts elements the block holds (L0 +
// L1 + staging + in flight) and whose low half counts L2 reads not yet
// published.  When the high half reaches zero the low half is added to
// ctrl.done.  An idle warp reads done THEN reserve; equality proves that no
// element is live anywhere.
//
// Every wait is bounded by a globaltimer deadline; on expiry the kernel
// records an error word and every warp returns.
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

namespace sssp {

constexpr int kWarp = 32;
constexpr uint32_t kFull = 0xffffffffu;
constexpr int kChunk = 32;          // elements per L2 chunk
#ifndef SSSP_FAR_CAP
#define SSSP_FAR_CAP 64
#endif
#ifndef SSSP_STAGE_CAP
#define SSSP_STAGE_CAP 64
#endif
constexpr int kFarCap = SSSP_FAR_CAP;  // per-warp far staging (elements)
constexpr int kMaxClaim = 32;       // chunks per L2 claim (upper bound, a power of two <= 32)
// claimed-chunk descriptors per block (a power of two): 256 against 64 took
// R-MAT-22 from 3.06 to 3.00 ms and 256 R-MAT-20 sources from 141 to 138 ms
#ifndef SSSP_DESC_CAP
#define SSSP_DESC_CAP 256
#endif
constexpr int kDescCap = SSSP_DESC_CAP;
constexpr int kStageCap = SSSP_STAGE_CAP;  // block staging per L2 bucket (elements, a power of two >= 64)
#ifndef SSSP_WINDOW_GUARD
#define SSSP_WINDOW_GUARD 8
#endif
#ifndef SSSP_FRONT_BOUND
#define SSSP_FRONT_BOUND 1
#endif
constexpr uint32_t kWindowGuard = SSSP_WINDOW_GUARD;  // buckets kept clear at the far end of the L2 window
constexpr uint32_t kInfU32 = 0xffffffffu;
constexpr uint32_t kEmptyKey = 0xffffffffu;  // a free L1 slot (never a valid element key)
constexpr uint32_t kSatU32 = 0xfffffffeu;
constexpr uint32_t kInfF32 = 0x7f800000u;

// error words (ctrl.error)
enum : int {
    kErrNone = 0,
    kErrTimeout = 1,      // a bounded wait or the solve watchdog expired
    kErrOverflow = 2,     // every L2 bucket ring was full
    kErrState = 3,        // queue metadata inconsistent at seeding
    kErrElement = 4,      // a popped element names a vertex or query out of range
};

// statistics slots (ctrl.stats)
enum : int {
    kStPopL0 = 0, kStPopL1, kStPopL2, kStRefill, kStRelax, kStImproved, kStStale,
    kStChunks, kStFlush, kStFar, kStCasFail, kStDeferred, kStRelaxShadow,
    // SM clock cycles spent per phase (lane 0 of every warp, summed)
    kCyRelax, kCyL1, kCyL2Write, kCyGlobalRead, kCyIdle, kCyL0,
    kStLockSpin, kStWaitSpin, kStIdleIter, kStRefillTry, kStIter, kStRounds,
    kStPullBack, kStLowWrite, kStAdvance,
    kStDup,           // improved arcs of a round whose target another improved arc of the round shares
    kCyRound,         // SSSP_FINE_CYCLES: loads and relaxation of the rounds
    kCyPush,          // SSSP_FINE_CYCLES: push_round (routing to L0 / far staging, their flushes)
    kCyBatch,         // SSSP_FINE_CYCLES: batch set-up (stale filter, row offsets, prefix sum)
    kStMarked,        // improvements not queued: the vertex was pending at an earlier-or-equal bucket
    kCyFarFlush,      // SSSP_FINE_CYCLES: far_flush (staging, its L2 writes and lock waits)
    kCyLock,          // SSSP_FINE_CYCLES: waiting for block locks
    kCyClaim,         // SSSP_FINE_CYCLES: l2_claim (window, probes, read-ticket CAS)
    kCyChunks,        // SSSP_FINE_CYCLES: waiting for and reading claimed chunks (incl. L1 writes)
    kCyStage,         // SSSP_FINE_CYCLES: stage_flush
    kStPopL2Desc,     // claimed chunks read through a descriptor by another warp of the block
    kStCount
};

static_assert(kStCount <= 40, "Ctrl::stats holds 40 counters");

struct __align__(128) Ctrl {
    unsigned long long reserve;          // elements ever written to L2
    unsigned long long pad0[15];
    unsigned long long done;             // elements read from L2 whose work completed
    unsigned long long pad1[15];
    unsigned long long window;           // W: lowest absolute bucket floor(d / delta) that may hold L2 work
    unsigned long long pad2[15];
    int finished;
    int error;
    int err_where;
    int err_info;
    unsigned long long slice_end;        // serving: globaltimer value at which the current slice ends (0 = unset)
    unsigned long long processed;        // run-time sampling: elements taken for relaxation
    int pad3[24];
    unsigned long long stats[40];
};

// The L2 rings: ring r = bucket * shards + shard uses rt[r * 32], wt[r * 32]
// (each on its own 128-byte line), seq/cnt[r * nch + s] and
// data[(r * nch + s) * kChunk + i].
struct Rings {
    uint32_t* rt;
    uint32_t* wt;
    uint32_t* seq;
    uint32_t* cnt;
    uint2* data;
    uint32_t nch;      // chunks per ring (power of two)
    uint32_t margin;   // free chunks that must remain before a writer may take a ticket
};

struct KParams {
    const int32_t* row_ptr;  // [nv + 1], shadow layout
    const uint2* adj;        // (col, weight bits) per arc
    const int32_t* owner;    // [nv - n]: real vertex owning shadow n + i
    int32_t n;               // real vertices
    int32_t nv;              // vertices including shadows (stride of a query slice)
    int32_t nq;              // number of queries (dist slices)
    void* dist;              // uint32_t[nq * nv] or unsigned long long[nq * nv]
    int32_t vbits;           // multi-query: key = (query << vbits) | v
    uint32_t vmask;
    Rings l2;
    int32_t shards;          // rings per bucket (power of two, <= 32)
    Ctrl* ctrl;
    uint32_t delta;          // u32 width, or f32 bits
    int32_t bnum, bmax;      // bmax <= 32
    int32_t l1_type, l1_cap, wb;
    float filter_deltas;     // L1FQ window
    uint32_t near_w;         // light-arc bound: writes through arcs with weight <= near_w stay
                             // local (L0/L1), heavier ones go to their L2 bucket (kInfU32 = all local)
    int32_t max_arcs;        // arcs per warp batch before the rest is deferred
    int32_t claim;           // chunks per L2 claim (1..kMaxClaim)
    int32_t refillers;       // warps of a block that may refill L1 from L2 at the same time
    int32_t stage;           // 1: heavy-arc writes are pooled per bucket in the block before L2
    int32_t l2_only;         // 1: single-queue baseline (every write to L2, one chunk per read)
    int32_t unit_w;          // 1: breadth-first search: every real arc weighs 1, a shadow link 0
    int32_t hub_bnum;        // > 0: shadow vertices (hub slices) use their own rings (the upper half
                             // of each bucket's shards) and are read only from the first hub_bnum
                             // non-empty buckets; 0: they share the rings
    int32_t dedup;           // 1: one write per improved target of a warp round
    uint32_t direct;         // block staging: writes to the window's first `direct` buckets go to L2 at once
    int32_t desc;            // 1: claimed chunks beyond the first go to the block as descriptors (else into L1)
    uint32_t* pend;          // pending marks (or null): per distance slot, the lowest bucket at which
                             // the vertex has a queued element, kInfU32 = none (see relax_batch)
    int32_t scratch_off, far_off, stat_off, stage_off, l1_off;  // byte offsets in dynamic shared memory
    unsigned long long timeout_ns;
    unsigned long long slice_ns;   // serving: end the launch after this long, draining local queues to L2 (0 = run to completion)
    const uint32_t* qoff;          // serving: per-query bucket offset (the window position when the query was admitted), or null
    int* qlive;                    // serving: per-query count of elements in L2 (writes add, reads subtract), or null
    unsigned long long* trace;   // debug only: per-lane (location << 48 | iteration), mapped host memory
    unsigned long long* timeline; // run-time sampling (or null): kTimelineFields words per sample
    int32_t timeline_cap;         // samples that fit
    uint32_t timeline_ns;         // sampling period
};

// Run-time sampling (one lane of block 0): time since start (ns), elements
// written to L2 (reserve), L2 elements completed (done, published per block
// and so lagging), elements taken for relaxation from any level, the window
// W, and the warps of block 0 holding a batch at the sampling instant.
constexpr int kTimelineFields = 6;

// ------------------------------------------------------------------ PTX --

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ unsigned long long gtime() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile_int(const int* p) {
    return *(const volatile int*)p;
}

// 64-bit volatile shared-memory element access (L1 is only touched under the lock)
__device__ __forceinline__ void vst(volatile uint2* p, uint2 v) {
    *(volatile unsigned long long*)p = ((unsigned long long)v.y << 32) | v.x;
}
__device__ __forceinline__ uint2 vld(const volatile uint2* p) {
    unsigned long long x = *(const volatile unsigned long long*)p;
    return make_uint2((uint32_t)x, (uint32_t)(x >> 32));
}

// A slot of a lock-free shared-memory ring (L1, block staging) as a
// one-element mailbox: kEmptySlot (key kEmptyKey, distance 0) or an
// element.  A writer deposits with a 64-bit CAS from empty and a taker
// withdraws with a 64-bit exchange to empty, so two writers of consecutive
// laps of the ring cannot both fill one slot, nor two takers both empty it
// (with plain stores, "empty" cannot tell "cleared by the previous lap's
// taker" from "not yet filled by the previous lap's writer").
constexpr unsigned long long kEmptySlot = 0x00000000ffffffffull;
__device__ __forceinline__ bool slot_try_put(volatile uint2* p, uint2 e) {
    if (vld(p).x != kEmptyKey) return false;
    const unsigned long long v = ((unsigned long long)e.y << 32) | e.x;
    return atomicCAS(const_cast<unsigned long long*>(reinterpret_cast<volatile unsigned long long*>(p)), kEmptySlot,
                     v) == kEmptySlot;
}
__device__ __forceinline__ bool slot_try_take(volatile uint2* p, uint2& e) {
    if (vld(p).x == kEmptyKey) return false;
    const unsigned long long y =
        atomicExch(const_cast<unsigned long long*>(reinterpret_cast<volatile unsigned long long*>(p)), kEmptySlot);
    if (y == kEmptySlot) return false;
    e = make_uint2((uint32_t)y, (uint32_t)(y >> 32));
    return true;
}

// Mailbox slots of the descriptor ring: the deposit releases, and the
// withdrawal acquires, at CTA scope, so that a warp that takes a descriptor
// sees everything the depositing warp saw (the chunk it acquired in L2).
__device__ __forceinline__ bool desc_try_put(unsigned long long* p, unsigned long long v) {
    if (*(volatile unsigned long long*)p != kEmptySlot) return false;
    unsigned long long old;
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("atom.release.cta.shared::cta.cas.b64 %0, [%1], %2, %3;"
                 : "=l"(old) : "r"(a), "l"(kEmptySlot), "l"(v) : "memory");
    return old == kEmptySlot;
}
__device__ __forceinline__ bool desc_try_take(unsigned long long* p, unsigned long long& v) {
    if (*(volatile unsigned long long*)p == kEmptySlot) return false;
    unsigned long long old;
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("atom.acquire.cta.shared::cta.exch.b64 %0, [%1], %2;" : "=l"(old) : "r"(a), "l"(kEmptySlot) : "memory");
    if (old == kEmptySlot) return false;
    v = old;
    return true;
}

// Ticket w is ahead of ticket r (wrap-safe): some writer holds ticket r.
// Any observed w with w - r > 0 proves ticket r was taken, whatever the order
// in which the two relaxed loads were performed.
__device__ __forceinline__ bool ahead(uint32_t w, uint32_t r) { return (int32_t)(w - r) > 0; }

// L2 residency.  The adjacency (8 bytes per arc) is streamed once per
// expansion and is far larger than L2; the distance words, row offsets and
// queue chunks are the reused working set.  With SSSP_L2_HINTS the arc loads
// carry an evict-first L2 policy (and skip L1), and the distance loads, the
// distance atomics and the row-offset loads an evict-last one, so the stream
// does not push the working set out of L2.
#ifndef SSSP_L2_HINTS
#define SSSP_L2_HINTS 0
#endif
#ifndef SSSP_FINE_CYCLES
#define SSSP_FINE_CYCLES 0
#endif
#ifndef SSSP_BULK_REFILL
#define SSSP_BULK_REFILL 0
#endif
#ifndef SSSP_LF_STAGE
#define SSSP_LF_STAGE 1
#endif
#ifndef SSSP_SHADOW_OWNER
#define SSSP_SHADOW_OWNER 1
#endif
#ifndef SSSP_SPEC_ROW
#define SSSP_SPEC_ROW 0
#endif
#ifndef SSSP_PIPELINE
#define SSSP_PIPELINE 0
#endif
// Publication of a chunk (its sequence number) and of a warp's element count
// (the block account) rely on release semantics alone: st.release.gpu orders
// the warp's chunk stores and loads before the sequence number (the other
// lanes' accesses through the __syncwarp before it), and the account update is
// an atom.release.cta that the block's flusher observes before its own fence
// and its add to ctrl.done.  SSSP_PUB_FENCE=1 adds a full fence before each
// (on GB300: R-MAT-22 single source 1%, 256-query batch 2%, road 4096^2 5%
// slower).
#ifndef SSSP_PUB_FENCE
#define SSSP_PUB_FENCE 0
#endif
#ifndef SSSP_CHUNK_DESC
#define SSSP_CHUNK_DESC 1
#endif
#ifndef SSSP_CLAIM_HINT
#define SSSP_CLAIM_HINT 0
#endif
#ifndef SSSP_NOINLINE
#define SSSP_NOINLINE __noinline__
#endif
#ifndef SSSP_CLAIM_TRIES
#define SSSP_CLAIM_TRIES 4
#endif
__device__ __forceinline__ unsigned long long pol_stream() {
    unsigned long long p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ unsigned long long pol_keep() {
    unsigned long long p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
// one arc (column, weight bits); the graph is read-only during a solve
__device__ __forceinline__ uint2 ld_arc(const uint2* p) {
#if SSSP_L2_HINTS
    uint2 r;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;"
                 : "=r"(r.x), "=r"(r.y) : "l"(p), "l"(pol_stream()));
    return r;
#else
    return __ldg(p);
#endif
}
// a row offset
__device__ __forceinline__ int32_t ld_row(const int32_t* p) {
#if SSSP_L2_HINTS
    int32_t r;
    asm("ld.global.nc.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(r) : "l"(p), "l"(pol_keep()));
    return r;
#else
    return __ldg(p);
#endif
}
// L2 load of a distance word (bypasses L1 so the filter sees recent values)
__device__ __forceinline__ uint32_t ld_dist(const uint32_t* p) {
#if SSSP_L2_HINTS
    uint32_t r;
    asm volatile("ld.global.cg.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(r) : "l"(p), "l"(pol_keep()));
    return r;
#else
    return __ldcg(p);
#endif
}
__device__ __forceinline__ unsigned long long ld_dist(const unsigned long long* p) {
#if SSSP_L2_HINTS
    unsigned long long r;
    asm volatile("ld.global.cg.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(r) : "l"(p), "l"(pol_keep()));
    return r;
#else
    return __ldcg(p);
#endif
}
// Adds v to a shared-memory word with release semantics at CTA scope.
__device__ __forceinline__ unsigned long long atom_add_release_cta(unsigned long long* p, unsigned long long v) {
    unsigned long long old;
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("atom.release.cta.shared::cta.add.u64 %0, [%1], %2;" : "=l"(old) : "r"(a), "l"(v) : "memory");
    return old;
}
// Pending-mark atomics: an improvement lowers the mark with release order
// (its distance write is visible to whoever takes the mark later); a read
// takes the mark with acquire order and only then loads the distance.
__device__ __forceinline__ uint32_t atom_min_release(uint32_t* p, uint32_t v) {
    uint32_t old;
    asm volatile("atom.release.gpu.global.min.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ uint32_t atom_exch_acquire(uint32_t* p, uint32_t v) {
    uint32_t old;
    asm volatile("atom.acquire.gpu.global.exch.b32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// distance minimum whose old value is not needed (a reduction)
__device__ __forceinline__ void red_min(uint32_t* p, uint32_t v) {
#if SSSP_L2_HINTS
    asm volatile("red.relaxed.gpu.global.min.L2::cache_hint.u32 [%0], %1, %2;" ::"l"(p), "r"(v), "l"(pol_keep()));
#else
    atomicMin(p, v);
#endif
}
__device__ __forceinline__ void red_min(unsigned long long* p, unsigned long long v) {
#if SSSP_L2_HINTS
    asm volatile("red.relaxed.gpu.global.min.L2::cache_hint.u64 [%0], %1, %2;" ::"l"(p), "l"(v), "l"(pol_keep()));
#else
    atomicMin(p, v);
#endif
}

// ------------------------------------------------------------ arithmetic --

template <int WT> struct Arith;

// u32 lengths: saturating add (never wraps; 0xFFFFFFFF stays "unreachable").
template <> struct Arith<0> {
    static __device__ __forceinline__ uint32_t add(uint32_t d, uint32_t w) {
        uint32_t s = d + w;
        return (s < d || s == kInfU32) ? kSatU32 : s;
    }
    // absolute bucket of distance d: floor(d / delta)
    static __device__ __forceinline__ uint32_t bucket(uint32_t d, uint32_t delta) { return d / delta; }
    // distance bound (W + mult) * delta of the window's first buckets
    static __device__ __forceinline__ uint32_t upper(uint32_t W, uint32_t delta, float mult) {
        double b = ((double)W + (double)mult) * (double)delta;
        return b >= (double)kSatU32 ? kSatU32 : (uint32_t)b;
    }
    static __device__ __forceinline__ uint32_t plus_delta(uint32_t d, uint32_t delta) {
        return add(d, delta);
    }
};

// f32 lengths as IEEE bit patterns: one round-to-nearest add per arc.  For
// non-negative floats the bit pattern orders like the value, so atomicMin
// on the bits is a min on the values.
template <> struct Arith<1> {
    static __device__ __forceinline__ uint32_t add(uint32_t d, uint32_t w) {
        return __float_as_uint(__fadd_rn(__uint_as_float(d), __uint_as_float(w)));
    }
    static __device__ __forceinline__ uint32_t bucket(uint32_t d, uint32_t delta) {
        float x = __uint_as_float(d) / __uint_as_float(delta);
        if (!(x > 0.0f)) return 0u;
        if (x >= 4.0e9f) return 4000000000u;
        return (uint32_t)x;
    }
    static __device__ __forceinline__ uint32_t upper(uint32_t W, uint32_t delta, float mult) {
        return __float_as_uint(((float)W + mult) * __uint_as_float(delta));
    }
    static __device__ __forceinline__ uint32_t plus_delta(uint32_t d, uint32_t delta) {
        return __float_as_uint(__uint_as_float(d) + __uint_as_float(delta));
    }
};

// ------------------------------------------------------ block shared state --

struct BlockShared {
    int lock;                     // L1 lock of the near-far and SLF policies (one warp at a time)
    int slock;                    // far-write staging lock
    int refill;                   // one warp of the block refills L1 from L2
    uint32_t head, tail;          // L1 ring (V, FQ, SLF) or the near ring (NF)
    uint32_t fhead, ftail;        // NF far ring
    uint32_t nf;                  // NF threshold (distance bits)
    uint32_t writes;              // L1 write calls (periodic flush)
    unsigned long long acct;      // (held elements << 32) | unpublished L2 reads
    uint32_t scnt[32];            // staging per L2 bucket ring index: elements staged (lock-free
                                  // staging: the ring's tail)
    uint32_t shead[32];           // lock-free staging: the ring's head (slots taken for L2)
    unsigned long long slice_end; // serving: end of this launch's slice (globaltimer), ~0 = none
    unsigned long long deadline;  // watchdog: globaltimer value after which waits give up
    unsigned long long t0;        // launch start (globaltimer), for run-time sampling
    unsigned long long next_sample;
    uint32_t nsamples;
    uint32_t wcache;              // the window base as last read from ctrl.window by a warp of the block
    uint32_t dhead, dtail;        // claimed-chunk descriptor ring (SSSP_CHUNK_DESC)
    unsigned long long desc[kDescCap];  // (ticket << 32) | (count << 16) | ring, kEmptySlot = free
    uint32_t busy;                // warps of the block holding a batch (sampling only)
    KParams params;               // the launch parameters, read by the workers from here
};
static_assert(sizeof(KParams) % 4 == 0, "the prologue copies KParams in 4-byte words");

// ------------------------------------------------------------- watchdog --

__device__ __forceinline__ void raise_error(Ctrl* C, int code, int where, int info) {
    if (atomicCAS(&C->error, 0, code) == 0) {
        C->err_where = where;
        C->err_info = info;
    }
    __threadfence();
}

// Release/acquire fence at GPU scope between a warp's queue writes and the
// word that publishes them (chunk sequence numbers, the block count, done).
// SSSP_FENCE_SC=1 uses the sequentially consistent __threadfence instead.
#ifndef SSSP_FENCE_SC
#define SSSP_FENCE_SC 1
#endif
__device__ __forceinline__ void fence_gpu() {
#if SSSP_FENCE_SC
    __threadfence();
#else
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
#endif
}

// ---------------------------------------------------------------- kernel --

// The dynamic shared memory of mlmq_kernel (BlockShared, then the regions at
// the byte offsets in KParams).
//
// Code size: the L2 write, the far-staging flush and the block-staging
// flush are called from many places and are kept out of line
// (__noinline__), so one copy of each sits in the instruction cache; the
// relaxation round and the L0/L1 paths stay inline.
extern __shared__ __align__(16) unsigned char mlmq_smem[];

template <int WT, int PRED, bool MQ, int R, bool X>
struct Worker {
    // PRED: 0 = distances only (uint32 words), 1 = (dist, pred) words with the
    // smallest-index tight predecessor, 2 = (dist, pred) words set only on a
    // strict improvement.
    using DistT = typename std::conditional<PRED == 0, uint32_t, unsigned long long>::type;
    using A = Arith<WT>;

    const KParams& P;   // the launch parameters (the block's shared-memory copy)
    uint32_t lane;

    // L0 ring
    uint2 l0[R];
    uint32_t l0h, l0t;
    uint32_t nfar;                // elements in farbuf (warp-uniform)
    // deferred accounting (see acct_apply)
    int unc;                      // private pushes (L0, far staging) not yet counted in S()->acct
    int dec;                      // completed / exported elements not yet subtracted

    // Block and warp state in shared memory, addressed from the dynamic
    // shared array and the byte offsets in P (not kept in registers).
    __device__ __forceinline__ uint32_t warp_id() const { return threadIdx.x >> 5; }
    __device__ __forceinline__ BlockShared* S() const { return reinterpret_cast<BlockShared*>(mlmq_smem); }
    // this warp's 32-element staging area
    __device__ __forceinline__ uint2* scratch() const {
        return reinterpret_cast<uint2*>(mlmq_smem + P.scratch_off) + warp_id() * 32u;
    }
    // this warp's far staging (kFarCap elements)
    __device__ __forceinline__ uint2* farbuf() const {
        return reinterpret_cast<uint2*>(mlmq_smem + P.far_off) + warp_id() * (uint32_t)kFarCap;
    }
    // block staging, kStageCap elements per L2 bucket ring index
    __device__ __forceinline__ uint2* stg() const { return reinterpret_cast<uint2*>(mlmq_smem + P.stage_off); }
    // block L1 buffer
    __device__ __forceinline__ volatile uint2* L1() const {
        return reinterpret_cast<volatile uint2*>(mlmq_smem + P.l1_off);
    }
    // statistics of this warp (lane 0 updates)
    __device__ __forceinline__ unsigned long long* sst() const {
        return reinterpret_cast<unsigned long long*>(mlmq_smem + P.stat_off) + warp_id() * (uint32_t)kStCount;
    }
    __device__ __forceinline__ DistT* dist() const { return reinterpret_cast<DistT*>(P.dist); }

    __device__ explicit Worker(const KParams& p)
        : P(p), lane(lane_id()), l0h(0), l0t(0), nfar(0), unc(0), dec(0) {
        if (lane == 0)
            for (int i = 0; i < kStCount; i++) sst()[i] = 0;
#pragma unroll
        for (int r = 0; r < R; r++) l0[r] = make_uint2(0, 0);
    }

    // warp-uniform statistic update (lane 0 writes)
    __device__ __forceinline__ void stat(int i, unsigned long long v) const {
        if (lane == 0) sst()[i] += v;
    }

    __device__ __forceinline__ bool expired() const { return gtime() > S()->deadline; }

    __device__ __forceinline__ bool aborted() const {
        return ld_volatile_int(&P.ctrl->error) != 0 || ld_volatile_int(&P.ctrl->finished) != 0;
    }

    // debug trace of where each lane is (no-op unless P.trace is set)
    __device__ __forceinline__ void mark(uint32_t code, uint32_t iter = 0) const {
        if (X && P.trace) {
            const uint32_t gt = blockIdx.x * blockDim.x + threadIdx.x;
            *(volatile unsigned long long*)(P.trace + gt) =
                ((unsigned long long)code << 48) | (unsigned long long)(iter & 0xffffffffffffull);
            __threadfence_system();
        }
    }

    // ---- element helpers
    __device__ __forceinline__ uint32_t key_query(uint32_t key) const { return MQ ? key >> P.vbits : 0u; }
    __device__ __forceinline__ uint32_t key_vertex(uint32_t key) const { return MQ ? key & P.vmask : key; }
    __device__ __forceinline__ size_t dist_index(uint32_t key) const {
        return MQ ? (size_t)key_query(key) * (size_t)P.nv + key_vertex(key) : (size_t)key;
    }
    static __device__ __forceinline__ uint32_t dpart(uint32_t w) { return w; }
    static __device__ __forceinline__ uint32_t dpart(unsigned long long w) { return (uint32_t)(w >> 32); }

    // warp-uniform read of a shared-memory word: lane 0 reads, all lanes get
    // the same value (control flow that depends on it stays convergent)
    __device__ __forceinline__ uint32_t sread(const uint32_t* p) const {
        uint32_t v = 0;
        if (lane == 0) v = *(const volatile uint32_t*)p;
        return __shfl_sync(kFull, v, 0);
    }

    // ---- block accounting -----------------------------------------------
    // Increments (elements becoming visible to other warps) are applied before
    // the elements can be seen; decrements may be deferred.  When the held
    // count reaches zero, the unpublished L2 reads are added to ctrl.done.
    __device__ void try_flush() {
        unsigned long long v = *(volatile unsigned long long*)&S()->acct;
        while ((uint32_t)(v >> 32) == 0u && (uint32_t)v != 0u) {
            unsigned long long old = atomicCAS(&S()->acct, v, 0ull);
            if (old == v) {
                fence_gpu();
                atomicAdd(&P.ctrl->done, (unsigned long long)(uint32_t)v);
                return;
            }
            v = old;
        }
    }

    __device__ void acct_apply() {
        int delta = unc - dec;
        unc = 0;
        dec = 0;
        if (lane == 0 && delta != 0) {
            unsigned long long add = ((unsigned long long)(uint32_t)delta) << 32;
#if SSSP_PUB_FENCE
            fence_gpu();
            unsigned long long old = atomicAdd(&S()->acct, add);
#else
            unsigned long long old = atom_add_release_cta(&S()->acct, add);
#endif
            if ((uint32_t)(old >> 32) + (uint32_t)delta == 0u) try_flush();
        }
        __syncwarp();
    }

    // ---- block locks ----------------------------------------------------------
    // One warp at a time: the L1 ring (word = &S()->lock) and the far-write
    // staging (word = &S()->slock) have separate locks.  Lane 0 spins on a
    // plain read and only then tries the atomic (test-and-test-and-set),
    // with a growing sleep, so waiters do not flood the shared-memory
    // atomic unit while the holder works.
    __device__ bool lock(int* word) {
        int ok = 1;
        mark(2);
#if SSSP_FINE_CYCLES
        const long long cl0 = clock64();
#endif
        if (lane == 0) {
            uint32_t spins = 0, ns = 16;
            for (;;) {
                if (*(volatile int*)word == 0 && atomicCAS(word, 0, 1) == 0) break;
                if ((++spins & 255u) == 0 && expired()) {
                    raise_error(P.ctrl, kErrTimeout, 1, 0);
                    ok = 0;
                    break;
                }
                __nanosleep(ns);
                ns = ns < 256u ? ns * 2u : 256u;
            }
            sst()[kStLockSpin] += spins;
#if SSSP_FINE_CYCLES
            sst()[kCyLock] += (unsigned long long)(clock64() - cl0);
#endif
        }
        ok = __shfl_sync(kFull, ok, 0);
        __threadfence_block();
        return ok != 0;
    }
    __device__ void unlock(int* word) {
        __threadfence_block();
        __syncwarp();
        if (lane == 0) atomicExch(word, 0);
        __syncwarp();
    }
    __device__ __forceinline__ bool lock() { return lock(&S()->lock); }
    __device__ __forceinline__ void unlock() { unlock(&S()->lock); }
    __device__ __forceinline__ bool slock() { return lock(&S()->slock); }
    __device__ __forceinline__ void sunlock() { unlock(&S()->slock); }

    // ---- L2: sharded bucket rings -----------------------------------------
    // The window base.  No data is published through it (it only steers
    // where elements are written and read), so the load is relaxed and later
    // loads need not wait for it.  window() reads ctrl.window and refreshes
    // the block's copy; window_hint() returns the copy, for decisions that
    // only group or route elements (the staging bucket, the local front, the
    // L1 filter), where a slightly stale base costs nothing.
#ifndef SSSP_WIN_HINT
#define SSSP_WIN_HINT 1
#endif
#if SSSP_WIN_HINT
    __device__ __forceinline__ unsigned long long window() const {
        const unsigned long long w = ld_relaxed64(&P.ctrl->window);
        S()->wcache = (uint32_t)w;
        return w;
    }
    __device__ __forceinline__ uint32_t window_hint() const { return *(volatile uint32_t*)&S()->wcache; }
#else
    __device__ __forceinline__ unsigned long long window() const { return ld_acquire64(&P.ctrl->window); }
    __device__ __forceinline__ uint32_t window_hint() const { return (uint32_t)ld_acquire64(&P.ctrl->window); }
#endif
    __device__ __forceinline__ uint32_t home_shard() const {
        return (blockIdx.x + (threadIdx.x >> 5)) & (uint32_t)(P.shards - 1);
    }
    // The shard an element is written to: its home shard, or with hub rings
    // (hub_bnum > 0) the lower half of the shards for ordinary vertices and
    // the upper half for shadow vertices.
    __device__ __forceinline__ uint32_t write_shard(bool shadow) const {
        if (P.hub_bnum <= 0) return home_shard();
        const uint32_t half = (uint32_t)P.shards >> 1;
        return (shadow ? half : 0u) + (home_shard() & (half - 1u));
    }
    __device__ __forceinline__ bool hub_ring(uint32_t shard) const {
        return P.hub_bnum > 0 && shard >= ((uint32_t)P.shards >> 1);
    }

    // Serving: adds `sign` per valid element to its query's L2 count, one
    // atomic per distinct query of the warp.  At the end of a slice every
    // element is in L2, so a count of zero means the query is complete.
    __device__ __forceinline__ void count_live(bool valid, uint32_t key, int sign) {
        if (!MQ || !P.qlive) return;
        const uint32_t q = valid ? key_query(key) : 0xffffffffu;
        const uint32_t grp = __match_any_sync(kFull, q);
        if (valid && (grp & lanemask_lt()) == 0u) atomicAdd(P.qlive + q, sign * __popc(grp));
    }

    // Writes the valid lanes' elements to the L2 bucket of their distance
    // (this warp's shard of it).  Lanes are grouped per bucket with
    // __match_any_sync and every group fills one chunk with a single ticket
    // (atomicAdd) on its ring; the group leaders take their tickets and
    // publish concurrently, so a write costs about two round trips whatever
    // the number of groups.  A shadow vertex (a slice of a hub's arcs) is a
    // chunk of its own.  ctrl.reserve grows BEFORE any chunk is published.
    // Returns the number of elements written (warp-uniform); the caller
    // defers the decrement.
    __device__ SSSP_NOINLINE int l2_write(bool valid, uint2 e) {
        const uint32_t vm = __ballot_sync(kFull, valid);
        if (vm == 0) return 0;
        const long long cw0 = clock64();
        mark(3);
        const int total = __popc(vm);
        unsigned long long win = 0;
        if (lane == 0) {
            atomicAdd(&P.ctrl->reserve, (unsigned long long)total);
            win = window();
        }
        win = __shfl_sync(kFull, win, 0);
        const uint32_t W = (uint32_t)win;
        // absolute bucket (clamp_bucket: beyond the window's reach -> its far end)
        uint32_t ab = valid ? abs_bucket(e.x, e.y) : W;
        ab = clamp_bucket(ab, W);
        const uint32_t b = ab % (uint32_t)P.bmax;
        const uint32_t below = __reduce_min_sync(kFull, valid ? ab : 0xffffffffu);
        const bool shadow = valid && key_vertex(e.x) >= (uint32_t)P.n;
        const uint32_t shard = write_shard(shadow);
        const uint32_t gkey = !valid ? 0xffffffffu : (shadow ? (0x80000000u | lane) : b);
        const uint32_t grp = __match_any_sync(kFull, gkey);
        const bool leader = valid && (grp & lanemask_lt()) == 0u;
        uint32_t t = 0, ring = b * (uint32_t)P.shards + shard;
        int okw = 1;
        if (leader) {
            // take a ticket on the first ring (from b towards the window end)
            // with `margin` free chunks; diverting an element to a later bucket
            // only delays it (results are order independent).
            uint32_t tries = 0, bucket = b;
            for (;;) {
                uint32_t* wtp = P.l2.wt + (size_t)ring * 32;
                uint32_t* rtp = P.l2.rt + (size_t)ring * 32;
                // read r before w (acquire) so w - r over-estimates the occupancy
                const uint32_t r0 = ld_acquire(rtp);
                const uint32_t w0 = ld_relaxed(wtp);
                if (w0 - r0 + P.l2.margin < P.l2.nch) {
                    t = atomicAdd(wtp, 1u);
                    break;
                }
                if (++tries >= (uint32_t)P.bmax) {
                    raise_error(P.ctrl, kErrOverflow, 2, (int)bucket);
                    okw = 0;
                    break;
                }
                bucket = (bucket + 1u) % (uint32_t)P.bmax;
                ring = bucket * (uint32_t)P.shards + shard;
            }
            if (okw) {
                // wait until the chunk slot of ticket t is free (normally immediate)
                uint32_t* sp = P.l2.seq + (size_t)ring * P.l2.nch + (t & (P.l2.nch - 1u));
                uint32_t spins = 0;
                while (ld_acquire(sp) != t) {
                    if ((++spins & 255u) == 0 && expired()) {
                        raise_error(P.ctrl, kErrTimeout, 3, (int)ring);
                        okw = 0;
                        break;
                    }
                    __nanosleep(32);
                }
                if (spins) atomicAdd(&sst()[kStWaitSpin], (unsigned long long)spins);
            }
        }
        const int ldr = __ffs(grp) - 1;
        t = __shfl_sync(kFull, t, ldr);
        ring = __shfl_sync(kFull, ring, ldr);
        okw = __shfl_sync(kFull, okw, ldr);
        if (!__all_sync(kFull, okw || !valid)) return total;
        count_live(valid, e.x, 1);
        const size_t slot = (size_t)ring * P.l2.nch + (t & (P.l2.nch - 1u));
        if (valid) P.l2.data[slot * kChunk + __popc(grp & lanemask_lt())] = e;
        __syncwarp();
        if (leader) {
            P.l2.cnt[slot] = (uint32_t)__popc(grp);
            if (SSSP_PUB_FENCE) fence_gpu();
            st_release(P.l2.seq + slot, t + 1u);
        }
        stat(kStChunks, (unsigned long long)__popc(__ballot_sync(kFull, leader)));
        __syncwarp();
        // written below the window: work held in the local queues (L0/L1),
        // which the window does not see, has smaller distances than the L2
        // front; pull the window back so readers see these buckets first
        if (lane == 0 && below < W) atomicMin(&P.ctrl->window, (unsigned long long)below);
        stat(kStPullBack, below < W ? 1u : 0u);
        stat(kStLowWrite, (unsigned long long)__popc(__ballot_sync(kFull, valid && ab < 2u)));
        stat(kCyL2Write, (unsigned long long)(clock64() - cw0));
        return total;
    }

    // Probes the L2 rings of the window, lowest absolute bucket first: lane i
    // looks at absolute bucket W + round * (32 / S) + i / S, shard
    // (home + i) % S.  When the lowest buckets are empty a reader moves the
    // window up to the lowest non-empty one (the base advance of Section
    // 4.2); a writer below the window pulls it back (l2_write).  Writers keep
    // every element inside the window's reach (clamp_bucket), and every ring
    // lies inside it, so no element is left behind.  Claims up to `want`
    // chunks of the lowest non-empty ring among the first bnum buckets (hub
    // rings: the first hub_bnum) with one CAS on its read ticket.  Returns the
    // number of chunks claimed (warp-uniform) with their ring and first ticket.
    __device__ uint32_t l2_claim(uint32_t want, uint32_t& ring_out, uint32_t& t_out) {
#if SSSP_CLAIM_HINT
        // the first probe starts from the block's copy of the window base
        // while the current base is loaded; a stale copy means one more probe
        unsigned long long win = 0;
        if (lane == 0) win = ld_relaxed64(&P.ctrl->window);
        uint32_t W = window_hint();
        bool checked = false;
#else
        unsigned long long win = 0;
        if (lane == 0) win = window();
        win = __shfl_sync(kFull, win, 0);
        const uint32_t W = (uint32_t)win;
#endif
        const uint32_t S_ = (uint32_t)P.shards, per = 32u / S_;
        const uint32_t home = home_shard();
        for (uint32_t r0 = 0; r0 < (uint32_t)P.bmax; r0 += per) {
            const uint32_t rel = r0 + lane / S_;
            const bool probe = rel < (uint32_t)P.bmax;
            const uint32_t ring = ((W + rel) % (uint32_t)P.bmax) * S_ + ((home + lane) & (S_ - 1u));
            uint32_t r = 0, w = 0;
            if (probe) {
                r = ld_relaxed(P.l2.rt + (size_t)ring * 32);
                w = ld_relaxed(P.l2.wt + (size_t)ring * 32);
            }
#if SSSP_CLAIM_HINT
            if (!checked) {
                checked = true;
                win = __shfl_sync(kFull, win, 0);
                if ((uint32_t)win != W) {
                    W = (uint32_t)win;
                    if (lane == 0) S()->wcache = W;
                    r0 = 0u - per;  // probe again from bucket W
                    continue;
                }
            }
#endif
            const bool ne = probe && ahead(w, r);
            const uint32_t nonempty = __ballot_sync(kFull, ne);
            if (nonempty == 0) continue;
            const int first = __ffs(nonempty) - 1;
            const uint32_t first_rel = r0 + (uint32_t)first / S_;
            if (first_rel > 0 && lane == 0)
                if (atomicCAS(&P.ctrl->window, win, (unsigned long long)(W + first_rel)) == win) {
                    sst()[kStAdvance]++;
                    S()->wcache = W + first_rel;
                }
            // candidates: non-empty rings of buckets within bnum of the first
            // one; hub rings only within hub_bnum of it (a hub slice is
            // relaxed once its distance is near the front, so it is rarely
            // relaxed again)
            const uint32_t lim = hub_ring((home + lane) & (S_ - 1u)) ? (uint32_t)P.hub_bnum : (uint32_t)P.bnum;
            uint32_t cand = __ballot_sync(kFull, ne && rel < first_rel + lim);
            while (cand) {
                int c = __ffs(cand) - 1;
                uint32_t got = 0, t = 0;
                if (lane == (uint32_t)c) {
                    uint32_t rr = r;
                    uint32_t* rtp = P.l2.rt + (size_t)ring * 32;
                    for (int k = 0; k < SSSP_CLAIM_TRIES && ahead(w, rr); k++) {
                        uint32_t avail = w - rr;
                        uint32_t take = avail < want ? avail : want;
                        uint32_t old = atomicCAS(rtp, rr, rr + take);
                        if (old == rr) { got = take; t = rr; break; }
                        rr = old;
                        w = ld_relaxed(P.l2.wt + (size_t)ring * 32);
                    }
                    if (!got) atomicAdd((unsigned long long*)&sst()[kStCasFail], 1ull);
                }
                got = __shfl_sync(kFull, got, c);
                if (got) {
                    t_out = __shfl_sync(kFull, t, c);
                    ring_out = __shfl_sync(kFull, ring, c);
                    return got;
                }
                cand &= ~(1u << c);
            }
            return 0;  // the lowest buckets are contended: back off and retry later
        }
        return 0;
    }

    // Waits for the claimed chunks t .. t + got - 1 of `ring` (lane j watches
    // chunk j, all in parallel) and returns their element counts in the
    // lanes (cnt of chunk j in lane j).  okr = false on a timeout.
    __device__ uint32_t l2_wait_chunks(uint32_t ring, uint32_t t, uint32_t got, bool& okr) {
        uint32_t cnt = 0;
        int ok = 1;
        mark(4);
        if (lane < got) {
            const size_t slot = (size_t)ring * P.l2.nch + ((t + lane) & (P.l2.nch - 1u));
            uint32_t spins = 0;
            while (ld_acquire(P.l2.seq + slot) != t + lane + 1u) {
                if ((++spins & 255u) == 0 && expired()) {
                    raise_error(P.ctrl, kErrTimeout, 5, (int)ring);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
            if (spins) atomicAdd(&sst()[kStWaitSpin], (unsigned long long)spins);
            if (ok) cnt = P.l2.cnt[slot];
        }
        okr = __all_sync(kFull, ok != 0);
        return cnt;
    }

    // Reads chunk t + j (count c) into the lanes and frees its slot.
    // CG: load through L2 only (a chunk claimed by another warp of the block).
    template <bool CG = false>
    __device__ void l2_read_chunk(uint32_t ring, uint32_t tj, uint32_t c, bool& valid, uint2& e) {
        const size_t slot = (size_t)ring * P.l2.nch + (tj & (P.l2.nch - 1u));
        valid = lane < c;
        if (valid) e = CG ? __ldcg(P.l2.data + slot * kChunk + lane) : P.l2.data[slot * kChunk + lane];
        count_live(valid, e.x, -1);
        __syncwarp();
        if (lane == 0) {
            if (SSSP_PUB_FENCE) fence_gpu();
            st_release(P.l2.seq + slot, tj + P.l2.nch);
        }
        __syncwarp();
    }

    // ---- L1 ------------------------------------------------------------------
    __device__ __forceinline__ uint32_t l1_mask() const { return (uint32_t)P.l1_cap - 1u; }

    // Places the valid elements (K per lane) into L1 under the block lock, per
    // the L1 policy; elements that do not fit or are filtered out get their
    // `out` flag set and must go to L2.  `count_add` elements are added to the
    // block count before the lock is released (they become visible here).
    template <int K>
    __device__ void l1_place(uint2 (&e)[K], bool (&valid)[K], bool (&out)[K], uint32_t fthr,
                             int count_add) {
        const int type = P.l1_type;
        const uint32_t cap = (uint32_t)P.l1_cap;
        if (type == 1) {
            // near-far: two rings of cap/2
            const uint32_t half = cap >> 1;
            uint32_t nf = sread(&S()->nf);
#pragma unroll
            for (int k = 0; k < K; k++) {
                bool nearv = valid[k] && e[k].y < nf;
                bool farv = valid[k] && !nearv;
                uint32_t nm = __ballot_sync(kFull, nearv), fm = __ballot_sync(kFull, farv);
                uint32_t h = sread(&S()->head), t = sread(&S()->tail);
                uint32_t fh = sread(&S()->fhead), ft = sread(&S()->ftail);
                uint32_t nspace = half - (t - h), fspace = half - (ft - fh);
                uint32_t nr = __popc(nm & lanemask_lt()), fr = __popc(fm & lanemask_lt());
                out[k] = false;
                if (nearv) {
                    if (nr < nspace) vst(&L1()[(t + nr) & (half - 1u)], e[k]);
                    else out[k] = true;
                }
                if (farv) {
                    if (fr < fspace) vst(&L1()[half + ((ft + fr) & (half - 1u))], e[k]);
                    else out[k] = true;
                }
                __syncwarp();
                if (lane == 0) {
                    uint32_t nn = __popc(nm), fn = __popc(fm);
                    *(volatile uint32_t*)&S()->tail = t + (nn < nspace ? nn : nspace);
                    *(volatile uint32_t*)&S()->ftail = ft + (fn < fspace ? fn : fspace);
                }
                __syncwarp();
            }
        } else if (type == 3) {
            // SLF deque: dist <= head element -> push front, else push back
#pragma unroll
            for (int k = 0; k < K; k++) {
                uint32_t h = sread(&S()->head), t = sread(&S()->tail);
                uint32_t hd = 0;
                if (lane == 0 && t != h) hd = vld(&L1()[h & l1_mask()]).y;
                hd = __shfl_sync(kFull, hd, 0);
                bool front = valid[k] && t != h && e[k].y <= hd;
                bool back = valid[k] && !front;
                uint32_t fm = __ballot_sync(kFull, front), bm = __ballot_sync(kFull, back);
                uint32_t space = cap - (t - h);
                uint32_t fn = __popc(fm), bn = __popc(bm);
                uint32_t ftake = fn < space ? fn : space;
                uint32_t btake = bn < space - ftake ? bn : space - ftake;
                uint32_t fr = __popc(fm & lanemask_lt()), br = __popc(bm & lanemask_lt());
                out[k] = false;
                if (front) {
                    if (fr < ftake) vst(&L1()[(h - 1u - fr) & l1_mask()], e[k]);
                    else out[k] = true;
                }
                if (back) {
                    if (br < btake) vst(&L1()[(t + br) & l1_mask()], e[k]);
                    else out[k] = true;
                }
                __syncwarp();
                if (lane == 0) {
                    *(volatile uint32_t*)&S()->head = h - ftake;
                    *(volatile uint32_t*)&S()->tail = t + btake;
                }
                __syncwarp();
            }
        } else {
            // vector (type 0) / filter (type 2, keep dist <= fthr)
#pragma unroll
            for (int k = 0; k < K; k++) {
                // with admission offsets (serving) the filter compares
                // absolute buckets: fthr then holds the last bucket kept
                bool want = valid[k] &&
                            (type != 2 || (MQ && P.qoff ? abs_bucket(e[k].x, e[k].y) <= fthr : e[k].y <= fthr));
                uint32_t wm = __ballot_sync(kFull, want);
                uint32_t h = sread(&S()->head), t = sread(&S()->tail);
                uint32_t space = cap - (t - h);
                uint32_t rank = __popc(wm & lanemask_lt());
                out[k] = valid[k] && !want;
                if (want) {
                    if (rank < space) vst(&L1()[(t + rank) & l1_mask()], e[k]);
                    else out[k] = true;
                }
                __syncwarp();
                if (lane == 0) {
                    uint32_t c = __popc(wm);
                    *(volatile uint32_t*)&S()->tail = t + (c < space ? c : space);
                }
                __syncwarp();
            }
        }
        if (lane == 0 && count_add != 0)
            atomicAdd(&S()->acct, ((unsigned long long)(uint32_t)count_add) << 32);
    }

    // Moves everything in L1 to L2 (periodic flush of L1V, Section 3.4).
    // Called with the lock held.
    __device__ void l1_flush_locked() {
        const uint32_t cap = (uint32_t)P.l1_cap;
        if (P.l1_type == 1) {
            const uint32_t half = cap >> 1;
            for (int rg = 0; rg < 2; rg++) {
                uint32_t* hp = rg ? &S()->fhead : &S()->head;
                uint32_t* tp = rg ? &S()->ftail : &S()->tail;
                uint32_t h = sread(hp), t = sread(tp);
                while (h != t) {
                    uint32_t c = t - h < 32u ? t - h : 32u;
                    bool v = lane < c;
                    uint2 x = make_uint2(0, 0);
                    if (v) x = vld(&L1()[(rg ? half : 0u) + ((h + lane) & (half - 1u))]);
                    h += c;
                    dec += l2_write(v, x);
                }
                __syncwarp();
                if (lane == 0) *(volatile uint32_t*)hp = h;
                __syncwarp();
            }
        } else {
            uint32_t h = sread(&S()->head), t = sread(&S()->tail);
            while (h != t) {
                uint32_t c = t - h < 32u ? t - h : 32u;
                bool v = lane < c;
                uint2 x = make_uint2(0, 0);
                if (v) x = vld(&L1()[(h + lane) & l1_mask()]);
                h += c;
                dec += l2_write(v, x);
            }
            __syncwarp();
            if (lane == 0) *(volatile uint32_t*)&S()->head = h;
            __syncwarp();
        }
        stat(kStFlush, 1);
    }

    // ---- L1 vector / filter policies: lock-free ring ------------------------
    // Slots are one-element mailboxes (slot_try_put / slot_try_take).
    // Writers reserve slots by CAS on tail (bounded by head + cap) and deposit
    // into each reserved slot once it is empty (its reader of the previous
    // lap has taken the element); readers reserve up to 32 slots by CAS on
    // head (bounded by tail) and withdraw from each once it is full.  Both
    // waits are on warps that are already inside the same operation, so they
    // are short; they are bounded by the deadline.
    // the lean kernel (X = false) runs the lock-free policies only
    __device__ __forceinline__ bool l1_lockfree() const { return !X || P.l1_type == 0 || P.l1_type == 2; }

    template <int K>
    __device__ void l1_write_lf(uint2 (&e)[K], bool (&valid)[K], int count_add, uint32_t fthr) {
        const uint32_t cap = (uint32_t)P.l1_cap;
        // the elements become visible to other warps: count them first
        if (lane == 0 && count_add != 0)
            atomicAdd(&S()->acct, ((unsigned long long)(uint32_t)count_add) << 32);
        __syncwarp();
        bool out[K];
#pragma unroll
        for (int k = 0; k < K; k++) {
            const bool want = valid[k] && (P.l1_type != 2 ||
                                           (MQ && P.qoff ? abs_bucket(e[k].x, e[k].y) <= fthr : e[k].y <= fthr));
            const uint32_t wm = __ballot_sync(kFull, want);
            out[k] = valid[k] && !want;
            if (!wm) continue;
            const uint32_t c = __popc(wm);
            uint32_t base = 0, take = 0;
            if (lane == 0) {
                uint32_t t = *(volatile uint32_t*)&S()->tail;
                for (;;) {
                    const uint32_t h = *(volatile uint32_t*)&S()->head;
                    const uint32_t used = t - h;
                    take = used < cap ? min(c, cap - used) : 0u;
                    if (take == 0) break;
                    const uint32_t old = atomicCAS(&S()->tail, t, t + take);
                    if (old == t) break;
                    t = old;
                }
                base = t;
            }
            base = __shfl_sync(kFull, base, 0);
            take = __shfl_sync(kFull, take, 0);
            const uint32_t rank = __popc(wm & lanemask_lt());
            const bool placed = want && rank < take;
            out[k] = out[k] || (want && !placed);
            int ok = 1;
            if (placed) {
                volatile uint2* slot = &L1()[(base + rank) & l1_mask()];
                uint32_t spins = 0;
                while (!slot_try_put(slot, e[k])) {
                    if ((++spins & 255u) == 0 && expired()) {
                        raise_error(P.ctrl, kErrTimeout, 10, 0);
                        ok = 0;
                        break;
                    }
                }
            }
            __syncwarp();
        }
#pragma unroll
        for (int k = 0; k < K; k++) dec += l2_write(out[k], e[k]);
    }

    __device__ bool l1_read_lf(bool& valid, uint2& e) {
        valid = false;
        uint32_t h = 0, c = 0;
        if (lane == 0) {
            h = *(volatile uint32_t*)&S()->head;
            for (;;) {
                const uint32_t t = *(volatile uint32_t*)&S()->tail;
                c = t - h < 32u ? t - h : 32u;
                if (c == 0) break;
                const uint32_t old = atomicCAS(&S()->head, h, h + c);
                if (old == h) break;
                h = old;
            }
        }
        c = __shfl_sync(kFull, c, 0);
        if (c == 0) return false;
        h = __shfl_sync(kFull, h, 0);
        if (lane < c) {
            volatile uint2* slot = &L1()[(h + lane) & l1_mask()];
            uint32_t spins = 0;
            uint2 x = make_uint2(kEmptyKey, 0u);
            while (!slot_try_take(slot, x)) {
                if ((++spins & 255u) == 0 && expired()) {
                    raise_error(P.ctrl, kErrTimeout, 11, 0);
                    break;
                }
            }
            valid = x.x != kEmptyKey;
            e = x;
        }
        __syncwarp();
        stat(kStPopL1, 1);
        return true;
    }

    // Write primitive of the L1 level for K elements per lane; `count_add`
    // of them are not yet in the block count (see l1_place).  `filter`
    // applies the L1FQ threshold.
    template <int K>
    __device__ void l1_write(uint2 (&e)[K], bool (&valid)[K], int count_add, bool filter = true) {
        const long long c0 = clock64();
        uint32_t fthr = kInfU32;
        if (P.l1_type == 2 && filter) {
            const uint32_t win = window_hint();
            fthr = MQ && P.qoff ? win + (uint32_t)P.filter_deltas       // bucket W + F
                                : A::upper(win, P.delta, P.filter_deltas);  // (W + F) * delta
        }
        if (l1_lockfree()) {
            l1_write_lf<K>(e, valid, count_add, fthr);
            if (P.wb > 0) {
                // L1V periodic flush (Section 3.4): every wb-th write moves L1 to L2
                uint32_t wc = 0;
                if (lane == 0) wc = atomicAdd(&S()->writes, 1u) + 1u;
                wc = __shfl_sync(kFull, wc, 0);
                if (wc % (uint32_t)P.wb == 0u) {
                    bool v = false;
                    uint2 x = make_uint2(0, 0);
                    for (uint32_t n = 0; n <= (uint32_t)P.l1_cap / 32u && l1_read_lf(v, x); n++)
                        dec += l2_write(v, x);
                    stat(kStFlush, 1);
                }
            }
            stat(kCyL1, (unsigned long long)((unsigned long long)(clock64() - c0)));
            return;
        }
        bool out[K];
        if (!lock()) return;
        l1_place<K>(e, valid, out, fthr, count_add);
        bool flush = false;
        if (P.wb > 0) {
            uint32_t wcount = 0;
            if (lane == 0) {
                wcount = *(volatile uint32_t*)&S()->writes + 1u;
                *(volatile uint32_t*)&S()->writes = wcount;
            }
            wcount = __shfl_sync(kFull, wcount, 0);
            flush = (wcount % (uint32_t)P.wb) == 0u;
        }
        if (flush) l1_flush_locked();
        unlock();
        stat(kCyL1, (unsigned long long)((unsigned long long)(clock64() - c0)));
#pragma unroll
        for (int k = 0; k < K; k++) dec += l2_write(out[k], e[k]);
    }

    // Read primitive of the L1 level: up to 32 elements, one per lane.
    __device__ bool l1_read(bool& valid, uint2& e) {
        valid = false;
        // cheap unlocked emptiness test first (lane 0 decides for the warp)
        uint32_t any = 0;
        if (lane == 0) {
            any = *(volatile uint32_t*)&S()->head != *(volatile uint32_t*)&S()->tail;
            if (X && P.l1_type == 1) any |= *(volatile uint32_t*)&S()->fhead != *(volatile uint32_t*)&S()->ftail;
        }
        if (!__shfl_sync(kFull, any, 0)) return false;
        if (l1_lockfree()) return l1_read_lf(valid, e);
        if (!lock()) return false;
        const uint32_t cap = (uint32_t)P.l1_cap;
        uint32_t h = sread(&S()->head), t = sread(&S()->tail);
        if (P.l1_type == 1 && h == t) {
            // near vector drained: NF = min(far) + delta, then re-partition far
            const uint32_t half = cap >> 1;
            uint32_t fh = sread(&S()->fhead), ft = sread(&S()->ftail);
            if (fh != ft) {
                uint32_t mn = kInfU32;
                for (uint32_t i = fh + lane; i - fh < ft - fh; i += 32)
                    mn = min(mn, vld(&L1()[half + (i & (half - 1u))]).y);
                mn = __reduce_min_sync(kFull, mn);
                uint32_t nf = A::plus_delta(mn, P.delta);
                uint32_t nt = t, nft = ft;
                uint32_t count = ft - fh;
                for (uint32_t base = 0; base < count; base += 32) {
                    bool v = base + lane < count;
                    uint2 x = make_uint2(0, 0);
                    if (v) x = vld(&L1()[half + ((fh + base + lane) & (half - 1u))]);
                    __syncwarp();
                    bool nearv = v && x.y < nf;
                    bool farv = v && !nearv;
                    uint32_t nm = __ballot_sync(kFull, nearv), fm = __ballot_sync(kFull, farv);
                    if (nearv) vst(&L1()[(nt + __popc(nm & lanemask_lt())) & (half - 1u)], x);
                    if (farv) vst(&L1()[half + ((nft + __popc(fm & lanemask_lt())) & (half - 1u))], x);
                    __syncwarp();
                    nt += __popc(nm);
                    nft += __popc(fm);
                }
                if (lane == 0) {
                    *(volatile uint32_t*)&S()->nf = nf;
                    *(volatile uint32_t*)&S()->tail = nt;
                    *(volatile uint32_t*)&S()->fhead = fh + count;
                    *(volatile uint32_t*)&S()->ftail = nft;
                }
                __syncwarp();
                t = nt;
            }
        }
        uint32_t c = t - h < 32u ? t - h : 32u;
        valid = lane < c;
        if (valid) {
            uint32_t idx = P.l1_type == 1 ? ((h + lane) & ((cap >> 1) - 1u)) : ((h + lane) & l1_mask());
            e = vld(&L1()[idx]);
        }
        __syncwarp();
        if (lane == 0) *(volatile uint32_t*)&S()->head = h + c;
        unlock();
        if (c) stat(kStPopL1, 1);
        return c != 0;
    }

    // Free L1 slots (estimate, no lock).
    __device__ uint32_t l1_free() const {
        uint32_t f = 0;
        if (lane == 0) {
            uint32_t h = *(volatile uint32_t*)&S()->head, t = *(volatile uint32_t*)&S()->tail;
            uint32_t cap = (uint32_t)P.l1_cap >> (X && P.l1_type == 1 ? 1 : 0);
            uint32_t used = t - h;
            f = used < cap ? cap - used : 0u;
        }
        return __shfl_sync(kFull, f, 0);
    }

    // The claimed chunks t .. t + got - 1 of `ring` (counts: chunk j's in lane
    // j) read together: chunk 0 becomes this warp's batch, chunks 1 .. got - 1
    // go to the lock-free L1 in one reservation.  The chunk loads are issued
    // in groups of four, then every chunk slot is released at once (lane j
    // releases chunk j).  Returns false, having read nothing, when L1 has no
    // room for all of them (the caller reads chunk by chunk instead).
    __device__ bool read_chunks_bulk(uint32_t ring, uint32_t t, uint32_t got, uint32_t cnt, bool& valid, uint2& e) {
        // exclusive prefix of the counts of chunks 1 .. got - 1 (lane j)
        const uint32_t mine = (lane >= 1u && lane < got) ? cnt : 0u;
        uint32_t incl = mine;
#pragma unroll
        for (int o = 1; o < kMaxClaim; o <<= 1) {
            const uint32_t x = __shfl_up_sync(kFull, incl, o);
            if (lane >= (uint32_t)o) incl += x;
        }
        const uint32_t rest = __shfl_sync(kFull, incl, kMaxClaim - 1);
        const uint32_t pre = incl - mine;
        // all-or-nothing reservation of `rest` L1 slots
        uint32_t base = 0;
        int ok = 1;
        if (lane == 0 && rest) {
            const uint32_t cap = (uint32_t)P.l1_cap;
            uint32_t tl = *(volatile uint32_t*)&S()->tail;
            for (;;) {
                const uint32_t h = *(volatile uint32_t*)&S()->head;
                if (tl - h + rest > cap) {
                    ok = 0;
                    break;
                }
                const uint32_t old = atomicCAS(&S()->tail, tl, tl + rest);
                if (old == tl) break;
                tl = old;
            }
            base = tl;
        }
        if (!__shfl_sync(kFull, ok, 0)) return false;
        base = __shfl_sync(kFull, base, 0);
        const size_t slot0 = (size_t)ring * P.l2.nch;
        const uint32_t mask = P.l2.nch - 1u;
        // chunk 0: this warp's batch
        {
            const uint32_t c0 = __shfl_sync(kFull, cnt, 0);
            valid = lane < c0;
            if (valid) e = P.l2.data[(slot0 + (t & mask)) * kChunk + lane];
            count_live(valid, e.x, -1);
        }
        // chunks 1 .. got - 1 into L1, four loads in flight per lane
#pragma unroll
        for (uint32_t j0 = 1; j0 < (uint32_t)kMaxClaim; j0 += 4) {
            uint2 x[4];
            bool v[4];
#pragma unroll
            for (uint32_t k = 0; k < 4; k++) {
                const uint32_t j = j0 + k;
                const uint32_t cj = __shfl_sync(kFull, cnt, j & 31u);
                v[k] = j < got && lane < cj;
                x[k] = v[k] ? P.l2.data[(slot0 + ((t + j) & mask)) * kChunk + lane] : make_uint2(0u, 0u);
            }
#pragma unroll
            for (uint32_t k = 0; k < 4; k++) {
                const uint32_t j = j0 + k;
                const uint32_t pj = __shfl_sync(kFull, pre, j & 31u);
                count_live(v[k], x[k].x, -1);
                if (v[k]) {
                    volatile uint2* sl = &L1()[(base + pj + lane) & l1_mask()];
                    uint32_t spins = 0;
                    while (!slot_try_put(sl, x[k])) {
                        if ((++spins & 255u) == 0 && expired()) {
                            raise_error(P.ctrl, kErrTimeout, 12, 0);
                            break;
                        }
                    }
                }
            }
        }
        __syncwarp();
        if (lane < got) {
            if (SSSP_PUB_FENCE) fence_gpu();
            st_release(P.l2.seq + slot0 + ((t + lane) & mask), t + lane + P.l2.nch);
        }
        __syncwarp();
        return true;
    }

    // L1 is empty: up to `refillers` warps of the block at a time refill it
    // from L2 (Section 3.2: an empty level triggers a read of the next level).
    // The first claimed chunk becomes this warp's batch, the rest go to L1.
    // Returns 1 with a batch in the lanes, 2 if only L1 received elements, 0
    // if L2 had nothing, -1 if enough warps of the block are already refilling.
    // ---- claimed-chunk descriptors (SSSP_CHUNK_DESC) ------------------------
    // A refill keeps the first claimed chunk as its own batch and hands the
    // others to the block as descriptors (ring, ticket, count) instead of
    // copying their elements into L1: another warp of the block takes a
    // descriptor and reads the chunk itself, so the chunks of one claim are
    // read by several warps at once, and their elements skip the L1 ring.
    // The elements are in the block count from the claim on.
    __device__ __forceinline__ uint32_t desc_free() const {
        uint32_t f = 0;
        if (lane == 0) {
            const uint32_t used = *(volatile uint32_t*)&S()->dtail - *(volatile uint32_t*)&S()->dhead;
            f = used < (uint32_t)kDescCap ? (uint32_t)kDescCap - used : 0u;
        }
        return __shfl_sync(kFull, f, 0);
    }

    // Deposits descriptors for chunks 1 .. got - 1 of a claim (lane j: the
    // count of chunk j); returns k: chunks 1 .. k were handed over, the rest
    // did not fit.
    __device__ uint32_t desc_put(uint32_t ring, uint32_t t, uint32_t got, uint32_t cnt) {
        uint32_t base = 0, take = 0;
        if (lane == 0) {
            uint32_t tl = *(volatile uint32_t*)&S()->dtail;
            for (;;) {
                const uint32_t h = *(volatile uint32_t*)&S()->dhead;
                const uint32_t used = tl - h;
                take = used < (uint32_t)kDescCap ? min(got - 1u, (uint32_t)kDescCap - used) : 0u;
                if (take == 0) break;
                const uint32_t old = atomicCAS(&S()->dtail, tl, tl + take);
                if (old == tl) break;
                tl = old;
            }
            base = tl;
        }
        take = __shfl_sync(kFull, take, 0);
        base = __shfl_sync(kFull, base, 0);
        if (lane >= 1u && lane <= take) {
            const unsigned long long d = ((unsigned long long)(t + lane) << 32) | (unsigned long long)(ring | (cnt << 16));
            unsigned long long* sl = &S()->desc[(base + lane - 1u) & (uint32_t)(kDescCap - 1)];
            uint32_t spins = 0;
            while (!desc_try_put(sl, d)) {
                if ((++spins & 255u) == 0 && expired()) {
                    raise_error(P.ctrl, kErrTimeout, 15, 0);
                    break;
                }
            }
        }
        __syncwarp();
        return take;
    }

    // Takes one descriptor and reads its chunk into the lanes (the warp's
    // batch).  False if there is none.
    __device__ bool desc_read(bool& valid, uint2& e) {
        valid = false;
        uint32_t h = 0;
        int got = 0;
        if (lane == 0) {
            h = *(volatile uint32_t*)&S()->dhead;
            for (;;) {
                if (*(volatile uint32_t*)&S()->dtail == h) break;
                const uint32_t old = atomicCAS(&S()->dhead, h, h + 1u);
                if (old == h) {
                    got = 1;
                    break;
                }
                h = old;
            }
        }
        if (!__shfl_sync(kFull, got, 0)) return false;
        unsigned long long d = kEmptySlot;
        if (lane == 0) {
            unsigned long long* sl = &S()->desc[h & (uint32_t)(kDescCap - 1)];
            uint32_t spins = 0;
            while (!desc_try_take(sl, d)) {
                if ((++spins & 255u) == 0 && expired()) {
                    raise_error(P.ctrl, kErrTimeout, 16, 0);
                    break;
                }
            }
        }
        d = __shfl_sync(kFull, d, 0);
        if (d == kEmptySlot) return true;  // timed out: the error stops the launch
        const uint32_t lo = (uint32_t)d;
        l2_read_chunk<true>(lo & 0xffffu, (uint32_t)(d >> 32), lo >> 16, valid, e);
        stat(kStPopL2Desc, 1);
        return true;
    }

    __device__ int refill(bool& valid, uint2& e) {
        valid = false;
        int role = 0;
        if (lane == 0) {
            role = atomicAdd(&S()->refill, 1) < P.refillers;
            if (!role) atomicSub(&S()->refill, 1);
        }
        role = __shfl_sync(kFull, role, 0);
        if (!role) return -1;
        stat(kStRefillTry, 1);
#if SSSP_FINE_CYCLES
        const long long cs0 = clock64();
        stage_flush(false);
        stat(kCyStage, (unsigned long long)(clock64() - cs0));
#else
        stage_flush(false);
#endif
        uint32_t want = (uint32_t)P.claim;
        uint32_t room = l1_free() / kChunk;
        if (SSSP_CHUNK_DESC && P.desc) room = max(room, desc_free());
        if (want > room + 1u) want = room + 1u;
        uint32_t ring = 0, t = 0;
#if SSSP_FINE_CYCLES
        const long long cc0 = clock64();
#endif
        const uint32_t got = l2_claim(want, ring, t);
#if SSSP_FINE_CYCLES
        const long long cc1 = clock64();
        stat(kCyClaim, (unsigned long long)(cc1 - cc0));
#endif
        int result = 0;
        if (got) {
            bool okr = true;
            const uint32_t cnt = l2_wait_chunks(ring, t, got, okr);
            if (okr) {
                // the claimed elements are held by this block from now on: count
                // them before they can be handed to other warps through L1
                const uint32_t total = __reduce_add_sync(kFull, cnt);
                if (lane == 0)
                    atomicAdd(&S()->acct, ((unsigned long long)total << 32) | (unsigned long long)total);
                const uint32_t c0 = __shfl_sync(kFull, cnt, 0);
                if (!(SSSP_BULK_REFILL && got > 1 && l1_lockfree() && read_chunks_bulk(ring, t, got, cnt, valid, e))) {
                    l2_read_chunk(ring, t, c0, valid, e);
                    const uint32_t j0 = SSSP_CHUNK_DESC && P.desc && got > 1u ? 1u + desc_put(ring, t, got, cnt) : 1u;
                    for (uint32_t j = j0; j < got; j++) {
                        const uint32_t cj = __shfl_sync(kFull, cnt, j);
                        bool v2 = false;
                        uint2 x[1] = {make_uint2(0, 0)};
                        l2_read_chunk(ring, t + j, cj, v2, x[0]);
                        bool vv[1] = {v2};
                        // chunks taken from L2 for processing bypass the L1 filter
                        l1_write<1>(x, vv, 0, false);
                    }
                }
                stat(kStPopL2, (unsigned long long)got);
                stat(kStRefill, 1);
#if SSSP_FINE_CYCLES
                stat(kCyChunks, (unsigned long long)(clock64() - cc1));
#endif
                result = c0 ? 1 : (total ? 2 : 0);
            }
        }
        __syncwarp();
        if (lane == 0) atomicSub(&S()->refill, 1);
        __syncwarp();
        return result;
    }

    // ---- L0 ------------------------------------------------------------------
    __device__ __forceinline__ uint2 l0_get(uint32_t r) const {
        uint2 x = l0[0];
#pragma unroll
        for (int i = 1; i < R; i++)
            if (r == (uint32_t)i) x = l0[i];
        return x;
    }
    __device__ __forceinline__ void l0_set(uint32_t r, uint2 x) {
#pragma unroll
        for (int i = 0; i < R; i++)
            if (r == (uint32_t)i) l0[i] = x;
    }

    // L0 is full: its whole content moves down to L1 (the L0 overflow rule of
    // Section 3.4).
    __device__ void l0_spill() {
        uint2 e[R];
        bool v[R];
        const uint32_t len = l0t - l0h;
#pragma unroll
        for (int r = 0; r < R; r++) {
            uint32_t want = 32u * (uint32_t)r + lane;
            uint32_t p = l0h + ((want - l0h) & (32u * R - 1u));
            v[r] = (p - l0h) < len;
            e[r] = l0[r];
        }
        l0h = l0t = 0;
        if (X && P.l2_only) {
            // single-queue baseline: no L1, the elements go to L2
#pragma unroll
            for (int r = 0; r < R; r++) dec += l2_write(v[r], e[r]);
            return;
        }
        // the elements become visible: count every private push now (the
        // far-staged ones too -- counting early only delays the block's
        // done flush, counting late could end the solve too soon)
        const int add = unc;
        unc = 0;
        l1_write<R>(e, v, add);
    }

    // Appends c (<= 32) staged elements scratch()[0..c) to L0.  `counted`:
    // they are already in the block count (a deferred batch element).
    __device__ void l0_push(uint32_t c, bool counted = false) {
        if (c == 0) return;
        if (l0t - l0h + c > 32u * R) l0_spill();
        uint32_t k = (lane - l0t) & 31u;
        if (k < c) {
            uint32_t p = l0t + k;
            l0_set((p >> 5) & (R - 1u), scratch()[k]);
        }
        l0t += c;
        if (!counted) unc += (int)c;
        __syncwarp();
    }

    __device__ bool l0_read(bool& valid, uint2& e) {
        uint32_t len = l0t - l0h;
        if (len == 0) return false;
        uint32_t c = len < 32u ? len : 32u;
        uint32_t k = (lane - l0h) & 31u;
        valid = k < c;
        if (valid) e = l0_get(((l0h + k) >> 5) & (R - 1u));
        l0h += c;
        if (l0h == l0t) l0h = l0t = 0;
        stat(kStPopL0, 1);
        return true;
    }

    // ---- far staging -------------------------------------------------------
    // Heavy-arc writes wait in a per-warp buffer.  Without block staging they
    // go to L2 in groups of up to 32.  With block staging (P.stage) the warps
    // of a block pool them per L2 bucket in shared memory under the staging lock,
    // and only full 32-element chunks go to L2 -- one warp's writes spread
    // over many buckets, so this is what keeps the chunks full.  Writes for
    // the window's first P.direct buckets (and hub slices) are urgent and go
    // to L2 at once; partial buckets are flushed when they become urgent (a
    // refill sends those of the first P.direct buckets) or the block runs dry.

    // absolute bucket of an element: floor(d / delta), shifted by the query's
    // admission offset when queries started at different times (serving)
    __device__ __forceinline__ uint32_t abs_bucket(uint32_t key, uint32_t d) const {
        uint32_t ab = A::bucket(d, P.delta);
        if (MQ && P.qoff) ab += __ldg(P.qoff + key_query(key));
        return ab;
    }

    // The bucket an element is written to.  Ring k serves buckets k, k + bmax,
    // ...; elements beyond the window's reach go to bucket W + reach - 1 with
    // reach = bmax - kWindowGuard, so that after the window is pulled back by
    // up to kWindowGuard buckets no ring holds elements of two buckets of the
    // window.  Elements below W keep their bucket (the writer pulls W back).
    __device__ __forceinline__ uint32_t clamp_bucket(uint32_t ab, uint32_t W) const {
        const uint32_t reach = (uint32_t)P.bmax > 2u * kWindowGuard ? (uint32_t)P.bmax - kWindowGuard
                                                                  : (uint32_t)P.bmax;
        if (ab > W && ab - W >= reach) return W + reach - 1u;
        return ab;
    }

    __device__ __forceinline__ uint32_t ring_bucket(uint32_t key, uint32_t d, uint32_t W, uint32_t& ab) const {
        ab = clamp_bucket(abs_bucket(key, d), W);
        return ab % (uint32_t)P.bmax;
    }

    // ---- lock-free block staging (SSSP_LF_STAGE) ----------------------------
    // One ring of kStageCap slots per L2 bucket ring index b, tail scnt[b] and
    // head shead[b], with mailbox slots as in the lock-free L1.  Writers
    // reserve slots with a CAS on the tail bounded by head + kStageCap and
    // deposit; a taker reserves up to 32 slots with a CAS on the head and
    // withdraws.  No block lock.
    __device__ __forceinline__ volatile uint2* stg_slot(uint32_t b, uint32_t i) const {
        return reinterpret_cast<volatile uint2*>(stg()) + b * (uint32_t)kStageCap + (i & (uint32_t)(kStageCap - 1));
    }

    // Reads the reserved slots h .. h + c - 1 of bucket b into the lanes and clears them.
    __device__ void stage_read(uint32_t b, uint32_t h, uint32_t c, bool& v, uint2& x) {
        v = lane < c;
        if (v) {
            volatile uint2* sl = stg_slot(b, h + lane);
            uint2 y = make_uint2(kEmptyKey, 0u);
            uint32_t spins = 0;
            while (!slot_try_take(sl, y)) {
                if ((++spins & 255u) == 0 && expired()) {
                    raise_error(P.ctrl, kErrTimeout, 13, (int)b);
                    break;
                }
            }
            v = y.x != kEmptyKey;
            x = y;
        }
        __syncwarp();
    }

    // Takes up to 32 staged elements of bucket b (lock-free); returns the count.
    __device__ uint32_t stage_take_lf(uint32_t b, bool& v, uint2& x) {
        uint32_t h = 0, c = 0;
        if (lane == 0) {
            h = *(volatile uint32_t*)&S()->shead[b];
            for (;;) {
                const uint32_t t = *(volatile uint32_t*)&S()->scnt[b];
                c = t - h < 32u ? t - h : 32u;
                if (c == 0) break;
                const uint32_t old = atomicCAS(&S()->shead[b], h, h + c);
                if (old == h) break;
                h = old;
            }
        }
        c = __shfl_sync(kFull, c, 0);
        h = __shfl_sync(kFull, h, 0);
        v = false;
        if (c) stage_read(b, h, c, v, x);
        return c;
    }

    // Places the lanes' staged elements sv (bucket b each) in their buckets'
    // rings; elements that do not fit go to L2 at once.  The leaders of the
    // bucket groups reserve their slots concurrently (a CAS on the ring's
    // tail, bounded by head + kStageCap), every lane then deposits its
    // element in its mailbox slot, and only after all deposits are the full
    // chunks taken and shipped to L2, one ring at a time.  No wait can close
    // a cycle: a writer lane waits only for its own slot to be emptied by the
    // taker of the previous lap (at least 33 slots behind its reservation), a
    // taker only for deposits into the slots it took (at most 31 ahead, with
    // kStageCap = 64 and at most 32 per take); no lane's deposit is ordered
    // after another lane's wait, and a warp takes chunks only while it holds
    // no reservation, so no wait depends on a second ring.
    __device__ void stage_place(bool sv, uint2 x, uint32_t b) {
        const uint32_t grp = __match_any_sync(kFull, sv ? b : 0xffffffffu);
        const uint32_t rank = __popc(grp & lanemask_lt());
        const bool leader = sv && rank == 0u;
        uint32_t base = 0, take = 0;
        if (leader) {
            const uint32_t k = (uint32_t)__popc(grp);
            uint32_t t = *(volatile uint32_t*)&S()->scnt[b];
            for (;;) {
                const uint32_t h = *(volatile uint32_t*)&S()->shead[b];
                const uint32_t used = t - h;
                take = used < (uint32_t)kStageCap ? min(k, (uint32_t)kStageCap - used) : 0u;
                if (take == 0) break;
                const uint32_t old = atomicCAS(&S()->scnt[b], t, t + take);
                if (old == t) break;
                t = old;
            }
            base = t;
        }
        const int ldr = __ffs(grp) - 1;
        base = __shfl_sync(kFull, base, ldr);
        take = __shfl_sync(kFull, take, ldr);
        const bool placed = sv && rank < take;
        const bool over = sv && !placed;
        if (placed) {
            volatile uint2* sl = stg_slot(b, base + rank);
            uint32_t spins = 0;
            while (!slot_try_put(sl, x)) {
                if ((++spins & 255u) == 0 && expired()) {
                    raise_error(P.ctrl, kErrTimeout, 14, (int)b);
                    break;
                }
            }
        }
        __syncwarp();
        // full chunks of the buckets this warp wrote go to L2
        uint32_t full = 0;
        if (leader) {
            const uint32_t t = *(volatile uint32_t*)&S()->scnt[b];
            const uint32_t h = *(volatile uint32_t*)&S()->shead[b];
            full = t - h >= 32u;
        }
        uint32_t fm = __ballot_sync(kFull, full != 0u);
        while (fm) {
            const uint32_t bg = __shfl_sync(kFull, b, __ffs(fm) - 1);
            fm &= fm - 1u;
            uint32_t h = 0;
            int own = 0;
            if (lane == 0) {
                h = *(volatile uint32_t*)&S()->shead[bg];
                const uint32_t t = *(volatile uint32_t*)&S()->scnt[bg];
                own = t - h >= 32u && atomicCAS(&S()->shead[bg], h, h + 32u) == h;
            }
            if (__shfl_sync(kFull, own, 0)) {
                h = __shfl_sync(kFull, h, 0);
                bool vy = false;
                uint2 y = make_uint2(0, 0);
                stage_read(bg, h, 32u, vy, y);
                dec += l2_write(vy, y);
            }
        }
        dec += l2_write(over, x);
    }

    // Takes up to 32 staged elements of bucket ring index b (lock held).
    __device__ uint32_t stage_take(uint32_t b, bool& v, uint2& x) {
        const uint32_t c0 = sread(&S()->scnt[b]);
        const uint32_t c = c0 < 32u ? c0 : 32u;
        v = lane < c;
        if (v) x = stg()[b * kStageCap + (c0 - c) + lane];
        __syncwarp();
        if (lane == 0) S()->scnt[b] = c0 - c;
        __syncwarp();
        return c;
    }

    // Moves staged elements to L2: all buckets (all = true, the block ran
    // dry) or only those of the window's first P.direct buckets.
    __device__ SSSP_NOINLINE void stage_flush(bool all) {
        if (!P.stage || (!all && P.direct == 0u)) return;
        const uint32_t W = window_hint();
        for (int guard = 0; guard < 64; guard++) {
            // unlocked look for a non-empty candidate bucket
            uint32_t cnt = 0;
            const uint32_t b = lane;
            const bool cand = b < (uint32_t)P.bmax &&
                              (all || ((b + (uint32_t)P.bmax - W % (uint32_t)P.bmax) % (uint32_t)P.bmax) < P.direct);
            if (cand) {
                cnt = *(volatile uint32_t*)&S()->scnt[b];
                if (SSSP_LF_STAGE) cnt -= *(volatile uint32_t*)&S()->shead[b];
            }
            const uint32_t m = __ballot_sync(kFull, cand && cnt > 0u);
            if (!m) return;
            const uint32_t bf = (uint32_t)(__ffs(m) - 1);
            bool v = false;
            uint2 x = make_uint2(0, 0);
#if SSSP_LF_STAGE
            stage_take_lf(bf, v, x);
#else
            if (!slock()) return;
            stage_take(bf, v, x);
            sunlock();
#endif
            dec += l2_write(v, x);
        }
    }

    __device__ SSSP_NOINLINE void far_flush(uint32_t upto) {
        if (nfar <= upto) return;
        const uint32_t W = P.stage ? window_hint() : 0u;
        while (nfar > upto) {
            const uint32_t take = nfar - upto < 32u ? nfar - upto : 32u;
            const bool v = lane < take;
            uint2 x = make_uint2(0, 0);
            if (v) x = farbuf()[nfar - take + lane];
            __syncwarp();
            nfar -= take;
            if (!P.stage) {
                dec += l2_write(v, x);
                continue;
            }
            uint32_t ab = 0;
            const uint32_t b = v ? ring_bucket(x.x, x.y, W, ab) : 0u;
            const bool urgent = v && (ab < W + P.direct || key_vertex(x.x) >= (uint32_t)P.n);
            dec += l2_write(urgent, x);
            const bool sv = v && !urgent;
            if (!__any_sync(kFull, sv)) continue;
#if SSSP_LF_STAGE
            // the staged elements become visible to the block: count every
            // private push now (counting early only delays the done flush)
            if (lane == 0 && unc != 0) atomicAdd(&S()->acct, ((unsigned long long)(uint32_t)unc) << 32);
            unc = 0;
            __syncwarp();
            stage_place(sv, x, b);
            continue;
#endif
            bool vy = false, over = false;
            uint2 y = make_uint2(0, 0);
            if (!slock()) return;
            // the staged elements become visible to the block: count every
            // private push now (counting early only delays the done flush)
            if (lane == 0 && unc != 0) atomicAdd(&S()->acct, ((unsigned long long)(uint32_t)unc) << 32);
            unc = 0;
            const uint32_t grp = __match_any_sync(kFull, sv ? b : 0xffffffffu);
            const int ldr = __ffs(grp) - 1;
            uint32_t base = 0;
            if (sv && lane == (uint32_t)ldr) base = S()->scnt[b];
            base = __shfl_sync(kFull, base, ldr);
            const uint32_t rank = __popc(grp & lanemask_lt());
            over = sv && base + rank >= (uint32_t)kStageCap;
            if (sv && !over) stg()[b * kStageCap + base + rank] = x;
            const uint32_t placed = min((uint32_t)__popc(grp), (uint32_t)kStageCap - min(base, (uint32_t)kStageCap));
            const bool full = sv && lane == (uint32_t)ldr && base + placed >= 32u;
            if (sv && lane == (uint32_t)ldr) S()->scnt[b] = base + placed;
            __syncwarp();
            const uint32_t fm = __ballot_sync(kFull, full);
            if (fm) {
                const uint32_t bf = __shfl_sync(kFull, b, __ffs(fm) - 1);
                stage_take(bf, vy, y);
            }
            sunlock();
            dec += l2_write(vy, y);
            dec += l2_write(over, x);
        }
    }

    __device__ void far_push(bool f, uint2 x) {
        uint32_t m = __ballot_sync(kFull, f);
        if (!m) return;
        uint32_t c = __popc(m);
#if SSSP_FINE_CYCLES
        const long long cf0 = clock64();
#endif
        if (nfar + c > (uint32_t)kFarCap) far_flush(0);
        if (f) farbuf()[nfar + __popc(m & lanemask_lt())] = x;
        __syncwarp();
        nfar += c;
        unc += (int)c;
        stat(kStFar, (unsigned long long)(c));
        if (nfar >= 32u) far_flush(nfar & 31u);
#if SSSP_FINE_CYCLES
        stat(kCyFarFlush, (unsigned long long)(clock64() - cf0));
#endif
    }

    // ---- relaxation ---------------------------------------------------------
    // Relaxes arc (u -> v, w) with u at distance du: nd = du (+) w; if nd
    // beats dist[v], atomicMin.  Returns true if dist[v] strictly improved
    // (the vertex must be written back, Listing 2).
    __device__ __forceinline__ bool relax(size_t vidx, uint32_t u, uint32_t du, uint32_t wbits,
                                          uint32_t& nd) {
        nd = A::add(du, wbits);
        if (PRED == 0) {
            uint32_t* p = reinterpret_cast<uint32_t*>(dist()) + vidx;
            uint32_t cur = ld_dist(p);
            if (nd >= cur) return false;
            uint32_t old = atomicMin(p, nd);
            return old > nd;
        } else if (PRED == 1) {
            unsigned long long* p = reinterpret_cast<unsigned long long*>(dist()) + vidx;
            unsigned long long cand = ((unsigned long long)nd << 32) | u;
            unsigned long long cur = ld_dist(p);
            if (cand >= cur) return false;
            unsigned long long old = atomicMin(p, cand);
            return (uint32_t)(old >> 32) > nd;
        } else {
            unsigned long long* p = reinterpret_cast<unsigned long long*>(dist()) + vidx;
            unsigned long long cand = ((unsigned long long)nd << 32) | u;
            unsigned long long cur = ld_dist(p);
            while ((uint32_t)(cur >> 32) > nd) {
                unsigned long long old = atomicCAS(p, cur, cand);
                if (old == cur) return true;
                cur = old;
            }
            return false;
        }
    }

    // relax() with dist[v] already loaded (cur).  Without predecessors, and
    // with the packed (dist, pred) minimum, the update is a reduction whose
    // old value is not waited for: the element is pushed when nd beat the
    // loaded value.  Every write that lowers dist[v] saw a larger value
    // when it loaded, so the final value is always pushed; a push that
    // lost the race carries a larger distance and is dropped as stale.
    __device__ __forceinline__ bool relax_cur(size_t vidx, uint32_t u, uint32_t du, uint32_t wbits, DistT cur,
                                              uint32_t& nd) {
        nd = A::add(du, wbits);
        if (PRED == 0) {
            if (nd >= (uint32_t)cur) return false;
            red_min(reinterpret_cast<uint32_t*>(dist()) + vidx, nd);
            return true;
        } else if (PRED == 1) {
            const unsigned long long cand = ((unsigned long long)nd << 32) | u;
            if (cand >= (unsigned long long)cur) return false;
            red_min(reinterpret_cast<unsigned long long*>(dist()) + vidx, cand);
            return (uint32_t)((unsigned long long)cur >> 32) > nd;
        } else {
            unsigned long long* p = reinterpret_cast<unsigned long long*>(dist()) + vidx;
            const unsigned long long cand = ((unsigned long long)nd << 32) | u;
            unsigned long long c = (unsigned long long)cur;
            while ((uint32_t)(c >> 32) > nd) {
                const unsigned long long old = atomicCAS(p, c, cand);
                if (old == c) return true;
                c = old;
            }
            return false;
        }
    }

    // route the improved elements of one round: writes through light arcs
    // (w <= near_w, the light/heavy split of delta-stepping) go to L0, the
    // others to the far staging and then their L2 bucket
    // `front` bounds what stays local: a light-arc write whose distance is
    // beyond the window front (W + F) * delta belongs to a later bucket and
    // goes to L2 like a heavy one (delta-stepping relaxes light arcs within
    // the current bucket only).  With admission offsets (serving) front is a
    // bucket, otherwise a distance.
    // n_imp / n_mark: per-batch counts of improvements and of improvements not
    // queued (pending marks), added to the statistics once per batch
    __device__ __forceinline__ void push_round(bool imp, uint32_t key, uint32_t nd, uint32_t w, uint32_t front,
                                               uint32_t& n_imp, uint32_t& n_mark) {
        n_imp += (uint32_t)__popc(__ballot_sync(kFull, imp));
        if (X && P.pend) {
            // an improved vertex already queued at an earlier-or-equal bucket
            // is not queued again: its queued element is relaxed with the
            // distance current when it is read
            bool q = false;
            if (imp) {
                const uint32_t b = abs_bucket(key, nd);
                q = atom_min_release(P.pend + dist_index(key), b) > b;
            }
            n_mark += (uint32_t)__popc(__ballot_sync(kFull, imp && !q));
            imp = q;
        }
        if (X && P.dedup) {
            // in-warp duplicates (Listing 1's write of a warp's improved
            // vertices): lanes whose arcs improved the same target this round
            // are matched; one write per target is enough, the one with the
            // smallest distance (ties: lowest lane) -- the others carry larger
            // or equal distances and would be dropped as stale when read
            const unsigned long long mk = imp ? (unsigned long long)key : (0x100000000ull | lane);
            const uint32_t grp = __match_any_sync(kFull, mk);
            const bool dup = imp && (grp & (grp - 1u)) != 0u;
            const uint32_t dm = __ballot_sync(kFull, dup);
            if (dm) {
                stat(kStDup, (unsigned long long)__popc(dm));
                const uint32_t mn = __reduce_min_sync(grp, imp ? nd : 0xffffffffu);
                const uint32_t at_min = __ballot_sync(kFull, imp && nd == mn) & grp;
                if (dup && lane != (uint32_t)(__ffs(at_min) - 1)) imp = false;
            }
        }
        // a shadow vertex (a slice of a hub's arcs) always goes to L2 so that
        // the slices of one hub spread over all blocks
        const bool inside = MQ && P.qoff ? abs_bucket(key, nd) <= front : nd <= front;
        const bool nearv = imp && (!X || !P.l2_only) && w <= P.near_w && inside && key_vertex(key) < (uint32_t)P.n;
        const uint32_t m = __ballot_sync(kFull, nearv);
        if (m) {
            if (nearv) scratch()[__popc(m & lanemask_lt())] = make_uint2(key, nd);
            __syncwarp();
            l0_push(__popc(m));
        }
        far_push(imp && !nearv, make_uint2(key, nd));
    }

    // One lane's arc of a relaxation round: the adjacency entry (col,
    // weight bits) and its source's distance, query and predecessor id.
    struct RoundIn {
        uint2 a;
        uint32_t du, q, pu;
        bool in;
    };

    // Arc g = g0 + lane of the batch's concatenated adjacency: its owner
    // is the largest lane j with ex[j] <= g; issues the adjacency load.
    __device__ __forceinline__ RoundIn round_in(int32_t g0, int32_t total, int32_t ex, int32_t rs, uint32_t du,
                                                uint32_t myq, uint32_t pu) const {
        RoundIn r;
        const int32_t g = g0 + (int32_t)lane;
        int j = 0;
#pragma unroll
        for (int s = 16; s >= 1; s >>= 1) {
            int32_t t = __shfl_sync(kFull, ex, j + s);
            if (t <= g) j += s;
        }
        const int32_t oex = __shfl_sync(kFull, ex, j);
        const int32_t ors = __shfl_sync(kFull, rs, j);
        r.du = __shfl_sync(kFull, du, j);
        r.q = MQ ? __shfl_sync(kFull, myq, j) : 0u;
        r.pu = PRED != 0 ? __shfl_sync(kFull, pu, j) : 0u;
        r.in = g < total;
        r.a = r.in ? ld_arc(P.adj + (ors + (g - oex))) : make_uint2(0u, 0u);
        if (P.unit_w) r.a.y = r.a.x >= (uint32_t)P.n ? 0u : 1u;
        return r;
    }

    // Relaxes a batch of up to 32 vertices (one per lane).  Stale elements are
    // dropped (Listing 2: u.dist > dist[u]); the arcs are spread evenly over
    // the lanes by a warp prefix sum over degrees (Section 4.1 hybrid load
    // balancing: a high-degree vertex is scanned by the whole warp, low-degree
    // vertices' arcs are packed together).  Vertices whose arcs start beyond
    // max_arcs go back to L0 for the next batch.  Returns the number of
    // elements consumed.
    __device__ int relax_batch(bool valid, uint2 el) {
#if SSSP_FINE_CYCLES
        const long long cb0 = clock64();
#endif
        uint32_t key = el.x, du = el.y;
        int32_t rs = 0, deg = 0;
        bool stale = false;
        if (valid && (key_vertex(key) >= (uint32_t)P.nv || key_query(key) >= (uint32_t)P.nq)) {
            raise_error(P.ctrl, kErrElement, 8, (int)key);
            valid = false;
        }
        if (X && valid && P.pend) {
            // pending marks: the read takes the vertex's mark; a mark already
            // taken by an earlier read means no improvement since that read's
            // relaxation, so the element is stale.  Otherwise the arcs are
            // relaxed from the current distance (never above the element's).
            const uint32_t v = key_vertex(key);
            const int32_t r0 = ld_row(P.row_ptr + v), r1 = ld_row(P.row_ptr + v + 1);
            const uint32_t mark = atom_exch_acquire(P.pend + dist_index(key), kInfU32);
            if (mark == kInfU32) {
                valid = false;
                stale = true;
            } else {
                du = dpart(ld_dist(dist() + dist_index(key)));
                el.y = du;
                rs = r0;
                deg = r1 - r0;
            }
        } else if (valid) {
#if SSSP_SPEC_ROW
            // the row offsets are loaded alongside the distance (one memory
            // round trip instead of two); a stale vertex ignores them
            const uint32_t v = key_vertex(key);
            const uint32_t cur = dpart(ld_dist(dist() + dist_index(key)));
            const int32_t r0 = ld_row(P.row_ptr + v), r1 = ld_row(P.row_ptr + v + 1);
            if (du > cur) {
                valid = false;
                stale = true;
            } else {
                rs = r0;
                deg = r1 - r0;
            }
#else
            uint32_t cur = dpart(ld_dist(dist() + dist_index(key)));
            if (du > cur) {
                valid = false;
                stale = true;
            } else {
                uint32_t v = key_vertex(key);
                rs = ld_row(P.row_ptr + v);
                deg = ld_row(P.row_ptr + v + 1) - rs;
#if SSSP_SHADOW_OWNER
                if (v >= (uint32_t)P.n) {
                    // a hub slice: when the hub has improved since the slice was
                    // queued, relax from the hub's current distance and give the
                    // slice that distance, so the hub's next relaxation of its
                    // zero-weight links finds nothing to improve and queues no
                    // second copy of the slice
                    const uint32_t ow = (uint32_t)__ldg(P.owner + (v - (uint32_t)P.n));
                    const size_t oidx = MQ ? (size_t)key_query(key) * (size_t)P.nv + ow : (size_t)ow;
                    const uint32_t dO = dpart(ld_dist(dist() + oidx));
                    if (dO < du) {
                        du = dO;
                        el.y = dO;
                        if (PRED == 0)
                            red_min(reinterpret_cast<uint32_t*>(dist()) + dist_index(key), dO);
                        else
                            red_min(reinterpret_cast<unsigned long long*>(dist()) + dist_index(key),
                                    ((unsigned long long)dO << 32) | ow);
                    }
                }
#endif
            }
#endif
        }
        int consumed = __popc(__ballot_sync(kFull, valid || stale));
        stat(kStStale, (unsigned long long)(__popc(__ballot_sync(kFull, stale))));
        // exclusive prefix sum of degrees
        int32_t incl = deg;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t x = __shfl_up_sync(kFull, incl, o);
            if (lane >= (uint32_t)o) incl += x;
        }
        int32_t ex = incl - deg;
        // defer vertices starting beyond max_arcs (never the first one)
        const bool defer = valid && ex >= P.max_arcs;
        const uint32_t dm = __ballot_sync(kFull, defer);
        if (dm) {
            // a deferred vertex is queued again (in L0): it gets its mark back
            if (X && defer && P.pend) atomicMin(P.pend + dist_index(key), abs_bucket(key, el.y));
            if (defer) scratch()[__popc(dm & lanemask_lt())] = el;
            __syncwarp();
            l0_push(__popc(dm), true);
            consumed -= __popc(dm);
            stat(kStDeferred, (unsigned long long)(__popc(dm)));
            if (defer) {
                valid = false;
                deg = 0;
            }
            incl = deg;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int32_t x = __shfl_up_sync(kFull, incl, o);
                if (lane >= (uint32_t)o) incl += x;
            }
            ex = incl - deg;
        }
        const int32_t total = __shfl_sync(kFull, incl, 31);
        const uint32_t myq = MQ ? key_query(key) : 0u;
        // the window front for this batch (see push_round); no bound when
        // every write is local (near_deltas = 0, as in Listing 1)
        uint32_t front = kInfU32;
        if (SSSP_FRONT_BOUND && P.near_w != kInfU32) {
            const uint32_t W = window_hint();
            front = MQ && P.qoff ? W + (uint32_t)P.filter_deltas : A::upper(W, P.delta, P.filter_deltas);
        }
        // predecessor id: a shadow vertex stands for its owner
        uint32_t pu = 0;
        if (PRED != 0 && valid) {
            uint32_t v = key_vertex(key);
            pu = v < (uint32_t)P.n ? v : (uint32_t)__ldg(P.owner + (v - (uint32_t)P.n));
        }
        stat(kStRelax, (unsigned long long)((uint32_t)total));
#if SSSP_FINE_CYCLES
        stat(kCyBatch, (unsigned long long)(clock64() - cb0));
#endif
        {
            const int32_t sh = valid && key_vertex(key) >= (uint32_t)P.n ? deg : 0;
            const int32_t shs = __reduce_add_sync(kFull, (uint32_t)sh);
            if (shs) stat(kStRelaxShadow, (unsigned long long)shs);
        }
        uint32_t n_imp = 0, n_mark = 0, n_rounds = 0;
#if SSSP_PIPELINE
        // the next round's arcs are loaded while this round's distances are
        RoundIn nx = round_in(0, total, ex, rs, du, myq, pu);
#endif
        for (int32_t g0 = 0; g0 < total; g0 += 32) {
            if (g0 && (g0 & 4095) == 0) {
                int stop = 0;
                if (lane == 0) stop = expired() || ld_volatile_int(&P.ctrl->error) != 0;
                if (__shfl_sync(kFull, stop, 0)) break;
            }
#if SSSP_FINE_CYCLES
            const long long cr0 = clock64();
#endif
#if SSSP_PIPELINE
            const RoundIn cu = nx;
            if (g0 + 32 < total) nx = round_in(g0 + 32, total, ex, rs, du, myq, pu);
#else
            const RoundIn cu = round_in(g0, total, ex, rs, du, myq, pu);
#endif
            uint32_t nd = 0;
            bool imp = false;
            if (cu.in) {
                const size_t vidx = MQ ? (size_t)cu.q * (size_t)P.nv + cu.a.x : (size_t)cu.a.x;
                imp = relax_cur(vidx, cu.pu, cu.du, cu.a.y, ld_dist(dist() + vidx), nd);
            }
#if SSSP_FINE_CYCLES
            const long long cr1 = clock64();
            stat(kCyRound, (unsigned long long)__shfl_sync(kFull, (unsigned long long)(cr1 - cr0), 0));
#endif
            push_round(imp, MQ ? ((cu.q << P.vbits) | cu.a.x) : cu.a.x, nd, cu.a.y, front, n_imp, n_mark);
            n_rounds++;
#if SSSP_FINE_CYCLES
            stat(kCyPush, (unsigned long long)(clock64() - cr1));
#endif
        }
        stat(kStRounds, n_rounds);
        stat(kStImproved, n_imp);
        if (n_mark) stat(kStMarked, n_mark);
        return consumed;
    }

    __device__ __noinline__ void publish_stats() {
        if (lane == 0) {
            for (int i = 0; i < kStCount; i++)
                if (sst()[i]) atomicAdd(&P.ctrl->stats[i], sst()[i]);
        }
    }

    // ---- run-time sampling ----------------------------------------------------
    __device__ __noinline__ void sample() {
        const unsigned long long now = gtime();
        BlockShared* B = S();
        if (now < B->next_sample || B->nsamples >= (uint32_t)P.timeline_cap) return;
        B->next_sample = now + P.timeline_ns;
        unsigned long long* o = P.timeline + (size_t)B->nsamples * kTimelineFields;
        o[0] = now - B->t0;
        o[2] = ld_acquire64(&P.ctrl->done);      // done before reserve: done <= reserve
        o[1] = ld_acquire64(&P.ctrl->reserve);
        o[3] = ld_acquire64(&P.ctrl->processed);
        o[4] = ld_acquire64(&P.ctrl->window);
        o[5] = *(volatile uint32_t*)&B->busy;
        B->nsamples++;
    }

    // ---- the worker loop (Listing 2, work_kernel) ---------------------------
    __device__ void run() {
        uint32_t idle_ns = 0;
        uint32_t iter = 0;
        for (;;) {
            mark(1, iter);
            stat(kStIter, 1);
            if (X && P.timeline && blockIdx.x == 0 && threadIdx.x == 0) sample();
            if ((++iter & 7u) == 0 || idle_ns || P.slice_ns) {
                int stop = 0;
                if (lane == 0) {
                    stop = aborted();
                    if (!stop && expired()) {
                        raise_error(P.ctrl, kErrTimeout, 7, 0);
                        stop = 1;
                    }
                    if (!stop && gtime() > S()->slice_end) stop = 2;  // end of a serving slice
                }
                stop = __shfl_sync(kFull, stop, 0);
                if (stop) break;
            }
            bool valid = false;
            uint2 e = make_uint2(0, 0);
            bool got = false;
            const long long c0 = clock64();
            got = l0_read(valid, e);
            const long long c1 = clock64();
            stat(kCyL0, (unsigned long long)((unsigned long long)(c1 - c0)));
            if (!got) got = l1_read(valid, e);
            if (SSSP_CHUNK_DESC && !got) got = desc_read(valid, e);
            const long long c2 = clock64();
            int rf = 1;
            if (!got) {
                // local levels are empty: hand the far staging to L2 first
                if (nfar) {
                    far_flush(0);
                    acct_apply();
                }
                rf = refill(valid, e);
                got = rf == 1;
            }
            const long long c3 = clock64();
            stat(kCyGlobalRead, (unsigned long long)((unsigned long long)(c3 - c2)));
            if (!got) {
                if (rf == 2) continue;  // L1 received elements
                if (rf == 0) {
                    // nothing in L2 for this block: publish everything it staged
                    stage_flush(true);
                    acct_apply();
                }
                mark(9, iter);
                int fin = 0;
                if (rf == 0 && lane == 0) {
                    // L2 looked empty to this block's refiller: test termination
                    unsigned long long d = ld_acquire64(&P.ctrl->done);
                    unsigned long long r = ld_acquire64(&P.ctrl->reserve);
                    if (d == r) {
                        atomicExch(&P.ctrl->finished, 1);
                        fin = 1;
                    }
                }
                fin = __shfl_sync(kFull, fin, 0);
                if (fin) break;
                stat(kStIdleIter, 1);
                idle_ns = idle_ns ? min(idle_ns * 2u, 1024u) : 64u;
                __nanosleep(idle_ns);
                stat(kCyIdle, (unsigned long long)((unsigned long long)(clock64() - c3)));
                continue;
            }
            idle_ns = 0;
            mark(7, iter);
            if (X && P.timeline) {
                // run-time sampling only: the batch's elements, and block 0's busy warps
                const uint32_t nb = (uint32_t)__popc(__ballot_sync(kFull, valid));
                if (lane == 0) atomicAdd(&P.ctrl->processed, (unsigned long long)nb);
                if (blockIdx.x == 0 && lane == 0) atomicAdd(&S()->busy, 1u);
            }
            dec += relax_batch(valid, e);
            if (X && P.timeline && blockIdx.x == 0 && lane == 0) atomicSub(&S()->busy, 1u);
            stat(kCyRelax, (unsigned long long)((unsigned long long)(clock64() - c3)));
            mark(10, iter);
            acct_apply();
        }
        mark(13, iter);
        drain_warp();
        publish_stats();
    }

    // End of a launch: move everything this warp holds (L0, far staging) to
    // L2.  After a normal termination there is nothing left and this is a
    // no-op; at the end of a serving slice the work continues from L2 in the
    // next launch.
    __device__ __noinline__ void drain_warp() {
        if (ld_volatile_int(&P.ctrl->error) != 0) return;
        const uint32_t len = l0t - l0h;
        if (len) {
#pragma unroll
            for (int r = 0; r < R; r++) {
                const uint32_t want = 32u * (uint32_t)r + lane;
                const uint32_t p = l0h + ((want - l0h) & (32u * R - 1u));
                dec += l2_write((p - l0h) < len, l0[r]);
            }
            l0h = l0t = 0;
        }
        if (nfar) far_flush(0);
        acct_apply();
    }

    // End of a launch, one warp per block after every warp drained: move L1
    // and the block staging to L2, then publish the block's count.
    __device__ __noinline__ void drain_block() {
        if (ld_volatile_int(&P.ctrl->error) != 0) return;
        if (SSSP_CHUNK_DESC) {
            // claimed chunks not read yet go back to L2
            bool v = false;
            uint2 x = make_uint2(0, 0);
            while (desc_read(v, x)) {
                dec += l2_write(v, x);
                if (ld_volatile_int(&P.ctrl->error) != 0) return;
            }
        }
        if (l1_lockfree()) {
            bool v = false;
            uint2 x = make_uint2(0, 0);
            while (l1_read_lf(v, x)) dec += l2_write(v, x);
        } else if (lock()) {
            if (P.l1_type == 1) {
                const uint32_t half = (uint32_t)P.l1_cap >> 1;
                for (int rg = 0; rg < 2; rg++) {
                    uint32_t* hp = rg ? &S()->fhead : &S()->head;
                    uint32_t* tp = rg ? &S()->ftail : &S()->tail;
                    uint32_t h = sread(hp), t = sread(tp);
                    while (h != t) {
                        const uint32_t c = t - h < 32u ? t - h : 32u;
                        const bool v = lane < c;
                        uint2 x = make_uint2(0, 0);
                        if (v) x = vld(&L1()[(rg ? half : 0u) + ((h + lane) & (half - 1u))]);
                        h += c;
                        dec += l2_write(v, x);
                    }
                    if (lane == 0) *(volatile uint32_t*)hp = h;
                    __syncwarp();
                }
            } else {
                uint32_t h = sread(&S()->head), t = sread(&S()->tail);
                while (h != t) {
                    const uint32_t c = t - h < 32u ? t - h : 32u;
                    const bool v = lane < c;
                    uint2 x = make_uint2(0, 0);
                    if (v) x = vld(&L1()[(h + lane) & l1_mask()]);
                    h += c;
                    dec += l2_write(v, x);
                }
                if (lane == 0) *(volatile uint32_t*)&S()->head = h;
                __syncwarp();
            }
            unlock();
        }
        stage_flush(true);
        acct_apply();
        if (lane == 0) {
            // nothing may stay behind in the block: its count must be zero,
            // and the L2 reads it finished are published to ctrl.done
            const unsigned long long v = *(volatile unsigned long long*)&S()->acct;
            if ((uint32_t)(v >> 32) != 0u) raise_error(P.ctrl, kErrState, 9, (int)(v >> 32));
            else try_flush();
        }
        __syncwarp();
    }
};

// The parameters are a grid constant (no local copy is made when their
// address is taken); the prologue copies them to shared memory, from where
// the workers read them: with a local copy every field read was a
// local-memory load, and through the grid constant the out-of-line queue
// functions read them with generic loads.
// X: the extended kernel, with the optional paths (pending marks, the
// in-warp duplicate filter, the single-queue baseline, run-time sampling,
// the debug trace, the L1 policies with a block lock).  X = false compiles
// them out: a smaller kernel, which runs every configuration that uses none
// of them.
template <int WT, int PRED, bool MQ, int R, bool X>
#ifndef SSSP_LB_THREADS
#define SSSP_LB_THREADS 1024
#endif
#ifndef SSSP_LB_MIN_BLOCKS
#define SSSP_LB_MIN_BLOCKS 1
#endif
__global__ void __launch_bounds__(SSSP_LB_THREADS, SSSP_LB_MIN_BLOCKS) mlmq_kernel(const __grid_constant__ KParams P) {
    BlockShared* S = reinterpret_cast<BlockShared*>(mlmq_smem);
    volatile uint2* l1 = reinterpret_cast<volatile uint2*>(mlmq_smem + P.l1_off);
    if (threadIdx.x == 0) {
        S->lock = 0;
        S->slock = 0;
        S->refill = 0;
        S->head = S->tail = S->fhead = S->ftail = 0;
        S->writes = 0;
        S->acct = 0ull;
        for (int i = 0; i < 32; i++) S->scnt[i] = S->shead[i] = 0;
        unsigned long long win = ld_acquire64(&P.ctrl->window);
        S->nf = Arith<WT>::upper((uint32_t)win, P.delta, 1.0f);
        S->wcache = (uint32_t)win;
        S->dhead = S->dtail = 0;
        for (int i = 0; i < kDescCap; i++) S->desc[i] = kEmptySlot;
        S->deadline = gtime() + P.timeout_ns;
        S->t0 = gtime();
        S->next_sample = 0;
        S->nsamples = 0;
        S->busy = 0;
        S->slice_end = ~0ull;
        if (P.slice_ns) {
            // the first block to start fixes the slice's end for all blocks
            const unsigned long long mine = gtime() + P.slice_ns;
            const unsigned long long prev = atomicCAS(&P.ctrl->slice_end, 0ull, mine);
            S->slice_end = prev ? prev : mine;
        }
    }
    for (int i = threadIdx.x; i < P.l1_cap; i += blockDim.x) vst(l1 + i, make_uint2(kEmptyKey, 0u));
    if (SSSP_LF_STAGE && P.stage) {
        volatile uint2* st = reinterpret_cast<volatile uint2*>(mlmq_smem + P.stage_off);
        for (int i = threadIdx.x; i < P.bmax * kStageCap; i += blockDim.x) vst(st + i, make_uint2(kEmptyKey, 0u));
    }
    {
        const uint32_t* src = reinterpret_cast<const uint32_t*>(&P);
        uint32_t* dst = reinterpret_cast<uint32_t*>(&S->params);
        for (int i = threadIdx.x; i < (int)(sizeof(KParams) / 4); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    Worker<WT, PRED, MQ, R, X> w(S->params);
    w.run();
    if (P.slice_ns) {
        // serving slice: every warp has drained its private state; one warp
        // now drains what the block shares
        __syncthreads();
        if ((threadIdx.x >> 5) == 0) w.drain_block();
    }
}

}  // namespace sssp
