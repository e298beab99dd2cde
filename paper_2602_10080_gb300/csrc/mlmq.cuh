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
//   L1  per thread block, in shared memory, behind a warp-granular lock:
//       Vector / Near-far / Filter / SLF policies (Section 3.4, Fig. 7).
//   L2  whole grid, in global memory: bmax circular delta-buckets
//       (Section 4.2, "L2 Bucket queue"), each a ring of 32-element chunks
//       moved with ONE atomic per chunk (Section 4.2, "L2 FIFO queue",
//       Listing 3), plus a ring of arc-range tasks for very high degree
//       vertices (the load balancing of Section 4.1, widened across warps).
//
// Spill and refill follow the cache-like collaboration of Section 3.2: the
// worker touches L0; an empty level refills from the next one down, a full
// level writes back to it.
//
// Termination (Section 4.1, delayed counting): every element written to L2
// (or the task ring) first adds to ctrl.reserve; elements read from L2 are
// counted in the block's `acct` word, whose high half counts elements the
// block holds (L0 + L1 + in flight) and whose low half counts L2 reads not
// yet published.  When the high half reaches zero the low half is added to
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
constexpr uint32_t kInfU32 = 0xffffffffu;
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
    kStPopL0 = 0, kStPopL1, kStPopL2, kStPopHeavy, kStRelax, kStImproved, kStStale,
    kStChunks, kStFlush, kStTasks, kStCount
};

struct __align__(128) Ctrl {
    unsigned long long reserve;          // elements ever written to L2 / tasks
    unsigned long long pad0[15];
    unsigned long long done;             // elements read from L2 whose work completed
    unsigned long long pad1[15];
    unsigned long long window;           // (bucket index << 32) | base distance bits
    unsigned long long pad2[15];
    int finished;
    int error;
    int err_where;
    int err_info;
    int pad3[28];
    unsigned long long stats[16];
};

// A set of rings: bucket b uses rt[b * 32], wt[b * 32] (own 128-byte line),
// seq/cnt[b * nch + s], data[(b * nch + s) * kChunk + i].
struct Rings {
    uint32_t* rt;
    uint32_t* wt;
    uint32_t* seq;
    uint32_t* cnt;
    uint2* data;
    uint32_t nch;      // chunks per ring (power of two)
    uint32_t margin;   // free chunks that must remain before a writer may take a ticket
};

// Arc-range task ring (one task per slot): (key, dist, arc_lo, arc_hi).
struct TaskRing {
    uint32_t* rt;
    uint32_t* wt;
    uint32_t* seq;
    uint4* data;
    uint32_t nslot;    // power of two
    uint32_t margin;
};

struct KParams {
    const int32_t* row_ptr;
    const uint2* adj;        // (col, weight bits) per arc
    int32_t n;
    void* dist;              // uint32_t[nq * n] or unsigned long long[nq * n]
    int32_t nq;              // number of queries (dist slices)
    int32_t vbits;           // multi-query: key = (query << vbits) | v
    uint32_t vmask;
    Rings l2;
    TaskRing hv;
    Ctrl* ctrl;
    uint32_t delta;          // u32 width, or f32 bits
    int32_t bnum, bmax;        // bmax <= 32
    int32_t l1_type, l1_cap, wb;
    float filter_deltas;
    int32_t th_heavy, split;
    int32_t l1_off;          // byte offset of the L1 buffer in dynamic shared memory
    unsigned long long timeout_ns;
    unsigned long long* trace;   // debug only: per-warp (location << 48 | iteration), mapped host memory
};

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
__device__ __forceinline__ unsigned long long ld_relaxed64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
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

// Ticket w is ahead of ticket r (wrap-safe): some writer holds ticket r.
// Any observed w with w - r > 0 proves ticket r was taken, whatever the order
// in which the two relaxed loads were performed.
__device__ __forceinline__ bool ahead(uint32_t w, uint32_t r) { return (int32_t)(w - r) > 0; }

// relaxed L2 load of a distance word (bypasses L1 so the filter sees recent values)
__device__ __forceinline__ uint32_t ld_dist(const uint32_t* p) { return __ldcg(p); }
__device__ __forceinline__ unsigned long long ld_dist(const unsigned long long* p) { return __ldcg(p); }

// ------------------------------------------------------------ arithmetic --

template <int WT> struct Arith;

// u32 lengths: saturating add (never wraps; 0xFFFFFFFF stays "unreachable").
template <> struct Arith<0> {
    static __device__ __forceinline__ uint32_t add(uint32_t d, uint32_t w) {
        uint32_t s = d + w;
        return (s < d || s == kInfU32) ? kSatU32 : s;
    }
    // bucket offset of distance d from the window base (0 .. bmax-1)
    static __device__ __forceinline__ uint32_t offset(uint32_t d, uint32_t base, uint32_t delta,
                                                      uint32_t last) {
        if (d <= base) return 0;
        uint32_t q = (d - base) / delta;
        return q < last ? q : last;
    }
    static __device__ __forceinline__ uint32_t advance(uint32_t base, uint32_t delta, uint32_t k) {
        unsigned long long b = (unsigned long long)base + (unsigned long long)delta * k;
        return b > kSatU32 ? kSatU32 : (uint32_t)b;
    }
    static __device__ __forceinline__ uint32_t upper(uint32_t base, uint32_t delta, float mult) {
        unsigned long long b = (unsigned long long)base + (unsigned long long)((double)delta * mult);
        return b > kSatU32 ? kSatU32 : (uint32_t)b;
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
    static __device__ __forceinline__ uint32_t offset(uint32_t d, uint32_t base, uint32_t delta,
                                                      uint32_t last) {
        float x = (__uint_as_float(d) - __uint_as_float(base)) / __uint_as_float(delta);
        if (!(x > 0.0f)) return 0;
        if (x >= (float)last) return last;
        return (uint32_t)x;
    }
    static __device__ __forceinline__ uint32_t advance(uint32_t base, uint32_t delta, uint32_t k) {
        return __float_as_uint(__uint_as_float(base) + __uint_as_float(delta) * (float)k);
    }
    static __device__ __forceinline__ uint32_t upper(uint32_t base, uint32_t delta, float mult) {
        return __float_as_uint(__uint_as_float(base) + __uint_as_float(delta) * mult);
    }
    static __device__ __forceinline__ uint32_t plus_delta(uint32_t d, uint32_t delta) {
        return __float_as_uint(__uint_as_float(d) + __uint_as_float(delta));
    }
};

// ------------------------------------------------------ block shared state --

struct BlockShared {
    int lock;
    uint32_t head, tail;          // L1 ring (V, FQ, SLF) or the near ring (NF)
    uint32_t fhead, ftail;        // NF far ring
    uint32_t nf;                  // NF threshold (distance bits)
    uint32_t writes;              // L1 write calls (periodic flush)
    uint32_t pad;
    unsigned long long acct;      // (held elements << 32) | unpublished L2 reads
};

// ------------------------------------------------------------- watchdog --

__device__ __forceinline__ void raise_error(Ctrl* C, int code, int where, int info) {
    if (atomicCAS(&C->error, 0, code) == 0) {
        C->err_where = where;
        C->err_info = info;
    }
    __threadfence();
}

// ---------------------------------------------------------------- kernel --

template <int WT, int PRED, bool MQ, int R>
struct Worker {
    // PRED: 0 = distances only (uint32 words), 1 = (dist, pred) words with the
    // smallest-index tight predecessor, 2 = (dist, pred) words set only on a
    // strict improvement.
    using DistT = typename std::conditional<PRED == 0, uint32_t, unsigned long long>::type;
    using A = Arith<WT>;

    const KParams& P;
    BlockShared* S;
    uint2* scratch;               // this warp's 32-element staging area
    volatile uint2* L1;           // block L1 buffer
    DistT* dist;
    uint32_t lane;
    unsigned long long deadline;

    // L0 ring
    uint2 l0[R];
    uint32_t l0h, l0t;
    // deferred accounting (see acct_apply)
    int unc;                      // L0 pushes not yet counted in S->acct
    int dec;                      // completed / exported elements not yet subtracted
    // statistics (per warp)
    uint32_t st[kStCount];

    __device__ Worker(const KParams& p, BlockShared* s, uint2* scr, uint2* l1, unsigned long long dl)
        : P(p), S(s), scratch(scr), L1(l1), dist(reinterpret_cast<DistT*>(p.dist)),
          lane(lane_id()), deadline(dl), l0h(0), l0t(0), unc(0), dec(0) {
#pragma unroll
        for (int i = 0; i < kStCount; i++) st[i] = 0;
#pragma unroll
        for (int r = 0; r < R; r++) l0[r] = make_uint2(0, 0);
    }

    __device__ __forceinline__ bool expired() const { return gtime() > deadline; }

    __device__ __forceinline__ bool aborted() const {
        return ld_volatile_int(&P.ctrl->error) != 0 || ld_volatile_int(&P.ctrl->finished) != 0;
    }

    // debug trace of where this warp is (no-op unless P.trace is set)
    __device__ __forceinline__ void mark(uint32_t code, uint32_t iter = 0) const {
        if (P.trace) {
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
        return MQ ? (size_t)key_query(key) * (size_t)P.n + key_vertex(key) : (size_t)key;
    }
    static __device__ __forceinline__ uint32_t dpart(uint32_t w) { return w; }
    static __device__ __forceinline__ uint32_t dpart(unsigned long long w) { return (uint32_t)(w >> 32); }

    // ---- block accounting -----------------------------------------------
    // Increments (elements becoming visible to other warps) are applied before
    // the elements can be seen; decrements may be deferred.  When the held
    // count reaches zero, the unpublished L2 reads are added to ctrl.done.
    __device__ void try_flush() {
        unsigned long long v = *(volatile unsigned long long*)&S->acct;
        while ((uint32_t)(v >> 32) == 0u && (uint32_t)v != 0u) {
            unsigned long long old = atomicCAS(&S->acct, v, 0ull);
            if (old == v) {
                __threadfence();
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
            __threadfence();
            unsigned long long add = ((unsigned long long)(uint32_t)delta) << 32;
            unsigned long long old = atomicAdd(&S->acct, add);
            if ((uint32_t)(old >> 32) + (uint32_t)delta == 0u) try_flush();
        }
        __syncwarp();
    }

    // warp-uniform read of a shared-memory word: lane 0 reads, all lanes get
    // the same value (control flow that depends on it stays convergent)
    __device__ __forceinline__ uint32_t sread(const uint32_t* p) const {
        uint32_t v = 0;
        if (lane == 0) v = *(const volatile uint32_t*)p;
        return __shfl_sync(kFull, v, 0);
    }

    // ---- L1 lock -----------------------------------------------------------
    __device__ bool lock() {
        int ok = 1;
        mark(2);
        if (lane == 0) {
            uint32_t spins = 0;
            while (atomicCAS(&S->lock, 0, 1) != 0) {
                if ((++spins & 1023u) == 0 && expired()) {
                    raise_error(P.ctrl, kErrTimeout, 1, 0);
                    ok = 0;
                    break;
                }
                __nanosleep(20);
            }
        }
        mark(42);
        ok = __shfl_sync(kFull, ok, 0);
        mark(43);
        __threadfence_block();
        return ok != 0;
    }
    __device__ void unlock() {
        __threadfence_block();
        __syncwarp();
        if (lane == 0) atomicExch(&S->lock, 0);
        __syncwarp();
    }

    // ---- L2: bucket rings -------------------------------------------------
    __device__ __forceinline__ unsigned long long window() const {
        return ld_acquire64(&P.ctrl->window);
    }

    // Writes the valid lanes' elements to the L2 bucket of their distance.
    // Lanes are grouped per bucket with __match_any_sync; each group fills
    // one chunk with a single ticket (atomicAdd) on that bucket's ring.
    // ctrl.reserve grows BEFORE any chunk is published.  Returns the number
    // of elements written (warp-uniform); the caller defers the decrement.
    __device__ int l2_write(bool valid, uint2 e) {
        uint32_t vm = __ballot_sync(kFull, valid);
        if (vm == 0) return 0;
        int total = __popc(vm);
        unsigned long long win = 0;
        if (lane == 0) {
            atomicAdd(&P.ctrl->reserve, (unsigned long long)total);
            win = window();
        }
        win = __shfl_sync(kFull, win, 0);
        const uint32_t cur = (uint32_t)(win >> 32), base = (uint32_t)win;
        const uint32_t last = (uint32_t)P.bmax - 1u;
        uint32_t off = valid ? A::offset(e.y, base, P.delta, last) : 0u;
        uint32_t b = (cur + off) % (uint32_t)P.bmax;
        uint32_t pending = vm;
        while (pending) {
            int leader = __ffs(pending) - 1;
            uint32_t bl = __shfl_sync(kFull, b, leader);
            uint32_t grp = __ballot_sync(kFull, valid && b == bl) & pending;
            uint32_t t = 0, bucket = bl;
            int okw = 1;
            if (lane == (uint32_t)leader) {
                // take a ticket on the first ring (from bl towards the window end)
                // that still has `margin` free chunks; diverting an element to a
                // later bucket only delays it (results are order independent).
                uint32_t tries = 0;
                for (;;) {
                    uint32_t* wtp = P.l2.wt + (size_t)bucket * 32;
                    uint32_t* rtp = P.l2.rt + (size_t)bucket * 32;
                    // read r before w (acquire) so w - r over-estimates the occupancy
                    uint32_t r0 = ld_acquire(rtp);
                    uint32_t w0 = ld_relaxed(wtp);
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
                }
                mark(3);
                if (okw) {
                    // wait until the chunk slot of ticket t is free (normally immediate)
                    uint32_t* sp = P.l2.seq + (size_t)bucket * P.l2.nch + (t & (P.l2.nch - 1u));
                    uint32_t spins = 0;
                    while (ld_acquire(sp) != t) {
                        if ((++spins & 255u) == 0 && expired()) {
                            raise_error(P.ctrl, kErrTimeout, 3, (int)bucket);
                            okw = 0;
                            break;
                        }
                        __nanosleep(32);
                    }
                }
            }
            okw = __shfl_sync(kFull, okw, leader);
            if (!okw) return total;
            t = __shfl_sync(kFull, t, leader);
            bucket = __shfl_sync(kFull, bucket, leader);
            const size_t slot = (size_t)bucket * P.l2.nch + (t & (P.l2.nch - 1u));
            if (grp & (1u << lane)) {
                int rank = __popc(grp & lanemask_lt());
                P.l2.data[slot * kChunk + rank] = e;
            }
            __syncwarp();
            if (lane == (uint32_t)leader) {
                P.l2.cnt[slot] = (uint32_t)__popc(grp);
                __threadfence();
                st_release(P.l2.seq + slot, t + 1u);
            }
            st[kStChunks]++;
            pending &= ~grp;
        }
        __syncwarp();
        return total;
    }

    // Reads one chunk from the bucket queue, or one arc-range task from the
    // task ring (probed by lane 31; tasks first).  Lane i probes bucket
    // cur + i of the circular window (bmax <= 32, so one warp sees every
    // bucket in one round trip).  Readers take from the non-empty buckets
    // among the first bnum (Section 4.2, "the first bnum buckets are
    // checked"), lowest first; when the first bucket is empty the window
    // moves up to the lowest non-empty bucket ("base is increased by delta
    // when the first bucket is empty"), even if that is beyond bnum.
    // Returns 0 (nothing), 1 (chunk: elements in lanes) or 2 (task).
    __device__ int global_read(bool& valid, uint2& e, uint4& task) {
        valid = false;
        unsigned long long win = 0;
        if (lane == 0) win = window();
        win = __shfl_sync(kFull, win, 0);
        const uint32_t cur = (uint32_t)(win >> 32), base = (uint32_t)win;
        uint32_t b = (cur + lane) % (uint32_t)P.bmax;
        uint32_t r = 0, w = 0;
        bool probe = lane < (uint32_t)P.bmax;
        if (probe) {
            r = ld_relaxed(P.l2.rt + (size_t)b * 32);
            w = ld_relaxed(P.l2.wt + (size_t)b * 32);
        }
        uint32_t hr = 0, hw = 0;
        if (lane == 31 && P.hv.nslot) {
            hr = ld_relaxed(P.hv.rt);
            hw = ld_relaxed(P.hv.wt);
        }
        mark(30);
        bool have_task = __shfl_sync(kFull, ahead(hw, hr), 31);
        mark(31);
        if (have_task) {
            int got = 0;
            uint32_t t = 0;
            if (lane == 31) {
                uint32_t rr = hr;
                for (int k = 0; k < 8 && ahead(hw, rr); k++) {
                    uint32_t old = atomicCAS(P.hv.rt, rr, rr + 1u);
                    if (old == rr) { got = 1; t = rr; break; }
                    rr = old;
                    hw = ld_relaxed(P.hv.wt);
                }
                if (got) {
                    uint32_t* sp = P.hv.seq + (t & (P.hv.nslot - 1u));
                    uint32_t spins = 0;
                    while (ld_acquire(sp) != t + 1u) {
                        if ((++spins & 255u) == 0 && expired()) {
                            raise_error(P.ctrl, kErrTimeout, 4, 0);
                            got = 0;
                            break;
                        }
                        __nanosleep(32);
                    }
                    if (got) {
                        task = P.hv.data[t & (P.hv.nslot - 1u)];
                        atomicAdd(&S->acct, (1ull << 32) | 1ull);
                        __threadfence();
                        st_release(sp, t + P.hv.nslot);
                    }
                }
            }
            got = __shfl_sync(kFull, got, 31);
            if (got) {
                task.x = __shfl_sync(kFull, task.x, 31);
                task.y = __shfl_sync(kFull, task.y, 31);
                task.z = __shfl_sync(kFull, task.z, 31);
                task.w = __shfl_sync(kFull, task.w, 31);
                st[kStPopHeavy]++;
                return 2;
            }
        }
        mark(32);
        uint32_t nonempty = __ballot_sync(kFull, probe && ahead(w, r));
        mark(33);
        if (nonempty == 0) return 0;
        const int first = __ffs(nonempty) - 1;
        uint32_t cand = nonempty & (P.bnum >= 32 ? kFull : ((1u << P.bnum) - 1u));
        if (first > 0) {
            // the first bucket is empty: move the window to the lowest non-empty one
            if (lane == 0) {
                unsigned long long nw =
                    ((unsigned long long)((cur + (uint32_t)first) % (uint32_t)P.bmax) << 32) |
                    A::advance(base, P.delta, (uint32_t)first);
                atomicCAS(&P.ctrl->window, win, nw);
            }
            if (cand == 0) cand = 1u << first;
        }
        // claim a ticket in the lowest candidate bucket (CAS only while w is ahead of r)
        int got = 0;
        uint32_t t = 0, cnt = 0, bb = 0;
        while (cand) {
            int c = __ffs(cand) - 1;
            if (lane == (uint32_t)c) {
                uint32_t rr = r;
                uint32_t* rtp = P.l2.rt + (size_t)b * 32;
                for (int k = 0; k < 8 && ahead(w, rr); k++) {
                    uint32_t old = atomicCAS(rtp, rr, rr + 1u);
                    if (old == rr) { got = 1; t = rr; break; }
                    rr = old;
                    w = ld_relaxed(P.l2.wt + (size_t)b * 32);
                }
                bb = b;
            }
            got = __shfl_sync(kFull, got, c);
            if (got) {
                t = __shfl_sync(kFull, t, c);
                bb = __shfl_sync(kFull, bb, c);
                break;
            }
            cand &= ~(1u << c);
        }
        if (!got) return 0;
        const size_t slot = (size_t)bb * P.l2.nch + (t & (P.l2.nch - 1u));
        int okr = 1;
        mark(4);
        if (lane == 0) {
            uint32_t spins = 0;
            while (ld_acquire(P.l2.seq + slot) != t + 1u) {
                if ((++spins & 255u) == 0 && expired()) {
                    raise_error(P.ctrl, kErrTimeout, 5, (int)bb);
                    okr = 0;
                    break;
                }
                __nanosleep(32);
            }
            if (okr) cnt = P.l2.cnt[slot];
        }
        okr = __shfl_sync(kFull, okr, 0);
        if (!okr) return 0;
        cnt = __shfl_sync(kFull, cnt, 0);
        valid = lane < cnt;
        if (valid) e = P.l2.data[slot * kChunk + lane];
        __syncwarp();
        if (lane == 0) {
            // count the elements as held by this block BEFORE freeing the slot
            atomicAdd(&S->acct, ((unsigned long long)cnt << 32) | (unsigned long long)cnt);
            __threadfence();
            st_release(P.l2.seq + slot, t + P.l2.nch);
        }
        __syncwarp();
        st[kStPopL2]++;
        return 1;
    }

    // ---- L1 ------------------------------------------------------------------
    __device__ __forceinline__ uint32_t l1_mask() const { return (uint32_t)P.l1_cap - 1u; }

    // Places the valid elements (K per lane) into L1 under the block lock, per
    // the L1 policy; elements that do not fit or are filtered out get their
    // `out` flag set and must go to L2.  Adds `unc` (uncounted L0 pushes) to
    // the block count before the lock is released.
    template <int K>
    __device__ void l1_place(uint2 (&e)[K], bool (&valid)[K], bool (&out)[K], uint32_t fthr) {
        const int type = P.l1_type;
        const uint32_t cap = (uint32_t)P.l1_cap;
        if (type == 1) {
            // near-far: two rings of cap/2
            const uint32_t half = cap >> 1;
            uint32_t nf = sread(&S->nf);
#pragma unroll
            for (int k = 0; k < K; k++) {
                bool nearv = valid[k] && e[k].y < nf;
                bool farv = valid[k] && !nearv;
                uint32_t nm = __ballot_sync(kFull, nearv), fm = __ballot_sync(kFull, farv);
                uint32_t h = sread(&S->head), t = sread(&S->tail);
                uint32_t fh = sread(&S->fhead), ft = sread(&S->ftail);
                uint32_t nspace = half - (t - h), fspace = half - (ft - fh);
                uint32_t nr = __popc(nm & lanemask_lt()), fr = __popc(fm & lanemask_lt());
                out[k] = false;
                if (nearv) {
                    if (nr < nspace) vst(&L1[(t + nr) & (half - 1u)], e[k]);
                    else out[k] = true;
                }
                if (farv) {
                    if (fr < fspace) vst(&L1[half + ((ft + fr) & (half - 1u))], e[k]);
                    else out[k] = true;
                }
                __syncwarp();
                if (lane == 0) {
                    uint32_t nn = __popc(nm), fn = __popc(fm);
                    *(volatile uint32_t*)&S->tail = t + (nn < nspace ? nn : nspace);
                    *(volatile uint32_t*)&S->ftail = ft + (fn < fspace ? fn : fspace);
                }
                __syncwarp();
            }
        } else if (type == 3) {
            // SLF deque: dist <= head element -> push front, else push back
#pragma unroll
            for (int k = 0; k < K; k++) {
                uint32_t h = sread(&S->head), t = sread(&S->tail);
                uint32_t hd = (t != h) ? vld(&L1[h & l1_mask()]).y : 0u;
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
                    if (fr < ftake) vst(&L1[(h - 1u - fr) & l1_mask()], e[k]);
                    else out[k] = true;
                }
                if (back) {
                    if (br < btake) vst(&L1[(t + br) & l1_mask()], e[k]);
                    else out[k] = true;
                }
                __syncwarp();
                if (lane == 0) {
                    *(volatile uint32_t*)&S->head = h - ftake;
                    *(volatile uint32_t*)&S->tail = t + btake;
                }
                __syncwarp();
            }
        } else {
            // vector (type 0) / filter (type 2, keep dist <= fthr)
#pragma unroll
            for (int k = 0; k < K; k++) {
                bool want = valid[k] && (type != 2 || e[k].y <= fthr);
                uint32_t wm = __ballot_sync(kFull, want);
                uint32_t h = sread(&S->head), t = sread(&S->tail);
                uint32_t space = cap - (t - h);
                uint32_t rank = __popc(wm & lanemask_lt());
                out[k] = valid[k] && !want;
                if (want) {
                    if (rank < space) vst(&L1[(t + rank) & l1_mask()], e[k]);
                    else out[k] = true;
                }
                __syncwarp();
                if (lane == 0) {
                    uint32_t c = __popc(wm);
                    *(volatile uint32_t*)&S->tail = t + (c < space ? c : space);
                }
                __syncwarp();
            }
        }
        // every element that was in L0 is now visible: count the uncounted ones
        if (lane == 0 && unc != 0) {
            atomicAdd(&S->acct, ((unsigned long long)(uint32_t)unc) << 32);
        }
        unc = 0;
    }

    // Moves everything in L1 to L2 (periodic flush of L1V, Section 3.4).
    // Called with the lock held.
    __device__ void l1_flush_locked() {
        const uint32_t cap = (uint32_t)P.l1_cap;
        if (P.l1_type == 1) {
            const uint32_t half = cap >> 1;
            for (int ring = 0; ring < 2; ring++) {
                uint32_t* hp = ring ? &S->fhead : &S->head;
                uint32_t* tp = ring ? &S->ftail : &S->tail;
                uint32_t h = sread(hp), t = sread(tp);
                while (h != t) {
                    uint32_t c = t - h < 32u ? t - h : 32u;
                    bool v = lane < c;
                    uint2 x = make_uint2(0, 0);
                    if (v) x = vld(&L1[(ring ? half : 0u) + ((h + lane) & (half - 1u))]);
                    h += c;
                    dec += l2_write(v, x);
                }
                __syncwarp();
                if (lane == 0) *(volatile uint32_t*)hp = h;
                __syncwarp();
            }
        } else {
            uint32_t h = sread(&S->head), t = sread(&S->tail);
            while (h != t) {
                uint32_t c = t - h < 32u ? t - h : 32u;
                bool v = lane < c;
                uint2 x = make_uint2(0, 0);
                if (v) x = vld(&L1[(h + lane) & l1_mask()]);
                h += c;
                dec += l2_write(v, x);
            }
            __syncwarp();
            if (lane == 0) *(volatile uint32_t*)&S->head = h;
            __syncwarp();
        }
        st[kStFlush]++;
    }

    // Write primitive of the L1 level for K elements per lane.
    template <int K>
    __device__ void l1_write(uint2 (&e)[K], bool (&valid)[K]) {
        uint32_t fthr = kInfU32;
        if (P.l1_type == 2) {
            unsigned long long win = 0;
            if (lane == 0) win = window();
            win = __shfl_sync(kFull, win, 0);
            fthr = A::upper((uint32_t)win, P.delta, P.filter_deltas);
        }
        bool out[K];
        if (!lock()) return;
        l1_place<K>(e, valid, out, fthr);
        bool flush = false;
        if (P.wb > 0) {
            uint32_t wcount = 0;
            if (lane == 0) {
                wcount = *(volatile uint32_t*)&S->writes + 1u;
                *(volatile uint32_t*)&S->writes = wcount;
            }
            wcount = __shfl_sync(kFull, wcount, 0);
            flush = (wcount % (uint32_t)P.wb) == 0u;
        }
        if (flush) l1_flush_locked();
        unlock();
#pragma unroll
        for (int k = 0; k < K; k++) dec += l2_write(out[k], e[k]);
    }

    // Read primitive of the L1 level: up to 32 elements, one per lane.
    __device__ bool l1_read(bool& valid, uint2& e) {
        valid = false;
        // cheap unlocked emptiness test first
        uint32_t h0 = *(volatile uint32_t*)&S->head, t0 = *(volatile uint32_t*)&S->tail;
        bool any = h0 != t0;
        if (P.l1_type == 1) {
            uint32_t fh0 = *(volatile uint32_t*)&S->fhead, ft0 = *(volatile uint32_t*)&S->ftail;
            any = any || fh0 != ft0;
        }
        mark(40);
        if (!__any_sync(kFull, any)) return false;
        mark(41);
        if (!lock()) return false;
        const uint32_t cap = (uint32_t)P.l1_cap;
        uint32_t h = sread(&S->head), t = sread(&S->tail);
        if (P.l1_type == 1 && h == t) {
            // near vector drained: NF = min(far) + delta, then re-partition far
            const uint32_t half = cap >> 1;
            uint32_t fh = sread(&S->fhead), ft = sread(&S->ftail);
            if (fh != ft) {
                uint32_t mn = kInfU32;
                for (uint32_t i = fh + lane; i - fh < ft - fh; i += 32)
                    mn = min(mn, vld(&L1[half + (i & (half - 1u))]).y);
                mn = __reduce_min_sync(kFull, mn);
                uint32_t nf = A::plus_delta(mn, P.delta);
                uint32_t nt = t, nft = ft;
                uint32_t count = ft - fh;
                for (uint32_t base = 0; base < count; base += 32) {
                    bool v = base + lane < count;
                    uint2 x = make_uint2(0, 0);
                    if (v) x = vld(&L1[half + ((fh + base + lane) & (half - 1u))]);
                    __syncwarp();
                    bool nearv = v && x.y < nf;
                    bool farv = v && !nearv;
                    uint32_t nm = __ballot_sync(kFull, nearv), fm = __ballot_sync(kFull, farv);
                    if (nearv) vst(&L1[(nt + __popc(nm & lanemask_lt())) & (half - 1u)], x);
                    if (farv) vst(&L1[half + ((nft + __popc(fm & lanemask_lt())) & (half - 1u))], x);
                    __syncwarp();
                    nt += __popc(nm);
                    nft += __popc(fm);
                }
                if (lane == 0) {
                    *(volatile uint32_t*)&S->nf = nf;
                    *(volatile uint32_t*)&S->tail = nt;
                    *(volatile uint32_t*)&S->fhead = fh + count;
                    *(volatile uint32_t*)&S->ftail = nft;
                }
                __syncwarp();
                t = nt;
            }
        }
        uint32_t c = t - h < 32u ? t - h : 32u;
        valid = lane < c;
        if (valid) {
            uint32_t idx = P.l1_type == 1 ? ((h + lane) & ((cap >> 1) - 1u)) : ((h + lane) & l1_mask());
            e = vld(&L1[idx]);
        }
        __syncwarp();
        if (lane == 0) *(volatile uint32_t*)&S->head = h + c;
        unlock();
        if (c) st[kStPopL1]++;
        return c != 0;
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

    // L0 is full: write all of it to L1 (Section 3.4: "when the L0 queue is
    // full, all its elements are transferred to the L1 queue").
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
        l1_write<R>(e, v);
    }

    // Appends c (<= 32) staged elements scratch[0..c) to L0.
    __device__ void l0_push(uint32_t c) {
        if (c == 0) return;
        if (l0t - l0h + c > 32u * R) l0_spill();
        uint32_t k = (lane - l0t) & 31u;
        if (k < c) {
            uint32_t p = l0t + k;
            l0_set((p >> 5) & (R - 1u), scratch[k]);
        }
        l0t += c;
        unc += (int)c;
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
        st[kStPopL0]++;
        return true;
    }

    // ---- relaxation ---------------------------------------------------------
    // Relaxes arc (u -> v, w) with u at distance du: nd = du (+) w; if nd
    // beats dist[v], atomicMin.  Returns true if dist[v] strictly improved
    // (the vertex must be written back, Listing 2).
    __device__ __forceinline__ bool relax(size_t vidx, uint32_t u, uint32_t du, uint32_t wbits,
                                          uint32_t& nd) {
        nd = A::add(du, wbits);
        if (PRED == 0) {
            uint32_t* p = reinterpret_cast<uint32_t*>(dist) + vidx;
            uint32_t cur = ld_dist(p);
            if (nd >= cur) return false;
            uint32_t old = atomicMin(p, nd);
            return old > nd;
        } else if (PRED == 1) {
            unsigned long long* p = reinterpret_cast<unsigned long long*>(dist) + vidx;
            unsigned long long cand = ((unsigned long long)nd << 32) | u;
            unsigned long long cur = ld_dist(p);
            if (cand >= cur) return false;
            unsigned long long old = atomicMin(p, cand);
            return (uint32_t)(old >> 32) > nd;
        } else {
            unsigned long long* p = reinterpret_cast<unsigned long long*>(dist) + vidx;
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

    // stage improved elements of one round and push them to L0
    __device__ __forceinline__ void push_round(bool imp, uint32_t key, uint32_t nd) {
        uint32_t m = __ballot_sync(kFull, imp);
        if (m == 0) return;
        if (imp) scratch[__popc(m & lanemask_lt())] = make_uint2(key, nd);
        __syncwarp();
        st[kStImproved] += __popc(m);
        l0_push(__popc(m));
    }

    // Relaxes arcs [lo, hi) of one vertex with the whole warp (task path).
    __device__ void relax_range(uint32_t key, uint32_t du, int32_t lo, int32_t hi) {
        const uint32_t u = key_vertex(key);
        const uint32_t qhi = MQ ? (key_query(key) << P.vbits) : 0u;
        const size_t qoff = MQ ? (size_t)key_query(key) * (size_t)P.n : 0;
        for (int32_t e0 = lo; e0 < hi; e0 += 64) {
            int32_t ea = e0 + (int32_t)lane, eb = ea + 32;
            bool va = ea < hi, vb = eb < hi;
            uint2 aa = make_uint2(0, 0), ab = make_uint2(0, 0);
            if (va) aa = __ldg(P.adj + ea);
            if (vb) ab = __ldg(P.adj + eb);
            uint32_t nda = 0, ndb = 0;
            bool ia = va && relax(qoff + aa.x, u, du, aa.y, nda);
            bool ib = vb && relax(qoff + ab.x, u, du, ab.y, ndb);
            st[kStRelax] += __popc(__ballot_sync(kFull, va)) + __popc(__ballot_sync(kFull, vb));
            push_round(ia, qhi | aa.x, nda);
            push_round(ib, qhi | ab.x, ndb);
        }
    }

    // Relaxes a batch of up to 32 vertices (one per lane).  Stale elements are
    // dropped (Listing 2: u.dist > dist[u]); vertices above th_heavy become
    // arc-range tasks; the remaining arcs are spread evenly over the lanes by
    // a warp prefix sum over degrees (Section 4.1 hybrid load balancing: a
    // high-degree vertex is scanned by the whole warp, low-degree vertices'
    // arcs are packed together).
    __device__ void relax_batch(bool valid, uint2 el) {
        uint32_t key = el.x, du = el.y;
        int32_t rs = 0, deg = 0;
        bool stale = false;
        if (valid && (key_vertex(key) >= (uint32_t)P.n || key_query(key) >= (uint32_t)P.nq)) {
            raise_error(P.ctrl, kErrElement, 8, (int)key);
            valid = false;
        }
        if (valid) {
            uint32_t cur = dpart(ld_dist(dist + dist_index(key)));
            if (du > cur) {
                valid = false;
                stale = true;
            } else {
                uint32_t v = key_vertex(key);
                rs = __ldg(P.row_ptr + v);
                deg = __ldg(P.row_ptr + v + 1) - rs;
            }
        }
        st[kStStale] += __popc(__ballot_sync(kFull, stale));
        // heavy vertices -> tasks
        uint32_t hm = __ballot_sync(kFull, valid && deg > P.th_heavy);
        while (hm) {
            int hl = __ffs(hm) - 1;
            hm &= hm - 1u;
            uint32_t hkey = __shfl_sync(kFull, key, hl);
            uint32_t hdu = __shfl_sync(kFull, du, hl);
            int32_t hrs = __shfl_sync(kFull, rs, hl);
            int32_t hdeg = __shfl_sync(kFull, deg, hl);
            uint32_t ntask = ((uint32_t)hdeg + (uint32_t)P.split - 1u) / (uint32_t)P.split;
            uint32_t t0 = 0;
            int ok = 0;
            if (lane == 0) {
                uint32_t r0 = ld_acquire(P.hv.rt);
                uint32_t w0 = ld_relaxed(P.hv.wt);
                if (w0 - r0 + ntask + P.hv.margin <= P.hv.nslot) {
                    atomicAdd(&P.ctrl->reserve, (unsigned long long)ntask);
                    t0 = atomicAdd(P.hv.wt, ntask);
                    ok = 1;
                }
            }
            ok = __shfl_sync(kFull, ok, 0);
            if (!ok) continue;   // ring busy: the warp scans this vertex itself
            t0 = __shfl_sync(kFull, t0, 0);
            for (uint32_t i = lane; i < ntask; i += 32) {
                uint32_t t = t0 + i;
                uint32_t* sp = P.hv.seq + (t & (P.hv.nslot - 1u));
                uint32_t spins = 0;
                bool okw = true;
                while (ld_acquire(sp) != t) {
                    if ((++spins & 255u) == 0 && expired()) {
                        raise_error(P.ctrl, kErrTimeout, 6, 0);
                        okw = false;
                        break;
                    }
                    __nanosleep(32);
                }
                if (!okw) break;
                int32_t lo = hrs + (int32_t)(i * (uint32_t)P.split);
                int32_t hi = min(lo + P.split, hrs + hdeg);
                P.hv.data[t & (P.hv.nslot - 1u)] = make_uint4(hkey, hdu, (uint32_t)lo, (uint32_t)hi);
                __threadfence();
                st_release(sp, t + 1u);
            }
            st[kStTasks] += ntask;
            if ((uint32_t)hl == lane) deg = 0;
        }
        // exclusive prefix sum of degrees
        int32_t incl = deg;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t x = __shfl_up_sync(kFull, incl, o);
            if (lane >= (uint32_t)o) incl += x;
        }
        const int32_t total = __shfl_sync(kFull, incl, 31);
        const int32_t ex = incl - deg;
        const uint32_t myq = MQ ? key_query(key) : 0u;
        st[kStRelax] += (uint32_t)total;
        for (int32_t g0 = 0; g0 < total; g0 += 32) {
            if ((g0 & 4095) == 4064) {
                int stop = 0;
                if (lane == 0) stop = expired() || ld_volatile_int(&P.ctrl->error) != 0;
                if (__shfl_sync(kFull, stop, 0)) break;
            }
            const int32_t g = g0 + (int32_t)lane;
            // owner: the largest lane j with ex[j] <= g
            int j = 0;
#pragma unroll
            for (int s = 16; s >= 1; s >>= 1) {
                int32_t t = __shfl_sync(kFull, ex, j + s);
                if (t <= g) j += s;
            }
            const int32_t oex = __shfl_sync(kFull, ex, j);
            const int32_t ors = __shfl_sync(kFull, rs, j);
            const uint32_t odu = __shfl_sync(kFull, du, j);
            const uint32_t okey = __shfl_sync(kFull, key, j);
            const uint32_t oq = __shfl_sync(kFull, myq, j);
            bool imp = false;
            uint32_t nd = 0, v = 0;
            if (g < total) {
                uint2 a = __ldg(P.adj + (ors + (g - oex)));
                v = a.x;
                size_t vidx = MQ ? (size_t)oq * (size_t)P.n + v : (size_t)v;
                imp = relax(vidx, key_vertex(okey), odu, a.y, nd);
            }
            push_round(imp, MQ ? ((oq << P.vbits) | v) : v, nd);
        }
    }

    __device__ void publish_stats() {
        if (lane == 0) {
#pragma unroll
            for (int i = 0; i < kStCount; i++)
                if (st[i]) atomicAdd(&P.ctrl->stats[i], (unsigned long long)st[i]);
        }
    }

    // ---- the worker loop (Listing 2, work_kernel) ---------------------------
    __device__ void run() {
        uint32_t idle_ns = 0;
        uint32_t iter = 0;
        for (;;) {
            mark(1, iter);
            if ((++iter & 7u) == 0 || idle_ns) {
                int stop = 0;
                if (lane == 0) {
                    stop = aborted();
                    if (!stop && expired()) {
                        raise_error(P.ctrl, kErrTimeout, 7, 0);
                        stop = 1;
                    }
                }
                stop = __shfl_sync(kFull, stop, 0);
                if (stop) break;
            }
            bool valid = false;
            uint2 e = make_uint2(0, 0);
            uint4 task = make_uint4(0, 0, 0, 0);
            int kind = 0;  // 0 none, 1 batch, 2 task
            int nb = 0;
            mark(20, iter);
            if (l0_read(valid, e)) kind = 1;
            mark(21, iter);
            if (!kind && l1_read(valid, e)) kind = 1;
            mark(22, iter);
            if (!kind) kind = global_read(valid, e, task);
            if (kind == 0) {
                mark(9, iter);
                // idle: publish deferred decrements, then test termination
                acct_apply();
                int fin = 0;
                if (lane == 0) {
                    unsigned long long d = ld_acquire64(&P.ctrl->done);
                    unsigned long long r = ld_acquire64(&P.ctrl->reserve);
                    if (d == r) {
                        atomicExch(&P.ctrl->finished, 1);
                        fin = 1;
                    }
                }
                fin = __shfl_sync(kFull, fin, 0);
                if (fin) break;
                idle_ns = idle_ns ? min(idle_ns * 2u, 2048u) : 64u;
                __nanosleep(idle_ns);
                continue;
            }
            idle_ns = 0;
            mark(kind == 2 ? 8 : 7, iter);
            if (kind == 2 && (key_vertex(task.x) >= (uint32_t)P.n || key_query(task.x) >= (uint32_t)P.nq ||
                              (int32_t)task.z < 0 || (int32_t)task.w < (int32_t)task.z)) {
                raise_error(P.ctrl, kErrElement, 9, (int)task.x);
                break;
            }
            if (kind == 2) {
                // one lane decides staleness for the whole warp: dist[u] may move
                // between per-lane loads, and relax_range is warp-collective
                uint32_t cur = 0;
                if (lane == 0) cur = dpart(ld_dist(dist + dist_index(task.x)));
                cur = __shfl_sync(kFull, cur, 0);
                if (task.y <= cur) relax_range(task.x, task.y, (int32_t)task.z, (int32_t)task.w);
                else st[kStStale]++;
                nb = 1;
            } else {
                nb = __popc(__ballot_sync(kFull, valid));
                relax_batch(valid, e);
            }
            dec += nb;
            mark(10, iter);
            acct_apply();
        }
        mark(13, iter);
        // drop anything still held (only on abort paths)
        publish_stats();
    }
};

template <int WT, int PRED, bool MQ, int R>
__global__ void __launch_bounds__(1024, 1) mlmq_kernel(KParams P) {
    extern __shared__ __align__(16) unsigned char smem[];
    BlockShared* S = reinterpret_cast<BlockShared*>(smem);
    const int nw = blockDim.x >> 5;
    uint2* scratch_all = reinterpret_cast<uint2*>(smem + sizeof(BlockShared));
    uint2* l1 = reinterpret_cast<uint2*>(smem + P.l1_off);
    if (threadIdx.x == 0) {
        S->lock = 0;
        S->head = S->tail = S->fhead = S->ftail = 0;
        S->nf = 0;
        S->writes = 0;
        S->acct = 0ull;
        unsigned long long win = ld_acquire64(&P.ctrl->window);
        S->nf = Arith<WT>::plus_delta((uint32_t)win, P.delta);
    }
    __syncthreads();
    const unsigned long long deadline = gtime() + P.timeout_ns;
    const int warp = threadIdx.x >> 5;
    (void)nw;
    Worker<WT, PRED, MQ, R> w(P, S, scratch_all + warp * 32, l1, deadline);
    w.run();
}

// ------------------------------------------------------------- seeding --

// Fills `count` 32-bit words with `value` (dist initialisation).
__global__ void fill_u32_kernel(uint32_t* p, size_t count, uint32_t value);
__global__ void fill_u64_kernel(unsigned long long* p, size_t count, unsigned long long value);

}  // namespace sssp
