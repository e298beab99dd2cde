// sssp_noalloc.cu -- a single-source solve that allocates no memory.
//
// Some callers cannot allocate device memory at the time they want a
// shortest-path answer: code running under a memory pool or arena that owns
// every allocation of the process, plugins or real-time loops whose
// allocation budget is fixed up front, and code that must not call
// cudaMalloc/cudaFree because those calls can synchronise the device.  The
// regular entry points create a graph handle and a per-graph workspace; this
// one runs the same persistent relaxation kernel with all of its scratch
// state (control block, L2 bucket rings, packed distance/predecessor words)
// in one fixed-size array that is part of the library image.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds it (kNoAllocBytes, about 25 MiB) until the process exits.
// Host code cannot use the array's name as a device address, so the first
// call on each device resolves it with cudaGetSymbolAddress (with that device
// current).  All calls share the array and it keeps the previous call's
// contents: every call first re-initialises what must start empty (the
// queue metadata and control block, then the distance words), so no call
// depends on how the previous one ended.  Calls that overlap on the GPU
// would race on the array; this file serialises the calls it issues with a
// process-wide mutex and returns only after the GPU work has finished.  A
// call reads results back and synchronises its stream part-way, so it must
// not be issued on a stream that is being captured into a CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/sssp.h"
#include "internal.h"

namespace sssp {

// kernels shared with the regular solve path (defined in sssp_api.cu)
__global__ void fill_u32_kernel(uint32_t* p, size_t count, uint32_t value);
__global__ void fill_u64_kernel(unsigned long long* p, size_t count, unsigned long long value);
__global__ void ring_reset_kernel(Rings r, uint32_t nrings, Ctrl* ctrl);
__global__ void seed_kernel(KParams P, const int32_t* srcs, int32_t src0, int32_t nq, int packed);
__global__ void unpack_kernel(const void* work, int packed, int32_t nq, int32_t n, int32_t nv,
                              uint32_t* dist, int32_t* pred, int f32);
__global__ void validate_rows_kernel(const int32_t* row_ptr, int32_t n, int64_t m, int* flags);

namespace {

// fixed shape of the no-allocation solve
constexpr int kNaBuckets = 8;                  // L2 buckets (one ring each)
constexpr uint32_t kNaChunks = 4096;           // chunks per ring
constexpr int kNaThreads = 256;                // threads per block, one block per SM
constexpr int kNaL1 = 1024;                    // L1 elements per block
constexpr size_t kCtrlBytes = 4096;
constexpr size_t kFlagBytes = 256;
constexpr size_t kTicketBytes = (size_t)kNaBuckets * 32 * sizeof(uint32_t);
constexpr size_t kMetaBytes = (size_t)kNaBuckets * kNaChunks * sizeof(uint32_t);
constexpr size_t kDataBytes = (size_t)kNaBuckets * kNaChunks * kChunk * sizeof(uint2);
constexpr size_t kWorkBytes = (size_t)SSSP_NOALLOC_MAX_VERTICES * sizeof(unsigned long long);
constexpr size_t kNoAllocBytes =
    kCtrlBytes + kFlagBytes + 2 * kTicketBytes + 2 * kMetaBytes + kDataBytes + kWorkBytes;

static_assert(sizeof(Ctrl) <= kCtrlBytes, "control block does not fit");

// The scratch array.  Device code could name it directly; host code only
// ever uses the address returned by cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Validation flags and graph statistics for the launch configuration.
struct NaFlags {
    int bad;                  // bit 0 row_ptr, bit 1 column range, bit 2 f32 weight
    unsigned int min_w;       // u32 value or f32 bits
    double sum_w;
};

// Checks the interleaved (column, weight) arcs and gathers min / sum of the
// weights (for the predecessor rule and the bucket width).
__global__ void na_check_arcs_kernel(const uint2* arcs, int64_t m, int32_t n, int f32, NaFlags* fl) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned int mn = 0xffffffffu;
    double sw = 0.0;
    int bad = 0;
    for (; i < m; i += stride) {
        const uint2 a = arcs[i];
        if ((int32_t)a.x < 0 || (int32_t)a.x >= n) bad |= 2;
        uint32_t wb = a.y;
        if (f32) {
            if (wb == 0x80000000u) wb = 0u;  // -0.0 adds like +0.0
            if ((wb & 0x80000000u) || (wb & 0x7f800000u) == 0x7f800000u) bad |= 4;
            sw += (double)__uint_as_float(wb);
        } else {
            sw += (double)wb;
        }
        mn = min(mn, wb);
    }
    for (int o = 16; o > 0; o >>= 1) {
        sw += __shfl_down_sync(kFull, sw, o);
        mn = min(mn, __shfl_down_sync(kFull, mn, o));
        bad |= __shfl_down_sync(kFull, bad, o);
    }
    if ((threadIdx.x & 31u) == 0) {
        if (bad) atomicOr(&fl->bad, bad);
        atomicMin(&fl->min_w, mn);
        atomicAdd(&fl->sum_w, sw);
    }
}

__global__ void na_flags_init_kernel(NaFlags* fl) {
    fl->bad = 0;
    fl->min_w = 0xffffffffu;
    fl->sum_w = 0.0;
}

struct NaDevice {
    bool ready = false;
    unsigned char* base = nullptr;   // device address of g_noalloc_scratch
};

std::mutex g_na_mu;
NaDevice g_na_dev[64];

struct NaLayout {
    Ctrl* ctrl;
    NaFlags* flags;
    Rings rings;
    unsigned long long* work;
};

NaLayout na_layout(unsigned char* base) {
    NaLayout L;
    unsigned char* p = base;
    L.ctrl = reinterpret_cast<Ctrl*>(p);
    p += kCtrlBytes;
    L.flags = reinterpret_cast<NaFlags*>(p);
    p += kFlagBytes;
    L.rings.rt = reinterpret_cast<uint32_t*>(p);
    p += kTicketBytes;
    L.rings.wt = reinterpret_cast<uint32_t*>(p);
    p += kTicketBytes;
    L.rings.seq = reinterpret_cast<uint32_t*>(p);
    p += kMetaBytes;
    L.rings.cnt = reinterpret_cast<uint32_t*>(p);
    p += kMetaBytes;
    L.rings.data = reinterpret_cast<uint2*>(p);
    p += kDataBytes;
    L.work = reinterpret_cast<unsigned long long*>(p);
    L.rings.nch = kNaChunks;
    L.rings.margin = 0;
    return L;
}

bool device_memory(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace sssp

using namespace sssp;

extern "C" int sssp_solve_noalloc(const int32_t* row_ptr, const uint32_t* arcs, int32_t n, int64_t m,
                                  int32_t wtype, int32_t src, void* dist_out, int32_t* pred_out,
                                  void* stream_ptr) {
    if (!row_ptr || !dist_out || (m > 0 && !arcs)) return SSSP_E_INVAL;
    if (n < 1 || n > SSSP_NOALLOC_MAX_VERTICES || m < 0 || m > 2147483647LL) return SSSP_E_INVAL;
    if (wtype != SSSP_W_U32 && wtype != SSSP_W_F32) return SSSP_E_INVAL;
    if (src < 0 || src >= n) return SSSP_E_INVAL;
    if (!device_memory(row_ptr) || !device_memory(dist_out) || (m > 0 && !device_memory(arcs)) ||
        (pred_out && !device_memory(pred_out)))
        return SSSP_E_INVAL;
    cudaStream_t stream = (cudaStream_t)stream_ptr;
    std::lock_guard<std::mutex> lk(g_na_mu);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SSSP_E_CUDA;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    NaDevice& D = g_na_dev[dev];
    if (!D.ready) {
        // once per device, with this device current: the array's device address
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
            cudaGetLastError();
            return SSSP_E_CUDA;
        }
        D.base = static_cast<unsigned char*>(ptr);
        D.ready = true;
    }
    NaLayout L = na_layout(D.base);
    const bool f32 = wtype == SSSP_W_F32;

    // validate the CSR (a bad column would make the kernel touch memory out of range)
    NaFlags hf;
    std::memset(&hf, 0, sizeof(hf));
    na_flags_init_kernel<<<1, 1, 0, stream>>>(L.flags);
    validate_rows_kernel<<<std::max(1, sms * 4), 256, 0, stream>>>(row_ptr, n, m, &L.flags->bad);
    if (m > 0)
        na_check_arcs_kernel<<<std::max(1, sms * 8), 256, 0, stream>>>(reinterpret_cast<const uint2*>(arcs), m, n,
                                                                      f32 ? 1 : 0, L.flags);
    if (cudaMemcpyAsync(&hf, L.flags, sizeof(hf), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return SSSP_E_CUDA;
    if (hf.bad) return SSSP_E_BADGRAPH;

    // configuration: L1 filter queue over an 8-bucket L2, block staging
    const int pred_mode = pred_out ? ((!f32 && m > 0 && hf.min_w >= 1u) ? 1 : 2) : 0;
    const KernelKey key{f32 ? 1 : 0, pred_mode, 0};
    const double avg_w = m > 0 ? hf.sum_w / (double)m : 1.0;
    const double avg_deg = std::max(1.0, (double)m / (double)n);
    const double dlt = std::max(f32 ? 1e-6 : 1.0, avg_w * 4.0 / avg_deg);
    const int warps_per_block = kNaThreads / 32;
    const size_t scratch_off = (sizeof(BlockShared) + 15) & ~size_t(15);
    const size_t far_off = scratch_off + (size_t)warps_per_block * 32 * sizeof(uint2);
    const size_t stat_off = far_off + (size_t)warps_per_block * kFarCap * sizeof(uint2);
    const size_t stage_off = stat_off + (size_t)warps_per_block * kStCount * sizeof(unsigned long long);
    const size_t l1_off = stage_off + (size_t)kNaBuckets * kStageCap * sizeof(uint2);
    const size_t smem = l1_off + (size_t)kNaL1 * sizeof(uint2);
    const int grid = sms;  // one block per SM
    const uint32_t warps = (uint32_t)(grid * warps_per_block);
    if (2 * warps >= kNaChunks) return SSSP_E_INVAL;

    KParams P;
    std::memset(&P, 0, sizeof(P));
    P.row_ptr = row_ptr;
    P.adj = reinterpret_cast<const uint2*>(arcs);
    P.owner = nullptr;
    P.n = n;
    P.nv = n;
    P.nq = 1;
    P.dist = pred_mode ? (void*)L.work : dist_out;
    P.vbits = 0;
    P.vmask = 0xffffffffu;
    P.l2 = L.rings;
    P.l2.margin = warps;
    P.shards = 1;
    P.ctrl = L.ctrl;
    if (f32) {
        float df = (float)dlt;
        std::memcpy(&P.delta, &df, 4);
        float nw = df;
        std::memcpy(&P.near_w, &nw, 4);
    } else {
        P.delta = (uint32_t)std::min(dlt, 4.0e9);
        P.near_w = P.delta;
    }
    P.bnum = 2;
    P.bmax = kNaBuckets;
    P.l1_type = SSSP_L1_FILTER;
    P.l1_cap = kNaL1;
    P.wb = 0;
    P.filter_deltas = 1.0f;
    P.max_arcs = 4096;
    P.claim = 4;
    P.refillers = 4;
    P.stage = 1;
    P.direct = 2;
    P.desc = 1;
    P.scratch_off = (int32_t)scratch_off;
    P.far_off = (int32_t)far_off;
    P.stat_off = (int32_t)stat_off;
    P.stage_off = (int32_t)stage_off;
    P.l1_off = (int32_t)l1_off;
    P.timeout_ns = 20000ull * 1000000ull;

    const size_t cells = (size_t)n;
    // empty queue metadata and control block, whatever the previous call left
    ring_reset_kernel<<<std::max(1, sms * 4), 256, 0, stream>>>(L.rings, kNaBuckets, L.ctrl);
    if (pred_mode)
        fill_u64_kernel<<<std::max(1, sms * 8), 256, 0, stream>>>(L.work, cells, ~0ull);
    else
        fill_u32_kernel<<<std::max(1, sms * 8), 256, 0, stream>>>((uint32_t*)dist_out, cells,
                                                                  f32 ? kInfF32 : kInfU32);
    seed_kernel<<<1, 32, 0, stream>>>(P, nullptr, src, 1, pred_mode ? 1 : 0);
    cudaError_t ce = launch_mlmq(key, dim3(grid), dim3(kNaThreads), smem, stream, P);
    if (ce != cudaSuccess) return SSSP_E_CUDA;
    if (pred_mode)
        unpack_kernel<<<std::max(1, sms * 8), 256, 0, stream>>>(L.work, 1, 1, n, n, (uint32_t*)dist_out, pred_out,
                                                                f32 ? 1 : 0);
    Ctrl hc;
    if (cudaMemcpyAsync(&hc, L.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return SSSP_E_CUDA;
    if (hc.error == kErrNone && hc.finished) return SSSP_OK;
    if (hc.error == kErrOverflow) return SSSP_E_NOMEM;
    if (hc.error == kErrTimeout) return SSSP_E_TIMEOUT;
    return SSSP_E_CUDA;
}
