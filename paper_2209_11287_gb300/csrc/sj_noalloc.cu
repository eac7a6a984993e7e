// sj_self_join_noalloc: a self-join that allocates no memory at all.
//
// Who needs it: callers that cannot allocate device memory while they run,
// e.g. a process whose device memory is fully reserved up front by another
// allocator, or an embedding runtime that forbids cudaMalloc / cudaFree after
// initialisation.  They still pass the input points and the output buffer;
// every working array this join needs lives in one fixed file-scope device
// array below, which each GPU that loads the library holds until the process
// exits.
//
// What it computes: the same result set as sj_join with the plain FP64 kernel
// (the decision rule of simjoin.h), without a grid: all points form a single
// cell, so every query is tiled against every point (brute force).  Limits:
// n <= SJ_NOALLOC_MAX_N points of dimension d <= SJ_NOALLOC_MAX_D.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "sj_internal.cuh"

namespace sj {

int launch_extent_raw(const double* pts, int64_t n, int d, unsigned long long* ext, cudaStream_t s);
size_t pack_params_size();
int pack_params_fill(void* host_pp, const double* lo, int d, int dp, double eps, double pbound, double delta);
int launch_pack_f64_raw(const double* pts, const int32_t* perm, int64_t n, const void* host_pp, double* xs, double* y,
                        double* h, double* to, double* ti, cudaStream_t s);

namespace {

constexpr int64_t kMaxN = SJ_NOALLOC_MAX_N;
constexpr int kMaxD = SJ_NOALLOC_MAX_D;
constexpr int kDp = 8;                                 // padded dimension of the packed rows
constexpr int64_t kMaxItems = (kMaxN + kQMax - 1) / kQMax;
constexpr int64_t kBandCap = int64_t(1) << 17;          // deferred-recheck queue entries
constexpr size_t kAlign = 256;

constexpr size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// Layout of the scratch array (byte offsets).
constexpr size_t kOffCounters = 0;                                         // 4 x u64
constexpr size_t kOffExt = align_up(kOffCounters + 4 * 8);                 // (2 d + 1) x u64
constexpr size_t kParamsBytes = 2048;                                      // host copy, >= sizeof(PackParams)
constexpr size_t kOffPerm = align_up(kOffExt + (2 * SJ_MAX_D + 1) * 8);    // n x i32
constexpr size_t kOffXs = align_up(kOffPerm + kMaxN * 4);                  // n x kDp f64
constexpr size_t kOffY = align_up(kOffXs + kMaxN * kDp * 8);               // n x kDp f64
constexpr size_t kOffH = align_up(kOffY + kMaxN * kDp * 8);                // n f64
constexpr size_t kOffTo = align_up(kOffH + kMaxN * 8);                     // n f64
constexpr size_t kOffTi = align_up(kOffTo + kMaxN * 8);                    // n f64
constexpr size_t kOffItems = align_up(kOffTi + kMaxN * 8);                 // items
constexpr size_t kOffRuns = align_up(kOffItems + kMaxItems * sizeof(Item));
constexpr size_t kOffBand = align_up(kOffRuns + sizeof(Run));             // band queue
constexpr size_t kScratchBytes = align_up(kOffBand + kBandCap * sizeof(int2));

}  // namespace

// The scratch itself: one static device array shared by every call on a
// device.  In host code its name is only a stand-in; its device address is
// obtained with cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[64];

// Device address of the scratch on the current device, resolved once per
// device (the first call on a device does this; make that call before any
// stream capture).
static int scratch_address(unsigned char** out) {
    int dev = 0;
    SJ_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        set_error("device ordinal %d out of range", dev);
        return SJ_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error("cudaGetSymbolAddress of the no-alloc scratch failed: %s", cudaGetErrorString(e));
            return SJ_ERR_CUDA;
        }
        g_noalloc_addr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_noalloc_addr[dev]);
    return SJ_OK;
}

__global__ void k_noalloc_setup(int32_t* perm, int64_t n, Item* items, int64_t n_items, Run* run) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) perm[i] = (int32_t)i;
    if (i < n_items) {
        Item it;
        it.q0 = (int32_t)(i * kQMax);
        it.q1 = (int32_t)std::min<int64_t>((i + 1) * kQMax, n);
        it.r0 = 0;
        it.r1 = 1;
        items[i] = it;
    }
    if (i == 0) {
        Run r;
        r.start = 0;
        r.end_flags = (uint32_t)n;  // one run over all points, no mirroring
        *run = r;
    }
}

}  // namespace sj

using namespace sj;

extern "C" int sj_self_join_noalloc(const double* pts, int64_t n, int32_t d, double eps, int32_t* pairs_out,
                                    int64_t capacity, int64_t* count_out, void* stream) {
    clear_error();
    if (!pts || !pairs_out || !count_out || n < 1 || d < 1 || !(eps > 0) || !isfinite(eps) || capacity < 0) {
        set_error("invalid argument: pts=%p n=%lld d=%d eps=%g pairs_out=%p capacity=%lld count_out=%p",
                  (const void*)pts, (long long)n, (int)d, eps, (void*)pairs_out, (long long)capacity,
                  (void*)count_out);
        return SJ_ERR_ARG;
    }
    if (n > kMaxN || d > kMaxD) {
        set_error("sj_self_join_noalloc supports n <= %lld points of dimension d <= %d (got n=%lld, d=%d)",
                  (long long)kMaxN, kMaxD, (long long)n, (int)d);
        return SJ_ERR_ARG;
    }
    if (!is_device_pointer(pts) || !is_device_pointer(pairs_out)) {
        set_error("sj_self_join_noalloc needs device pointers for pts and pairs_out");
        return SJ_ERR_ARG;
    }
    if (pack_params_size() > kParamsBytes) {
        set_error("internal: packing parameters larger than their host buffer");
        return SJ_ERR_UNSUPPORTED;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned char* base = nullptr;
    SJ_TRY(scratch_address(&base));
    unsigned long long* counters = reinterpret_cast<unsigned long long*>(base + kOffCounters);
    unsigned long long* ext = reinterpret_cast<unsigned long long*>(base + kOffExt);

    // extent and finiteness (the scratch keeps the previous call's values:
    // everything that must start from a fixed value is reset here)
    unsigned long long init[2 * kMaxD + 1];
    for (int k = 0; k < d; ++k) {
        init[k] = ~0ull;
        init[d + k] = 0ull;
    }
    init[2 * d] = 0ull;
    SJ_CK(cudaMemcpyAsync(ext, init, (2 * d + 1) * sizeof(unsigned long long), cudaMemcpyHostToDevice, s));
    SJ_TRY(launch_extent_raw(pts, n, d, ext, s));
    unsigned long long got[2 * kMaxD + 1];
    SJ_CK(cudaMemcpyAsync(got, ext, (2 * d + 1) * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    SJ_CK(cudaStreamSynchronize(s));
    if (got[2 * d] != 0) {
        set_error("non-finite coordinate in the input points");
        return SJ_ERR_ARG;
    }
    double lo[kMaxD], pbound = 0.0, rmax = 0.0;
    for (int k = 0; k < d; ++k) {
        const unsigned long long a = got[k], b = got[d + k];
        const unsigned long long ba = (a >> 63) ? (a & 0x7FFFFFFFFFFFFFFFull) : ~a;
        const unsigned long long bb = (b >> 63) ? (b & 0x7FFFFFFFFFFFFFFFull) : ~b;
        double va, vb;
        memcpy(&va, &ba, 8);
        memcpy(&vb, &bb, 8);
        lo[k] = va;
        const double r = vb - va;
        pbound += r * r;
        rmax = std::max(rmax, r);
    }
    pbound *= 1.0 + ldexp(1.0, -20);

    // packing parameters, identity order, one item per 16 queries, one run
    alignas(16) unsigned char pp[kParamsBytes];
    SJ_TRY(pack_params_fill(pp, lo, d, kDp, eps, pbound, 1.01 * ldexp(1.0, -53) * rmax));
    const int64_t n_items = (n + kQMax - 1) / kQMax;
    int32_t* perm = reinterpret_cast<int32_t*>(base + kOffPerm);
    Item* items = reinterpret_cast<Item*>(base + kOffItems);
    Run* run = reinterpret_cast<Run*>(base + kOffRuns);
    k_noalloc_setup<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(perm, n, items, n_items, run);
    note_launch();
    SJ_CK(cudaGetLastError());
    double* xs = reinterpret_cast<double*>(base + kOffXs);
    double* y = reinterpret_cast<double*>(base + kOffY);
    double* h = reinterpret_cast<double*>(base + kOffH);
    double* to = reinterpret_cast<double*>(base + kOffTo);
    double* ti = reinterpret_cast<double*>(base + kOffTi);
    SJ_TRY(launch_pack_f64_raw(pts, perm, n, pp, xs, y, h, to, ti, s));

    // the plain FP64 join kernel and its deferred recheck on the scratch
    Index ix;  // a view of the scratch (its host vectors stay empty)
    SJ_CK(cudaGetDevice(&ix.device));
    ix.stream = s;
    ix.kernel = SJ_KERNEL_FP64_FMA;
    ix.n = n;
    ix.d = d;
    ix.dp = kDp;
    ix.eps = eps;
    ix.e2 = eps * eps;
    ix.xs = xs;
    ix.y = y;
    ix.h = h;
    ix.thr_out = to;
    ix.thr_in = ti;
    ix.perm = perm;
    ix.items = items;
    ix.runs = run;
    ix.n_items = n_items;
    ix.n_runs = 1;
    ix.n_cells = 1;
    ix.counters = counters;
    JoinOut jo;
    jo.out_pairs = reinterpret_cast<int2*>(pairs_out);
    jo.out_dist = nullptr;
    jo.capacity = (unsigned long long)capacity;
    jo.band = reinterpret_cast<int2*>(base + kOffBand);
    jo.band_cap = (unsigned long long)kBandCap;
    SJ_CK(cudaMemsetAsync(counters, 0, 4 * sizeof(unsigned long long), s));
    SJ_TRY(launch_join_cc(&ix, jo, 0));
    SJ_TRY(launch_recheck(&ix, jo, 0));
    unsigned long long c[4];
    SJ_CK(cudaMemcpyAsync(c, counters, sizeof c, cudaMemcpyDeviceToHost, s));
    SJ_CK(cudaStreamSynchronize(s));
    *count_out = (int64_t)c[1];
    if (c[1] > (unsigned long long)capacity) {
        set_error("result of %llu pairs exceeds the output capacity of %lld pairs", c[1], (long long)capacity);
        return SJ_ERR_RESULT_OVERFLOW;
    }
    return SJ_OK;
}
