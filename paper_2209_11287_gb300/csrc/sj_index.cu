// Grid index of the similarity self-join (Sec. III-B): extent, cell keys,
// LSD radix sort, cell table, packing in cell order with norms and certified
// thresholds, neighbour-run enumeration and work items.
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <type_traits>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "sj_internal.cuh"

namespace sj {

// ---------------------------------------------------------------------------
// order-preserving map double -> uint64 (for atomic min / max)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long ord_of(double v) {
    unsigned long long b = __double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
static double from_ord(unsigned long long o) {
    unsigned long long b = (o >> 63) ? (o & 0x7FFFFFFFFFFFFFFFull) : ~o;
    double v;
    memcpy(&v, &b, sizeof v);
    return v;
}

// Per-dim min / max of the points and a flag for any non-finite coordinate.
// The block size and the grid stride are multiples of d, so every element a
// thread visits belongs to dim threadIdx.x % d and the thread keeps one
// running min / max; all comparisons are on integer order keys.
__global__ void k_extent(const double* __restrict__ x, int64_t total, int d, unsigned long long* lo,
                         unsigned long long* hi, int* bad) {
    extern __shared__ unsigned long long s_ext[];  // [2 * d]
    for (int k = threadIdx.x; k < d; k += blockDim.x) {
        s_ext[k] = ~0ull;
        s_ext[d + k] = 0ull;
    }
    __syncthreads();
    unsigned long long mn = ~0ull, mx = 0ull;
    int local_bad = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += stride) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(x[i]);
        if (((b >> 52) & 0x7FFull) == 0x7FFull) {  // Inf or NaN
            local_bad = 1;
            continue;
        }
        const unsigned long long o = (b >> 63) ? ~b : (b | 0x8000000000000000ull);
        mn = o < mn ? o : mn;
        mx = o > mx ? o : mx;
    }
    if (local_bad) atomicOr(bad, 1);
    const int k = threadIdx.x % d;
    if (mn <= mx) {
        atomicMin(&s_ext[k], mn);
        atomicMax(&s_ext[d + k], mx);
    }
    __syncthreads();
    for (int k2 = threadIdx.x; k2 < d; k2 += blockDim.x) {
        atomicMin(&lo[k2], s_ext[k2]);
        atomicMax(&hi[k2], s_ext[d + k2]);
    }
}

// Per-dim sum and sum of squares (binary64) of the points, for the
// variance order of the short-circuit (an order only: its rounding changes no
// result).  Same thread layout as k_extent.
__global__ void k_moments(const double* __restrict__ x, int64_t total, int d, double* mom) {
    extern __shared__ double s_mom[];  // [2 * d]
    for (int k = threadIdx.x; k < 2 * d; k += blockDim.x) s_mom[k] = 0.0;
    __syncthreads();
    double s1 = 0.0, s2 = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += stride) {
        const double v = x[i];
        s1 += v;
        s2 = fma(v, v, s2);
    }
    const int k = threadIdx.x % d;
    atomicAdd(&s_mom[k], s1);
    atomicAdd(&s_mom[d + k], s2);
    __syncthreads();
    for (int k2 = threadIdx.x; k2 < 2 * d; k2 += blockDim.x) atomicAdd(&mom[k2], s_mom[k2]);
}

struct GridParams {
    int m;
    int dims[kMaxM];
    double lo[kMaxM];
    int64_t ncell[kMaxM];
    unsigned long long stride[kMaxM];
    double inv_w;
};

// Cell coordinate of one value: floor((x - lo) * (1 / w)), clamped to the
// grid.  (1 / w is rounded once; the relative margin of w over eps absorbs
// the three roundings, see choose_grid.)
__device__ __forceinline__ int64_t cell_coord(double v, double lo, double inv_w, int64_t ncell) {
    // floor and conversion in one instruction (binary64 work is scarce here)
    const int64_t c = __double2ll_rd(__dmul_rn(__dsub_rn(v, lo), inv_w));
    return c < 0 ? 0 : (c >= ncell ? ncell - 1 : c);
}

__global__ void k_cell_keys(const double* __restrict__ x, int64_t n, int d, GridParams g,
                            unsigned long long* keys, int32_t* ids) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned long long key = 0;
    for (int k = 0; k < g.m; ++k) {
        int64_t c = cell_coord(x[i * d + g.dims[k]], g.lo[k], g.inv_w, g.ncell[k]);
        key += (unsigned long long)c * g.stride[k];
    }
    keys[i] = key;
    ids[i] = (int32_t)i;
}

// ---------------------------------------------------------------------------
// counting sort by cell key, for key spaces of at most a few times n keys
// ---------------------------------------------------------------------------
// One count per key, a scan of the counts, a scatter; the key's first
// position then stands for its cell (no table of non-empty cells is
// built: the neighbour runs are read per key, k_denum).  Lanes of a warp with the same key
// share one atomic (match_any), so a crowded cell costs one atomic per warp.
// Inside a cell the points follow the order in which warps reach it, not the
// input order: every result of the join is a set and does not depend on it.
constexpr uint32_t kNoKey = 0xFFFFFFFFu;  // keys of the dense path are below 2^31

__global__ void k_key_count(const double* __restrict__ x, int64_t n, int d, GridParams g, uint32_t* key32,
                            uint32_t* cnt) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool valid = i < n;
    uint32_t key = kNoKey;
    if (valid) {
        unsigned long long k64 = 0;
        for (int k = 0; k < g.m; ++k)
            k64 += (unsigned long long)cell_coord(x[i * d + g.dims[k]], g.lo[k], g.inv_w, g.ncell[k]) * g.stride[k];
        key = (uint32_t)k64;
        key32[i] = key;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const int lane = threadIdx.x & 31;
    if (valid && lane == __ffs(peers) - 1) atomicAdd(&cnt[key], (uint32_t)__popc(peers));
}


// ---------------------------------------------------------------------------
// exclusive scan (reduce-then-scan over tiles of 4096), of uint32 or of
// uint64 values produced by a load functor
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* s_warp, T* total) {
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        T w = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        s_warp[lane] = w;
    }
    __syncthreads();
    T warp_base = wid ? s_warp[wid - 1] : T(0);
    *total = s_warp[(blockDim.x >> 5) - 1];
    T r = warp_base + x - v;
    __syncthreads();
    return r;
}

struct LoadU32 {
    const uint32_t* p;
    __device__ __forceinline__ uint32_t operator()(int64_t i) const { return p[i]; }
};
struct LoadU64 {
    const unsigned long long* p;
    __device__ __forceinline__ unsigned long long operator()(int64_t i) const { return p[i]; }
};
// A key's point count c in the high half and its work items ceil(c / qmax)
// in the low half: one scan gives each key's first sorted position and its
// first work item.
struct LoadCountItems {
    const uint32_t* cnt;
    uint32_t qmax;
    __device__ __forceinline__ unsigned long long operator()(int64_t i) const {
        const uint32_t c = cnt[i];
        return ((unsigned long long)c << 32) | (unsigned long long)((c + qmax - 1u) / qmax);
    }
};

template <typename T, typename L>
__global__ void k_scan_tile_sums(L in, int64_t n, T* sums) {
    __shared__ T s_warp[32];
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    T acc = 0;
    for (int i = 0; i < kScanItems; ++i) {
        int64_t idx = base + (int64_t)i * kScanThreads + threadIdx.x;
        if (idx < n) acc += in(idx);
    }
    T tot;
    block_exclusive_scan<T>(acc, s_warp, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// Scans one tile (thread t owns items t*kScanItems .. +kScanItems, a
// contiguous chunk) and adds the tile's base offset; the last tile writes
// the total to out[n] when `with_total`.
template <typename T, typename L>
__global__ void k_scan_tiles(L in, T* out, int64_t n, const T* __restrict__ tile_base, int with_total) {
    __shared__ T s_warp[32];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    T v[kScanItems];
    T acc = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t idx = base + i;
        v[i] = idx < n ? in(idx) : T(0);
        acc += v[i];
    }
    T tot;
    T run = block_exclusive_scan<T>(acc, s_warp, &tot) + (tile_base ? tile_base[blockIdx.x] : T(0));
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t idx = base + i;
        if (idx < n) out[idx] = run;
        run += v[i];
    }
    if (with_total && blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) out[n] = run;
}

template <typename T, typename L>
static int scan_exclusive(L in, T* out, int64_t n, bool with_total, cudaStream_t s) {
    if (n <= 0) {
        if (with_total) SJ_CK(cudaMemsetAsync(out, 0, sizeof(T), s));
        return SJ_OK;
    }
    int64_t tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles == 1) {
        k_scan_tiles<T, L><<<1, kScanThreads, 0, s>>>(in, out, n, nullptr, with_total ? 1 : 0);
        note_launch();
        SJ_CK(cudaGetLastError());
        return SJ_OK;
    }
    Scratch tmp(s);
    T* sums = nullptr;
    SJ_TRY(tmp.alloc(&sums, (size_t)tiles * 2));
    T* sums_scan = sums + tiles;
    k_scan_tile_sums<T, L><<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, sums);
    note_launch();
    SJ_CK(cudaGetLastError());
    int st = SJ_OK;
    if constexpr (sizeof(T) == 4)
        st = scan_exclusive<T, LoadU32>(LoadU32{sums}, sums_scan, tiles, false, s);
    else
        st = scan_exclusive<T, LoadU64>(LoadU64{sums}, sums_scan, tiles, false, s);
    if (st == SJ_OK) {
        k_scan_tiles<T, L><<<(unsigned)tiles, kScanThreads, 0, s>>>(in, out, n, sums_scan, with_total ? 1 : 0);
        note_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            set_error("scan launch: %s", cudaGetErrorString(e));
            st = SJ_ERR_CUDA;
        }
    }
    return st;
}

int scan_exclusive_u32(const uint32_t* in, uint32_t* out, int64_t n, cudaStream_t s) {
    return scan_exclusive<uint32_t, LoadU32>(LoadU32{in}, out, n, false, s);
}

int scan_exclusive_u32_total(const uint32_t* in, uint32_t* out, int64_t n, cudaStream_t s) {
    return scan_exclusive<uint32_t, LoadU32>(LoadU32{in}, out, n, true, s);
}

// ---------------------------------------------------------------------------
// LSD radix sort of (uint64 key, int32 value), 8-bit digits, stable passes
// ---------------------------------------------------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortRounds = 16;
constexpr int kSortTile = kSortThreads * kSortRounds;  // elements per tile

// hist[digit * tiles + tile] = count of `digit` in the tile.
__global__ void k_sort_hist(const unsigned long long* __restrict__ keys, int64_t n, int shift, uint32_t* hist,
                            int64_t tiles) {
    __shared__ uint32_t s_h[256];
    s_h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int r = 0; r < kSortRounds; ++r) {
        int64_t i = base + (int64_t)r * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&s_h[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * tiles + blockIdx.x] = s_h[threadIdx.x];
}

// Stable scatter: element order within the tile is round-major then thread
// order, i.e. the input order, and ranks follow it.
__global__ void k_sort_scatter(const unsigned long long* __restrict__ keys_in, const int32_t* __restrict__ vals_in,
                               unsigned long long* keys_out, int32_t* vals_out, int64_t n, int shift,
                               const uint32_t* __restrict__ offs, int64_t tiles) {
    __shared__ uint32_t s_base[256];           // running output position per digit
    __shared__ uint32_t s_wcnt[kSortThreads / 32][256];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    s_base[threadIdx.x] = offs[(int64_t)threadIdx.x * tiles + blockIdx.x];
    int64_t base = (int64_t)blockIdx.x * kSortTile;
    const unsigned lt = (1u << lane) - 1u;
    for (int r = 0; r < kSortRounds; ++r) {
        for (int w = 0; w < kSortThreads / 32; ++w) s_wcnt[w][threadIdx.x] = 0;
        __syncthreads();
        int64_t i = base + (int64_t)r * kSortThreads + threadIdx.x;
        bool valid = i < n;
        unsigned long long k = valid ? keys_in[i] : 0ull;
        int32_t v = valid ? vals_in[i] : 0;
        unsigned dig = valid ? (unsigned)((k >> shift) & 255u) : 256u;  // 256 = padding
        unsigned peers = __match_any_sync(0xffffffffu, dig);
        unsigned rank_in_warp = __popc(peers & lt);
        bool leader = rank_in_warp == 0;
        if (valid && leader) s_wcnt[wid][dig] = __popc(peers);
        __syncthreads();
        {   // per digit: exclusive prefix over warps, advance the running base
            unsigned dg = threadIdx.x;
            uint32_t run = s_base[dg];
            for (int w = 0; w < kSortThreads / 32; ++w) {
                uint32_t c = s_wcnt[w][dg];
                s_wcnt[w][dg] = run;
                run += c;
            }
            s_base[dg] = run;
        }
        __syncthreads();
        if (valid) {
            uint32_t pos = s_wcnt[wid][dig] + rank_in_warp;
            keys_out[pos] = k;
            vals_out[pos] = v;
        }
        __syncthreads();
    }
}

int radix_sort_pairs(uint64_t* keys, int32_t* vals, int64_t n, int key_bits, cudaStream_t s) {
    if (n <= 1 || key_bits <= 0) return SJ_OK;
    int64_t tiles = (n + kSortTile - 1) / kSortTile;
    if ((int64_t)tiles * 256 >= (int64_t(1) << 32)) {
        set_error("radix sort: input too large");
        return SJ_ERR_ARG;
    }
    Scratch tmp(s);
    unsigned long long* k2 = nullptr;
    int32_t* v2 = nullptr;
    uint32_t* hist = nullptr;
    int st = SJ_OK;
    SJ_TRY(tmp.alloc(&k2, (size_t)n));
    SJ_TRY(tmp.alloc(&v2, (size_t)n));
    SJ_TRY(tmp.alloc(&hist, (size_t)tiles * 256 * 2));
    uint32_t* offs = hist + tiles * 256;
    unsigned long long* ka = reinterpret_cast<unsigned long long*>(keys);
    int32_t* va = vals;
    unsigned long long* kb = k2;
    int32_t* vb = v2;
    int passes = (key_bits + 7) / 8;
    for (int p = 0; p < passes && st == SJ_OK; ++p) {
        int shift = 8 * p;
        k_sort_hist<<<(unsigned)tiles, kSortThreads, 0, s>>>(ka, n, shift, hist, tiles);
        note_launch();
        st = scan_exclusive_u32(hist, offs, tiles * 256, s);
        if (st != SJ_OK) break;
        k_sort_scatter<<<(unsigned)tiles, kSortThreads, 0, s>>>(ka, va, kb, vb, n, shift, offs, tiles);
        note_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            set_error("radix sort launch: %s", cudaGetErrorString(e));
            st = SJ_ERR_CUDA;
        }
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (st == SJ_OK && ka != reinterpret_cast<unsigned long long*>(keys)) {
        cudaError_t e1 = cudaMemcpyAsync(keys, ka, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s);
        cudaError_t e2 = cudaMemcpyAsync(vals, va, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
        if (e1 != cudaSuccess || e2 != cudaSuccess) {
            set_error("radix sort copy-back failed");
            st = SJ_ERR_CUDA;
        }
    }
    return st;
}

// ---------------------------------------------------------------------------
// cell table
// ---------------------------------------------------------------------------
__global__ void k_heads(const unsigned long long* __restrict__ keys, int64_t n, uint32_t* flags) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) flags[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1u : 0u;
}

__global__ void k_cells(const unsigned long long* __restrict__ keys, const uint32_t* __restrict__ flags,
                        const uint32_t* __restrict__ idx, int64_t n, unsigned long long* cell_key,
                        int32_t* cell_start, unsigned long long* n_cells) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (flags[i]) {
        cell_key[idx[i]] = keys[i];
        cell_start[idx[i]] = (int32_t)i;
    }
    if (i == n - 1) {
        uint32_t m = idx[i] + flags[i];
        *n_cells = m;
        cell_start[m] = (int32_t)n;
    }
}

// ---------------------------------------------------------------------------
// packing in cell order, kernel coordinates and certified thresholds
// ---------------------------------------------------------------------------
struct PackParams {
    double lo[SJ_MAX_D];
    // thresholds as affine functions of the computed norm pc (see below)
    double a_out, b_out, a_in, b_in;
    // the same coefficients rounded outward to binary32 once (FP32 kernels)
    float af_out, bf_out, af_in, bf_in;
    int has_in;
    int d, dp;
    // kernel coordinate k is input dim order[k] (identity unless the
    // short-circuit orders dims by variance)
    uint8_t order[SJ_MAX_D];
    // short-circuit: the checkpoint (kernel dims before it; 0: off) and the
    // margin coefficient (see pack_one)
    int sc_b;
    double sc_coef, sc_p;
    // kernel coordinates y = (x - lo) * scale, a power of two (1 except for
    // the FP16x2 filter, whose fp16 terms need |y_k| <= 2^15)
    double scale = 1.0;
    // (eps (1 + g) + eta)^2 rounded up, and its binary32 copy rounded up: a
    // squared distance of kernel coordinates above it is out for the decision
    // rule (the small-d FP32 filter's bounding-box prune)
    double prune_r2 = INFINITY;
    float prune_r2f = INFINITY;
};

__host__ __device__ inline double gamma_n(double u, int k) { return k * u / (1.0 - k * u); }

// Scale of binary32 kernel coordinates: S = 2^e, the largest power of two
// with S^2 P <= 2^30, so S^2 P is in (2^28, 2^30] (1 when P = 0).  Then no
// norm, product, threshold or accumulator overflows binary32 (all below
// 2^31), every coordinate is below 2^15 (an fp16 value: FP16x2), and a
// coordinate or partial product that underflows is off by at most 2^-149
// absolute, far below the bound c1 (P + pc) with P > 2^28; eps, P and delta
// scale with S and every threshold relation of pack_coefficients is
// unchanged (scaling by a power of two is exact).  False when no such e in
// [-500, 500] exists (P below about 2^-970 or not finite).
bool binary32_scale(double pbound, double* scale) {
    *scale = 1.0;
    if (pbound == 0.0) return true;
    if (!(pbound > 0.0) || !std::isfinite(pbound)) return false;
    int e = (int)std::floor(0.5 * (30.0 - std::log2(pbound)));
    e = std::min(500, std::max(-500, e));
    while (e > -500 && ldexp(pbound, 2 * e) > ldexp(1.0, 30)) --e;
    while (e < 500 && ldexp(pbound, 2 * (e + 1)) <= ldexp(1.0, 30)) ++e;
    const double ps = ldexp(pbound, 2 * e);
    if (!(ps > ldexp(1.0, 28) && ps <= ldexp(1.0, 30))) return false;
    *scale = ldexp(1.0, e);
    return true;
}

// Thresholds on a = y_q.y_c - ||y_q||^2/2 computed in T (fma chain over the
// padded dims, started at -||y_q||^2/2) for candidate c with computed norm
// pc.  With s_y = ||y_q - y_c||^2 = ||y_c||^2 - 2 a_exact, the evaluation
// error satisfies |s_y - (pc - 2 a)| <= 3 gamma_T(dp) (||y_q||^2 + ||y_c||^2)
// (norm chains and the dot-product chain); doubled for safety:
//   E_s = c1 (P + pc),  c1 = 6.2 gamma_T(dp + 1),  P >= every ||y||^2.
// The coordinates carry |y_k - (x_k - lo_k)| <= delta, so
// |sqrt(s_y) - sqrt(s)| <= eta = 2 delta sqrt(d), s the exact squared
// distance of the inputs.  The decision rule's s differs from the exact one by
// at most gamma_64(d + 3) s; g = 2 gamma_64(d + 3) covers it.  Then
//   a <  thr_out  =>  s > e2 (1 + g)     => out for the decision rule,
//   a >= thr_in   =>  s <= e2 (1 - g)    => in for the decision rule,
// with, S_o = (eps (1 + g) + eta)^2 and S_i = (eps (1 - g) - eta)^2,
//   thr_out = (pc - S_o - E_s) / 2 - 4 u_T (pc + S_o + E_s)  = a_out pc - b_out
//   thr_in  = (pc - S_i + E_s) / 2 + 4 u_T (pc + S_i + E_s)  = a_in pc + b_in
// (thr_in = +inf when eps (1 - g) <= eta).  The affine coefficients are
// formed on the host in binary64, rounded outward to T, and each threshold is
// one fma rounded down (thr_out) or up (thr_in), so the stored values are on
// the safe side of the exact ones.
//
// `c1_override` > 0 replaces c1 for arithmetic with another error model (the
// tensor-core filter, see build_index).
void pack_coefficients(double eps, double pbound, double delta, double u_t, int d, int dp, PackParams* pp,
                       double c1_override = -1.0) {
    const double g = 2.0 * gamma_n(ldexp(1.0, -53), d + 3);
    const double eta = 2.0 * delta * sqrt((double)d) * (1.0 + ldexp(1.0, -40));
    const double c1 = c1_override > 0 ? c1_override : 6.2 * gamma_n(u_t, dp + 1);
    const double so_r = eps * (1.0 + g) + eta;
    const double so = so_r * so_r * (1.0 + ldexp(1.0, -50));
    const double m = 4.0 * u_t;
    // thr_out = pc (1/2 - c1/2 - m (1 + c1)) - ((so + c1 P)/2 + m (so + c1 P))
    pp->a_out = nextafter(0.5 - 0.5 * c1 - m * (1.0 + c1), 0.0);
    pp->b_out = nextafter((so + c1 * pbound) * 0.5 + m * (so + c1 * pbound), INFINITY);
    const double si_r = eps * (1.0 - g) - eta;
    pp->has_in = si_r > 0 ? 1 : 0;
    const double si = si_r * si_r * (1.0 - ldexp(1.0, -50));
    // thr_in = pc (1/2 + c1/2 + m (1 + c1)) + ((c1 P - si)/2 + m (si + c1 P))
    pp->a_in = nextafter(0.5 + 0.5 * c1 + m * (1.0 + c1), INFINITY);
    pp->b_in = nextafter((c1 * pbound - si) * 0.5 + m * (si + c1 * pbound), INFINITY);
    // binary32 copies, rounded down (a_out) or up (the others), as the
    // device's __double2float_rd / _ru would round them
    auto down = [](double v) {
        float f = (float)v;
        if ((double)f > v) f = nextafterf(f, -INFINITY);
        return f;
    };
    auto up = [](double v) {
        float f = (float)v;
        if ((double)f < v) f = nextafterf(f, INFINITY);
        return f;
    };
    pp->af_out = down(pp->a_out);
    pp->bf_out = up(pp->b_out);
    pp->af_in = up(pp->a_in);
    pp->bf_in = up(pp->b_in);
    pp->prune_r2 = so;
    pp->prune_r2f = up(so);
}

// The two thresholds of a point with computed norm pc, one fma each, rounded
// outward (see pack_coefficients).
__device__ __forceinline__ float pack_thr_out(const PackParams& pp, float pc) {
    return __fmaf_rd(pp.af_out, pc, -pp.bf_out);
}
__device__ __forceinline__ double pack_thr_out(const PackParams& pp, double pc) {
    return __fma_rd(pp.a_out, pc, -pp.b_out);
}
__device__ __forceinline__ float pack_thr_in(const PackParams& pp, float pc) {
    return __fmaf_ru(pp.af_in, pc, pp.bf_in);
}
__device__ __forceinline__ double pack_thr_in(const PackParams& pp, double pc) { return __fma_ru(pp.a_in, pc, pp.b_in); }

__device__ __forceinline__ float fma_pack(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_pack(double a, double b, double c) { return __fma_rn(a, b, c); }
// outward-rounded affine thresholds
__device__ __forceinline__ float thr_down(double a, float pc, double b) {
    return __fmaf_rd(__double2float_rd(a), pc, -__double2float_ru(b));
}
__device__ __forceinline__ double thr_down(double a, double pc, double b) { return __fma_rd(a, pc, -b); }
__device__ __forceinline__ float thr_up(double a, float pc, double b) {
    return __fmaf_ru(__double2float_ru(a), pc, __double2float_ru(b));
}
__device__ __forceinline__ double thr_up(double a, double pc, double b) { return __fma_ru(a, pc, b); }

// One thread per point: its row is gathered through perm and written in cell
// order, with its kernel coordinates, norm and thresholds (and, for the
// small-d FP32 filter, its 16-byte record: both thresholds and the input
// index).  The parameters travel by value.
// Output arrays of the packing (cell order).
template <typename T>
struct PackOut {
    double* xs;
    T* y;
    T* h;
    T* thr_out;
    T* thr_in;
    float4* aux;   // or null
    double* sc_w;  // or null
};

// Packs input point src_i (row xr) at sorted position p: its original row,
// its kernel coordinates (in the kernel dim order), norm and thresholds
// (and, for the small-d FP32 filter, its 16-byte record: both thresholds and
// the input index; for the short-circuit, its checkpoint bounds).
template <typename T>
__device__ __forceinline__ void pack_one(const double* __restrict__ xr, int32_t src_i, int64_t p, const PackParams& pp,
                                         const PackOut<T>& o) {
    const int d = pp.d, dp = pp.dp;
    for (int k = 0; k < dp; ++k) o.xs[p * dp + k] = k < d ? xr[k] : 0.0;  // input order
    T nrm = T(0), nrm_b = T(0);
    for (int k = 0; k < dp; ++k) {
        const int ok = k < d ? pp.order[k] : k;
        const T yk = k < d ? T((xr[ok] - pp.lo[ok]) * pp.scale) : T(0);
        o.y[p * dp + k] = yk;
        nrm = fma_pack(yk, yk, nrm);
        if (k + 1 == pp.sc_b) nrm_b = nrm;  // the partial norm at the short-circuit checkpoint
    }
    o.h[p] = -nrm * T(0.5);
    const T to = pack_thr_out(pp, nrm);
    const T ti = pp.has_in ? pack_thr_in(pp, nrm) : T(INFINITY);
    o.thr_out[p] = to;
    o.thr_in[p] = ti;
    if (o.aux) o.aux[p] = make_float4((float)to, (float)ti, __int_as_float(src_i), 0.f);
    if (o.sc_w) {
        // w = half the norm over the dims after the checkpoint (rounded up)
        // plus E_sc / 2, E_sc = sc_coef (P + pc): the remaining products satisfy
        // y_q y_c <= (y_q^2 + y_c^2) / 2, so a pair's accumulator at the
        // checkpoint plus w of both points (the margins covering every
        // rounding involved) bounds its full filter value from above
        const double full = (double)nrm;
        const double e_half = 0.5 * __dmul_ru(pp.sc_coef, __dadd_ru(pp.sc_p, full));
        o.sc_w[p] = __dadd_ru(0.5 * __dsub_ru(full, (double)nrm_b), e_half);
    }
}

// One thread per sorted position: the point is gathered through perm.
template <typename T>
__global__ void k_pack(const double* __restrict__ x, const int32_t* __restrict__ perm, int64_t n, const PackParams pp,
                       PackOut<T> o) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int32_t src_i = perm[p];
    pack_one<T>(x + (int64_t)src_i * pp.d, src_i, p, pp, o);
}

// k_pack for d == dp in {2, 4, 8} with the input dim order and no
// short-circuit bounds: the same arithmetic as pack_one in the same order
// (so the same bits), the rows moved with 16-byte loads and stores.
template <typename T, int DP>
__device__ __forceinline__ void store_row(T* dst, const T (&v)[DP]) {
    if constexpr (sizeof(T) == 8) {
#pragma unroll
        for (int h = 0; h < DP / 2; ++h) reinterpret_cast<double2*>(dst)[h] = make_double2(v[2 * h], v[2 * h + 1]);
    } else if constexpr (DP == 2) {
        *reinterpret_cast<float2*>(dst) = make_float2(v[0], v[1]);
    } else {
#pragma unroll
        for (int h = 0; h < DP / 4; ++h)
            reinterpret_cast<float4*>(dst)[h] = make_float4(v[4 * h], v[4 * h + 1], v[4 * h + 2], v[4 * h + 3]);
    }
}

template <typename T, int DP>
__global__ void k_pack_dp(const double* __restrict__ x, const int32_t* __restrict__ perm, int64_t n,
                          const PackParams pp, PackOut<T> o) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int32_t src_i = perm[p];
    double xv[DP];
#pragma unroll
    for (int h = 0; h < DP / 2; ++h) {
        const double2 v = reinterpret_cast<const double2*>(x + (int64_t)src_i * DP)[h];
        xv[2 * h] = v.x;
        xv[2 * h + 1] = v.y;
    }
    store_row<double, DP>(o.xs + p * DP, xv);
    T yv[DP];
    T nrm = T(0);
#pragma unroll
    for (int k = 0; k < DP; ++k) {
        yv[k] = T((xv[k] - pp.lo[k]) * pp.scale);
        nrm = fma_pack(yv[k], yv[k], nrm);
    }
    store_row<T, DP>(o.y + p * DP, yv);
    o.h[p] = -nrm * T(0.5);
    const T to = pack_thr_out(pp, nrm);
    const T ti = pp.has_in ? pack_thr_in(pp, nrm) : T(INFINITY);
    o.thr_out[p] = to;
    o.thr_in[p] = ti;
    if (o.aux) o.aux[p] = make_float4((float)to, (float)ti, __int_as_float(src_i), 0.f);
}

// The counting sort's scatter: one thread per input point takes its sorted
// position, off64[key] >> 32 plus its rank among the key's points (in the
// order warps reach the key).  (Fusing the packing into this scatter was
// measured slower: its scattered row writes cost more than k_pack's gather.)
__global__ void k_key_scatter(const uint32_t* __restrict__ key32, int64_t n,
                              const unsigned long long* __restrict__ off64, uint32_t* fill, int32_t* perm) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool valid = i < n;
    const uint32_t key = valid ? key32[i] : kNoKey;
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(peers) - 1;
    uint32_t b = 0;
    if (valid && lane == leader) b = atomicAdd(&fill[key], (uint32_t)__popc(peers));
    b = __shfl_sync(0xffffffffu, b, leader);
    if (valid) perm[(uint32_t)(off64[key] >> 32) + b + (uint32_t)__popc(peers & ((1u << lane) - 1u))] = (int32_t)i;
}

// Per-point records of the small-d FP32 filter: its two thresholds and its
// input index in one 16-byte load.
__global__ void k_aux(const float* __restrict__ to, const float* __restrict__ ti, const int32_t* __restrict__ perm,
                      int64_t n, float4* aux) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p < n) aux[p] = make_float4(to[p], ti[p], __int_as_float(perm[p]), 0.f);
}

int build_aux(Index* ix) {
    cudaStream_t s = ix->stream;
    float4* aux = nullptr;
    SJ_TRY(dev_alloc_t(&aux, (size_t)std::max<int64_t>(ix->n, 1), s));
    ix->aux = aux;
    k_aux<<<(unsigned)((ix->n + 255) / 256), 256, 0, s>>>(static_cast<const float*>(ix->thr_out),
                                                          static_cast<const float*>(ix->thr_in), ix->perm, ix->n, aux);
    note_launch();
    SJ_CK(cudaGetLastError());
    return SJ_OK;
}

// Pair evaluations of one work item: its queries times the candidates of
// its runs (a self-cell run starts at the item's first query when the join
// evaluates self-cell triangles, as the tile kernels load it).
__device__ __forceinline__ long long item_evals(const Item& I, const Run* __restrict__ runs, int tri) {
    long long c = 0;
    for (int32_t r = I.r0; r < I.r1; ++r) {
        const Run R = runs[r];
        const bool mirror = (R.end_flags & kMirrorBit) != 0u;
        const int32_t end = (int32_t)(R.end_flags & ~kMirrorBit);
        const int32_t start = (tri && !mirror) ? I.q0 : R.start;
        c += (long long)(end - start);
    }
    return c * (long long)(I.q1 - I.q0);
}

// Work per cell, reported at the cell's first work item (0 at its other
// items).  The items of one cell are consecutive and share their run list
// (the same r0), so a cell's first item is the one whose predecessor has
// another r0.
__global__ void k_item_work(const Item* __restrict__ items, const Run* __restrict__ runs, int64_t n_items, int tri,
                            long long* work) {
    const int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (it >= n_items) return;
    const Item I = items[it];
    if (it > 0 && items[it - 1].r0 == I.r0) {
        work[it] = 0;
        return;
    }
    long long c = item_evals(I, runs, tri);
    for (int64_t k = it + 1; k < n_items; ++k) {
        const Item J = items[k];
        if (J.r0 != I.r0) break;
        c += item_evals(J, runs, tri);
    }
    work[it] = c;
}

int launch_item_work(Index* ix, long long* work) {
    if (ix->n_items <= 0) return SJ_OK;
    k_item_work<<<(unsigned)((ix->n_items + 255) / 256), 256, 0, ix->stream>>>(ix->items, ix->runs, ix->n_items,
                                                                            uses_triangle(ix) ? 1 : 0, work);
    note_launch();
    SJ_CK(cudaGetLastError());
    return SJ_OK;
}

// ---------------------------------------------------------------------------
// neighbour runs and work items
// ---------------------------------------------------------------------------
struct EnumParams {
    int m;
    int64_t ncell[kMaxM];
    unsigned long long stride[kMaxM];
    int symmetric;
    int qmax;
    // a cell key is prefix | local key: the grid arithmetic uses the local
    // part (key & local_mask), neighbour keys keep the prefix (a batched
    // index puts the instance number there; a single index has no prefix)
    unsigned long long local_mask;
};

__device__ __forceinline__ int64_t lower_bound_u64(const unsigned long long* a, int64_t n, unsigned long long v) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] < v)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// Non-empty cells with keys in [k_lo, k_hi] (at most three consecutive
// keys): the index range [ca, cb) of the cell table.
__device__ __forceinline__ void cells_in_key_range(const EnumParams& e, const unsigned long long* __restrict__ cell_key,
                                                   int64_t n_cells, unsigned long long k_lo, unsigned long long k_hi,
                                                   int64_t& ca, int64_t& cb) {
    ca = lower_bound_u64(cell_key, n_cells, k_lo);
    cb = lower_bound_u64(cell_key, n_cells, k_hi + 1);
}

// Visits the candidate runs of cell c: for every offset vector o of the
// first m-1 indexed dims in {-1,0,1} inside the grid, the cells whose last
// coordinate is within one of c's form one contiguous key range, hence one
// contiguous range of sorted points.  In symmetric mode only offset vectors
// that are lexicographically positive keep their whole range; the zero vector
// keeps the cell itself (no mirroring) and the next cell along the last dim.
template <typename F>
__device__ void visit_runs(const EnumParams& e, const unsigned long long* __restrict__ cell_key,
                           const int32_t* __restrict__ cell_start, int64_t n_cells, int64_t c, F&& f) {
    if (e.m == 0) {  // a single cell holding every point
        f(cell_start[0], cell_start[n_cells], false);
        return;
    }
    const unsigned long long key = cell_key[c] & e.local_mask;
    const unsigned long long prefix = cell_key[c] & ~e.local_mask;
    int64_t cc[kMaxM];
    for (int k = 0; k < e.m; ++k) cc[k] = (int64_t)((key / e.stride[k]) % (unsigned long long)e.ncell[k]);
    const int mm = e.m - 1;
    int nvec = 1;
    for (int k = 0; k < mm; ++k) nvec *= 3;
    const int64_t last = cc[mm];
    const int64_t lo_l = last > 0 ? last - 1 : 0;
    const int64_t hi_l = last + 1 < e.ncell[mm] ? last + 1 : e.ncell[mm] - 1;
    for (int vi = 0; vi < nvec; ++vi) {
        // offset digit k is (vi / 3^k) % 3 - 1; the lexicographic sign is
        // that of the first non-zero digit in k order
        int rem = vi;
        long long delta = 0;
        int sign = 0;
        bool inside = true;
        for (int k = 0; k < mm; ++k) {
            const int o = rem % 3 - 1;
            rem /= 3;
            if (sign == 0 && o != 0) sign = o;
            if (cc[k] + o < 0 || cc[k] + o >= e.ncell[k]) inside = false;
            delta += (long long)o * (long long)e.stride[k];
        }
        if (!inside) continue;
        if (e.symmetric && sign < 0) continue;
        const unsigned long long base = prefix | (unsigned long long)((long long)key + delta);
        auto emit_range = [&](int64_t a_l, int64_t b_l, bool mirror) {
            if (a_l > b_l) return;
            int64_t ca, cb;
            cells_in_key_range(e, cell_key, n_cells, base - (unsigned long long)(last - a_l),
                               base + (unsigned long long)(b_l - last), ca, cb);
            if (ca >= cb) return;
            f(cell_start[ca], cell_start[cb], mirror);
        };
        if (!e.symmetric) {
            emit_range(lo_l, hi_l, false);
        } else if (sign > 0) {
            emit_range(lo_l, hi_l, true);
        } else {
            emit_range(last, last, false);
            emit_range(last + 1, hi_l, true);
        }
    }
}

struct EnumTotals {
    unsigned long long n_runs, n_items, n_evaluated, sum_sq, tri_skip;
};

// Evaluations a symmetric join saves by starting each work item's self-cell
// candidates at its own first query (the triangle of the self cell): item t
// of a cell (queries [t qmax, t qmax + Q_t)) skips the t qmax self-cell
// points before it.
__device__ __forceinline__ unsigned long long tri_skip(int64_t q, int qmax) {
    // sum over items t of t qmax Q_t: T full items, then one of r queries
    const unsigned long long T = (unsigned long long)(q / qmax), r = (unsigned long long)(q % qmax);
    const unsigned long long m = (unsigned long long)qmax;
    return m * m * (T * (T - (T > 0 ? 1ull : 0ull)) / 2) + T * m * r;
}

// Per cell: its run count, its item count, and the pair evaluations of its
// queries.  The canonical candidate count (full neighbourhoods, ordered) is
// the evaluations when not symmetric, else 2 * evaluations - sum_c |c|^2
// (each unordered pair of distinct adjacent cells is evaluated once and
// stands for both orders; a cell with itself is evaluated once).
__global__ void k_enum_count(EnumParams e, const unsigned long long* __restrict__ cell_key,
                             const int32_t* __restrict__ cell_start, int64_t n_cells, uint32_t* run_cnt,
                             uint32_t* item_cnt, EnumTotals* tot) {
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    unsigned long long my_sq = 0, my_eval = 0, my_runs = 0, my_items = 0, my_skip = 0;
    if (c < n_cells) {
        const int64_t q = cell_start[c + 1] - cell_start[c];
        uint32_t nr = 0;
        unsigned long long ev = 0;
        visit_runs(e, cell_key, cell_start, n_cells, c, [&](int32_t a, int32_t b, bool) {
            ++nr;
            ev += (unsigned long long)(b - a);
        });
        run_cnt[c] = nr;
        uint32_t ni = (uint32_t)((q + e.qmax - 1) / e.qmax);
        item_cnt[c] = ni;
        my_sq = (unsigned long long)q * (unsigned long long)q;
        my_eval = ev * (unsigned long long)q;
        my_runs = nr;
        my_items = ni;
        if (e.symmetric) my_skip = tri_skip(q, e.qmax);
    }
    // warp reduction then one atomic per warp
    for (int o = 16; o > 0; o >>= 1) {
        my_skip += __shfl_down_sync(0xffffffffu, my_skip, o);
        my_sq += __shfl_down_sync(0xffffffffu, my_sq, o);
        my_eval += __shfl_down_sync(0xffffffffu, my_eval, o);
        my_runs += __shfl_down_sync(0xffffffffu, my_runs, o);
        my_items += __shfl_down_sync(0xffffffffu, my_items, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&tot->sum_sq, my_sq);
        atomicAdd(&tot->tri_skip, my_skip);
        atomicAdd(&tot->n_evaluated, my_eval);
        atomicAdd(&tot->n_runs, my_runs);
        atomicAdd(&tot->n_items, my_items);
    }
}

__global__ void k_enum_fill(EnumParams e, const unsigned long long* __restrict__ cell_key,
                            const int32_t* __restrict__ cell_start, int64_t n_cells,
                            const uint32_t* __restrict__ run_off, const uint32_t* __restrict__ item_off,
                            Run* runs, Item* items) {
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= n_cells) return;
    uint32_t r = run_off[c];
    const uint32_t r0 = r;
    visit_runs(e, cell_key, cell_start, n_cells, c, [&](int32_t a, int32_t b, bool mirror) {
        Run rr;
        rr.start = a;
        rr.end_flags = (uint32_t)b | (mirror ? kMirrorBit : 0u);
        runs[r++] = rr;
    });
    const int32_t q0 = cell_start[c], q1 = cell_start[c + 1];
    uint32_t it = item_off[c];
    for (int32_t q = q0; q < q1; q += e.qmax) {
        Item x;
        x.q0 = q;
        x.q1 = q + e.qmax < q1 ? q + e.qmax : q1;
        x.r0 = (int32_t)r0;
        x.r1 = (int32_t)r;
        items[it++] = x;
    }
}

// ---------------------------------------------------------------------------
// neighbour runs and work items from the counting sort (dense key spaces)
// ---------------------------------------------------------------------------
// The counting sort gives, for every key k of the grid, its first sorted
// position start(k) = off64[k] >> 32 and its first work item off64[k] &
// 0xFFFFFFFF.  A range of consecutive keys [a, b] (a run of cells along the
// last indexed dim) is then the range of sorted points [start(a),
// start(b + 1)) directly: no table of non-empty cells is needed.  One thread
// per key; the run arithmetic is visit_runs' (same offsets, same order).
struct DenseEnum {
    int m;
    uint32_t ncell[kMaxM];
    uint32_t stride[kMaxM];
    int symmetric;
    uint32_t qmax;
    int64_t K;
};

struct DenseTotals {
    unsigned long long n_evaluated, sum_sq, tri_skip, n_cells, n_runs;
};

// MODE 0: count the runs of every key (run_cnt) and the totals; MODE 1: write
// runs at run_off[key] and the items; MODE 2: both in one pass, the runs of
// key k in fixed slots from k * slots (no count pass, no scan).
template <int MODE>
__global__ void k_denum(DenseEnum e, const unsigned long long* __restrict__ off64, uint32_t* run_cnt,
                        const uint32_t* __restrict__ run_off, Run* runs, Item* items, DenseTotals* tot,
                        uint32_t slots) {
    constexpr bool FILL = MODE >= 1;
    constexpr bool COUNT = MODE != 1;
    const int64_t key = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    unsigned long long my_eval = 0, my_sq = 0, my_skip = 0, my_cells = 0, my_runs = 0;
    if (key < e.K) {
        const unsigned long long a0 = off64[key], a1 = off64[key + 1];
        const uint32_t s0 = (uint32_t)(a0 >> 32);
        const uint32_t q = (uint32_t)(a1 >> 32) - s0;
        uint32_t nr = 0;
        unsigned long long ev = 0;
        const uint32_t r0 = MODE == 1 ? run_off[key] : MODE == 2 ? (uint32_t)key * slots : 0u;
        auto emit = [&](uint32_t ka, uint32_t kb, bool mirror) {  // keys [ka, kb]
            const int32_t a = (int32_t)(off64[ka] >> 32), b = (int32_t)(off64[kb + 1] >> 32);
            if (a >= b) return;
            if (FILL) {
                Run rr;
                rr.start = a;
                rr.end_flags = (uint32_t)b | (mirror ? kMirrorBit : 0u);
                runs[r0 + nr] = rr;
            }
            ++nr;
            ev += (unsigned long long)(b - a);
        };
        if (q > 0) {
            if (e.m == 0) {
                emit(0u, 0u, false);  // one cell holding every point
            } else {
                const uint32_t k32 = (uint32_t)key;
                uint32_t cc[kMaxM];
                for (int k = 0; k < e.m; ++k) cc[k] = (k32 / e.stride[k]) % e.ncell[k];
                const int mm = e.m - 1;
                int nvec = 1;
                for (int k = 0; k < mm; ++k) nvec *= 3;
                const uint32_t last = cc[mm];
                const uint32_t lo_l = last > 0 ? last - 1 : 0;
                const uint32_t hi_l = last + 1 < e.ncell[mm] ? last + 1 : e.ncell[mm] - 1;
#pragma unroll 3
                for (int vi = 0; vi < nvec; ++vi) {
                    int rem = vi, sign = 0;
                    long long delta = 0;
                    bool inside = true;
                    for (int k = 0; k < mm; ++k) {
                        const int o = rem % 3 - 1;
                        rem /= 3;
                        if (sign == 0 && o != 0) sign = o;
                        const long long c = (long long)cc[k] + o;
                        if (c < 0 || c >= (long long)e.ncell[k]) inside = false;
                        delta += (long long)o * (long long)e.stride[k];
                    }
                    if (!inside || (e.symmetric && sign < 0)) continue;
                    const uint32_t base = (uint32_t)((long long)k32 + delta);
                    if (!e.symmetric) {
                        emit(base - (last - lo_l), base + (hi_l - last), false);
                    } else if (sign > 0) {
                        emit(base - (last - lo_l), base + (hi_l - last), true);
                    } else {
                        emit(base, base, false);
                        if (hi_l > last) emit(base + 1, base + (hi_l - last), true);
                    }
                }
            }
        }
        if (FILL) {
            const uint32_t it0 = (uint32_t)(a0 & 0xFFFFFFFFull);
            for (uint32_t t = 0; t * e.qmax < q; ++t) {
                Item x;
                x.q0 = (int32_t)(s0 + t * e.qmax);
                x.q1 = (int32_t)(s0 + min(q, (t + 1) * e.qmax));
                x.r0 = (int32_t)r0;
                x.r1 = (int32_t)(r0 + nr);
                items[it0 + t] = x;
            }
        }
        if (COUNT) {
            if (MODE == 0) run_cnt[key] = nr;
            if (q > 0) {
                my_eval = ev * (unsigned long long)q;
                my_sq = (unsigned long long)q * (unsigned long long)q;
                if (e.symmetric) my_skip = tri_skip((int64_t)q, (int)e.qmax);
                my_cells = 1;
                my_runs = nr;
            }
        }
    }
    if (COUNT) {
        for (int o = 16; o > 0; o >>= 1) {
            my_eval += __shfl_down_sync(0xffffffffu, my_eval, o);
            my_sq += __shfl_down_sync(0xffffffffu, my_sq, o);
            my_skip += __shfl_down_sync(0xffffffffu, my_skip, o);
            my_cells += __shfl_down_sync(0xffffffffu, my_cells, o);
            my_runs += __shfl_down_sync(0xffffffffu, my_runs, o);
        }
        if ((threadIdx.x & 31) == 0 && my_cells) {
            atomicAdd(&tot->n_evaluated, my_eval);
            atomicAdd(&tot->sum_sq, my_sq);
            atomicAdd(&tot->tri_skip, my_skip);
            atomicAdd(&tot->n_cells, my_cells);
            atomicAdd(&tot->n_runs, my_runs);
        }
    }
}

// ---------------------------------------------------------------------------
// host orchestration
// ---------------------------------------------------------------------------
static int choose_grid(Index* ix) {
    const int d = ix->d;
    // w >= eps with a relative margin that absorbs the rounding of
    // (x - lo) * (1 / w), so two coordinates within eps are never two cells
    // apart; dims with 2^30 cells or more are not indexed (there the margin
    // would no longer cover the rounding).
    ix->w = ix->eps * (1.0 + ldexp(1.0, -20));
    const double inv_w = 1.0 / ix->w;
    struct Cand {
        int k;
        int64_t ncell;
    };
    std::vector<Cand> cand;
    for (int k = 0; k < d; ++k) {
        double r = ix->hi[k] - ix->lo[k];
        double cells = floor(r * inv_w) + 1.0;
        if (!(cells < ldexp(1.0, 30))) continue;  // too fine for a safe cell coordinate
        cand.push_back({k, (int64_t)cells});
    }
    // most selective dims first (most cells); ties keep the input order
    std::stable_sort(cand.begin(), cand.end(), [](const Cand& a, const Cand& b) { return a.ncell > b.ncell; });
    // SJ_NO_INDEX: no indexed dims, one cell, every pair evaluated (brute force)
    int want = ix->opt.indexed_dims > 0   ? std::min(ix->opt.indexed_dims, kMaxM)
               : ix->opt.indexed_dims < 0 ? 0
                                          : std::min(d, kMaxM);
    std::vector<Cand> take;
    long double prod = 1;
    for (const Cand& c : cand) {
        if ((int)take.size() >= want) break;
        if (ix->opt.indexed_dims <= 0 && c.ncell < 3) continue;  // no pruning from <3 cells
        if (prod * (long double)c.ncell > ldexpl(1.0L, ix->key_bits_cap)) continue;
        prod *= (long double)c.ncell;
        take.push_back(c);
    }
    // Batched instances (uniform data assumed): fewer indexed dims when that
    // costs less.  The distance kernels run work items of up to qmax queries
    // against every point of the item's neighbourhood: with M = min(n, cells
    // of the first m dims) cells of q = n / M points, and a dim of c cells
    // keeping the fraction (3c - 2) / c^2 of the points within +-1 cell, the
    // work is about M ceil(q / qmax) qmax n prod_k (3 c_k - 2) / c_k^2.  The
    // tensor-core filter's large items pay for few big cells.
    if (ix->trim_dims && ix->opt.indexed_dims <= 0 && !take.empty()) {
        const int qmax = item_qmax(ix);
        const double nn = (double)ix->n;
        int best = 0;
        double best_cost = 0, cells = 1, frac = 1;
        for (int j = 0; j <= (int)take.size(); ++j) {
            if (j > 0) {
                const double c = (double)take[j - 1].ncell;
                cells *= c;
                frac *= (3.0 * c - 2.0) / (c * c);
            }
            const double M = std::min(nn, cells), q = nn / M;
            const double cost = M * std::ceil(q / qmax) * qmax * nn * frac;
            if (j == 0 || cost < best_cost) {
                best = j;
                best_cost = cost;
            }
        }
        take.resize(best);
    }
    // keep the input order of the chosen dims (row-major keys)
    std::sort(take.begin(), take.end(), [](const Cand& a, const Cand& b) { return a.k < b.k; });
    ix->m = (int)take.size();
    unsigned long long stride = 1;
    for (int i = ix->m - 1; i >= 0; --i) {
        ix->dims[i] = take[i].k;
        ix->ncell[i] = take[i].ncell;
        ix->stride[i] = stride;
        stride *= (unsigned long long)take[i].ncell;
    }
    unsigned long long maxkey = stride - 1;
    ix->key_bits = 0;
    while (ix->key_bits < 64 && (maxkey >> ix->key_bits) != 0) ++ix->key_bits;
    return SJ_OK;
}

template <typename T>
static int pack_points(Index* ix, const double* pts, const PackParams& hp) {
    cudaStream_t s = ix->stream;
    const int64_t n = ix->n;
    // each array goes into the index as soon as it exists (released with it)
    PackOut<T> o{};
    SJ_TRY(dev_alloc_t(&ix->xs, (size_t)n * ix->dp, s));
    o.xs = ix->xs;
    SJ_TRY(dev_alloc_t(&o.y, (size_t)n * ix->dp, s));
    ix->y = o.y;
    SJ_TRY(dev_alloc_t(&o.h, (size_t)n, s));
    ix->h = o.h;
    SJ_TRY(dev_alloc_t(&o.thr_out, (size_t)n, s));
    ix->thr_out = o.thr_out;
    SJ_TRY(dev_alloc_t(&o.thr_in, (size_t)n, s));
    ix->thr_in = o.thr_in;
    if (std::is_same<T, float>::value && wants_aux(ix)) {
        SJ_TRY(dev_alloc_t(&o.aux, (size_t)n, s));
        ix->aux = o.aux;
    }
    if (std::is_same<T, double>::value && hp.sc_b > 0) {
        SJ_TRY(dev_alloc_t(&o.sc_w, (size_t)n, s));
        ix->sc_w = o.sc_w;
        ix->sc_b = hp.sc_b;
    }
    bool identity = true;
    for (int k = 0; k < ix->d; ++k) identity = identity && hp.order[k] == k;
    const bool rows16 = ix->d == ix->dp && identity && !o.sc_w && (reinterpret_cast<uintptr_t>(pts) & 15u) == 0;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    if (rows16 && ix->dp == 2)
        k_pack_dp<T, 2><<<blocks, 256, 0, s>>>(pts, ix->perm, n, hp, o);
    else if (rows16 && ix->dp == 4)
        k_pack_dp<T, 4><<<blocks, 256, 0, s>>>(pts, ix->perm, n, hp, o);
    else if (rows16 && ix->dp == 8)
        k_pack_dp<T, 8><<<blocks, 256, 0, s>>>(pts, ix->perm, n, hp, o);
    else
        k_pack<T><<<blocks, 256, 0, s>>>(pts, ix->perm, n, hp, o);
    note_launch();
    SJ_CK(cudaGetLastError());
    return SJ_OK;
}

// Split of an FP32 value into three 16-bit terms, each the round-to-nearest
// term of what is left (each difference is exact in FP32).  bf16 (8
// significant bits, FP32's exponent range): y = t1 + t2 + t3 exactly.  fp16
// (11 significant bits, normal down to 2^-14, subnormal spacing 2^-24): the
// terms keep 33 bits, and each remainder is at most 2^-11 of what it splits
// plus 2^-25 (a subnormal term's rounding).
__device__ __forceinline__ __nv_bfloat16 to_term(float v, __nv_bfloat16) { return __float2bfloat16_rn(v); }
__device__ __forceinline__ __half to_term(float v, __half) { return __float2half_rn(v); }
__device__ __forceinline__ float from_term(__nv_bfloat16 t) { return __bfloat162float(t); }
__device__ __forceinline__ float from_term(__half t) { return __half2float(t); }
template <typename H>
__device__ __forceinline__ void split3(float y, H& t1, H& t2, H& t3) {
    t1 = to_term(y, H());
    const float r1 = y - from_term(t1);
    t2 = to_term(r1, H());
    const float r2 = r1 - from_term(t2);
    t3 = to_term(r2, H());
}

// Operand rows of the tensor-core filter for every packed point: K slot
// 6k .. 6k+5 of dim k holds (c1, c2, c1, c3, c2, c1) in the candidate row and
// (q1, q1, q2, q1, q2, q3) in the query row, so their dot product keeps the
// six split products with term indices summing to at most 4; slots 6 dp ..
// 6 dp + 2 hold the split of -||y||^2 / 2 (query row) against ones
// (candidate row); the rest is zero.
//
// Layout: K is cut into slices of 64 (the last one shorter); slice by slice,
// the rows in 8-row groups, each group the K-major core matrices of the MMA
// operand (8 rows x 16 bytes) in K order.  So one K-slice of a run of
// consecutive groups is one contiguous block that a bulk copy moves into
// shared memory in the layout the MMA reads.
__device__ __forceinline__ int64_t split_at(int64_t p, int k, int kp, int64_t nrows) {
    const int sl = k >> 6, kk = k & 63;
    const int ks = kp - sl * 64 < 64 ? kp - sl * 64 : 64;
    return (int64_t)sl * 64 * nrows + (((p >> 3) * (ks >> 3) + (kk >> 3)) * 8 + (p & 7)) * 8 + (kk & 7);
}

// One thread per 16-byte chunk (8 K slots of one row): consecutive threads
// write consecutive rows of a chunk, so a warp stores whole 128-byte lines.
// prod = 6 (BF16x3) or 3 (BF16x2 and FP16x2: per dim candidate (c1, c2, c1),
// query (q1, q1, q2) of the first two split terms, which t1 and t2 of split3
// are).  H: the term type (bf16, or fp16 for FP16x2).  The three h slots hold
// hs in the candidate row and the split of h / hs in the query row (hs a
// power of two: 1 for bf16, 2^15 for fp16, whose range stops at 65504).
template <typename H, int PROD, int KP>
__global__ void k_pack_split(const float* __restrict__ y, const float* __restrict__ h, int64_t n, int dp,
                             int64_t nrows, float hs, H* rows_a, H* rows_b) {
    constexpr int CH = KP / 8;  // 16-byte chunks per row (compile-time: no run-time division)
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t grp = t / (8 * CH);
    const int c = (int)((t >> 3) % CH);
    const int64_t p = grp * 8 + (t & 7);
    if (p >= nrows) return;
    const bool live = p < n;  // padding rows (p >= n) are written as zeros
    const H zero = to_term(0.f, H()), hterm = to_term(hs, H());
    __align__(16) H av[8], bv[8];
    int last = -1;  // the coordinate whose split t1 .. t3 hold
    H t1 = zero, t2 = zero, t3 = zero;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int k = c * 8 + u;
        H a = zero, b = zero;
        if (!live) {
        } else if (k < PROD * dp) {
            const int j = k / PROD, r = k - j * PROD;
            if (j != last) {  // each coordinate split once per thread
                split3(y[p * dp + j], t1, t2, t3);
                last = j;
            }
            if (PROD == 6) {
                switch (r) {  // candidate (c1, c2, c1, c3, c2, c1), query (q1, q1, q2, q1, q2, q3)
                    case 0: a = t1; b = t1; break;
                    case 1: a = t2; b = t1; break;
                    case 2: a = t1; b = t2; break;
                    case 3: a = t3; b = t1; break;
                    case 4: a = t2; b = t2; break;
                    default: a = t1; b = t3; break;
                }
            } else {
                switch (r) {  // candidate (c1, c2, c1), query (q1, q1, q2)
                    case 0: a = t1; b = t1; break;
                    case 1: a = t2; b = t1; break;
                    default: a = t1; b = t2; break;
                }
            }
        } else if (k < PROD * dp + 3) {
            H h1, h2, h3;
            split3(h[p] / hs, h1, h2, h3);  // (exact: hs is a power of two)
            a = hterm;
            b = k == PROD * dp ? h1 : (k == PROD * dp + 1 ? h2 : h3);
        }
        av[u] = a;
        bv[u] = b;
    }
    const int64_t o = split_at(p, c * 8, KP, nrows);
    *reinterpret_cast<uint4*>(rows_a + o) = *reinterpret_cast<const uint4*>(av);
    *reinterpret_cast<uint4*>(rows_b + o) = *reinterpret_cast<const uint4*>(bv);
}

template <typename H, int PROD, int KP>
static void launch_pack_split(const Index* ix, int64_t nrows, float hs, void* ra, void* rb, cudaStream_t s) {
    const int64_t threads = nrows * (KP / 8);
    k_pack_split<H, PROD, KP><<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(
        static_cast<const float*>(ix->y), static_cast<const float*>(ix->h), ix->n, ix->dp, nrows, hs,
        static_cast<H*>(ra), static_cast<H*>(rb));
}

template <typename H, int PROD>
static int launch_pack_split_k(const Index* ix, int64_t nrows, float hs, void* ra, void* rb, cudaStream_t s) {
    switch (ix->kp) {
        case 16: launch_pack_split<H, PROD, 16>(ix, nrows, hs, ra, rb, s); break;
        case 32: launch_pack_split<H, PROD, 32>(ix, nrows, hs, ra, rb, s); break;
        case 64: launch_pack_split<H, PROD, 64>(ix, nrows, hs, ra, rb, s); break;
        case 112: launch_pack_split<H, PROD, 112>(ix, nrows, hs, ra, rb, s); break;
        case 208: launch_pack_split<H, PROD, 208>(ix, nrows, hs, ra, rb, s); break;
        case 400: launch_pack_split<H, PROD, 400>(ix, nrows, hs, ra, rb, s); break;
        default:
            set_error("no split-row packing for K = %d", ix->kp);
            return SJ_ERR_UNSUPPORTED;
    }
    return SJ_OK;
}

static int pack_split_rows(Index* ix) {
    cudaStream_t s = ix->stream;
    const int64_t n = ix->n;
    ix->kp = tc_kp(ix->dp, ix->kernel);
    const int64_t nrows = ((n + 7) & ~int64_t(7)) + kTcPadRows;
    const size_t elems = (size_t)nrows * ix->kp;
    uint16_t *ra = nullptr, *rb = nullptr;  // 16-bit terms (bf16 or fp16)
    SJ_TRY(dev_alloc_t(&ra, elems, s));
    ix->rows_a = ra;
    SJ_TRY(dev_alloc_t(&rb, elems, s));
    ix->rows_b = rb;
    // every slot of every row is written (padding rows as zeros): no memset
    if (ix->kernel == SJ_KERNEL_FILTER_FP16X2)
        SJ_TRY((launch_pack_split_k<__half, 3>(ix, nrows, 32768.f, ra, rb, s)));
    else if (tc_products(ix->kernel) == 3)
        SJ_TRY((launch_pack_split_k<__nv_bfloat16, 3>(ix, nrows, 1.f, ra, rb, s)));
    else
        SJ_TRY((launch_pack_split_k<__nv_bfloat16, 6>(ix, nrows, 1.f, ra, rb, s)));
    note_launch();
    SJ_CK(cudaGetLastError());
    return SJ_OK;
}

// Tensor-core filter: |s_y - (pc - 2a)| <= gamma_32(dp) (Pq + Pc) for the
// FP32 norms plus twice the dot-product error.  The products of bf16 terms are
// exact in FP32; the FP32 accumulation of K products is taken to lose up to
// 2^-22 relative at every addition (truncation): at most 1.02 K 2^-22 (Pq+Pc).
// The split products left out add, relative to sum_k |yq_k| |yc_k| <=
// (Pq + Pc) / 2: BF16x3 (y = t1 + t2 + t3 exactly, 8 bits each; the three
// products whose term indices sum to 5 or 6) below 2^-23 in all, so at most
// 2^-23 (Pq + Pc); BF16x2 (y = t1 + t2 + r, |t2| <= 2^-8 |y|, |r| <= 2^-16 |y|;
// t2 t2', r (t1' + t2') and r' (t1 + t2) left out) at most 3.01 2^-16, so
// 1.51 2^-16 (Pq + Pc).  FP16x2 (the same three products of fp16 terms of the
// scaled coordinates v = y S, with S^2 P in (2^28, 2^30]): a term in fp16's
// subnormal range is off by at most a = 2^-14 whether the tensor core keeps
// it (2^-25) or flushes it to zero, so |v - t1| <= 2^-11 |v| + a,
// |r| <= 2^-22 |v| + 1.001 a and |t2| <= 2^-11 (1 + 2^-11) |v| + 2.001 a; the
// left-out products are at most 3.01 2^-22 |v| |v'| per dim
// (1.51 2^-22 (Pq + Pc) in all) plus an absolute part below
// 1.01 a sum_k (|v_k| + |v'_k|) + 5 a^2 dp <= 1.01 2^-13 sqrt(dp P) + 5 dp 2^-28
// <= 1.02 sqrt(dp) 2^-27 P (as P > 2^28); the query's -||v||^2 / 2 goes in as
// 2^15 times the 3 fp16 terms of its 2^-15 part (33 bits, each off by at most
// a), which miss at most 2^-33 of it plus 3 a 2^15 < 2^-25 P.  The sum is
// doubled (for 2a) and doubled again for safety.
double tc_c1(int dp, int kernel) {
    const int kp = tc_kp(dp, kernel);
    const double norms = 2.0 * gamma_n(ldexp(1.0, -24), dp);
    const double acc = 4.1 * kp * ldexp(1.0, -22);
    double split = 2.0 * ldexp(1.0, -22);  // BF16x3
    if (kernel == SJ_KERNEL_FILTER_BF16X2) split = 6.1 * ldexp(1.0, -16);
    if (kernel == SJ_KERNEL_FILTER_FP16X2)
        split = 4.0 * (1.51 * ldexp(1.0, -22) + 1.02 * std::sqrt((double)dp) * ldexp(1.0, -27) + ldexp(1.0, -25) +
                       ldexp(1.0, -33));
    return norms + acc + split;
}

// The dense path's enumeration: its parameters, the totals, and the item
// array (upper bound: at most q / qmax + 1 items per non-empty cell, at most
// min(n, K) cells); with fixed run slots (K (3^(m-1) + 1) runs in at most
// 512 MB) also the run array, so one pass fills both.
struct DensePlan {
    DenseEnum de;
    DenseTotals* dtot;
    unsigned eb;
    int64_t slots, cells_max, items_cap, runs_cap;
    bool fixed;
};

static int dense_enum_prepare(Index* ix, int64_t K, int qmax, Scratch& tmp, DensePlan* dp) {
    cudaStream_t s = ix->stream;
    const int64_t n = ix->n;
    DenseEnum& de = dp->de;
    de = DenseEnum{};
    de.m = ix->m;
    for (int i = 0; i < ix->m; ++i) {
        de.ncell[i] = (uint32_t)ix->ncell[i];
        de.stride[i] = (uint32_t)ix->stride[i];
    }
    de.symmetric = ix->opt.symmetric ? 1 : 0;
    de.qmax = (uint32_t)qmax;
    de.K = K;
    SJ_TRY(tmp.alloc(&dp->dtot, 1));
    SJ_CK(cudaMemsetAsync(dp->dtot, 0, sizeof(DenseTotals), s));
    dp->eb = (unsigned)((K + 127) / 128);
    // runs of a cell: at most 3^(m-1), one more when the self offset splits
    // (symmetric joins)
    int mm = ix->m > 0 ? ix->m - 1 : 0, per = 1;
    for (int k = 0; k < mm; ++k) per *= 3;
    dp->slots = per + 1;
    dp->cells_max = std::min<int64_t>(n, K);
    dp->items_cap = dp->cells_max + n / qmax + 1;
    SJ_TRY(dev_alloc_t(&ix->items, (size_t)std::max<int64_t>(dp->items_cap, 1), s));
    dp->fixed = K * dp->slots * (int64_t)sizeof(Run) <= (int64_t(512) << 20);
    dp->runs_cap = 0;
    if (dp->fixed) {
        dp->runs_cap = K * dp->slots;
        SJ_TRY(dev_alloc_t(&ix->runs, (size_t)std::max<int64_t>(dp->runs_cap, 1), s));
    }
    return SJ_OK;
}

int build_index(Index* ix, const double* pts) {
    cudaStream_t s = ix->stream;
    const int64_t n = ix->n;
    const int d = ix->d;
    Scratch tmp(s);  // temporaries, released on every return
    // side-stream work (below) is joined back into s on every return, before
    // the temporaries above or the index's arrays are released
    struct SideJoin {
        cudaStream_t s;
        cudaEvent_t ev = nullptr;
        ~SideJoin() {
            if (ev) cudaStreamWaitEvent(s, ev, 0);
        }
    } side_join{s};
    PhaseClock clock(s);
    clock.mark();
    // ---- extent and finiteness check (one sync) ----
    unsigned long long* ext = nullptr;
    SJ_TRY(tmp.alloc(&ext, (size_t)2 * d + 1));
    // minima start at all ones, maxima and the non-finite flag at zero
    SJ_CK(cudaMemsetAsync(ext, 0xFF, (size_t)d * 8, s));
    SJ_CK(cudaMemsetAsync(ext + d, 0, (size_t)(d + 1) * 8, s));
    {
        const int64_t total = n * d;
        const int bs = 256 - (256 % d);  // a multiple of d (d <= 128)
        const int blocks = (int)std::min<int64_t>((total + bs - 1) / bs, (int64_t)device_sm_count(ix->device) * 8);
        k_extent<<<blocks, bs, 2 * d * sizeof(unsigned long long), s>>>(
            pts, total, d, ext, ext + d, reinterpret_cast<int*>(ext + 2 * d));
        note_launch();
        SJ_CK(cudaGetLastError());
    }
    // the short-circuit of the FP64 tile orders the kernel dims by variance
    const bool short_circuit = ix->kernel == SJ_KERNEL_FP64_FMA && ix->opt.short_circuit && ix->dp >= 16;
    std::vector<double> mom(2 * d, 0.0);
    double* dmom = nullptr;
    if (short_circuit) {
        SJ_TRY(tmp.alloc(&dmom, (size_t)2 * d));
        SJ_CK(cudaMemsetAsync(dmom, 0, 2 * d * sizeof(double), s));
        const int64_t total = n * d;
        const int bs = 256 - (256 % d);
        const int blocks = (int)std::min<int64_t>((total + bs - 1) / bs, (int64_t)device_sm_count(ix->device) * 8);
        k_moments<<<blocks, bs, 2 * d * sizeof(double), s>>>(pts, total, d, dmom);
        note_launch();
        SJ_CK(cudaGetLastError());
        SJ_CK(cudaMemcpyAsync(mom.data(), dmom, 2 * d * sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    std::vector<unsigned long long> got(2 * d + 1);
    {
        void* hs = host_staging(got.size() * 8);  // pinned: a direct copy
        SJ_CK(cudaMemcpyAsync(hs ? hs : got.data(), ext, got.size() * 8, cudaMemcpyDeviceToHost, s));
        SJ_CK(cudaStreamSynchronize(s));
        if (hs) memcpy(got.data(), hs, got.size() * 8);
    }
    if (*reinterpret_cast<int*>(&got[2 * d]) != 0) {
        set_error("non-finite coordinate in the input points");
        return SJ_ERR_ARG;
    }
    ix->lo.resize(d);
    ix->hi.resize(d);
    for (int k = 0; k < d; ++k) {
        ix->lo[k] = from_ord(got[k]);
        ix->hi[k] = from_ord(got[d + k]);
    }
    SJ_TRY(choose_grid(ix));
    clock.mark();

    // ---- packing parameters ----
    // kernel coordinates y = x - centre of the extent: |y_k| <= R_k / 2, which
    // keeps the norms in the expanded form (and the certified band) small
    PackParams hp{};
    double pb = 0, rmax = 0;
    for (int k = 0; k < d; ++k) {
        hp.lo[k] = 0.5 * (ix->lo[k] + ix->hi[k]);
        const double r = 0.5 * (ix->hi[k] - ix->lo[k]) * (1.0 + ldexp(1.0, -40));
        pb += r * r;
        rmax = std::max(rmax, r);
    }
    const double pbound = pb * (1.0 + ldexp(1.0, -20));
    hp.d = d;
    hp.dp = ix->dp;
    // kernel dim order: input order, or decreasing variance (ties: input
    // order) for the short-circuit, so the partial sums grow fastest
    std::vector<int> order(d);
    std::iota(order.begin(), order.end(), 0);
    if (short_circuit) {
        std::vector<double> var(d);
        for (int k = 0; k < d; ++k) {
            const double mean = mom[k] / (double)n;
            var[k] = mom[d + k] / (double)n - mean * mean;
        }
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return var[a] > var[b]; });
        // one checkpoint at half the dims (a multiple of 8): a pair whose
        // partial distance there already exceeds eps is out
        hp.sc_b = std::max(8, ix->dp / 2 / 8 * 8);
        hp.sc_coef = 8.0 * gamma_n(ldexp(1.0, -53), ix->dp + 1);
        hp.sc_p = pbound;
    }
    for (int k = 0; k < d; ++k) hp.order[k] = (uint8_t)order[k];
    ix->dim_order = order;
    // binary32 kernel coordinates (the FP32 and tensor-core filters) are
    // scaled into binary32's range (binary32_scale); an extent that cannot be
    // scaled runs the binary64 tile under AUTO and is refused otherwise
    double scale = 1.0;
    if ((ix->kernel == SJ_KERNEL_FILTER_F32 || is_tensor_kernel(ix->kernel)) && !binary32_scale(pbound, &scale)) {
        if (ix->opt.kernel != SJ_KERNEL_AUTO) {
            set_error("binary32 kernel coordinates cannot hold an extent with P = %g (take an FP64 kernel)", pbound);
            return SJ_ERR_UNSUPPORTED;
        }
        ix->kernel = SJ_KERNEL_FP64_FMA;
    }
    const bool tensor = is_tensor_kernel(ix->kernel);
    const bool use_f32 = ix->kernel == SJ_KERNEL_FILTER_F32 || tensor;
    const double u_t = use_f32 ? ldexp(1.0, -24) : ldexp(1.0, -53);
    const double delta = 1.01 * u_t * rmax;
    double c1 = -1.0;  // (the tensor-core filter's bound: tc_c1)
    if (tensor) c1 = tc_c1(ix->dp, ix->kernel);
    hp.scale = scale;
    ix->kscale = scale;
    pack_coefficients(ix->eps * scale, pbound * scale * scale, delta * scale, u_t, d, ix->dp, &hp, c1);
    ix->prune_r2 = hp.prune_r2f;

    // ---- cell keys, sort and packing ----
    SJ_TRY(dev_alloc_t(&ix->perm, (size_t)n, s));
    GridParams gp{};
    gp.m = ix->m;
    gp.inv_w = 1.0 / ix->w;
    for (int i = 0; i < ix->m; ++i) {
        gp.dims[i] = ix->dims[i];
        gp.lo[i] = ix->lo[ix->dims[i]];
        gp.ncell[i] = ix->ncell[i];
        gp.stride[i] = ix->stride[i];
    }
    // the key space: small enough (at most max(4 n, 2^22) keys) for a
    // counting sort whose per-key first positions index the cells directly
    long double kspace = 1;
    for (int i = 0; i < ix->m; ++i) kspace *= (long double)ix->ncell[i];
    const bool dense = kspace <= (long double)std::max<int64_t>(4 * n, int64_t(1) << 22) &&
                       kspace < (long double)0x7FFFFFFF;
    const int qmax = item_qmax(ix);
    const int64_t K = dense ? (int64_t)kspace : 0;
    DensePlan dp{};  // dense path: the enumeration's parameters and arrays
    unsigned long long* off64 = nullptr;     // dense: K + 1 of (first position << 32 | first item)
    unsigned long long* ckey_tmp = nullptr;  // sparse: cell table before the cell count is known
    int32_t* cstart_tmp = nullptr;
    unsigned long long* dcount = nullptr;
    if (dense) {
        // ---- counting sort: per-key counts, one scan for first positions
        // and first work items, scatter ----
        uint32_t *key32 = nullptr, *bins = nullptr;
        SJ_TRY(tmp.alloc(&key32, (size_t)n));
        SJ_TRY(tmp.alloc(&bins, (size_t)K * 2));
        SJ_TRY(tmp.alloc(&off64, (size_t)K + 1));
        uint32_t *cnt = bins, *fill = bins + K;
        SJ_CK(cudaMemsetAsync(bins, 0, (size_t)K * 2 * sizeof(uint32_t), s));  // cnt and fill
        k_key_count<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(pts, n, d, gp, key32, cnt);
        note_launch();
        SJ_CK(cudaGetLastError());
        SJ_TRY((scan_exclusive<unsigned long long, LoadCountItems>(LoadCountItems{cnt, (uint32_t)qmax}, off64, K,
                                                                   true, s)));
        // the runs and items depend on the keys' first positions only, the
        // scatter and the packing on the order: with fixed run slots the
        // enumeration runs on a side stream beside them
        SJ_TRY(dense_enum_prepare(ix, K, qmax, tmp, &dp));
        if (dp.fixed) {
            cudaStream_t side = nullptr;
            SJ_TRY(side_stream(ix->device, &side));
            for (int e = 0; e < 2; ++e)
                if (!ix->ev_side[e]) SJ_CK(cudaEventCreateWithFlags(&ix->ev_side[e], cudaEventDisableTiming));
            SJ_CK(cudaEventRecord(ix->ev_side[0], s));
            SJ_CK(cudaStreamWaitEvent(side, ix->ev_side[0], 0));
            k_denum<2><<<dp.eb, 128, 0, side>>>(dp.de, off64, nullptr, nullptr, ix->runs, ix->items, dp.dtot,
                                                (uint32_t)dp.slots);
            note_launch();
            SJ_CK(cudaGetLastError());
            SJ_CK(cudaEventRecord(ix->ev_side[1], side));
            side_join.ev = ix->ev_side[1];
        }
        k_key_scatter<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(key32, n, off64, fill, ix->perm);
        note_launch();
        SJ_CK(cudaGetLastError());
    } else {
        // ---- radix sort and cell table ----
        unsigned long long* keys = nullptr;
        uint32_t *flags = nullptr, *idx = nullptr;
        SJ_TRY(tmp.alloc(&keys, (size_t)n));
        SJ_TRY(tmp.alloc(&dcount, 1));
        k_cell_keys<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(pts, n, d, gp, keys, ix->perm);
        note_launch();
        SJ_CK(cudaGetLastError());
        SJ_TRY(radix_sort_pairs(reinterpret_cast<uint64_t*>(keys), ix->perm, n, ix->key_bits, s));
        SJ_TRY(tmp.alloc(&flags, (size_t)n));
        SJ_TRY(tmp.alloc(&idx, (size_t)n));
        k_heads<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(keys, n, flags);
        note_launch();
        SJ_CK(cudaGetLastError());
        SJ_TRY(scan_exclusive_u32(flags, idx, n, s));
        SJ_TRY(tmp.alloc(&ckey_tmp, (size_t)n));
        SJ_TRY(tmp.alloc(&cstart_tmp, (size_t)n + 1));
        k_cells<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(keys, flags, idx, n, ckey_tmp, cstart_tmp, dcount);
        note_launch();
        SJ_CK(cudaGetLastError());
    }
    clock.mark();
    // ---- packing (gathered through perm) ----
    if (use_f32)
        SJ_TRY(pack_points<float>(ix, pts, hp));
    else
        SJ_TRY(pack_points<double>(ix, pts, hp));
    if (tensor) SJ_TRY(pack_split_rows(ix));
    ix->filter_band_rel = 2.0 * (c1 > 0 ? c1 : 6.2 * gamma_n(u_t, ix->dp + 1)) * 2.0 * pbound / ix->e2;
    ix->bound_c1 = c1 > 0 ? c1 : 6.2 * gamma_n(u_t, ix->dp + 1);
    ix->bound_p = pbound * scale * scale;  // in kernel coordinates
    clock.mark();

    if (dense) {
        // ---- neighbour runs and work items, per key; one read-back at the
        // end of the build ----
        const DenseEnum& de = dp.de;
        DenseTotals* dtot = dp.dtot;
        const unsigned eb = dp.eb;
        const int64_t slots = dp.slots, cells_max = dp.cells_max, items_cap = dp.items_cap;
        int64_t runs_cap = dp.runs_cap;
        uint32_t* run_off = nullptr;  // count pass: K + 1 run offsets
        if (dp.fixed) {
            // one pass (launched on the side stream above): the runs of key k
            // in the fixed slots k * slots ..
            SJ_CK(cudaStreamWaitEvent(s, ix->ev_side[1], 0));
        } else {
            // count pass, scan, fill pass; the run array sized by the upper
            // bound (non-empty cells <= min(n, K)) when that is moderate, else
            // by the exact count read back
            uint32_t* run_cnt = nullptr;  // K counts, then K + 1 offsets
            SJ_TRY(tmp.alloc(&run_cnt, (size_t)2 * K + 1));
            run_off = run_cnt + K;
            k_denum<0><<<eb, 128, 0, s>>>(de, off64, run_cnt, nullptr, nullptr, nullptr, dtot, 0u);
            note_launch();
            SJ_CK(cudaGetLastError());
            SJ_TRY((scan_exclusive<uint32_t, LoadU32>(LoadU32{run_cnt}, run_off, K, true, s)));
            runs_cap = cells_max * slots;
            if (runs_cap * (int64_t)sizeof(Run) > (int64_t(1) << 30)) {
                uint32_t total = 0;
                SJ_CK(cudaMemcpyAsync(&total, run_off + K, 4, cudaMemcpyDeviceToHost, s));
                SJ_CK(cudaStreamSynchronize(s));
                runs_cap = (int64_t)total;
            }
            SJ_TRY(dev_alloc_t(&ix->runs, (size_t)std::max<int64_t>(runs_cap, 1), s));
            k_denum<1><<<eb, 128, 0, s>>>(de, off64, nullptr, run_off, ix->runs, ix->items, nullptr, 0u);
            note_launch();
            SJ_CK(cudaGetLastError());
        }
        struct Got {
            DenseTotals t;
            unsigned long long last_off;
        } got{};
        // everything the join needs that does not depend on the totals is set
        // up before waiting for them: the counters, and the release of the
        // build's temporaries (stream-ordered, after the copies below)
        SJ_TRY(dev_alloc_t(&ix->counters, kCounters, s));
        Got* hg = static_cast<Got*>(host_staging(sizeof(Got)));  // pinned: direct copies
        Got* dst = hg ? hg : &got;
        SJ_CK(cudaMemcpyAsync(&dst->t, dtot, sizeof(DenseTotals), cudaMemcpyDeviceToHost, s));
        SJ_CK(cudaMemcpyAsync(&dst->last_off, off64 + K, 8, cudaMemcpyDeviceToHost, s));
        tmp.release();
        SJ_CK(cudaStreamSynchronize(s));
        if (hg) got = *hg;
        ix->n_cells = (int64_t)got.t.n_cells;
        ix->n_runs = (int64_t)got.t.n_runs;
        ix->n_items = (int64_t)(got.last_off & 0xFFFFFFFFull);
        ix->n_candidates =
            de.symmetric ? (int64_t)(2 * got.t.n_evaluated - got.t.sum_sq) : (int64_t)got.t.n_evaluated;
        ix->n_evaluated = (int64_t)(got.t.n_evaluated - (uses_triangle(ix) ? got.t.tri_skip : 0ull));
        if ((int64_t)(got.last_off >> 32) != n || (run_off && ix->n_runs > runs_cap) || ix->n_items > items_cap) {
            set_error("internal: dense index sizes inconsistent (%lld points, %lld runs, %lld items)",
                      (long long)(got.last_off >> 32), (long long)ix->n_runs, (long long)ix->n_items);
            return SJ_ERR_CUDA;
        }
        clock.mark();
        clock.finish(ix);
        return SJ_OK;
    }

    // ---- sparse key space: cell table, neighbour runs and items (one sync
    // for the cell count, one for the totals) ----
    unsigned long long M = 0;
    SJ_CK(cudaMemcpyAsync(&M, dcount, 8, cudaMemcpyDeviceToHost, s));
    SJ_CK(cudaStreamSynchronize(s));
    ix->n_cells = (int64_t)M;
    SJ_TRY(dev_alloc_t(&ix->cell_key, (size_t)M, s));
    SJ_TRY(dev_alloc_t(&ix->cell_start, (size_t)M + 1, s));
    SJ_CK(cudaMemcpyAsync(ix->cell_key, ckey_tmp, M * 8, cudaMemcpyDeviceToDevice, s));
    SJ_CK(cudaMemcpyAsync(ix->cell_start, cstart_tmp, (M + 1) * 4, cudaMemcpyDeviceToDevice, s));
    EnumParams ep{};
    ep.m = ix->m;
    for (int i = 0; i < ix->m; ++i) {
        ep.ncell[i] = ix->ncell[i];
        ep.stride[i] = ix->stride[i];
    }
    ep.symmetric = ix->opt.symmetric ? 1 : 0;
    ep.qmax = qmax;
    const int64_t Mc = (int64_t)M;
    ep.local_mask = ~0ull;
    uint32_t *run_cnt, *item_cnt, *run_off, *item_off;
    EnumTotals* dtot;
    SJ_TRY(tmp.alloc(&run_cnt, (size_t)Mc * 4));
    item_cnt = run_cnt + Mc;
    run_off = run_cnt + 2 * Mc;
    item_off = run_cnt + 3 * Mc;
    SJ_TRY(tmp.alloc(&dtot, 1));
    SJ_CK(cudaMemsetAsync(dtot, 0, sizeof(EnumTotals), s));
    const unsigned eb = (unsigned)((Mc + 127) / 128);
    k_enum_count<<<eb, 128, 0, s>>>(ep, ix->cell_key, ix->cell_start, Mc, run_cnt, item_cnt, dtot);
    note_launch();
    SJ_CK(cudaGetLastError());
    SJ_TRY(scan_exclusive_u32(run_cnt, run_off, Mc, s));
    SJ_TRY(scan_exclusive_u32(item_cnt, item_off, Mc, s));
    EnumTotals tot{};
    SJ_CK(cudaMemcpyAsync(&tot, dtot, sizeof tot, cudaMemcpyDeviceToHost, s));
    SJ_CK(cudaStreamSynchronize(s));
    ix->n_runs = (int64_t)tot.n_runs;
    ix->n_items = (int64_t)tot.n_items;
    ix->n_candidates = ep.symmetric ? (int64_t)(2 * tot.n_evaluated - tot.sum_sq) : (int64_t)tot.n_evaluated;
    // the CUDA-core kernels evaluate only the triangle of each self cell
    ix->n_evaluated = (int64_t)(tot.n_evaluated - (uses_triangle(ix) ? tot.tri_skip : 0ull));
    if (tot.n_runs >= 0xFFFFFFFFull || tot.n_items >= 0x7FFFFFFFull) {
        set_error("index too large: %llu runs, %llu items", tot.n_runs, tot.n_items);
        return SJ_ERR_ARG;
    }
    SJ_TRY(dev_alloc_t(&ix->runs, (size_t)std::max<int64_t>(ix->n_runs, 1), s));
    SJ_TRY(dev_alloc_t(&ix->items, (size_t)std::max<int64_t>(ix->n_items, 1), s));
    k_enum_fill<<<eb, 128, 0, s>>>(ep, ix->cell_key, ix->cell_start, Mc, run_off, item_off, ix->runs, ix->items);
    note_launch();
    SJ_CK(cudaGetLastError());
    SJ_TRY(dev_alloc_t(&ix->counters, kCounters, s));
    clock.mark();
    clock.finish(ix);
    return SJ_OK;
}

}  // namespace sj

namespace sj {

// Launchers used by the allocation-free entry point (sj_noalloc.cu): the
// extent reduction and the FP64 packing on caller-provided memory.
int launch_extent_raw(const double* pts, int64_t n, int d, unsigned long long* ext, cudaStream_t s) {
    const int64_t total = n * d;
    const int bs = 256 - (256 % d);
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((total + bs - 1) / bs, 152 * 8));
    k_extent<<<blocks, bs, 2 * d * sizeof(unsigned long long), s>>>(pts, total, d, ext, ext + d,
                                                                    reinterpret_cast<int*>(ext + 2 * d));
    note_launch();
    SJ_CK(cudaGetLastError());
    return SJ_OK;
}

size_t pack_params_size() { return sizeof(PackParams); }

int pack_params_fill(void* host_pp, const double* lo, int d, int dp, double eps, double pbound, double delta) {
    PackParams* pp = static_cast<PackParams*>(host_pp);
    *pp = PackParams{};  // zeros, scale 1
    for (int k = 0; k < d; ++k) {
        pp->lo[k] = lo[k];
        pp->order[k] = (uint8_t)k;
    }
    pp->d = d;
    pp->dp = dp;
    pack_coefficients(eps, pbound, delta, ldexp(1.0, -53), d, dp, pp);
    return SJ_OK;
}

int launch_pack_f64_raw(const double* pts, const int32_t* perm, int64_t n, const void* host_pp, double* xs, double* y,
                        double* h, double* to, double* ti, cudaStream_t s) {
    PackOut<double> o{xs, y, h, to, ti, nullptr, nullptr};
    k_pack<double><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(pts, perm, n, *static_cast<const PackParams*>(host_pp),
                                                             o);
    note_launch();
    SJ_CK(cudaGetLastError());
    return SJ_OK;
}

}  // namespace sj

// ===========================================================================
// Batched index (sj_join_batch): the instances of one group (same padded
// dimension) share one index whose cell keys are instance << S | local key,
// built with segmented versions of the kernels above.
// ===========================================================================
namespace sj {

// Grid and threshold parameters of one instance.
struct BInst {
    int m;
    int dims[kMaxM];
    double lo[kMaxM];
    int64_t ncell[kMaxM];
    unsigned long long stride[kMaxM];
    double inv_w;
    double a_out, b_out, a_in, b_in;
    int has_in;
    double scale;  // kernel coordinates (x - centre) * scale (binary32_scale; 1 for binary64)
};

__device__ __forceinline__ int inst_of_position(const long long* __restrict__ off, int n_inst, long long p) {
    int lo = 0, hi = n_inst - 1;  // last instance whose first point is <= p
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= p)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Instance of every point of the group (points are numbered instance by
// instance).
__global__ void k_binst(const long long* __restrict__ off, int n_inst, int64_t n, int32_t* inst_of) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n) return;
    inst_of[p] = inst_of_position(off, n_inst, p);
}

// Coordinate c of point p (group numbering) of instance k, read in place from
// the instance's own n_k x d_k array; zero in the padding dims.
__device__ __forceinline__ double bcoord(const double* const* __restrict__ src, const int32_t* __restrict__ d_of,
                                         const long long* __restrict__ off, int k, int64_t p, int c) {
    const int d = d_of[k];
    return c < d ? src[k][(p - off[k]) * d + c] : 0.0;
}

// Extents: block b covers points [blk_start[b], blk_start[b] + kBlkPts) of
// instance blk_inst[b] (capped at its end); per-dim min / max as order keys
// merged into ext[k] (2 d + 1 words: mins, maxes, non-finite flag) with
// atomics, so the result does not depend on the order of the blocks.
constexpr int kBlkPts = 2048;
__global__ void k_bextent(const double* const* __restrict__ src, const int32_t* __restrict__ d_of,
                          const long long* __restrict__ off, const int32_t* __restrict__ blk_inst,
                          const long long* __restrict__ blk_start, int dp, unsigned long long* ext) {
    extern __shared__ unsigned long long s_ext[];  // [2 * dp + 1]
    const int k = blk_inst[blockIdx.x];
    const int d = d_of[k];
    for (int c = threadIdx.x; c < dp; c += blockDim.x) {
        s_ext[c] = ~0ull;
        s_ext[dp + c] = 0ull;
    }
    if (threadIdx.x == 0) s_ext[2 * dp] = 0ull;
    __syncthreads();
    const long long p0 = blk_start[blockIdx.x];
    const long long p1 = p0 + kBlkPts < off[k + 1] ? p0 + kBlkPts : off[k + 1];
    const double* base = src[k] + (p0 - off[k]) * d;
    const long long m = (p1 - p0) * d;
    // a stride that is a multiple of d keeps every thread on one dim
    const int stride = (int)blockDim.x - (int)blockDim.x % d;
    if ((int)threadIdx.x < stride) {
        const int c = (int)threadIdx.x % d;
        unsigned long long mn = ~0ull, mx = 0ull;
        int bad = 0;
        for (long long i = threadIdx.x; i < m; i += stride) {
            const unsigned long long w = (unsigned long long)__double_as_longlong(base[i]);
            if (((w >> 52) & 0x7FFull) == 0x7FFull) {
                bad = 1;
                continue;
            }
            const unsigned long long o = (w >> 63) ? ~w : (w | 0x8000000000000000ull);
            mn = o < mn ? o : mn;
            mx = o > mx ? o : mx;
        }
        if (mn <= mx) {
            atomicMin(&s_ext[c], mn);
            atomicMax(&s_ext[dp + c], mx);
        }
        if (bad) atomicOr(&s_ext[2 * dp], 1ull);
    }
    __syncthreads();
    unsigned long long* e = ext + (int64_t)k * (2 * dp + 1);
    for (int c = threadIdx.x; c < dp; c += blockDim.x) {
        // padding dims hold zeros (key of +0)
        const unsigned long long zero = 0x8000000000000000ull;
        atomicMin(&e[c], c < d ? s_ext[c] : zero);
        atomicMax(&e[dp + c], c < d ? s_ext[dp + c] : zero);
    }
    if (threadIdx.x == 0 && s_ext[2 * dp]) atomicOr(&e[2 * dp], 1ull);
}

__global__ void k_bextent_init(unsigned long long* ext, int n_inst, int dp) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t w = 2 * dp + 1;
    if (i >= (int64_t)n_inst * w) return;
    const int64_t c = i % w;
    ext[i] = c < dp ? ~0ull : 0ull;
}

__global__ void k_bkeys(const double* const* __restrict__ src, const int32_t* __restrict__ d_of,
                        const long long* __restrict__ off, int64_t n, const int32_t* __restrict__ inst_of,
                        const BInst* __restrict__ P, int shift, unsigned long long* keys, int32_t* ids) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int k = inst_of[i];
    const BInst& g = P[k];
    unsigned long long key = 0;
    for (int t = 0; t < g.m; ++t) {
        const int64_t c = cell_coord(bcoord(src, d_of, off, k, i, g.dims[t]), g.lo[t], g.inv_w, g.ncell[t]);
        key += (unsigned long long)c * g.stride[t];
    }
    keys[i] = ((unsigned long long)k << shift) | key;
    ids[i] = (int32_t)i;
}

template <typename T>
__global__ void k_bpack(const double* const* __restrict__ srcp, const int32_t* __restrict__ d_of,
                        const long long* __restrict__ off, const int32_t* __restrict__ perm,
                        const int32_t* __restrict__ inst_of, const BInst* __restrict__ P,
                        const double* __restrict__ centre, int64_t n, int dp, double* xs, T* y, T* h, T* thr_out,
                        T* thr_in, int32_t* inst_of_sorted) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int64_t src = perm[p];
    const int k = inst_of[src];
    const BInst& g = P[k];
    T nrm = T(0);
    for (int c = 0; c < dp; ++c) {
        const double v = bcoord(srcp, d_of, off, k, src, c);
        xs[p * dp + c] = v;
        const T yc = T((v - centre[(int64_t)k * dp + c]) * g.scale);
        y[p * dp + c] = yc;
        nrm = fma_pack(yc, yc, nrm);
    }
    h[p] = -nrm * T(0.5);
    thr_out[p] = thr_down(g.a_out, nrm, g.b_out);
    thr_in[p] = g.has_in ? thr_up(g.a_in, nrm, g.b_in) : T(INFINITY);
    inst_of_sorted[p] = k;
}

// As k_bpack with dp threads per point (dp <= 32, a power of two): the row
// is read and written coalesced and the norm is summed by a shuffle tree over
// the point's dp lanes (the norm bound holds for any order of the sum).
template <typename T>
__global__ void k_bpack_lanes(const double* const* __restrict__ srcp, const int32_t* __restrict__ d_of,
                              const long long* __restrict__ off, const int32_t* __restrict__ perm,
                              const int32_t* __restrict__ inst_of, const BInst* __restrict__ P,
                              const double* __restrict__ centre, int64_t n, int dp, double* xs, T* y, T* h,
                              T* thr_out, T* thr_in, int32_t* inst_of_sorted) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t p = t / dp;
    const int c = (int)(t % dp);
    const bool live = p < n;
    int k = 0;
    T sq = T(0);
    if (live) {
        const int64_t src = perm[p];
        k = inst_of[src];
        const double v = bcoord(srcp, d_of, off, k, src, c);
        xs[p * dp + c] = v;
        const T yc = T((v - centre[(int64_t)k * dp + c]) * P[k].scale);
        y[p * dp + c] = yc;
        sq = yc * yc;
    }
    for (int o = dp >> 1; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o, dp);
    if (live && c == 0) {
        const BInst& g = P[k];
        h[p] = -sq * T(0.5);
        thr_out[p] = thr_down(g.a_out, sq, g.b_out);
        thr_in[p] = g.has_in ? thr_up(g.a_in, sq, g.b_in) : T(INFINITY);
        inst_of_sorted[p] = k;
    }
}

struct BEnum {
    int shift, symmetric, qmax;
};

__device__ __forceinline__ EnumParams benum_params(const BEnum& b, const BInst& g) {
    EnumParams e{};
    e.m = g.m;
    for (int t = 0; t < kMaxM; ++t) {
        e.ncell[t] = g.ncell[t];
        e.stride[t] = g.stride[t];
    }
    e.symmetric = b.symmetric;
    e.qmax = b.qmax;
    e.local_mask = (1ull << b.shift) - 1ull;
    return e;
}

__global__ void k_benum_count(BEnum b, const BInst* __restrict__ P, const unsigned long long* __restrict__ cell_key,
                              const int32_t* __restrict__ cell_start, int64_t n_cells, uint32_t* run_cnt,
                              uint32_t* item_cnt, unsigned long long* inst_eval, unsigned long long* inst_sq,
                              unsigned long long* inst_skip, EnumTotals* tot) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    unsigned long long my_runs = 0, my_items = 0;
    if (c < n_cells) {
        const int k = (int)(cell_key[c] >> b.shift);
        const EnumParams e = benum_params(b, P[k]);
        const int64_t q = cell_start[c + 1] - cell_start[c];
        uint32_t nr = 0;
        unsigned long long ev = 0;
        if (e.m == 0) {  // the instance is one cell: its own points
            nr = 1;
            ev = (unsigned long long)q;
        } else {
            visit_runs(e, cell_key, cell_start, n_cells, c, [&](int32_t a, int32_t z, bool) {
                ++nr;
                ev += (unsigned long long)(z - a);
            });
        }
        run_cnt[c] = nr;
        const uint32_t ni = (uint32_t)((q + e.qmax - 1) / e.qmax);
        item_cnt[c] = ni;
        atomicAdd(&inst_eval[k], ev * (unsigned long long)q);
        atomicAdd(&inst_sq[k], (unsigned long long)q * (unsigned long long)q);
        if (b.symmetric) atomicAdd(&inst_skip[k], tri_skip(q, e.qmax));
        my_runs = nr;
        my_items = ni;
    }
    for (int o = 16; o > 0; o >>= 1) {
        my_runs += __shfl_down_sync(0xffffffffu, my_runs, o);
        my_items += __shfl_down_sync(0xffffffffu, my_items, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&tot->n_runs, my_runs);
        atomicAdd(&tot->n_items, my_items);
    }
}

__global__ void k_benum_fill(BEnum b, const BInst* __restrict__ P, const unsigned long long* __restrict__ cell_key,
                             const int32_t* __restrict__ cell_start, int64_t n_cells,
                             const uint32_t* __restrict__ run_off, const uint32_t* __restrict__ item_off, Run* runs,
                             Item* items, int32_t* item_inst) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= n_cells) return;
    const int k = (int)(cell_key[c] >> b.shift);
    const EnumParams e = benum_params(b, P[k]);
    uint32_t r = run_off[c];
    const uint32_t r0 = r;
    if (e.m == 0) {
        Run rr;
        rr.start = cell_start[c];
        rr.end_flags = (uint32_t)cell_start[c + 1];
        runs[r++] = rr;
    } else {
        visit_runs(e, cell_key, cell_start, n_cells, c, [&](int32_t a, int32_t z, bool mirror) {
            Run rr;
            rr.start = a;
            rr.end_flags = (uint32_t)z | (mirror ? kMirrorBit : 0u);
            runs[r++] = rr;
        });
    }
    const int32_t q0 = cell_start[c], q1 = cell_start[c + 1];
    uint32_t it = item_off[c];
    for (int32_t q = q0; q < q1; q += e.qmax) {
        Item x;
        x.q0 = q;
        x.q1 = q + e.qmax < q1 ? q + e.qmax : q1;
        x.r0 = (int32_t)r0;
        x.r1 = (int32_t)r;
        items[it] = x;
        item_inst[it] = k;
        ++it;
    }
}

// Sorted keys -> cell table (cell_key, cell_start), with one read-back of
// the cell count.
static int build_cells(const unsigned long long* keys, int64_t n, unsigned long long** cell_key, int32_t** cell_start,
                       int64_t* n_cells, cudaStream_t s) {
    Scratch tmp(s);
    uint32_t *flags = nullptr, *idx = nullptr;
    unsigned long long* dcount = nullptr;
    unsigned long long* ck = nullptr;
    int32_t* cs = nullptr;
    SJ_TRY(tmp.alloc(&flags, (size_t)n));
    SJ_TRY(tmp.alloc(&idx, (size_t)n));
    SJ_TRY(tmp.alloc(&dcount, 1));
    SJ_TRY(dev_alloc_t(&ck, (size_t)n, s));
    *cell_key = ck;  // owned by the caller's index from here on
    SJ_TRY(dev_alloc_t(&cs, (size_t)n + 1, s));
    *cell_start = cs;
    k_heads<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(keys, n, flags);
    note_launch();
    SJ_CK(cudaGetLastError());
    SJ_TRY(scan_exclusive_u32(flags, idx, n, s));
    k_cells<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(keys, flags, idx, n, ck, cs, dcount);
    note_launch();
    SJ_CK(cudaGetLastError());
    unsigned long long M = 0;
    SJ_CK(cudaMemcpyAsync(&M, dcount, 8, cudaMemcpyDeviceToHost, s));
    SJ_CK(cudaStreamSynchronize(s));
    *cell_key = ck;
    *cell_start = cs;
    *n_cells = (int64_t)M;
    return SJ_OK;
}

int build_batch_group(BatchGroup* g, const double* const* src_dev_ptrs, const int32_t* d_of_host) {
    Index* ix = &g->ix;
    cudaStream_t s = ix->stream;
    Scratch tmp(s);  // temporaries, released on every return
    const int K = g->n_inst;
    const int dp = ix->dp;
    const int64_t n = ix->n;
    // ---- per-instance offsets, dims, source pointers ----
    SJ_TRY(dev_alloc_t(&g->d_off, (size_t)K + 1, s));
    SJ_CK(cudaMemcpyAsync(g->d_off, g->off.data(), (K + 1) * sizeof(long long), cudaMemcpyHostToDevice, s));
    int32_t* inst_of = nullptr;
    SJ_TRY(tmp.alloc(&inst_of, (size_t)n));
    // the instances' arrays are read in place
    const double** dsrc = nullptr;
    int32_t* dd = nullptr;
    SJ_TRY(tmp.alloc(&dsrc, (size_t)K));
    SJ_TRY(tmp.alloc(&dd, (size_t)K));
    SJ_CK(cudaMemcpyAsync(dsrc, src_dev_ptrs, K * sizeof(double*), cudaMemcpyHostToDevice, s));
    SJ_CK(cudaMemcpyAsync(dd, d_of_host, K * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    k_binst<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g->d_off, K, n, inst_of);
    note_launch();
    SJ_CK(cudaGetLastError());
    // ---- extents (blocks of up to kBlkPts points; one read-back) and per-instance grids ----
    std::vector<int32_t> hblk_inst;
    std::vector<long long> hblk_start;
    for (int k = 0; k < K; ++k)
        for (long long p = g->off[k]; p < g->off[k + 1]; p += kBlkPts) {
            hblk_inst.push_back(k);
            hblk_start.push_back(p);
        }
    const int nblk = (int)hblk_inst.size();
    int32_t* dblk_inst = nullptr;
    long long* dblk_start = nullptr;
    unsigned long long* ext = nullptr;
    SJ_TRY(tmp.alloc(&dblk_inst, (size_t)nblk));
    SJ_TRY(tmp.alloc(&dblk_start, (size_t)nblk));
    SJ_TRY(tmp.alloc(&ext, (size_t)K * (2 * dp + 1)));
    SJ_CK(cudaMemcpyAsync(dblk_inst, hblk_inst.data(), nblk * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    SJ_CK(cudaMemcpyAsync(dblk_start, hblk_start.data(), nblk * sizeof(long long), cudaMemcpyHostToDevice, s));
    {
        const int64_t w = (int64_t)K * (2 * dp + 1);
        k_bextent_init<<<(unsigned)((w + 255) / 256), 256, 0, s>>>(ext, K, dp);
        note_launch();
        SJ_CK(cudaGetLastError());
    }
    k_bextent<<<nblk, 256, (2 * dp + 1) * sizeof(unsigned long long), s>>>(dsrc, dd, g->d_off, dblk_inst, dblk_start,
                                                                         dp, ext);
    note_launch();
    SJ_CK(cudaGetLastError());
    std::vector<unsigned long long> hext((size_t)K * (2 * dp + 1));
    SJ_CK(cudaMemcpyAsync(hext.data(), ext, hext.size() * 8, cudaMemcpyDeviceToHost, s));
    SJ_CK(cudaStreamSynchronize(s));
    int inst_bits = 0;
    while ((1ll << inst_bits) < K) ++inst_bits;
    std::vector<BInst> hp((size_t)K);
    std::vector<double> centre((size_t)K * dp, 0.0);
    std::vector<double> e2((size_t)K);
    std::vector<float> r2((size_t)K);
    int shift = 0;
    const bool tensor = is_tensor_kernel(ix->kernel);
    const bool use_f32 = ix->kernel == SJ_KERNEL_FILTER_F32 || tensor;
    const double u_t = use_f32 ? ldexp(1.0, -24) : ldexp(1.0, -53);
    // the tensor-core filter's widened bound (as for a single join)
    const double c1 = tensor ? tc_c1(dp, ix->kernel) : -1.0;
    for (int k = 0; k < K; ++k) {
        const unsigned long long* e = hext.data() + (size_t)k * (2 * dp + 1);
        if (e[2 * dp] != 0) {
            set_error("non-finite coordinate in batch instance %d", g->gids[k]);
            return SJ_ERR_ARG;
        }
        Index t;
        t.d = dp;
        t.dp = dp;
        t.eps = g->eps[k];
        t.opt = ix->opt;
        t.kernel = ix->kernel;
        t.n = g->off[k + 1] - g->off[k];
        t.trim_dims = true;
        t.key_bits_cap = std::min(62, 64 - inst_bits);
        t.lo.resize(dp);
        t.hi.resize(dp);
        for (int c = 0; c < dp; ++c) {
            t.lo[c] = from_ord(e[c]);
            t.hi[c] = from_ord(e[dp + c]);
        }
        SJ_TRY(choose_grid(&t));
        BInst& b = hp[k];
        memset(&b, 0, sizeof b);
        b.m = t.m;
        ix->m = std::max(ix->m, t.m);  // the group's kernels size their run arrays by the largest m
        for (int i = 0; i < t.m; ++i) {
            b.dims[i] = t.dims[i];
            b.lo[i] = t.lo[t.dims[i]];
            b.ncell[i] = t.ncell[i];
            b.stride[i] = t.stride[i];
        }
        b.inv_w = 1.0 / t.w;
        shift = std::max(shift, t.key_bits);
        double pb = 0, rmax = 0;
        for (int c = 0; c < dp; ++c) {
            centre[(size_t)k * dp + c] = 0.5 * (t.lo[c] + t.hi[c]);
            const double r = 0.5 * (t.hi[c] - t.lo[c]) * (1.0 + ldexp(1.0, -40));
            pb += r * r;
            rmax = std::max(rmax, r);
        }
        const double pbk = pb * (1.0 + ldexp(1.0, -20));
        double sk = 1.0;  // binary32 kernels: the instance's scale (binary32_scale)
        if (use_f32 && !binary32_scale(pbk, &sk)) {
            set_error("batch instance %d: binary32 kernel coordinates cannot hold its extent (P = %g; take "
                      "SJ_KERNEL_FP64_FMA)", g->gids[k], pbk);
            return SJ_ERR_UNSUPPORTED;
        }
        b.scale = sk;
        PackParams pp{};
        pack_coefficients(t.eps * sk, pbk * sk * sk, 1.01 * u_t * rmax * sk, u_t, dp, dp, &pp, c1);
        r2[k] = pp.prune_r2f;
        b.a_out = pp.a_out;
        b.b_out = pp.b_out;
        b.a_in = pp.a_in;
        b.b_in = pp.b_in;
        b.has_in = pp.has_in;
        e2[k] = t.eps * t.eps;
    }
    if (shift + inst_bits > 64) {
        set_error("batched index keys need %d bits", shift + inst_bits);
        return SJ_ERR_ARG;
    }
    BInst* dP = nullptr;
    double* dcentre = nullptr;
    SJ_TRY(tmp.alloc(&dP, (size_t)K));
    SJ_TRY(tmp.alloc(&dcentre, (size_t)K * dp));
    SJ_TRY(dev_alloc_t(&g->d_e2, (size_t)K, s));
    SJ_CK(cudaMemcpyAsync(dP, hp.data(), K * sizeof(BInst), cudaMemcpyHostToDevice, s));
    SJ_CK(cudaMemcpyAsync(dcentre, centre.data(), centre.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    SJ_CK(cudaMemcpyAsync(g->d_e2, e2.data(), K * sizeof(double), cudaMemcpyHostToDevice, s));
    SJ_TRY(dev_alloc_t(&g->d_r2, (size_t)K, s));
    SJ_CK(cudaMemcpyAsync(g->d_r2, r2.data(), K * sizeof(float), cudaMemcpyHostToDevice, s));
    // ---- keys, sort, cells ----
    unsigned long long* keys = nullptr;
    SJ_TRY(tmp.alloc(&keys, (size_t)n));
    SJ_TRY(dev_alloc_t(&ix->perm, (size_t)n, s));
    k_bkeys<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(dsrc, dd, g->d_off, n, inst_of, dP, shift, keys, ix->perm);
    note_launch();
    SJ_CK(cudaGetLastError());
    SJ_TRY(radix_sort_pairs(reinterpret_cast<uint64_t*>(keys), ix->perm, n, shift + inst_bits, s));
    SJ_TRY(build_cells(keys, n, &ix->cell_key, &ix->cell_start, &ix->n_cells, s));
    // ---- packing ----
    SJ_TRY(dev_alloc_t(&ix->xs, (size_t)n * dp, s));
    SJ_TRY(dev_alloc_t(&g->d_inst_of_sorted, (size_t)n, s));
    if (use_f32) {
        float *y, *h, *to, *ti;
        SJ_TRY(dev_alloc_t(&y, (size_t)n * dp, s));
        ix->y = y;
        SJ_TRY(dev_alloc_t(&h, (size_t)n, s));
        ix->h = h;
        SJ_TRY(dev_alloc_t(&to, (size_t)n, s));
        ix->thr_out = to;
        SJ_TRY(dev_alloc_t(&ti, (size_t)n, s));
        ix->thr_in = ti;
        if (dp <= 32)
            k_bpack_lanes<float><<<(unsigned)((n * dp + 255) / 256), 256, 0, s>>>(
                dsrc, dd, g->d_off, ix->perm, inst_of, dP, dcentre, n, dp, ix->xs, y, h, to, ti, g->d_inst_of_sorted);
        else
            k_bpack<float><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(dsrc, dd, g->d_off, ix->perm, inst_of, dP,
                                                                       dcentre, n, dp, ix->xs, y, h, to, ti,
                                                                       g->d_inst_of_sorted);
    } else {
        double *y, *h, *to, *ti;
        SJ_TRY(dev_alloc_t(&y, (size_t)n * dp, s));
        ix->y = y;
        SJ_TRY(dev_alloc_t(&h, (size_t)n, s));
        ix->h = h;
        SJ_TRY(dev_alloc_t(&to, (size_t)n, s));
        ix->thr_out = to;
        SJ_TRY(dev_alloc_t(&ti, (size_t)n, s));
        ix->thr_in = ti;
        if (dp <= 32)
            k_bpack_lanes<double><<<(unsigned)((n * dp + 255) / 256), 256, 0, s>>>(
                dsrc, dd, g->d_off, ix->perm, inst_of, dP, dcentre, n, dp, ix->xs, y, h, to, ti, g->d_inst_of_sorted);
        else
            k_bpack<double><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(dsrc, dd, g->d_off, ix->perm, inst_of, dP,
                                                                        dcentre, n, dp, ix->xs, y, h, to, ti,
                                                                        g->d_inst_of_sorted);
    }
    note_launch();
    SJ_CK(cudaGetLastError());
    if (tensor) SJ_TRY(pack_split_rows(ix));
    if (wants_aux(ix)) SJ_TRY(build_aux(ix));
    // perm now maps packed points to their place in the group; the join
    // subtracts the instance's first position to get instance-local indices
    // ---- runs and items (one read-back) ----
    const int64_t M = ix->n_cells;
    BEnum be{shift, ix->opt.symmetric ? 1 : 0, item_qmax(ix)};
    uint32_t* cnt = nullptr;
    SJ_TRY(tmp.alloc(&cnt, (size_t)M * 4));
    uint32_t *run_cnt = cnt, *item_cnt = cnt + M, *run_off = cnt + 2 * M, *item_off = cnt + 3 * M;
    unsigned long long* ev = nullptr;
    SJ_TRY(tmp.alloc(&ev, (size_t)3 * K));
    SJ_CK(cudaMemsetAsync(ev, 0, 3 * K * sizeof(unsigned long long), s));
    EnumTotals* dtot = nullptr;
    SJ_TRY(tmp.alloc(&dtot, 1));
    SJ_CK(cudaMemsetAsync(dtot, 0, sizeof(EnumTotals), s));
    k_benum_count<<<(unsigned)((M + 127) / 128), 128, 0, s>>>(be, dP, ix->cell_key, ix->cell_start, M, run_cnt,
                                                              item_cnt, ev, ev + K, ev + 2 * K, dtot);
    note_launch();
    SJ_CK(cudaGetLastError());
    SJ_TRY(scan_exclusive_u32(run_cnt, run_off, M, s));
    SJ_TRY(scan_exclusive_u32(item_cnt, item_off, M, s));
    EnumTotals tot{};
    std::vector<unsigned long long> hev((size_t)3 * K);
    SJ_CK(cudaMemcpyAsync(&tot, dtot, sizeof tot, cudaMemcpyDeviceToHost, s));
    SJ_CK(cudaMemcpyAsync(hev.data(), ev, hev.size() * 8, cudaMemcpyDeviceToHost, s));
    SJ_CK(cudaStreamSynchronize(s));
    ix->n_runs = (int64_t)tot.n_runs;
    ix->n_items = (int64_t)tot.n_items;
    g->eval.assign(K, 0);
    g->cand.assign(K, 0);
    ix->n_evaluated = 0;
    ix->n_candidates = 0;
    for (int k = 0; k < K; ++k) {
        g->eval[k] = (int64_t)(hev[k] - hev[2 * K + k]);  // (the kernels evaluate self-cell triangles)
        g->cand[k] = ix->opt.symmetric ? (int64_t)(2 * hev[k] - hev[K + k]) : (int64_t)hev[k];
        ix->n_evaluated += g->eval[k];
        ix->n_candidates += g->cand[k];
    }
    if (tot.n_runs >= 0xFFFFFFFFull || tot.n_items >= 0x7FFFFFFFull) {
        set_error("batched index too large");
        return SJ_ERR_ARG;
    }
    SJ_TRY(dev_alloc_t(&ix->runs, (size_t)std::max<int64_t>(ix->n_runs, 1), s));
    SJ_TRY(dev_alloc_t(&ix->items, (size_t)std::max<int64_t>(ix->n_items, 1), s));
    SJ_TRY(dev_alloc_t(&g->d_item_inst, (size_t)std::max<int64_t>(ix->n_items, 1), s));
    k_benum_fill<<<(unsigned)((M + 127) / 128), 128, 0, s>>>(be, dP, ix->cell_key, ix->cell_start, M, run_off,
                                                             item_off, ix->runs, ix->items, g->d_item_inst);
    note_launch();
    SJ_CK(cudaGetLastError());
    SJ_TRY(dev_alloc_t(&ix->counters, kCounters, s));
    return SJ_OK;
}

}  // namespace sj
