// The distance tile as a standalone operation, and k nearest neighbours
// from a join's result.
//
// sj_sqdist_tile: every squared distance between two point sets, the
// brute-force tile of the paper's Fig. 3 experiment (Sec. IV), in the
// decision rule's own arithmetic (binary64, dimension order, subtraction,
// product and sum each rounded, no contraction), so each value is exactly
// the s the join decides with.
//
// sj_knn_from_join: the k nearest of every point's eps-neighbours (the
// reuse of the join for kNN the paper names as future work, Sec. V): the
// pairs of a result with distances are bucketed by their first point and
// each bucket's k smallest (distance, index) are selected.
#include <algorithm>

#include "sj_internal.cuh"

namespace sj {

namespace {

constexpr int kTileQ = 64;  // rows of A per block
constexpr int kTileC = 64;  // rows of B per block
constexpr int kDimChunk = 16;

// One 64 x 64 output tile per block of 256 threads (4 x 4 values each); A
// and B rows staged in shared memory 16 dims at a time.
__global__ void __launch_bounds__(256) k_sqdist_tile(const double* __restrict__ A, int64_t m,
                                                     const double* __restrict__ B, int64_t nb, int d, double* out) {
    __shared__ double sa[kDimChunk][kTileQ + 1];
    __shared__ double sb[kDimChunk][kTileC + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t i0 = (int64_t)blockIdx.y * kTileQ, j0 = (int64_t)blockIdx.x * kTileC;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < d; k0 += kDimChunk) {
        const int kc = min(kDimChunk, d - k0);
        for (int e = threadIdx.x; e < kDimChunk * kTileQ; e += 256) {
            const int r = e / kDimChunk, k = e % kDimChunk;
            const int64_t ia = i0 + r, jb = j0 + r;
            sa[k][r] = (k < kc && ia < m) ? A[ia * d + k0 + k] : 0.0;
            sb[k][r] = (k < kc && jb < nb) ? B[jb * d + k0 + k] : 0.0;
        }
        __syncthreads();
        for (int k = 0; k < kc; ++k) {  // dimension order, each operation rounded
            double a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = sa[k][ty + 16 * u];
                b[u] = sb[k][tx + 16 * u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const double t = __dsub_rn(a[u], b[v]);
                    acc[u][v] = __dadd_rn(acc[u][v], __dmul_rn(t, t));
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int64_t i = i0 + ty + 16 * u, j = j0 + tx + 16 * v;
            if (i < m && j < nb) out[i * nb + j] = acc[u][v];
        }
}

// kNN from a join: bucket sizes (self pairs left out) ...
__global__ void k_knn_degree(const int2* __restrict__ pairs, long long count, int32_t* deg) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < count;
         p += (long long)gridDim.x * blockDim.x) {
        const int2 e = pairs[p];
        if (e.x != e.y) atomicAdd(&deg[e.x], 1);
    }
}

// ... the pairs bucketed by their first point ...
__global__ void k_knn_bucket(const int2* __restrict__ pairs, const double* __restrict__ dist, long long count,
                             const uint32_t* __restrict__ off, uint32_t* fill, int32_t* nb_idx, double* nb_dist) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < count;
         p += (long long)gridDim.x * blockDim.x) {
        const int2 e = pairs[p];
        if (e.x == e.y) continue;
        const uint32_t slot = off[e.x] + atomicAdd(&fill[e.x], 1u);
        nb_idx[slot] = e.y;
        nb_dist[slot] = dist[p];
    }
}

// ... and, one warp per point, its k smallest (distance, index) in k rounds
// of a warp-wide minimum above the last one taken.
__global__ void k_knn_select(int64_t n, int k, const uint32_t* __restrict__ off, const int32_t* __restrict__ nb_idx,
                             const double* __restrict__ nb_dist, int32_t* idx_out, double* dist_out,
                             int32_t* found_out) {
    const int lane = threadIdx.x & 31;
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (i >= n) return;
    const uint32_t a = off[i], b = off[i + 1];
    double last_d = -1.0;
    int32_t last_j = -1;
    int found = 0;
    for (int r = 0; r < k; ++r) {
        double bd = INFINITY;
        int32_t bj = 0x7FFFFFFF;
        for (uint32_t s = a + lane; s < b; s += 32) {
            const double dd = nb_dist[s];
            const int32_t jj = nb_idx[s];
            const bool after = dd > last_d || (dd == last_d && jj > last_j);
            if (after && (dd < bd || (dd == bd && jj < bj))) {
                bd = dd;
                bj = jj;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double od = __shfl_xor_sync(0xffffffffu, bd, o);
            const int32_t oj = __shfl_xor_sync(0xffffffffu, bj, o);
            if (od < bd || (od == bd && oj < bj)) {
                bd = od;
                bj = oj;
            }
        }
        if (bj == 0x7FFFFFFF) break;  // the bucket is exhausted
        if (lane == 0) {
            idx_out[i * k + r] = bj;
            dist_out[i * k + r] = bd;
        }
        last_d = bd;
        last_j = bj;
        ++found;
    }
    if (lane == 0) {
        found_out[i] = found;
        for (int r = found; r < k; ++r) {
            idx_out[i * k + r] = -1;
            dist_out[i * k + r] = INFINITY;
        }
    }
}

unsigned grid_for(long long work, int device) {
    const long long cap = (long long)device_sm_count(device) * 16;
    long long b = (work + 255) / 256;
    return (unsigned)std::max<long long>(1, std::min(b, cap));
}

}  // namespace

}  // namespace sj

using namespace sj;

extern "C" int sj_sqdist_tile(const double* A, int64_t m, const double* B, int64_t nb, int32_t d, double* out,
                              void* stream) {
    clear_error();
    if (!A || !B || !out || m < 1 || nb < 1 || d < 1 || d > SJ_MAX_D || m > 0x7FFFFFFFll || nb > 0x7FFFFFFFll) {
        set_error("invalid argument");
        return SJ_ERR_ARG;
    }
    if (!is_device_pointer(A) || !is_device_pointer(B) || !is_device_pointer(out)) {
        set_error("sj_sqdist_tile needs device pointers");
        return SJ_ERR_ARG;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const dim3 grid((unsigned)((nb + kTileC - 1) / kTileC), (unsigned)((m + kTileQ - 1) / kTileQ));
    if (grid.y > 65535u) {
        set_error("m = %lld rows of A exceed one launch (at most %lld)", (long long)m, 65535ll * kTileQ);
        return SJ_ERR_ARG;
    }
    k_sqdist_tile<<<grid, 256, 0, s>>>(A, m, B, nb, d, out);
    note_launch();
    SJ_CK(cudaGetLastError());
    return SJ_OK;
}

extern "C" int sj_knn_from_join(const sj_result* r, int64_t n, int32_t k, int32_t* idx_out, double* dist_out,
                                int32_t* found_out) {
    clear_error();
    if (!r || !idx_out || !dist_out || !found_out || n < 1 || n > 0x7FFFFFFFll || k < 1 || k > 1024) {
        set_error("invalid argument");
        return SJ_ERR_ARG;
    }
    const ResultImpl* ri = static_cast<const ResultImpl*>(r->internal);
    if (r->count > 0 && (!ri || !ri->block || ri->shared_pool)) {
        set_error("sj_knn_from_join takes the result of a single join (sj_self_join / sj_join)");
        return SJ_ERR_ARG;
    }
    if (r->count > 0 && (!r->has_distances || !ri->dblock)) {
        set_error("sj_knn_from_join needs a result with distances (sj_options.emit_distances = 1)");
        return SJ_ERR_ARG;
    }
    if (r->count > (int64_t)r->n_pages * r->page_pairs) {
        set_error("the result holds only part of its pairs");
        return SJ_ERR_RESULT_OVERFLOW;
    }
    cudaStream_t s = ri ? ri->stream : nullptr;
    int dev = 0;
    SJ_CK(cudaGetDevice(&dev));
    const long long count = (long long)r->count;
    const int2* pairs = ri ? reinterpret_cast<const int2*>(ri->block) : nullptr;
    const double* dist = ri ? ri->dblock : nullptr;
    Scratch tmp(s);
    int32_t *deg = nullptr, *nb_idx = nullptr, *oi = nullptr, *of = nullptr;
    uint32_t *off = nullptr, *fill = nullptr;
    double *nb_dist = nullptr, *od = nullptr;
    SJ_TRY(tmp.alloc(&deg, (size_t)n));
    SJ_TRY(tmp.alloc(&off, (size_t)n + 1));
    SJ_TRY(tmp.alloc(&fill, (size_t)n));
    SJ_TRY(tmp.alloc(&nb_idx, (size_t)std::max<long long>(count, 1)));
    SJ_TRY(tmp.alloc(&nb_dist, (size_t)std::max<long long>(count, 1)));
    SJ_TRY(tmp.alloc(&oi, (size_t)n * k));
    SJ_TRY(tmp.alloc(&od, (size_t)n * k));
    SJ_TRY(tmp.alloc(&of, (size_t)n));
    SJ_CK(cudaMemsetAsync(deg, 0, (size_t)n * sizeof(int32_t), s));
    SJ_CK(cudaMemsetAsync(fill, 0, (size_t)n * sizeof(uint32_t), s));
    if (count > 0) {
        k_knn_degree<<<grid_for(count, dev), 256, 0, s>>>(pairs, count, deg);
        note_launch();
        SJ_CK(cudaGetLastError());
    }
    SJ_TRY(scan_exclusive_u32_total(reinterpret_cast<const uint32_t*>(deg), off, n, s));  // off[n]: the total
    if (count > 0) {
        k_knn_bucket<<<grid_for(count, dev), 256, 0, s>>>(pairs, dist, count, off, fill, nb_idx, nb_dist);
        note_launch();
        SJ_CK(cudaGetLastError());
    }
    k_knn_select<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(n, k, off, nb_idx, nb_dist, oi, od, of);
    note_launch();
    SJ_CK(cudaGetLastError());
    SJ_CK(cudaMemcpyAsync(idx_out, oi, (size_t)n * k * sizeof(int32_t), cudaMemcpyDefault, s));
    SJ_CK(cudaMemcpyAsync(dist_out, od, (size_t)n * k * sizeof(double), cudaMemcpyDefault, s));
    SJ_CK(cudaMemcpyAsync(found_out, of, (size_t)n * sizeof(int32_t), cudaMemcpyDefault, s));
    SJ_CK(cudaStreamSynchronize(s));
    return SJ_OK;
}
