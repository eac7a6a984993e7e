// DBSCAN on the result of a self-join: the join's eps-neighbourhoods reused
// for density-based clustering (the paper names this reuse of its join as
// future work, Sec. V).
//
// Definition (Ester et al. 1996, on the neighbourhoods the join returns): a
// point is core iff its neighbourhood, itself included, holds at least
// min_pts points; clusters are the connected components of the core points
// under the core-core pairs; a non-core point with a core neighbour is a
// border point and joins the smallest of its core neighbours' clusters; the
// rest is noise (-1).  Clusters are numbered by their smallest core point.
//
// Components come from a lock-free union-find over the core-core pairs:
// roots are always hooked under the smaller root (parent[x] <= x holds at
// every moment, so every find terminates and a component's root is its
// smallest core point), finds halve their paths, a failed hook retries.
#include <algorithm>

#include "sj_internal.cuh"

namespace sj {

namespace {

constexpr int32_t kNoLabel = 0x7FFFFFFF;
constexpr int kUnionTries = 1 << 20;  // retries of one union (each failure is another thread's progress)

__global__ void k_db_degree(const int2* __restrict__ pairs, long long count, int32_t* deg) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < count;
         p += (long long)gridDim.x * blockDim.x)
        atomicAdd(&deg[pairs[p].x], 1);
}

__global__ void k_db_init(int64_t n, int32_t* parent, int32_t* border) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) {
        parent[i] = (int32_t)i;
        border[i] = kNoLabel;
    }
}

__device__ __forceinline__ int32_t db_find(volatile int32_t* parent, int32_t x) {
    for (;;) {  // indices strictly decrease along the path: this ends
        const int32_t p = parent[x];
        if (p == x) return x;
        const int32_t gp = parent[p];
        if (gp != p) parent[x] = gp;  // path halving (x is not a root)
        x = p;
    }
}

__global__ void k_db_union(const int2* __restrict__ pairs, long long count, const int32_t* __restrict__ deg,
                           int32_t min_pts, int32_t* parent, unsigned long long* error) {
    volatile int32_t* par = parent;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < count;
         p += (long long)gridDim.x * blockDim.x) {
        const int2 e = pairs[p];
        if (e.x >= e.y || deg[e.x] < min_pts || deg[e.y] < min_pts) continue;  // each core-core pair once
        int tries = 0;
        for (;; ++tries) {
            if (tries == kUnionTries) {
                atomicExch(error, 1ull);
                break;
            }
            int32_t a = db_find(par, e.x), b = db_find(par, e.y);
            if (a == b) break;
            if (a > b) {
                const int32_t t = a;
                a = b;
                b = t;
            }
            if (atomicCAS(&parent[b], b, a) == b) break;  // the larger root under the smaller
        }
    }
}

__global__ void k_db_flatten(int64_t n, const int32_t* __restrict__ deg, int32_t min_pts, int32_t* parent) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n && deg[i] >= min_pts) parent[i] = db_find(parent, (int32_t)i);
}

__global__ void k_db_border(const int2* __restrict__ pairs, long long count, const int32_t* __restrict__ deg,
                            int32_t min_pts, const int32_t* __restrict__ parent, int32_t* border) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < count;
         p += (long long)gridDim.x * blockDim.x) {
        const int2 e = pairs[p];
        if (deg[e.x] < min_pts && deg[e.y] >= min_pts) atomicMin(&border[e.x], parent[e.y]);
    }
}

__global__ void k_db_roots(int64_t n, const int32_t* __restrict__ deg, int32_t min_pts,
                           const int32_t* __restrict__ parent, uint32_t* flag) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) flag[i] = (deg[i] >= min_pts && parent[i] == (int32_t)i) ? 1u : 0u;
}

__global__ void k_db_label(int64_t n, const int32_t* __restrict__ deg, int32_t min_pts,
                           const int32_t* __restrict__ parent, const int32_t* __restrict__ border,
                           const uint32_t* __restrict__ rank, int32_t* labels) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t l = -1;
    if (deg[i] >= min_pts)
        l = (int32_t)rank[parent[i]];
    else if (border[i] != kNoLabel)
        l = (int32_t)rank[border[i]];
    labels[i] = l;
}

unsigned grid_for(long long work, int device) {
    const long long cap = (long long)device_sm_count(device) * 16;
    long long b = (work + 255) / 256;
    return (unsigned)std::max<long long>(1, std::min(b, cap));
}

}  // namespace

}  // namespace sj

using namespace sj;

extern "C" int sj_dbscan(const sj_result* r, int64_t n, int32_t min_pts, int32_t* labels_out, int64_t* n_clusters) {
    clear_error();
    if (!r || !labels_out || n < 1 || n > 0x7FFFFFFFll || min_pts < 1) {
        set_error("invalid argument");
        return SJ_ERR_ARG;
    }
    const ResultImpl* ri = static_cast<const ResultImpl*>(r->internal);
    if (r->count > 0 && (!ri || !ri->block || ri->shared_pool)) {
        set_error("sj_dbscan takes the result of a single join (sj_self_join / sj_join)");
        return SJ_ERR_ARG;
    }
    if (r->count > (int64_t)r->n_pages * r->page_pairs) {
        set_error("the result holds %lld of its %lld pairs", (long long)r->n_pages * r->page_pairs,
                  (long long)r->count);
        return SJ_ERR_RESULT_OVERFLOW;
    }
    cudaStream_t s = ri ? ri->stream : nullptr;
    int dev = 0;
    SJ_CK(cudaGetDevice(&dev));
    const int2* pairs = ri ? reinterpret_cast<const int2*>(ri->block) : nullptr;
    const long long count = (long long)r->count;
    Scratch tmp(s);
    int32_t *deg = nullptr, *parent = nullptr, *border = nullptr, *labels = nullptr;
    uint32_t* flag = nullptr;  // n flags, then n + 1 ranks
    unsigned long long* error = nullptr;
    SJ_TRY(tmp.alloc(&deg, (size_t)n));
    SJ_TRY(tmp.alloc(&parent, (size_t)n));
    SJ_TRY(tmp.alloc(&border, (size_t)n));
    SJ_TRY(tmp.alloc(&labels, (size_t)n));
    SJ_TRY(tmp.alloc(&flag, (size_t)2 * n + 1));
    SJ_TRY(tmp.alloc(&error, 1));
    uint32_t* rank = flag + n;
    SJ_CK(cudaMemsetAsync(deg, 0, (size_t)n * sizeof(int32_t), s));
    SJ_CK(cudaMemsetAsync(error, 0, sizeof(unsigned long long), s));
    const unsigned gn = (unsigned)((n + 255) / 256);
    k_db_init<<<gn, 256, 0, s>>>(n, parent, border);
    note_launch();
    if (count > 0) {
        k_db_degree<<<grid_for(count, dev), 256, 0, s>>>(pairs, count, deg);
        note_launch();
        k_db_union<<<grid_for(count, dev), 256, 0, s>>>(pairs, count, deg, min_pts, parent, error);
        note_launch();
    }
    k_db_flatten<<<gn, 256, 0, s>>>(n, deg, min_pts, parent);
    note_launch();
    if (count > 0) {
        k_db_border<<<grid_for(count, dev), 256, 0, s>>>(pairs, count, deg, min_pts, parent, border);
        note_launch();
    }
    k_db_roots<<<gn, 256, 0, s>>>(n, deg, min_pts, parent, flag);
    note_launch();
    SJ_CK(cudaGetLastError());
    SJ_TRY(scan_exclusive_u32(flag, rank, n, s));
    k_db_label<<<gn, 256, 0, s>>>(n, deg, min_pts, parent, border, rank, labels);
    note_launch();
    SJ_CK(cudaGetLastError());
    uint32_t last[2] = {0, 0};
    unsigned long long err = 0;
    SJ_CK(cudaMemcpyAsync(&last[0], rank + n - 1, 4, cudaMemcpyDeviceToHost, s));
    SJ_CK(cudaMemcpyAsync(&last[1], flag + n - 1, 4, cudaMemcpyDeviceToHost, s));
    SJ_CK(cudaMemcpyAsync(&err, error, sizeof err, cudaMemcpyDeviceToHost, s));
    SJ_CK(cudaMemcpyAsync(labels_out, labels, (size_t)n * sizeof(int32_t), cudaMemcpyDefault, s));
    SJ_CK(cudaStreamSynchronize(s));
    if (err) {
        set_error("a union-find update ran out of retries");
        return SJ_ERR_TIMEOUT;
    }
    if (n_clusters) *n_clusters = (int64_t)last[0] + (int64_t)last[1];
    return SJ_OK;
}
