// Parts shared by the distance-tile kernels: parameters, the decision rule's
// direct form, the work-item prologue (queries and candidate runs in shared
// memory) and the warp-aggregated compaction into result pages.
#pragma once

#include <math.h>

#include "sj_internal.cuh"

namespace sj {

struct JoinParams {
    const void* y;        // n x dp kernel coordinates (double or float)
    const void* h;        // n: -||y||^2 / 2
    const void* thr_out;  // n: maybe-in threshold
    const void* thr_in;   // n: certain-in threshold
    const double* xs;     // n x dp original coordinates (cell order)
    const int32_t* perm;  // cell order -> input index
    const Item* items;
    const Run* runs;
    long long n_items;
    unsigned long long* counters;  // [0] item queue, [1] result cursor, [2] rechecked
    int2* const* pages;
    double* const* dpages;
    int page_log2;
    unsigned long long capacity;
    double e2;
    int d;
    int emit_dist;
};

JoinParams make_join_params(Index* ix, const JoinOut& out, int emit_dist);

// Squared distance in the decision rule's operation order: binary64, k
// ascending, subtraction, product and sum each rounded (no fma).
__device__ __forceinline__ double direct_sq(const double* __restrict__ a, const double* __restrict__ b, int d) {
    double s = 0.0;
    for (int k = 0; k < d; ++k) {
        double t = __dsub_rn(a[k], b[k]);
        s = __dadd_rn(s, __dmul_rn(t, t));
    }
    return s;
}

struct WarpStage {
    int2* pairs;   // kStage slots of this warp
    double* dist;  // kStage slots (used when distances are emitted)
    int cnt;       // warp-uniform fill
};

// Reserves room for the warp's staged pairs with one atomic on the result
// cursor and copies them to their pages (coalesced).  Positions past the
// pool's capacity are counted but not written.
__device__ __forceinline__ void stage_flush(WarpStage& st, const JoinParams& P, int lane) {
    __syncwarp();
    unsigned long long base = 0;
    if (lane == 0 && st.cnt > 0) base = atomicAdd(&P.counters[1], (unsigned long long)st.cnt);
    base = __shfl_sync(0xffffffffu, base, 0);
    const unsigned long long pmask = (1ull << P.page_log2) - 1ull;
    for (int i = lane; i < st.cnt; i += 32) {
        unsigned long long p = base + (unsigned long long)i;
        if (p < P.capacity) {
            unsigned long long pg = p >> P.page_log2, off = p & pmask;
            P.pages[pg][off] = st.pairs[i];
            if (P.emit_dist) P.dpages[pg][off] = st.dist[i];
        }
    }
    __syncwarp();
    st.cnt = 0;
}

// Warp-collective: each lane offers nout in {0, 1, 2} pairs ((qid, cid) and,
// when 2, the mirrored (cid, qid)); their slots follow lane order.
__device__ __forceinline__ void stage_emit(WarpStage& st, const JoinParams& P, int lane, int nout, int32_t qid,
                                           int32_t cid, double dist) {
    const unsigned lt = (1u << lane) - 1u;
    const unsigned b1 = __ballot_sync(0xffffffffu, nout >= 1);
    const unsigned b2 = __ballot_sync(0xffffffffu, nout == 2);
    const int tot = __popc(b1) + __popc(b2);
    if (tot == 0) return;
    if (st.cnt + tot > kStage) stage_flush(st, P, lane);
    const int pos = st.cnt + __popc(b1 & lt) + __popc(b2 & lt);
    if (nout >= 1) {
        st.pairs[pos] = make_int2(qid, cid);
        st.dist[pos] = dist;
    }
    if (nout == 2) {
        st.pairs[pos + 1] = make_int2(cid, qid);
        st.dist[pos + 1] = dist;
    }
    st.cnt += tot;
}

// Shared-memory image of one work item.
template <typename T, int DP>
struct ItemSmem {
    __align__(16) T qy[kQMax][DP];
    T qh[kQMax];
    int32_t qid[kQMax];
    int32_t rstart[kMaxRuns];
    uint32_t rpre[kMaxRuns + 1];  // prefix of run lengths
    uint8_t rmir[kMaxRuns];
};

// Loads item I into shared memory (all threads of the CTA); query rows past
// Q are zero.  Returns the candidate count C after a barrier.
template <typename T, int DP>
__device__ __forceinline__ uint32_t load_item(ItemSmem<T, DP>& S, const JoinParams& P, const Item& I) {
    const T* __restrict__ Y = static_cast<const T*>(P.y);
    const T* __restrict__ H = static_cast<const T*>(P.h);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int Q = I.q1 - I.q0;
    const int nr = I.r1 - I.r0;
    for (int i = threadIdx.x; i < kQMax * DP; i += blockDim.x)
        S.qy[i / DP][i % DP] = i < Q * DP ? Y[(int64_t)I.q0 * DP + i] : T(0);
    if (threadIdx.x < kQMax) {
        const int q = threadIdx.x;
        S.qh[q] = q < Q ? H[I.q0 + q] : T(0);
        S.qid[q] = q < Q ? P.perm[I.q0 + q] : 0;
    }
    for (int r = threadIdx.x; r < nr; r += blockDim.x) {
        const Run R = P.runs[I.r0 + r];
        S.rstart[r] = R.start;
        S.rpre[r + 1] = (uint32_t)((int32_t)(R.end_flags & ~kMirrorBit) - R.start);
        S.rmir[r] = (uint8_t)(R.end_flags >> 31);
    }
    __syncthreads();
    if (wid == 0) {  // inclusive prefix of the run lengths
        uint32_t carry = 0;
        for (int b = 0; b < nr; b += 32) {
            const int r = b + lane;
            uint32_t v = r < nr ? S.rpre[r + 1] : 0u;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += u;
            }
            if (r < nr) S.rpre[r + 1] = carry + v;
            carry += __shfl_sync(0xffffffffu, v, 31);
        }
        if (lane == 0) S.rpre[0] = 0;
    }
    __syncthreads();
    return S.rpre[nr];
}

// Candidate v (0 <= v < C) of the item: its sorted position and mirror flag.
template <typename T, int DP>
__device__ __forceinline__ int32_t map_candidate(const ItemSmem<T, DP>& S, int nr, uint32_t v, bool& mirror) {
    int lo = 0, hi = nr - 1;  // last r with rpre[r] <= v
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (S.rpre[mid] <= v)
            lo = mid;
        else
            hi = mid - 1;
    }
    mirror = S.rmir[lo] != 0;
    return S.rstart[lo] + (int32_t)(v - S.rpre[lo]);
}

}  // namespace sj
