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
    long long n_points;            // packed points (bound of every queued sorted position)
    unsigned long long* counters;  // [0] item queue, [1] result cursor, [2] rechecked
    int2* out_pairs;               // the result pool (pages are views of it)
    double* out_dist;              // distances, or null
    unsigned long long capacity;   // pairs the pool holds
    double e2;
    int d;
    int dp;            // padded dimension (row stride of xs)
    int emit_dist;
    int tri;           // symmetric join: evaluate only the triangle of each self cell
    // deferred re-decisions: pairs whose certified bound straddles eps (and,
    // when distances are emitted, every maybe-in pair) are queued here and
    // re-decided by k_recheck with whole warps.  Entry: (query sorted
    // position, candidate sorted position | kMirrorBit).  counters[3] counts
    // queued entries; past `band_cap` a pair is re-decided in place.
    int2* band;
    unsigned long long band_cap;
    const BatchJoin* batch;  // null for a single join
    const float4* aux;       // small-d FP32 filter: per point (thr_out, thr_in, input index bits, 0)
    // short-circuit of the FP64 tile (sj_options.short_circuit): per point, an
    // upper bound of half its norm over the dims after the checkpoint (the
    // first sc_b kernel dims) plus the error margin; null when off
    const double* sc_w;
    int sc_b;
    // test aid (sj_debug_filter_dump): when set, the FP32 filters record
    // every evaluated (query, candidate) pair with their filter value a as
    // (query sorted position, candidate sorted position, bits of a, 0);
    // counters[5] counts records, those past dbg_cap are dropped
    int4* dbg;
    unsigned long long dbg_cap;
    // small-d FP32 filter: a candidate whose squared distance to the bounding
    // box of an item's queries exceeds prune_r2 (kernel units) is out for
    // every query and is not evaluated (single joins; batched joins take the
    // per-instance value from BatchJoin::inst_r2); counters[6] counts the
    // pair evaluations this removes
    float prune_r2;
};

// Records one evaluated pair for the filter dump.
__device__ __forceinline__ void dbg_record(const JoinParams& P, int32_t qs, int32_t cs, float a) {
    const unsigned long long k = atomicAdd(&P.counters[5], 1ull);
    if (k < P.dbg_cap) P.dbg[k] = make_int4(qs, cs, __float_as_int(a), 0);
}
// Records one pair the bounding-box prune decided out without evaluating it
// (fourth field 1, no filter value).
__device__ __forceinline__ void dbg_record_pruned(const JoinParams& P, int32_t qs, int32_t cs) {
    const unsigned long long k = atomicAdd(&P.counters[5], 1ull);
    if (k < P.dbg_cap) P.dbg[k] = make_int4(qs, cs, 0, 1);
}

JoinParams make_join_params(Index* ix, const JoinOut& out, int emit_dist);

// Bounds checks of the debug build (compiled with -DSJ_DEBUG_BOUNDS): a
// failed check records its site number in counters[7] (the first one wins),
// evaluates to false so the caller skips the access it guards, and the host
// reports SJ_ERR_CUDA naming the site.  In the regular build they are no
// code at all.
#ifdef SJ_DEBUG_BOUNDS
#define SJ_BOUND(P, cond, site) \
    ((cond) ? true : (atomicCAS(&(P).counters[7], 0ull, (unsigned long long)(site)), false))
#else
#define SJ_BOUND(P, cond, site) true
#endif
// CUDA-core tile launch for padded dimension DP (sj_join_cc.cuh; explicit
// instantiations in sj_cc_d*.cu).
template <typename T, int DP>
int launch_cc_dp(Index* ix, const JoinParams& p);

// Fused multiply-add in the kernel type, one rounding (explicit intrinsics so
// a float chain never runs on the FP64 pipe).
__device__ __forceinline__ float fma_t(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return __fma_rn(a, b, c); }

// Order key of a binary64 value as a signed 64-bit integer: for non-NaN
// values, a < b  <=>  key(a) < key(b) (with -0 ordered just below +0).
// Comparing keys moves the threshold test of the FP64 kernels from the FP64
// pipe to the integer ALUs.
__device__ __forceinline__ long long order_key(double v) {
    const long long b = __double_as_longlong(v);
    return b ^ ((b >> 63) & 0x7FFFFFFFFFFFFFFFll);
}
// a >= t for a float / double against a threshold whose order key (double)
// or value (float) is given.
__device__ __forceinline__ bool ge_threshold(float a, float t) { return a >= t; }
__device__ __forceinline__ bool ge_threshold(double a, double t) { return order_key(a) >= order_key(t); }

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
    int2* pairs;   // cap slots of this warp
    double* dist;  // cap slots (used when distances are emitted)
    int cnt;       // warp-uniform fill
    int gid;       // batched join: the instance the staged pairs belong to
    int cap = kStage;  // slots
};

// Batched join: the slot of pair position p of instance gid in the shared
// pool, taking a fresh page for it on first use (a page-table slot is claimed
// with a compare-and-swap; a thread that loses the race leaves its page
// unused).  Returns null when the instance's table or the pool is exhausted
// (the pair is then counted but not stored).
// The pool page holding page `pg` of instance `gid`, taken from the pool on
// first use; -1 when pg is past the instance's page table or the pool is
// exhausted (the host sees both from the counters and reruns).  The first
// caller locks the table slot (-2) and takes the next pool page (or marks the
// slot exhausted, -3); later callers wait for it with a bounded spin whose
// expiry raises B.error.
__device__ __forceinline__ int32_t batch_page(const BatchJoin& B, int gid, unsigned long long pg) {
    if (pg >= (unsigned long long)B.max_pages[gid]) return -1;
    int32_t* slot = B.page_table + B.table_off[gid] + (long long)pg;
    volatile int32_t* vslot = slot;
    int32_t page = *vslot;
    if (page == -1) {
        const int32_t old = atomicCAS(slot, -1, -2);
        if (old == -1) {
            const unsigned long long fresh = atomicAdd(B.pool_next, 1ull);
            page = fresh < (unsigned long long)B.n_pages ? (int32_t)fresh : -3;
            atomicExch(slot, page);
        } else {
            page = old;
        }
    }
    for (int it = 0; page == -2; ++it) {
        if (it == (1 << 20)) {
            atomicExch(B.error, 1ull);
            return -1;
        }
        __nanosleep(64);
        page = *vslot;
    }
    return page >= 0 ? page : -1;
}

static_assert(kStage / 64 + 1 <= 32, "a warp's flush must touch at most 32 pages");
constexpr int kStageMax = 31 * 64;  // largest stage whose flush touches at most 32 pages of 64

// Pool slot of position p of instance gid's result, or -1.
__device__ __forceinline__ long long batch_slot(const BatchJoin& B, int gid, unsigned long long p) {
    const int32_t page = batch_page(B, gid, p >> B.page_log2);
    if (page < 0) return -1;
    return ((long long)page << B.page_log2) | (long long)(p & ((1ull << B.page_log2) - 1ull));
}

// Reserves room for the warp's staged pairs with one atomic on the result
// cursor and copies them to their pages (coalesced).  Positions past the
// pool's capacity are counted but not written.
__device__ __forceinline__ void stage_flush(WarpStage& st, const JoinParams& P, int lane) {
    __syncwarp();
    if (P.batch) {
        const BatchJoin& B = *P.batch;
        unsigned long long base = 0;
        if (lane == 0 && st.cnt > 0) base = atomicAdd(&B.cursor[st.gid], (unsigned long long)st.cnt);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (st.cnt > 0) {
            // pages of at least 64 pairs: a flush of <= kStageMax pairs
            // touches at most 32 pages, one lane resolves each
            const unsigned long long pg0 = base >> B.page_log2;
            const int npg = (int)(((base + (unsigned long long)st.cnt - 1ull) >> B.page_log2) - pg0) + 1;
            const int32_t mine = lane < npg ? batch_page(B, st.gid, pg0 + (unsigned long long)lane) : -1;
            const unsigned long long mask = (1ull << B.page_log2) - 1ull;
            for (int i0 = 0; i0 < st.cnt; i0 += 32) {
                const int i = i0 + lane;
                const unsigned long long p = base + (unsigned long long)i;
                const int src = i < st.cnt ? (int)((p >> B.page_log2) - pg0) : 0;
                const int32_t page = __shfl_sync(0xffffffffu, mine, src);
                if (i < st.cnt && page >= 0) {
                    const long long s = ((long long)page << B.page_log2) | (long long)(p & mask);
                    B.pool[s] = st.pairs[i];
                    if (P.emit_dist) B.dpool[s] = st.dist[i];
                }
            }
        }
        __syncwarp();
        st.cnt = 0;
        return;
    }
    unsigned long long base = 0;
    if (lane == 0 && st.cnt > 0) base = atomicAdd(&P.counters[1], (unsigned long long)st.cnt);
    base = __shfl_sync(0xffffffffu, base, 0);
    for (int i = lane; i < st.cnt; i += 32) {
        const unsigned long long p = base + (unsigned long long)i;
        if (p < P.capacity) {
            P.out_pairs[p] = st.pairs[i];
            if (P.emit_dist) P.out_dist[p] = st.dist[i];
        }
    }
    __syncwarp();
    st.cnt = 0;
}

// Batched join, per work item: the instance of item `it` (its number in the
// batch), its first point in the group and its eps^2.  The warp's stage is
// flushed when the instance changes.
struct ItemRoute {
    int gid;
    long long off;
    double e2;
    float r2;  // the bounding-box prune's radius^2 (small-d FP32 filter)
};
__device__ __forceinline__ ItemRoute item_route(WarpStage& st, const JoinParams& P, long long it, int lane) {
    ItemRoute r{0, 0, P.e2, P.prune_r2};
    if (P.batch) {
        const int li = P.batch->item_inst[it];
        r.gid = P.batch->inst_gid[li];
        r.off = P.batch->inst_off[li];
        r.e2 = P.batch->inst_e2[li];
        r.r2 = P.batch->inst_r2 ? P.batch->inst_r2[li] : INFINITY;
        if (st.cnt > 0 && st.gid != r.gid) stage_flush(st, P, lane);
        st.gid = r.gid;
    }
    return r;
}

// Batched join: one pair (and its mirror when nout == 2) written by a single
// lane (used by the recheck kernel, whose lanes may serve different instances).
__device__ __forceinline__ void batch_emit_one(const JoinParams& P, int gid, int nout, int32_t qid, int32_t cid,
                                               double dist) {
    const BatchJoin& B = *P.batch;
    const unsigned long long base = atomicAdd(&B.cursor[gid], (unsigned long long)nout);
    for (int k = 0; k < nout; ++k) {
        const long long s = batch_slot(B, gid, base + k);
        if (s >= 0) {
            B.pool[s] = k == 0 ? make_int2(qid, cid) : make_int2(cid, qid);
            if (P.emit_dist) B.dpool[s] = dist;
        }
    }
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
    if (st.cnt + tot > st.cap) stage_flush(st, P, lane);
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

// Warp-collective emission without distances (nothing of binary64 is touched).
__device__ __forceinline__ void stage_emit_pairs(WarpStage& st, const JoinParams& P, int lane, int nout,
                                                 int32_t qid, int32_t cid) {
    const unsigned lt = (1u << lane) - 1u;
    const unsigned b1 = __ballot_sync(0xffffffffu, nout >= 1);
    const unsigned b2 = __ballot_sync(0xffffffffu, nout == 2);
    const int tot = __popc(b1) + __popc(b2);
    if (tot == 0) return;
    if (st.cnt + tot > st.cap) stage_flush(st, P, lane);
    const int pos = st.cnt + __popc(b1 & lt) + __popc(b2 & lt);
    if (nout >= 1) st.pairs[pos] = make_int2(qid, cid);
    if (nout == 2) st.pairs[pos + 1] = make_int2(cid, qid);
    st.cnt += tot;
}

// Warp-collective: lanes with `want` queue (qs, cs | mirror) for the
// deferred recheck, one atomic per warp.  Returns, per lane, whether its entry
// found room (if not, the caller re-decides the pair itself).
__device__ __forceinline__ bool band_push(const JoinParams& P, int lane, bool want, int32_t qs, int32_t cs,
                                          bool mirror) {
    const unsigned m = __ballot_sync(0xffffffffu, want);
    if (m == 0) return false;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&P.counters[3], (unsigned long long)__popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (!want) return false;
    const unsigned long long pos = base + (unsigned long long)__popc(m & ((1u << lane) - 1u));
    if (pos >= P.band_cap) return false;
    P.band[pos] = make_int2(qs, (int32_t)((uint32_t)cs | (mirror ? kMirrorBit : 0u)));
    return true;
}

// Per-warp reservation in the recheck queue: a warp takes queue slots in
// chunks of kBandChunk with one atomic and fills them in order, so a tile
// waits on a queue atomic once per chunk rather than once per round of
// entries.  Slots a warp reserved but did not fill are closed with the
// sentinel (-1, -1) before the kernel ends; the recheck kernel skips entries
// outside [0, n).
constexpr int kBandChunk = 64;
struct BandQ {
    unsigned long long base;  // next reserved slot
    int left;                 // reserved slots left (warp-uniform)
};

// Warp-collective: lanes with `want` queue (qs, cs | mirror); returns, per
// lane, whether its entry found room (if not, the queue is full and the
// caller re-decides the pair itself).
__device__ __forceinline__ bool band_push_q(BandQ& bq, const JoinParams& P, int lane, bool want, int32_t qs,
                                            int32_t cs, bool mirror) {
    const unsigned m = __ballot_sync(0xffffffffu, want);
    if (m == 0) return false;
    const int n = __popc(m);
    const int r = __popc(m & ((1u << lane) - 1u));
    unsigned long long pos;
    if (n <= bq.left) {
        pos = bq.base + (unsigned long long)r;
        bq.base += (unsigned long long)n;
        bq.left -= n;
    } else {  // the rest of this chunk, then a fresh one (n <= 32 < kBandChunk)
        unsigned long long fresh = 0;
        if (lane == 0) fresh = atomicAdd(&P.counters[3], (unsigned long long)kBandChunk);
        fresh = __shfl_sync(0xffffffffu, fresh, 0);
        pos = r < bq.left ? bq.base + (unsigned long long)r : fresh + (unsigned long long)(r - bq.left);
        const int used = n - bq.left;
        bq.base = fresh + (unsigned long long)used;
        bq.left = kBandChunk - used;
    }
    if (!want || pos >= P.band_cap) return false;
    P.band[pos] = make_int2(qs, (int32_t)((uint32_t)cs | (mirror ? kMirrorBit : 0u)));
    return true;
}

// Closes the warp's reservation: its unfilled slots get the sentinel.
__device__ __forceinline__ void band_q_close(BandQ& bq, const JoinParams& P, int lane) {
    for (int i = lane; i < bq.left; i += 32) {
        const unsigned long long pos = bq.base + (unsigned long long)i;
        if (pos < P.band_cap) P.band[pos] = make_int2(-1, -1);
    }
    bq.left = 0;
}

// Warp-wide exclusive prefix sum of v; *total gets the sum.
__device__ __forceinline__ int warp_excl_scan(int v, int lane, int* total) {
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    *total = __shfl_sync(0xffffffffu, x, 31);
    return x - v;
}

// Shared-memory image of one work item (RUNS: run capacity, 3^(m-1) + 1 for
// a grid of m indexed dims).
template <typename T, int DP, int RUNS = kMaxRuns>
struct ItemSmem {
    __align__(16) T qy[kQMax][DP];
    T qh[kQMax];
    int32_t qid[kQMax];
    int32_t rstart[RUNS];
    uint32_t rpre[RUNS + 1];  // prefix of run lengths
    uint8_t rmir[RUNS];
};

// Loads item I into shared memory (all threads of the CTA); query rows past
// Q are zero.  Returns the candidate count C after a barrier.
template <typename T, int DP, int RUNS>
__device__ __forceinline__ uint32_t load_item(ItemSmem<T, DP, RUNS>& S, const JoinParams& P, const Item& I) {
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

// Warp-level variant of load_item: the calling warp alone fills S (its own
// copy) and the result is visible to the warp after the returned __syncwarp.
template <typename T, int DP, int RUNS>
// With P.tri the self-cell run (the one run without the mirror flag in a
// symmetric join) starts at the item's first query and is flagged 2: its
// pairs above the diagonal are emitted in both orders, those below skipped.
__device__ __forceinline__ uint32_t load_item_warp(ItemSmem<T, DP, RUNS>& S, const JoinParams& P, const Item& I,
                                                   int lane) {
    const T* __restrict__ Y = static_cast<const T*>(P.y);
    const T* __restrict__ H = static_cast<const T*>(P.h);
    const int Q = I.q1 - I.q0;
    const int nr = I.r1 - I.r0;
    for (int i = lane; i < kQMax * DP; i += 32) S.qy[i / DP][i % DP] = i < Q * DP ? Y[(int64_t)I.q0 * DP + i] : T(0);
    if (lane < kQMax) {
        S.qh[lane] = lane < Q ? H[I.q0 + lane] : T(0);
        S.qid[lane] = lane < Q ? P.perm[I.q0 + lane] : 0;
    }
    uint32_t carry = 0;
    for (int b = 0; b < nr; b += 32) {
        const int r = b + lane;
        uint32_t len = 0;
        if (r < nr) {
            const Run R = P.runs[I.r0 + r];
            const bool self = P.tri && !(R.end_flags & kMirrorBit);
            const int32_t start = self ? I.q0 : R.start;
            S.rstart[r] = start;
            S.rmir[r] = self ? (uint8_t)2 : (uint8_t)(R.end_flags >> 31);
            len = (uint32_t)((int32_t)(R.end_flags & ~kMirrorBit) - start);
        }
        uint32_t v = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += u;
        }
        if (r < nr) S.rpre[r + 1] = carry + v;
        carry += __shfl_sync(0xffffffffu, v, 31);
    }
    if (lane == 0) S.rpre[0] = 0;
    __syncwarp();
    return carry;
}

// Candidate v (0 <= v < C) of an item whose runs are (rstart, rpre, rmir).
__device__ __forceinline__ int32_t map_candidate_tc(const int32_t* rstart, const uint32_t* rpre, const uint8_t* rmir,
                                                    int nr, uint32_t v, bool& mirror) {
    int lo = 0, hi = nr - 1;  // last r with rpre[r] <= v
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (rpre[mid] <= v)
            lo = mid;
        else
            hi = mid - 1;
    }
    mirror = rmir[lo] != 0;
    return rstart[lo] + (int32_t)(v - rpre[lo]);
}

// Candidate v (0 <= v < C) of the item: its sorted position and mirror flag.
template <typename T, int DP, int RUNS>
__device__ __forceinline__ int32_t map_candidate(const ItemSmem<T, DP, RUNS>& S, int nr, uint32_t v, bool& mirror) {
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

// As map_candidate, with the run's flag (0 plain, 1 mirror, 2 self-cell triangle).
template <typename T, int DP, int RUNS>
__device__ __forceinline__ int32_t map_candidate_flag(const ItemSmem<T, DP, RUNS>& S, int nr, uint32_t v,
                                                      uint8_t& flag) {
    int lo = 0, hi = nr - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (S.rpre[mid] <= v)
            lo = mid;
        else
            hi = mid - 1;
    }
    flag = S.rmir[lo];
    return S.rstart[lo] + (int32_t)(v - S.rpre[lo]);
}

}  // namespace sj
