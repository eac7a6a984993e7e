// Certified FP32 distance tiles for small dimensions (padded d <= 8), without
// distances: the filter of the low-precision join on CUDA cores, fused with
// the eps threshold and the compaction into result pages.
//
// What a tile computes is the same as k_join_cc<float> (sj_join_cc.cu): per
// (query q, candidate c) of a work item (the queries of one grid cell and the
// candidate runs of its neighbourhood, Sec. III-B),
//     a = -||y_q||^2 / 2 + sum_k y_qk * y_ck        (fma chain, k ascending)
// the expanded form of Eq. 3 with the candidate's norm moved into its two
// certified thresholds: a < thr_out means out, a >= thr_in means in, and the
// pairs in between are re-decided by the binary64 decision rule (k_recheck).
// Only the instruction stream differs; the kernel is bound by instruction
// issue, so every step is shaped to spend few instructions per pair:
//
//  * each lane holds TC candidates in registers as pairs (paired FMA over two
//    candidates, one rounding per component as the scalar FMA), the query
//    rows sit in shared memory with every coordinate duplicated, so a query
//    coordinate is one operand of the paired FMA without repacking;
//  * the threshold tests are paired adds a + (-thr): the sign of a
//    round-to-nearest sum is the sign of the exact sum (zero only when the
//    operands cancel exactly, which gives +0 since -thr is never -0), so the
//    sign bit is the test a < thr; a funnel shift moves it into the lane's
//    miss mask (queries are visited last to first, so bit q is query q);
//  * a candidate's thresholds and input index come in one 16-byte record,
//    its coordinates in one more load (two for d = 8);
//  * candidates are first pruned against the bounding box of the item's
//    queries: a lane per candidate walks the item's runs with a cursor,
//    bounds the candidate's squared distance to the box from below (binary32,
//    every operation rounded down) and drops it when that bound exceeds the
//    radius^2 (eps (1 + g) + eta)^2 of the certified "out" threshold, so the
//    pair is out for every query of the item; the kept candidates are
//    compacted (ballot + popc) into a per-warp ring in shared memory.  On
//    uniform data about half of the half-neighbourhood's candidates go (a
//    cell's neighbours reach eps beyond its corners; the grid of Sec. III-B
//    keeps every point of the 3^m cells);
//  * chunks of 32 TC kept candidates from the ring;
//  * emission: one warp scan of the lanes' output counts, then each lane
//    writes its pairs straight into the warp's shared-memory stage; a pair
//    of adjacent cells or above the self-cell triangle's diagonal, which is
//    emitted in both orders, is staged once with a flag (bit 31 of the query
//    index) and its mirror is written at the flush, so the stage holds twice
//    the output and the lane stores half of it; a chunk whose entries would
//    not fit the stage takes a general path in stage-sized windows.
#include <atomic>

#include "sj_join_common.cuh"

namespace sj {

// Candidate slots per lane of the main chunks (register budget: 2 for d = 8)
// and pairs in a warp's stage (a main chunk emits about 32 TC x the mean
// queries per item x 13% x 2 pairs on the uniform workloads; the stage holds
// a typical chunk's output).  Compile-time tuning constants.
#ifndef SJ_F32S_TC_SMALL
#define SJ_F32S_TC_SMALL 2
#endif
#ifndef SJ_F32S_STAGE
#define SJ_F32S_STAGE 512
#endif
template <int DP>
constexpr int f32s_tc() { return DP <= 4 ? SJ_F32S_TC_SMALL : 2; }
constexpr int kF32sStage = SJ_F32S_STAGE;
static_assert(2 * kF32sStage <= kStageMax, "a stage flush (entries and mirrors) resolves at most 32 pages");
// Candidates per lane of a compaction step, and the ring of kept candidates:
// a chunk takes 32 TC of them once that many are queued, and a compaction
// step adds at most 32 G, so it never holds more than 32 TC - 1 + 32 G (a
// power of two, for the index arithmetic).  Compile-time tuning constant.
#ifndef SJ_F32S_GATHER
#define SJ_F32S_GATHER 2
#endif
constexpr int kF32sGather = SJ_F32S_GATHER;
template <int DP>
constexpr int f32s_ring() { return 32 * f32s_tc<DP>() - 1 + 32 * kF32sGather <= 128 ? 128 : 256; }

template <int DP, int RUNS>
struct F32sWarp {
    __align__(16) float2 qd[kQMax][DP];  // query coordinates, each as (v, v)
    float2 qh2[kQMax];     // (h, h), h = -||y_q||^2 / 2
    int32_t qid[kQMax];    // output index of each query (batched: instance-local)
    __align__(16) float blo[DP];  // bounding box of the item's queries
    __align__(16) float bhi[DP];
    int32_t rstart[RUNS];  // first sorted position of each run
    uint32_t rpre[RUNS + 1];  // prefix of the run lengths
    uint8_t rmir[RUNS];    // 0 plain, 1 mirrored, 2 self-cell triangle
    int32_t cid[32 * f32s_tc<DP>()];  // per slot of a chunk: output index
    int32_t ring_j[f32s_ring<DP>()];  // kept candidates: sorted position
    uint8_t ring_f[f32s_ring<DP>()];  // and run flag
    unsigned long long pruned;        // pair evaluations the prune removed (lane 0)
    unsigned long long rechecked;     // pairs re-decided in place, queue full (lane 0)
    float r2;                         // the item's prune radius^2
    int smir;                         // staged entries flagged for a mirrored copy (lane 0)
    int2 stage[kF32sStage];
};

// The bounding box of the item's queries, per dim, as two values (binary32).
template <int DP>
__device__ __forceinline__ void load_box(const float* b, float (&v)[DP]) {
    if constexpr (DP == 2) {
        const float2 u = *reinterpret_cast<const float2*>(b);
        v[0] = u.x;
        v[1] = u.y;
    } else {
#pragma unroll
        for (int h = 0; h < DP / 4; ++h) {
            const float4 u = reinterpret_cast<const float4*>(b)[h];
            v[4 * h] = u.x;
            v[4 * h + 1] = u.y;
            v[4 * h + 2] = u.z;
            v[4 * h + 3] = u.w;
        }
    }
}

// Candidate coordinates of one point as DP floats, loaded with vector loads.
template <int DP>
__device__ __forceinline__ void load_coords(const float* __restrict__ Y, int32_t j, float (&c)[DP]) {
    if constexpr (DP == 2) {
        const float2 v = reinterpret_cast<const float2*>(Y)[j];
        c[0] = v.x;
        c[1] = v.y;
    } else {
#pragma unroll
        for (int h = 0; h < DP / 4; ++h) {
            const float4 v = reinterpret_cast<const float4*>(Y)[(int64_t)j * (DP / 4) + h];
            c[4 * h] = v.x;
            c[4 * h + 1] = v.y;
            c[4 * h + 2] = v.z;
            c[4 * h + 3] = v.w;
        }
    }
}

// (mask << 1) | sign bit of v: one funnel shift.
__device__ __forceinline__ uint32_t push_sign(uint32_t mask, float v) {
    return __funnelshift_l(__float_as_uint(v), mask, 1);
}

// Stage entries: (query output index | kStageMirror if the pair is also
// emitted mirrored, candidate output index); output indices are below 2^31.
constexpr uint32_t kStageMirror = 0x80000000u;

// Copies the warp's staged entries out: one atomic on the result cursor (the
// instance's cursor in a batched join) reserves entries + mirrored pairs;
// entry i goes to base + i, the mirrored pairs after them in entry order.
// Positions past the pool's capacity (a batched instance's pages) are counted
// but not written.
template <int DP, int RUNS>
__device__ __forceinline__ void f32s_flush(F32sWarp<DP, RUNS>& W, WarpStage& st, const JoinParams& P, int lane) {
    __syncwarp();
    const int ne = st.cnt;
    const unsigned long long total = (unsigned long long)(ne + W.smir);
    const unsigned lt = (1u << lane) - 1u;
    unsigned long long base = 0;
    if (P.batch) {
        const BatchJoin& B = *P.batch;
        if (lane == 0 && total > 0) base = atomicAdd(&B.cursor[st.gid], total);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (total > 0) {
            // pages of at least 64 pairs: a flush of <= kStageMax pairs
            // touches at most 32 pages, one lane resolves each
            const unsigned long long pg0 = base >> B.page_log2;
            const int npg = (int)(((base + total - 1ull) >> B.page_log2) - pg0) + 1;
            const int32_t mine = lane < npg ? batch_page(B, st.gid, pg0 + (unsigned long long)lane) : -1;
            const unsigned long long mask = (1ull << B.page_log2) - 1ull;
            unsigned long long mb = base + (unsigned long long)ne;
            for (int i0 = 0; i0 < ne; i0 += 32) {
                const int i = i0 + lane;
                const int2 e = i < ne ? st.pairs[i] : make_int2(0, 0);
                const bool m = i < ne && ((uint32_t)e.x & kStageMirror) != 0u;
                const int32_t qi = (int32_t)((uint32_t)e.x & ~kStageMirror);
                const unsigned bm = __ballot_sync(0xffffffffu, m);
                const unsigned long long p1 = base + (unsigned long long)i;
                const unsigned long long p2 = mb + (unsigned long long)__popc(bm & lt);
                const int32_t pa = __shfl_sync(0xffffffffu, mine, i < ne ? (int)((p1 >> B.page_log2) - pg0) : 0);
                const int32_t pb = __shfl_sync(0xffffffffu, mine, m ? (int)((p2 >> B.page_log2) - pg0) : 0);
                if (i < ne && pa >= 0)
                    B.pool[((long long)pa << B.page_log2) | (long long)(p1 & mask)] = make_int2(qi, e.y);
                if (m && pb >= 0) B.pool[((long long)pb << B.page_log2) | (long long)(p2 & mask)] = make_int2(e.y, qi);
                mb += (unsigned long long)__popc(bm);
            }
        }
    } else {
        if (lane == 0 && total > 0) base = atomicAdd(&P.counters[1], total);
        base = __shfl_sync(0xffffffffu, base, 0);
        unsigned long long mb = base + (unsigned long long)ne;
        for (int i0 = 0; i0 < ne; i0 += 32) {
            const int i = i0 + lane;
            const int2 e = i < ne ? st.pairs[i] : make_int2(0, 0);
            const bool m = i < ne && ((uint32_t)e.x & kStageMirror) != 0u;
            const int32_t qi = (int32_t)((uint32_t)e.x & ~kStageMirror);
            const unsigned bm = __ballot_sync(0xffffffffu, m);
            const unsigned long long p1 = base + (unsigned long long)i;
            if (i < ne && p1 < P.capacity) P.out_pairs[p1] = make_int2(qi, e.y);
            const unsigned long long p2 = mb + (unsigned long long)__popc(bm & lt);
            if (m && p2 < P.capacity) P.out_pairs[p2] = make_int2(e.y, qi);
            mb += (unsigned long long)__popc(bm);
        }
    }
    __syncwarp();
    st.cnt = 0;
    if (lane == 0) W.smir = 0;
}

// Warp-collective: each lane offers nout in {0, 1, 2} pairs ((qid, cid) and,
// when 2, the mirrored (cid, qid)): one stage entry each, flagged when 2.
template <int DP, int RUNS>
__device__ __forceinline__ void f32s_emit(F32sWarp<DP, RUNS>& W, WarpStage& st, const JoinParams& P, int lane,
                                          int nout, int32_t qid, int32_t cid) {
    const unsigned lt = (1u << lane) - 1u;
    const unsigned b1 = __ballot_sync(0xffffffffu, nout >= 1);
    const unsigned b2 = __ballot_sync(0xffffffffu, nout == 2);
    const int ne = __popc(b1);
    if (ne == 0) return;
    if (st.cnt + ne > st.cap) f32s_flush(W, st, P, lane);
    if (nout >= 1)
        st.pairs[st.cnt + __popc(b1 & lt)] =
            make_int2((int32_t)((uint32_t)qid | (nout == 2 ? kStageMirror : 0u)), cid);
    st.cnt += ne;
    if (lane == 0) W.smir += __popc(b2);
}

// Compaction step: candidates [v0, v0 + 32 G) of the item (G per lane, `r`
// the lane's run cursor, kept across steps) are tested against the queries'
// bounding box and the kept ones appended to the ring after its `cnt`
// entries from `head`; the G coordinate loads of a lane are issued before
// any is used, so their latencies overlap.  The lower bound: per dim the gap
// max(lo - c, c - hi, 0) and the sum of the squared gaps, each operation
// rounded down, is at most the exact squared distance of the candidate to
// every query; above W.r2 the pair is out for every query (the argument of
// the certified "out" threshold, pack_coefficients).  Self-cell candidates
// (flag 2) are always kept.  W.pruned counts the pair evaluations removed.
template <int DP, int RUNS, bool DBG>
__device__ __forceinline__ void f32s_gather(F32sWarp<DP, RUNS>& W, const JoinParams& P, const Item& I,
                                            const ItemRoute& R, int Q, uint32_t C, uint32_t v0, int lane, int& r,
                                            uint32_t head, uint32_t& cnt) {
    constexpr uint32_t RING = (uint32_t)f32s_ring<DP>();
    constexpr int G = kF32sGather;
    const float* __restrict__ Y = static_cast<const float*>(P.y);
    int32_t jj[G];
    uint32_t f[G];
    bool test[G], keep[G];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const uint32_t v = v0 + (uint32_t)(32 * g + lane);
        jj[g] = 0;
        f[g] = 0;
        keep[g] = v < C;
        if (v < C) {
            while (W.rpre[r + 1] <= v) ++r;
            jj[g] = W.rstart[r] + (int32_t)(v - W.rpre[r]);
            if (!SJ_BOUND(P, jj[g] >= 0 && jj[g] < P.n_points && r < RUNS, 11)) jj[g] = 0;
            f[g] = W.rmir[r];
        }
        test[g] = keep[g] && f[g] != 2u;
    }
    float c[G][DP];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        if (test[g]) {
            load_coords<DP>(Y, jj[g], c[g]);
        } else {
#pragma unroll
            for (int k = 0; k < DP; ++k) c[g][k] = 0.f;
        }
    }
    float lo[DP], hi[DP];
    load_box<DP>(W.blo, lo);
    load_box<DP>(W.bhi, hi);
    const float r2 = W.r2;
#pragma unroll
    for (int g = 0; g < G; ++g) {
        float lb = 0.f;
#pragma unroll
        for (int k = 0; k < DP; ++k) {
            const float gap = fmaxf(fmaxf(__fsub_rd(lo[k], c[g][k]), __fsub_rd(c[g][k], hi[k])), 0.f);
            lb = __fmaf_rd(gap, gap, lb);
        }
        if (test[g] && lb > r2) keep[g] = false;
    }
    uint32_t kept = 0;
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const unsigned m = __ballot_sync(0xffffffffu, keep[g]);
        if (keep[g]) {
            const uint32_t e = (head + cnt + kept + (uint32_t)__popc(m & ((1u << lane) - 1u))) & (RING - 1u);
            W.ring_j[e] = jj[g];
            W.ring_f[e] = (uint8_t)f[g];
        }
        kept += (uint32_t)__popc(m);
    }
    const uint32_t nv = min((uint32_t)(32 * G), C - v0);
    if (lane == 0) W.pruned += (unsigned long long)(nv - kept) * (unsigned long long)Q;
    cnt += kept;
    if constexpr (DBG) {
#pragma unroll
        for (int g = 0; g < G; ++g)
            if (test[g] && !keep[g])
                for (int q = 0; q < Q; ++q) dbg_record_pruned(P, I.q0 + q, jj[g]);
    }
}

// One chunk of `ns` <= 32 TC kept candidates, ring entries [head, head + ns),
// against the item's Q queries (slot t 32 + lane is entry head + t 32 + lane).
template <int DP, int RUNS, int TC, bool DBG>
__device__ __forceinline__ void f32s_chunk(F32sWarp<DP, RUNS>& W, WarpStage& st, const JoinParams& P,
                                           const Item& I, const ItemRoute& R, int Q, uint32_t ns, uint32_t head,
                                           int lane) {
    static_assert(TC % 2 == 0, "candidates go in pairs");
    constexpr uint32_t RING = (uint32_t)f32s_ring<DP>();
    const float* __restrict__ Y = static_cast<const float*>(P.y);
    const float4* __restrict__ AUX = P.aux;

    float2 cy[TC / 2][DP];  // candidate pairs, per dim
    float2 nto[TC / 2], nti[TC / 2];  // negated thresholds, never -0
    // per slot, 8 bits: the run flag (bits 0-1) and, for a self-cell
    // candidate among the item's queries, 1 + its query index (bits 2-7)
    uint32_t meta = 0;
#pragma unroll
    for (int t = 0; t < TC; ++t) {
        const uint32_t sl = (uint32_t)(t * 32 + lane);
        float c[DP];
        float to = INFINITY, ti = INFINITY;
        if (sl < ns) {
            const uint32_t e = (head + sl) & (RING - 1u);
            const int32_t jj = W.ring_j[e];
            const uint32_t f = W.ring_f[e];
            load_coords<DP>(Y, jj, c);
            const float4 ax = AUX[jj];
            to = ax.x;
            ti = ax.y;
            W.cid[t * 32 + lane] = (int32_t)(__float_as_int(ax.z) - (int32_t)R.off);
            // self-cell triangle: queries q0 .. jj pair with jj
            const uint32_t dg1 = (f == 2 && jj < I.q1) ? (uint32_t)(jj - I.q0 + 1) : 0u;
            meta |= (f | (dg1 << 2)) << (8 * t);
        } else {
#pragma unroll
            for (int k = 0; k < DP; ++k) c[k] = 0.f;
        }
        const float nt_o = __fsub_rn(0.f, to), nt_i = __fsub_rn(0.f, ti);
        if (t & 1) {
#pragma unroll
            for (int k = 0; k < DP; ++k) cy[t / 2][k].y = c[k];
            nto[t / 2].y = nt_o;
            nti[t / 2].y = nt_i;
        } else {
#pragma unroll
            for (int k = 0; k < DP; ++k) cy[t / 2][k].x = c[k];
            nto[t / 2].x = nt_o;
            nti[t / 2].x = nt_i;
        }
    }

    // miss masks: bit q set <=> a(q, slot) < thr
    uint32_t mo[TC], mi[TC];
#pragma unroll
    for (int t = 0; t < TC; ++t) mo[t] = mi[t] = 0u;
    const float2* __restrict__ qrow = &W.qd[Q - 1][0];
    const float2* __restrict__ qh = &W.qh2[Q - 1];
#pragma unroll
    for (int qq = 0; qq < kQMax; ++qq) {
        if (qq >= Q) break;
        const float2 h2 = qh[-qq];
        float2 qv[DP];
        if constexpr (DP % 2 == 0) {  // rows of DP float2 are 16-byte aligned
            const float4* q4 = reinterpret_cast<const float4*>(qrow - qq * DP);
#pragma unroll
            for (int k = 0; k < DP / 2; ++k) {
                const float4 u = q4[k];
                qv[2 * k] = make_float2(u.x, u.y);
                qv[2 * k + 1] = make_float2(u.z, u.w);
            }
        } else {
#pragma unroll
            for (int k = 0; k < DP; ++k) qv[k] = qrow[k - qq * DP];
        }
#pragma unroll
        for (int p = 0; p < TC / 2; ++p) {
            float2 a = h2;
#pragma unroll
            for (int k = 0; k < DP; ++k) a = __ffma2_rn(qv[k], cy[p][k], a);
            const float2 dout = __fadd2_rn(a, nto[p]);
            const float2 din = __fadd2_rn(a, nti[p]);
            mo[2 * p] = push_sign(mo[2 * p], dout.x);
            mo[2 * p + 1] = push_sign(mo[2 * p + 1], dout.y);
            mi[2 * p] = push_sign(mi[2 * p], din.x);
            mi[2 * p + 1] = push_sign(mi[2 * p + 1], din.y);
            if constexpr (DBG) {
                const int q = Q - 1 - qq;
                const uint32_t s0 = (uint32_t)(2 * p * 32 + lane), s1 = s0 + 32u;
                if (s0 < ns) dbg_record(P, I.q0 + q, W.ring_j[(head + s0) & (RING - 1u)], a.x);
                if (s1 < ns) dbg_record(P, I.q0 + q, W.ring_j[(head + s1) & (RING - 1u)], a.y);
            }
        }
    }

    // classify: certain-in (emitted now) and uncertain (re-decided later)
    const uint32_t qm = (1u << Q) - 1u;  // Q <= 16
    uint32_t cin[TC], unc[TC];
    int nout = 0;
    uint32_t any_unc = 0;
#pragma unroll
    for (int t = 0; t < TC; ++t) {
        const uint32_t f = (meta >> (8 * t)) & 3u;
        const uint32_t dg1 = (meta >> (8 * t + 2)) & 63u;
        const uint32_t tri = dg1 ? (1u << dg1) - 1u : 0xFFFFFFFFu;
        const uint32_t mb = ~mo[t] & qm & tri;
        cin[t] = ~mi[t] & mb;
        unc[t] = mb & mi[t];
        any_unc |= unc[t];
        // entries (low 16 bits) and mirrored copies (high 16 bits; the
        // self-cell diagonal is emitted once)
        const int c = __popc(cin[t]);
        const int dgin = (dg1 && ((cin[t] >> (dg1 - 1u)) & 1u)) ? 1 : 0;
        nout += c + (f ? (c - dgin) << 16 : 0);
    }
    int total;
    const int off16 = warp_excl_scan(nout, lane, &total);
    const int tmir = total >> 16;
    total &= 0xFFFF;
    const int off = off16 & 0xFFFF;
    nout &= 0xFFFF;
    if (total > 0) {
        if (st.cnt + total > st.cap) f32s_flush(W, st, P, lane);
        if (st.cnt + total <= st.cap) {
            // the common case: the chunk's entries fit the stage
            int pos = st.cnt + off;
            if (!SJ_BOUND(P, pos >= 0 && pos + nout <= st.cap, 12)) {
                pos = 0;
                nout = 0;
#pragma unroll
                for (int t = 0; t < TC; ++t) cin[t] = 0u;  // (the debug build skips this lane's pairs)
            }
            if constexpr (TC == 2) {
                // both slots' pairs in one loop (Q <= 16: slot t's queries
                // at bits 16 t ..), so the warp runs max over lanes of the
                // lane's pairs, not the sum over slots of the maxima
                uint32_t b = cin[0] | (cin[1] << 16);
                if (b) {
                    uint32_t two = 0;  // bit set: the pair is also written mirrored
#pragma unroll
                    for (int t = 0; t < 2; ++t) {
                        const uint32_t f = (meta >> (8 * t)) & 3u;
                        const uint32_t dg1 = (meta >> (8 * t + 2)) & 63u;
                        const uint32_t tw = f ? (dg1 ? ~(1u << (dg1 - 1u)) : 0xFFFFu) & 0xFFFFu : 0u;
                        two |= tw << (16 * t);
                    }
                    const int32_t ci0 = W.cid[lane], ci1 = W.cid[32 + lane];
                    while (b) {
                        const int bit = __ffs(b) - 1;
                        b &= b - 1u;
                        const int32_t ci = bit >= 16 ? ci1 : ci0;
                        const uint32_t qi = (uint32_t)W.qid[bit & 15] | (((two >> bit) & 1u) << 31);
                        st.pairs[pos++] = make_int2((int32_t)qi, ci);
                    }
                }
            } else {
#pragma unroll
                for (int t = 0; t < TC; ++t) {
                    uint32_t b = cin[t];
                    if (!b) continue;
                    const bool two = ((meta >> (8 * t)) & 3u) != 0u;
                    const int dg = (int)((meta >> (8 * t + 2)) & 63u) - 1;
                    const int32_t ci = W.cid[t * 32 + lane];
                    while (b) {
                        const int q = __ffs(b) - 1;
                        b &= b - 1u;
                        const uint32_t qi = (uint32_t)W.qid[q] | (two && q != dg ? kStageMirror : 0u);
                        st.pairs[pos++] = make_int2((int32_t)qi, ci);
                    }
                }
            }
            st.cnt += total;
            if (lane == 0) W.smir += tmir;
        } else {
            // dense cells: the entries in stage-sized windows; each lane
            // writes the entries of its range [off, off + nout) that fall in
            // the window, the stage is flushed after each window
            for (int w0 = 0; w0 < total;) {  // warp-uniform
                const int w1 = min(total, w0 + (st.cap - st.cnt));
                int wm = 0;  // this lane's mirrored entries in the window
                if (off < w1 && off + nout > w0) {
                    int idx = off;
#pragma unroll
                    for (int t = 0; t < TC; ++t) {
                        uint32_t b = cin[t];
                        if (!b) continue;
                        const bool two = ((meta >> (8 * t)) & 3u) != 0u;
                        const int dg = (int)((meta >> (8 * t + 2)) & 63u) - 1;
                        const int32_t ci = W.cid[t * 32 + lane];
                        while (b) {
                            const int q = __ffs(b) - 1;
                            b &= b - 1u;
                            const bool mq = two && q != dg;
                            if (idx >= w0 && idx < w1) {
                                st.pairs[st.cnt + idx - w0] =
                                    make_int2((int32_t)((uint32_t)W.qid[q] | (mq ? kStageMirror : 0u)), ci);
                                wm += mq ? 1 : 0;
                            }
                            ++idx;
                        }
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) wm += __shfl_xor_sync(0xffffffffu, wm, o);
                st.cnt += w1 - w0;
                if (lane == 0) W.smir += wm;
                w0 = w1;
                if (st.cnt == st.cap) f32s_flush(W, st, P, lane);
            }
        }
    }
    if (!__any_sync(0xffffffffu, any_unc != 0u)) return;
    // uncertain pairs: queued for the binary64 recheck (or re-decided here
    // when the queue is full), one per lane per round
    for (;;) {
        bool want = false;
        int q = 0, t_sel = 0;
#pragma unroll
        for (int t = 0; t < TC; ++t)
            if (!want && unc[t]) {
                q = __ffs(unc[t]) - 1;
                unc[t] &= unc[t] - 1u;
                want = true;
                t_sel = t;
            }
        if (!__any_sync(0xffffffffu, want)) break;
        const uint32_t ms = (meta >> (8 * t_sel)) & 0xFFu;
        const int32_t jj = want ? W.ring_j[(head + (uint32_t)(t_sel * 32 + lane)) & (RING - 1u)] : 0;
        const int32_t ci = want ? W.cid[t_sel * 32 + lane] : 0;
        const bool mir = want && (ms & 3u) != 0u && q != (int)(ms >> 2) - 1;
        const bool queued = band_push(P, lane, want, I.q0 + q, jj, mir);
        int no = 0;
        int32_t qi = 0;
        const unsigned inplace = __ballot_sync(0xffffffffu, want && !queued);
        if (lane == 0 && inplace) W.rechecked += (unsigned long long)__popc(inplace);
        if (want && !queued) {
            const double s = direct_sq(P.xs + (int64_t)(I.q0 + q) * P.dp, P.xs + (int64_t)jj * P.dp, P.d);
            if (s <= R.e2) {
                no = mir ? 2 : 1;
                qi = W.qid[q];
            }
        }
        f32s_emit(W, st, P, lane, no, qi, ci);
    }
}

// Minimum resident CTAs per SM asked of the register allocator (4 warps
// each), per padded dimension.  Compile-time tuning constants.
#ifndef SJ_F32S_MIN_BLOCKS_D2
#define SJ_F32S_MIN_BLOCKS_D2 8
#endif
#ifndef SJ_F32S_MIN_BLOCKS_D4
#define SJ_F32S_MIN_BLOCKS_D4 8
#endif
#ifndef SJ_F32S_MIN_BLOCKS_D8
#define SJ_F32S_MIN_BLOCKS_D8 7
#endif
constexpr int kF32sWarps = 4;
template <int DP>
constexpr int f32s_min_blocks() {
    return DP == 2 ? SJ_F32S_MIN_BLOCKS_D2 : DP == 4 ? SJ_F32S_MIN_BLOCKS_D4 : SJ_F32S_MIN_BLOCKS_D8;
}

template <int DP, int RUNS, bool DBG>
__global__ void __launch_bounds__(kF32sWarps * 32, f32s_min_blocks<DP>()) k_join_f32s(JoinParams P) {
    constexpr int TC = f32s_tc<DP>();
    constexpr uint32_t SLOTS = 32u * TC;
    constexpr uint32_t RING = (uint32_t)f32s_ring<DP>();
    static_assert(SLOTS - 1u + 32u * kF32sGather <= RING, "the ring holds a chunk and one compaction step");
    __shared__ F32sWarp<DP, RUNS> smem[kF32sWarps];
    const float* __restrict__ Y = static_cast<const float*>(P.y);
    const float* __restrict__ H = static_cast<const float*>(P.h);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    F32sWarp<DP, RUNS>& W = smem[wid];
    WarpStage st{W.stage, nullptr, 0, 0, kF32sStage};
    if (lane == 0) {
        W.pruned = 0;
        W.rechecked = 0;
        W.smir = 0;
    }

    long long next = 0;
    if (lane == 0) next = (long long)atomicAdd(&P.counters[0], 1ull);
    next = __shfl_sync(0xffffffffu, next, 0);
    for (;;) {
        const long long it = next;
        if (it >= P.n_items) break;
        if (lane == 0) next = (long long)atomicAdd(&P.counters[0], 1ull);  // used next iteration
        next = __shfl_sync(0xffffffffu, next, 0);
        const Item I = P.items[it];
        const int Q = I.q1 - I.q0;
        const int nr = I.r1 - I.r0;
        if (!SJ_BOUND(P, I.q0 >= 0 && Q >= 1 && Q <= kQMax && I.q1 <= P.n_points && nr >= 0 && nr <= RUNS, 13))
            continue;
        // (batched: the stage holds one instance's entries; flushed here, in
        // its own format, before item_route would flush it)
        if (P.batch && st.cnt > 0 && P.batch->inst_gid[P.batch->item_inst[it]] != st.gid) f32s_flush(W, st, P, lane);
        const ItemRoute R = item_route(st, P, it, lane);
        // the item's queries (duplicated coordinates), their bounding box
        // (lane holds dim lane % DP, as 32 is a multiple of DP) and runs
        float bmin = INFINITY, bmax = -INFINITY;
        for (int i = lane; i < kQMax * DP; i += 32) {
            const int q = i / DP;
            const float v = q < Q ? Y[(int64_t)I.q0 * DP + i] : 0.f;
            W.qd[q][i % DP] = make_float2(v, v);
            if (q < Q) {
                bmin = fminf(bmin, v);
                bmax = fmaxf(bmax, v);
            }
        }
#pragma unroll
        for (int o = DP; o < 32; o <<= 1) {
            bmin = fminf(bmin, __shfl_xor_sync(0xffffffffu, bmin, o));
            bmax = fmaxf(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
        }
        if (lane < DP) {
            W.blo[lane] = bmin;
            W.bhi[lane] = bmax;
        }
        if (lane == 0) W.r2 = R.r2;
        if (lane < kQMax) {
            const float h = lane < Q ? H[I.q0 + lane] : -INFINITY;
            W.qh2[lane] = make_float2(h, h);
            W.qid[lane] = lane < Q ? (int32_t)(P.perm[I.q0 + lane] - R.off) : 0;
        }
        uint32_t carry = 0;
        for (int b = 0; b < nr; b += 32) {
            const int rr = b + lane;
            uint32_t len = 0;
            if (rr < nr) {
                const Run Rn = P.runs[I.r0 + rr];
                const bool self = P.tri && !(Rn.end_flags & kMirrorBit);
                const int32_t start = self ? I.q0 : Rn.start;
                W.rstart[rr] = start;
                W.rmir[rr] = self ? (uint8_t)2 : (uint8_t)(Rn.end_flags >> 31);
                len = (uint32_t)((int32_t)(Rn.end_flags & ~kMirrorBit) - start);
            }
            uint32_t v = len;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += u;
            }
            if (rr < nr) W.rpre[rr + 1] = carry + v;
            carry += __shfl_sync(0xffffffffu, v, 31);
        }
        if (lane == 0) W.rpre[0] = 0;
        __syncwarp();
        const uint32_t C = carry;
        // compaction steps of 32 G candidates into the ring, a chunk whenever
        // SLOTS kept candidates are queued, then the rest
        // (one call site each, so one inlined copy of the chunk's code)
        int r = 0;
        uint32_t head = 0, cnt = 0, v0 = 0;
        for (;;) {  // warp-uniform
            if (v0 < C) {
                f32s_gather<DP, RUNS, DBG>(W, P, I, R, Q, C, v0, lane, r, head, cnt);
                v0 += 32u * kF32sGather;
            }
            const bool more = v0 < C;
            if (cnt >= SLOTS || (!more && cnt > 0u)) {
                const uint32_t ns = min(cnt, SLOTS);
                __syncwarp();
                f32s_chunk<DP, RUNS, TC, DBG>(W, st, P, I, R, Q, ns, head, lane);
                head = (head + ns) & (RING - 1u);
                cnt -= ns;
            } else if (!more) {
                break;
            }
        }
        __syncwarp();
    }
    f32s_flush(W, st, P, lane);
    if (lane == 0 && W.rechecked) atomicAdd(&P.counters[2], W.rechecked);
    if (lane == 0 && W.pruned) atomicAdd(&P.counters[6], W.pruned);
}

template <int DP, int RUNS, bool DBG>
static int launch_f32s_dr(Index* ix, const JoinParams& p) {
    auto kern = k_join_f32s<DP, RUNS, DBG>;
    static std::atomic<int> cached{0};  // resident CTAs per SM (a property of the kernel)
    int per_sm = cached.load(std::memory_order_relaxed);
    if (per_sm == 0) {
        SJ_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kF32sWarps * 32, 0));
        if (per_sm < 1) per_sm = 1;
        cached.store(per_sm, std::memory_order_relaxed);
    }
    long long blocks = (long long)device_sm_count(ix->device) * per_sm;
    const long long need = (ix->n_items + kF32sWarps - 1) / kF32sWarps;
    if (blocks > need) blocks = need > 0 ? need : 1;
    kern<<<(unsigned)blocks, kF32sWarps * 32, 0, ix->stream>>>(p);
    note_launch();
    SJ_CK(cudaGetLastError());
    return SJ_OK;
}

template <int DP>
static int launch_f32s_d(Index* ix, const JoinParams& p) {
    if (p.dbg) return launch_f32s_dr<DP, kMaxRuns, true>(ix, p);  // the filter dump (test aid)
    return ix->m <= 4 ? launch_f32s_dr<DP, 28, false>(ix, p) : launch_f32s_dr<DP, kMaxRuns, false>(ix, p);
}

bool f32s_supported(const Index* ix, int emit_dist) {
    return ix->kernel == SJ_KERNEL_FILTER_F32 && !emit_dist && ix->dp <= 8 && ix->aux != nullptr;
}

int launch_join_f32s(Index* ix, const JoinOut& out) {
    const JoinParams p = make_join_params(ix, out, 0);
    switch (ix->dp) {
        case 2: return launch_f32s_d<2>(ix, p);
        case 4: return launch_f32s_d<4>(ix, p);
        case 8: return launch_f32s_d<8>(ix, p);
        default:
            set_error("no small-d FP32 kernel for padded dimension %d", ix->dp);
            return SJ_ERR_UNSUPPORTED;
    }
}

}  // namespace sj
