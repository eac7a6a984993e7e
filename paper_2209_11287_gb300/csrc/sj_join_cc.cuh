// Distance tiles on CUDA cores, fused with the eps threshold and the
// compaction into result pages (templates; each padded dimension is
// instantiated in a translation unit of its own, sj_cc_d*.cu, so the library
// compiles in parallel).
//
// One work item = up to kQMax queries of one grid cell and the candidate runs
// of that cell (Sec. III-B: the queries of a cell share their candidates).
// Per (query, candidate) pair the tile computes, in the kernel type T,
//     a = -||y_q||^2 / 2 + sum_k y_qk * y_ck          (fma chain, k ascending)
// which is the expanded form of Eq. 3 with the constant part moved to the
// candidate's threshold: ||y_q - y_c||^2 = ||y_c||^2 - 2 a.  Per-candidate
// thresholds (computed at packing) certify the decision: a < thr_out means
// out, a >= thr_in means in; pairs in between are re-decided with the
// decision rule itself (binary64 direct form, dimension order, no
// contraction) by k_recheck, so the returned set equals the rule's.
//
// T = double is the plain FP64 join (Eq. 3/4 evaluated on FP64 CUDA cores);
// T = float is the certified FP32 filter.
//
// Work decomposition: every warp takes work items on its own (an atomic
// queue, the next index fetched one item ahead), so no block-wide barrier
// ever stalls a tile.  A warp evaluates its item in chunks of 32 x TC
// candidates: each lane holds TC candidates in registers and walks the
// item's queries, broadcast from shared memory.  For d <= 8 the threshold
// test is fused into the query loop (and FP32 pairs of candidates use the
// paired FMA, one rounding per lane as for the scalar FMA); for larger d
// the accumulators of all queries are kept and tested after the d-loop.  The
// "maybe in" pairs of a chunk (a >= thr_out) are compacted into a per-warp
// list with one warp scan, and the list is classified 32 entries at a time,
// so the rare work (certain-in test, queueing for the recheck, emission)
// runs with every lane busy.
#pragma once

#include <type_traits>

#include "sj_join_common.cuh"

namespace sj {

// Warps per CTA (independent of each other): as many as keep the per-warp
// shared memory of a CTA within the 48 KB of static shared memory, at most 4.
template <typename WS>
constexpr int cc_warps() {
    return sizeof(WS) * 4 <= 46 * 1024 ? 4 : sizeof(WS) * 2 <= 46 * 1024 ? 2 : 1;
}

template <typename T, int DP, int TC, bool EMIT, int RUNS>
struct CcWarpSmem {
    ItemSmem<T, DP, RUNS> it;
    int32_t cj[EMIT ? 32 * TC : 1];    // sorted position of each candidate slot (with distances)
    int32_t cperm[32 * TC];            // its input index
    uint8_t cmir[32 * TC];             // its mirror flag
    uint16_t list[EMIT ? 32 * TC * (kQMax / 2) : 1];  // with distances: maybe-in entries of one half
                                                      // of the queries, slot << 4 | query
    int2 stage[kStage];
    double sdist[EMIT ? kStage : 1];
    double scq[DP >= 16 ? kQMax : 1];  // short-circuit: each query's w
};

// Maybe-in bitmasks of TC candidates against all queries of the item, d <= 8:
// the threshold test follows each query's fma chain.
template <typename T, int DP, int TC, int RUNS>
__device__ __forceinline__ void tile_fused(const ItemSmem<T, DP, RUNS>& S, int Q, const T (&c)[TC][DP], const T (&to)[TC],
                                           const T (&ti)[TC], uint32_t (&bits)[TC], uint32_t (&cbits)[TC]) {
#pragma unroll
    for (int t = 0; t < TC; ++t) bits[t] = cbits[t] = 0;
    if constexpr (std::is_same<T, float>::value && TC % 2 == 0) {
#pragma unroll
        for (int q = 0; q < kQMax; ++q) {
            if (q >= Q) break;
            const float h = S.qh[q];
#pragma unroll
            for (int t = 0; t < TC; t += 2) {
                float2 a = make_float2(h, h);
#pragma unroll
                for (int k = 0; k < DP; ++k) {
                    const float qv = S.qy[q][k];
                    a = __ffma2_rn(make_float2(qv, qv), make_float2(c[t][k], c[t + 1][k]), a);
                }
                if (a.x >= to[t]) bits[t] |= 1u << q;
                if (a.y >= to[t + 1]) bits[t + 1] |= 1u << q;
                if (a.x >= ti[t]) cbits[t] |= 1u << q;
                if (a.y >= ti[t + 1]) cbits[t + 1] |= 1u << q;
            }
        }
    } else {
#pragma unroll
        for (int q = 0; q < kQMax; ++q) {
            if (q >= Q) break;
            const T h = S.qh[q];
#pragma unroll
            for (int t = 0; t < TC; ++t) {
                T a = h;
#pragma unroll
                for (int k = 0; k < DP; ++k) a = fma_t(S.qy[q][k], c[t][k], a);
                if (ge_threshold(a, to[t])) bits[t] |= 1u << q;
                if (ge_threshold(a, ti[t])) cbits[t] |= 1u << q;
            }
        }
    }
}

// Emission of one chunk without distances.  Certain pairs (maybe-in and
// certain-in bits) go straight into the warp's stage: one warp scan of each
// lane's output count (two outputs for a mirrored pair, one for a self pair)
// gives every lane its slots, and each lane writes its pairs in query order.
// A chunk larger than the stage is written in stage-sized windows, each
// flushed when full.  Uncertain pairs (maybe-in, not certain-in: the
// certified bound straddles eps) are queued for the binary64 recheck, one
// per lane per round, or re-decided here when the queue is full.
template <int TC>
__device__ __forceinline__ void emit_direct(WarpStage& st, const JoinParams& P, const int32_t* cperm,
                                            const uint8_t* cmir, const int32_t* qids, const ItemRoute& R,
                                            const Item& I, int lane, const int32_t (&j)[TC],
                                            const uint32_t (&bits)[TC], const uint32_t (&cbits)[TC],
                                            unsigned long long& rechecked) {
    int nout = 0;
    uint32_t any_unc = 0;
#pragma unroll
    for (int t = 0; t < TC; ++t) {
        const uint32_t cin = bits[t] & cbits[t];
        any_unc |= bits[t] & ~cbits[t];
        if (cin) {
            const int fl = cmir[t * 32 + lane];
            const int c = __popc(cin);
            nout += fl ? 2 * c : c;
            const int qd = j[t] - I.q0;  // the diagonal of a self-cell candidate
            if (fl == 2 && qd >= 0 && qd < kQMax && ((cin >> qd) & 1u)) nout -= 1;
        }
    }
    int total;
    const int off = warp_excl_scan(nout, lane, &total);
    if (total > 0) {
        if (st.cnt + total > kStage) stage_flush(st, P, lane);
        for (int w0 = 0; w0 < total;) {  // warp-uniform
            const int w1 = min(total, w0 + (kStage - st.cnt));
            if (off < w1 && off + nout > w0) {
                int idx = off;
#pragma unroll
                for (int t = 0; t < TC; ++t) {
                    uint32_t b = bits[t] & cbits[t];
                    if (!b) continue;
                    const int slot = t * 32 + lane;
                    const int fl = cmir[slot];
                    const int32_t cid = (int32_t)(cperm[slot] - R.off);
                    const int qd = fl == 2 ? j[t] - I.q0 : -1;
                    while (b) {
                        const int q = __ffs(b) - 1;
                        b &= b - 1u;
                        const int32_t qid = (int32_t)(qids[q] - R.off);
                        if (idx >= w0 && idx < w1) st.pairs[st.cnt + idx - w0] = make_int2(qid, cid);
                        ++idx;
                        if (fl == 1 || (fl == 2 && q != qd)) {
                            if (idx >= w0 && idx < w1) st.pairs[st.cnt + idx - w0] = make_int2(cid, qid);
                            ++idx;
                        }
                    }
                }
            }
            st.cnt += w1 - w0;
            w0 = w1;
            if (st.cnt == kStage) stage_flush(st, P, lane);
        }
    }
    if (!__any_sync(0xffffffffu, any_unc != 0u)) return;
    uint32_t unc[TC];
#pragma unroll
    for (int t = 0; t < TC; ++t) unc[t] = bits[t] & ~cbits[t];
    for (;;) {
        bool want = false;
        int q = 0, slot = 0;
        int32_t jj = 0;
#pragma unroll
        for (int t = 0; t < TC; ++t)
            if (!want && unc[t]) {
                q = __ffs(unc[t]) - 1;
                unc[t] &= unc[t] - 1u;
                want = true;
                jj = j[t];
                slot = t * 32 + lane;
            }
        if (!__any_sync(0xffffffffu, want)) break;
        const int fl = want ? cmir[slot] : 0;
        const bool mir = fl == 1 || (fl == 2 && jj != I.q0 + q);
        const bool queued = band_push(P, lane, want, I.q0 + q, jj, mir);  // rare: no reservation
        int no = 0;
        int32_t qid = 0, cid = 0;
        if (want && !queued) {  // queue full: decide here
            const double s = direct_sq(P.xs + (int64_t)(I.q0 + q) * P.dp, P.xs + (int64_t)jj * P.dp, P.d);
            ++rechecked;
            if (s <= R.e2) {
                no = mir ? 2 : 1;
                qid = (int32_t)(qids[q] - R.off);
                cid = (int32_t)(cperm[slot] - R.off);
            }
        }
        stage_emit_pairs(st, P, lane, no, qid, cid);
    }
}

// Minimum resident CTAs per SM requested from the register allocator, and
// candidates per lane, of the FP32 small-d tile (d <= 8): it is
// latency-bound, so it runs with 2 candidates per lane and 9 CTAs of 4
// warps per SM (at most 56 registers).  Measured on the uniform 4-D
// workload (2M points), tile-kernel time: 2 candidates x 9 CTAs 1.196 ms,
// 2 x 10 1.218, 2 x 8 1.235, 2 x 12 1.521, 2 x 16 1.781, 4 x 8 1.323,
// 4 x 7 1.372, 4 x 6 1.428.  Compile-time tuning constants.
#ifndef SJ_CC_F32_MIN_BLOCKS
#define SJ_CC_F32_MIN_BLOCKS 9
#endif
#ifndef SJ_CC_TC_SMALL_D
#define SJ_CC_TC_SMALL_D 2
#endif
template <typename T, int DP>
constexpr int cc_min_blocks() {
    return std::is_same<T, float>::value && DP <= 8 ? SJ_CC_F32_MIN_BLOCKS : 1;
}

template <typename T, int DP, int TC, bool EMIT, int NW, int RUNS>
__global__ void __launch_bounds__(NW * 32, cc_min_blocks<T, DP>()) k_join_cc(JoinParams P) {
    constexpr bool FUSED = DP <= 8;
    constexpr int KC = DP < 8 ? DP : 8;  // dims per register chunk (unfused path)
    constexpr int SLOTS = 32 * TC;
    static_assert(SLOTS <= 2048, "slot index must fit in 11 bits");
    __shared__ CcWarpSmem<T, DP, TC, EMIT, RUNS> smem[NW];

    const T* __restrict__ Y = static_cast<const T*>(P.y);
    const T* __restrict__ TO = static_cast<const T*>(P.thr_out);
    const T* __restrict__ TI = static_cast<const T*>(P.thr_in);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    CcWarpSmem<T, DP, TC, EMIT, RUNS>& W = smem[wid];
    ItemSmem<T, DP, RUNS>& S = W.it;
    WarpStage st{W.stage, EMIT ? W.sdist : nullptr, 0, 0};
    BandQ bq{0, 0};
    unsigned long long rechecked = 0;

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
        const ItemRoute R = item_route(st, P, it, lane);
        const uint32_t C = load_item_warp<T, DP>(S, P, I, lane);
        if constexpr (std::is_same<T, double>::value && DP >= 16) {
            if (P.sc_w) {  // each query's remainder bound
                if (lane < kQMax) W.scq[lane] = lane < Q ? P.sc_w[I.q0 + lane] : 0.0;
                __syncwarp();
            }
        }

        for (uint32_t base = 0; base < C; base += (uint32_t)SLOTS) {
            int32_t j[TC];
            bool valid[TC];
            uint32_t tri_mask[TC];
            T to[TC], ti[TC];
#pragma unroll
            for (int t = 0; t < TC; ++t) {
                const int slot = t * 32 + lane;
                const uint32_t v = base + (uint32_t)slot;
                valid[t] = v < C;
                j[t] = 0;
                tri_mask[t] = 0xFFFFFFFFu;
                to[t] = T(INFINITY);  // an empty slot is never maybe-in
                ti[t] = T(INFINITY);
                if (valid[t]) {
                    uint8_t fl;
                    j[t] = map_candidate_flag<T, DP>(S, nr, v, fl);
                    if (!SJ_BOUND(P, j[t] >= 0 && j[t] < P.n_points, 21)) j[t] = 0;
                    to[t] = TO[j[t]];
                    ti[t] = TI[j[t]];
                    if constexpr (EMIT) W.cj[slot] = j[t];
                    W.cperm[slot] = P.perm[j[t]];
                    W.cmir[slot] = fl;
                    // self-cell triangle: candidate j pairs with queries q0 .. j only
                    tri_mask[t] = (fl == 2 && j[t] < I.q1) ? (2u << (j[t] - I.q0)) - 1u : 0xFFFFFFFFu;
                }
            }
            uint32_t bits[TC], cbits[TC];
            if constexpr (FUSED) {
                T c[TC][DP];
#pragma unroll
                for (int t = 0; t < TC; ++t)
#pragma unroll
                    for (int k = 0; k < DP; ++k) c[t][k] = valid[t] ? Y[(int64_t)j[t] * DP + k] : T(0);
                tile_fused<T, DP, TC, RUNS>(S, Q, c, to, ti, bits, cbits);
            } else {
                T acc[TC][kQMax];
#pragma unroll
                for (int q = 0; q < kQMax; ++q)
#pragma unroll
                    for (int t = 0; t < TC; ++t) acc[t][q] = S.qh[q];
                bool all_out = false;  // short-circuit taken: every pair of the tile is out
#pragma unroll
                for (int kc = 0; kc < DP; kc += KC) {
                    T c[TC][KC];
#pragma unroll
                    for (int t = 0; t < TC; ++t)
#pragma unroll
                        for (int kk = 0; kk < KC; ++kk) c[t][kk] = valid[t] ? Y[(int64_t)j[t] * DP + kc + kk] : T(0);
#pragma unroll
                    for (int q = 0; q < kQMax; ++q) {
                        if (q >= Q) break;
#pragma unroll
                        for (int kk = 0; kk < KC; ++kk) {
                            const T qv = S.qy[q][kc + kk];
#pragma unroll
                            for (int t = 0; t < TC; ++t) acc[t][q] = fma_t(qv, c[t][kk], acc[t][q]);
                        }
                    }
                    if constexpr (std::is_same<T, double>::value && DP >= 16) {
                        // short-circuit (Sec. III-B) at the checkpoint, after the
                        // first sc_b dims: with w bounding half the remaining norm
                        // of each point (plus the rounding margins),
                        // acc + w_q + w_c below thr_out means the full filter value
                        // is below it too, i.e. the pair is certainly out; when that
                        // holds for every pair of the warp's tile the remaining
                        // dims are skipped
                        // (a one-pair-per-lane pre-test first: the full test runs
                        // only when that already holds for the whole warp)
                        if (P.sc_w && kc + KC == P.sc_b &&
                            __all_sync(0xffffffffu,
                                       !valid[0] || order_key(__dadd_ru(acc[0][0], W.scq[0])) <
                                                        order_key(__dsub_rd(to[0], P.sc_w[j[0]])))) {
                            bool out = true;
#pragma unroll
                            for (int t = 0; t < TC; ++t) {
                                if (!valid[t]) continue;
                                const long long kr = order_key(__dsub_rd(to[t], P.sc_w[j[t]]));
#pragma unroll
                                for (int q = 0; q < kQMax; ++q)
                                    if (q < Q) out = out && order_key(__dadd_ru(acc[t][q], W.scq[q])) < kr;
                            }
                            if (__all_sync(0xffffffffu, out)) {
                                all_out = true;
                                break;
                            }
                        }
                    }
                }
#pragma unroll
                for (int t = 0; t < TC; ++t) {
                    uint32_t b = 0, cb = 0;
#pragma unroll
                    for (int q = 0; q < kQMax; ++q) {
                        if (!all_out && q < Q && ge_threshold(acc[t][q], to[t])) b |= 1u << q;
                        if (!all_out && q < Q && ge_threshold(acc[t][q], ti[t])) cb |= 1u << q;
                    }
                    bits[t] = b;
                    cbits[t] = cb;
                }
            }
#pragma unroll
            for (int t = 0; t < TC; ++t) {
                bits[t] &= tri_mask[t];
                cbits[t] &= tri_mask[t];
            }
            if constexpr (!EMIT) {
                emit_direct<TC>(st, P, W.cperm, W.cmir, S.qid, R, I, lane, j, bits, cbits, rechecked);
            } else {
            // with distances every maybe-in pair is re-decided in binary64: the
            // pairs are compacted with one warp scan per half of the queries and
            // queued 32 at a time
#pragma unroll 1
            for (int half = 0; half < 2; ++half) {
            const uint32_t hm = half ? 0xFF00u : 0x00FFu;
            int cnt = 0;
#pragma unroll
            for (int t = 0; t < TC; ++t) cnt += __popc(bits[t] & hm);
            int total;
            int off = warp_excl_scan(cnt, lane, &total);
            if (total == 0) continue;
#pragma unroll
            for (int t = 0; t < TC; ++t) {
                uint32_t b = bits[t] & hm;
                while (b) {
                    const int q = __ffs(b) - 1;
                    b &= b - 1u;
                    W.list[off++] = (uint16_t)(((t * 32 + lane) << 4) | q);
                }
            }
            __syncwarp();
            for (int e0 = 0; e0 < total; e0 += 32) {
                const int e = e0 + lane;
                int nout = 0;
                int32_t qid = 0, cid = 0;
                double dist = 0.0;
                bool band = false, mir = false;
                int q = 0;
                int64_t jj = 0;
                if (e < total) {
                    const int ent = W.list[e];
                    const int slot = (ent >> 4) & 0x7FF;
                    q = ent & 15;
                    jj = W.cj[slot];
                    const int fl = W.cmir[slot];
                    mir = fl == 1 || (fl == 2 && jj != (int64_t)(I.q0 + q));
                    band = true;
                }
                const bool queued = band_push_q(bq, P, lane, band, I.q0 + q, (int32_t)jj, mir);
                if (band && !queued) {  // queue full: decide here
                    const double s = direct_sq(P.xs + (int64_t)(I.q0 + q) * DP, P.xs + jj * DP, P.d);
                    ++rechecked;
                    if (s <= R.e2) {
                        nout = mir ? 2 : 1;
                        qid = (int32_t)(S.qid[q] - R.off);
                        cid = (int32_t)(W.cperm[(W.list[e] >> 4) & 0x7FF] - R.off);
                        dist = sqrt(s);
                    }
                }
                stage_emit(st, P, lane, nout, qid, cid, dist);
            }
            __syncwarp();
            }
            }
        }
        __syncwarp();
    }
    band_q_close(bq, P, lane);
    stage_flush(st, P, lane);
    for (int o = 16; o > 0; o >>= 1) rechecked += __shfl_down_sync(0xffffffffu, rechecked, o);
    if (lane == 0 && rechecked) atomicAdd(&P.counters[2], rechecked);
}

template <typename T, int DP, bool EMIT, int RUNS>
inline int launch_dper(Index* ix, const JoinParams& p) {
    constexpr int TC = DP > 8 ? 2 : std::is_same<T, float>::value ? SJ_CC_TC_SMALL_D : 4;
    constexpr int NW = cc_warps<CcWarpSmem<T, DP, TC, EMIT, RUNS>>();
    auto kern = k_join_cc<T, DP, TC, EMIT, NW, RUNS>;
    int per_sm = 0;
    SJ_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NW * 32, 0));
    if (per_sm < 1) per_sm = 1;
    long long blocks = (long long)device_sm_count(ix->device) * per_sm;
    const long long need = (ix->n_items + NW - 1) / NW;
    if (blocks > need) blocks = need > 0 ? need : 1;
    kern<<<(unsigned)blocks, NW * 32, 0, ix->stream>>>(p);
    note_launch();
    SJ_CK(cudaGetLastError());
    return SJ_OK;
}

// Run capacity of the item image: 3^(m-1) + 1 runs for m indexed dims; a
// grid of at most 4 dims needs 28, which keeps the per-warp shared memory of
// the small-d kernels small enough for 8 CTAs per SM.  Large-d kernels are
// bound by registers, so they keep the general capacity only.
template <typename T, int DP, bool EMIT>
inline int launch_dpe(Index* ix, const JoinParams& p) {
    if constexpr (DP <= 8)
        return ix->m <= 4 ? launch_dper<T, DP, EMIT, 28>(ix, p) : launch_dper<T, DP, EMIT, kMaxRuns>(ix, p);
    else
        return launch_dper<T, DP, EMIT, kMaxRuns>(ix, p);
}

// The tile launch for padded dimension DP.  The FP32 filter at DP <= 8
// without distances runs k_join_f32s (sj_join_f32s.cu) instead.
template <typename T, int DP>
int launch_cc_dp(Index* ix, const JoinParams& p) {
    if constexpr (std::is_same<T, float>::value && DP <= 8) {
        if (!p.emit_dist) {
            set_error("the FP32 filter at padded dimension %d without distances runs k_join_f32s", DP);
            return SJ_ERR_UNSUPPORTED;
        }
        return launch_dpe<T, DP, true>(ix, p);
    } else {
        return p.emit_dist ? launch_dpe<T, DP, true>(ix, p) : launch_dpe<T, DP, false>(ix, p);
    }
}


}  // namespace sj
