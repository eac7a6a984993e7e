// The recheck kernel, the join parameters and the dispatch of the CUDA-core
// distance tiles (the tile kernels themselves: sj_join_cc.cuh, instantiated
// per padded dimension in sj_cc_d*.cu; the small-d FP32 filter:
// sj_join_f32s.cu).
#include "sj_join_common.cuh"

namespace sj {

// Re-decides the queued pairs with the decision rule (binary64 direct form),
// 32 pairs per warp instruction, and emits the members (both orders for
// mirrored entries) with their distances when requested.
template <int DP, bool EMIT>
__global__ void __launch_bounds__(128) k_recheck(JoinParams P) {
    __shared__ int2 s_stage[4][kStage];
    __shared__ double s_sdist[4][EMIT ? kStage : 1];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    WarpStage st{s_stage[wid], EMIT ? s_sdist[wid] : nullptr, 0, 0};
    const unsigned long long queued = P.counters[3];
    const unsigned long long count = queued < P.band_cap ? queued : P.band_cap;
    const unsigned long long gw = (unsigned long long)blockIdx.x * 4 + wid;
    const unsigned long long nw = (unsigned long long)gridDim.x * 4;
    unsigned long long nvalid = 0;
    for (unsigned long long b = gw * 32; b < count; b += nw * 32) {
        const unsigned long long i = b + lane;
        int nout = 0;
        int32_t qid = 0, cid = 0;
        double dist = 0.0;
        const int2 e = i < count ? P.band[i] : make_int2(-1, -1);
        const int32_t qs = e.x;
        const int32_t cs = (int32_t)((uint32_t)e.y & ~kMirrorBit);
        // closed (unfilled) reservation slots hold (-1, -1)
        if (qs >= 0 && qs < P.n_points && cs >= 0 && cs < P.n_points) {
            ++nvalid;
            const bool mir = ((uint32_t)e.y & kMirrorBit) != 0;
            const double s = direct_sq(P.xs + (int64_t)qs * DP, P.xs + (int64_t)cs * DP, P.d);
            if (P.batch) {  // lanes may serve different instances: one lane, one write
                const int li = P.batch->inst_of_sorted[qs];
                if (s <= P.batch->inst_e2[li]) {
                    const long long off = P.batch->inst_off[li];
                    batch_emit_one(P, P.batch->inst_gid[li], mir ? 2 : 1, (int32_t)(P.perm[qs] - off),
                                   (int32_t)(P.perm[cs] - off), EMIT ? sqrt(s) : 0.0);
                }
            } else if (s <= P.e2) {
                nout = mir ? 2 : 1;
                qid = P.perm[qs];
                cid = P.perm[cs];
                if (EMIT) dist = sqrt(s);
            }
        }
        if (P.batch) continue;
        if (EMIT)
            stage_emit(st, P, lane, nout, qid, cid, dist);
        else
            stage_emit_pairs(st, P, lane, nout, qid, cid);
    }
    stage_flush(st, P, lane);
    for (int o = 16; o > 0; o >>= 1) nvalid += __shfl_down_sync(0xffffffffu, nvalid, o);
    if (lane == 0 && nvalid) atomicAdd(&P.counters[2], nvalid);
}

template <typename T>
static int launch_t(Index* ix, const JoinParams& p) {
    switch (ix->dp) {
        case 2: return launch_cc_dp<T, 2>(ix, p);
        case 4: return launch_cc_dp<T, 4>(ix, p);
        case 8: return launch_cc_dp<T, 8>(ix, p);
        case 16: return launch_cc_dp<T, 16>(ix, p);
        case 32: return launch_cc_dp<T, 32>(ix, p);
        case 64: return launch_cc_dp<T, 64>(ix, p);
        case 128: return launch_cc_dp<T, 128>(ix, p);
        default:
            set_error("no CUDA-core kernel for padded dimension %d", ix->dp);
            return SJ_ERR_UNSUPPORTED;
    }
}

template <int DP>
static int launch_recheck_dp(Index* ix, const JoinParams& p) {
    const unsigned blocks = (unsigned)device_sm_count(ix->device) * 4;
    if (p.emit_dist)
        k_recheck<DP, true><<<blocks, 128, 0, ix->stream>>>(p);
    else
        k_recheck<DP, false><<<blocks, 128, 0, ix->stream>>>(p);
    note_launch();
    SJ_CK(cudaGetLastError());
    return SJ_OK;
}

int launch_recheck(Index* ix, const JoinOut& out, int emit_dist) {
    const JoinParams p = make_join_params(ix, out, emit_dist);
    switch (ix->dp) {
        case 2: return launch_recheck_dp<2>(ix, p);
        case 4: return launch_recheck_dp<4>(ix, p);
        case 8: return launch_recheck_dp<8>(ix, p);
        case 16: return launch_recheck_dp<16>(ix, p);
        case 32: return launch_recheck_dp<32>(ix, p);
        case 64: return launch_recheck_dp<64>(ix, p);
        case 128: return launch_recheck_dp<128>(ix, p);
        default:
            set_error("no recheck kernel for padded dimension %d", ix->dp);
            return SJ_ERR_UNSUPPORTED;
    }
}

JoinParams make_join_params(Index* ix, const JoinOut& out, int emit_dist) {
    JoinParams p{};
    p.y = ix->y;
    p.h = ix->h;
    p.thr_out = ix->thr_out;
    p.thr_in = ix->thr_in;
    p.xs = ix->xs;
    p.perm = ix->perm;
    p.items = ix->items;
    p.runs = ix->runs;
    p.n_items = ix->n_items;
    p.n_points = ix->n;
    p.counters = ix->counters;
    p.out_pairs = out.out_pairs;
    p.out_dist = out.out_dist;
    p.capacity = out.capacity;
    p.e2 = ix->e2;
    p.d = ix->d;
    p.dp = ix->dp;
    p.emit_dist = emit_dist;
    p.tri = uses_triangle(ix) ? 1 : 0;
    p.band = out.band;
    p.band_cap = out.band_cap;
    p.batch = static_cast<const BatchJoin*>(out.batch);
    p.aux = static_cast<const float4*>(ix->aux);
    p.sc_w = ix->sc_w;
    p.sc_b = ix->sc_b;
    p.dbg = out.dbg;
    p.dbg_cap = out.dbg_cap;
    p.prune_r2 = ix->prune_r2;
    return p;
}

int launch_join_cc(Index* ix, const JoinOut& out, int emit_dist) {
    if (f32s_supported(ix, emit_dist)) return launch_join_f32s(ix, out);
    const JoinParams p = make_join_params(ix, out, emit_dist);
    if (ix->kernel == SJ_KERNEL_FILTER_F32) return launch_t<float>(ix, p);
    return launch_t<double>(ix, p);
}

}  // namespace sj
