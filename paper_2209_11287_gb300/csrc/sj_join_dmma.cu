// Distance tiles on the FP64 tensor cores: mma.sync.m8n8k4 f64 (the FP64 MMA
// shape the paper builds its algorithm on, Sec. II-B and Fig. 2).
//
// Fig. 2 computes T = A x B + C on the tensor cores with A the (scaled)
// query coordinates, B the candidate coordinates and C the candidates'
// squared norms, then adds the queries' norms on the CUDA cores.  Here the
// accumulator is initialised with the query term instead, so one MMA chain
// over ceil(d/4) k-steps gives, for 8 queries x 8 candidates,
//     a = -||y_q||^2 / 2 + y_q . y_c
// the same quantity as the CUDA-core kernel, compared with the same
// per-candidate certified thresholds (||y_q - y_c||^2 = ||y_c||^2 - 2 a).
//
// Fragment layout of m8n8k4 .f64 (PTX ISA): with g = lane / 4, t = lane % 4,
// A holds element (row g, k t), B element (k t, col g), C/D elements
// (row g, col 2t) and (row g, col 2t + 1).
#include "sj_join_common.cuh"

namespace sj {

__device__ __forceinline__ void dmma_8x8x4(double& d0, double& d1, double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                 : "+d"(d0), "+d"(d1)
                 : "d"(a), "d"(b));
}

template <int DP, bool EMIT>
__global__ void __launch_bounds__(kThreads) k_join_dmma(JoinParams P) {
    static_assert(DP % 4 == 0, "DMMA needs the padded dimension to be a multiple of 4");
    constexpr int KS = DP / 4;  // k-steps
    __shared__ ItemSmem<double, DP> S;
    __shared__ int2 s_stage[kThreads / 32][kStage];
    __shared__ double s_sdist[kThreads / 32][kStage];
    __shared__ long long s_item;

    const double* __restrict__ Y = static_cast<const double*>(P.y);
    const double* __restrict__ TO = static_cast<const double*>(P.thr_out);
    const double* __restrict__ TI = static_cast<const double*>(P.thr_in);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int g = lane >> 2, tq = lane & 3;
    WarpStage st{s_stage[wid], s_sdist[wid], 0, 0};
    unsigned long long rechecked = 0;

    for (;;) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(&P.counters[0], 1ull);
        __syncthreads();
        const long long it = s_item;
        if (it >= P.n_items) break;
        const Item I = P.items[it];
        const int Q = I.q1 - I.q0;
        const int nr = I.r1 - I.r0;
        const uint32_t C = load_item<double, DP>(S, P, I);
        const int RG = (Q + 7) >> 3;  // row groups of 8 queries (1 or 2)

        // A fragments of the item's queries (rows past Q are zero)
        double afr[2][KS];
#pragma unroll
        for (int rg = 0; rg < 2; ++rg)
#pragma unroll
            for (int ks = 0; ks < KS; ++ks) afr[rg][ks] = S.qy[rg * 8 + g][ks * 4 + tq];

        for (uint32_t cg = (uint32_t)wid * 8u; cg < C; cg += (uint32_t)(kThreads / 32) * 8u) {
            // B fragment: candidate cg + g, dims ks*4 + tq
            bool mb;
            const uint32_t vb = cg + (uint32_t)g;
            const int32_t jb = vb < C ? map_candidate<double, DP>(S, nr, vb, mb) : -1;
            double bfr[KS];
#pragma unroll
            for (int ks = 0; ks < KS; ++ks) bfr[ks] = jb >= 0 ? Y[(int64_t)jb * DP + ks * 4 + tq] : 0.0;
            // the two accumulator columns of this lane: candidates cg + 2 tq + i
            int32_t jc[2];
            bool mc[2];
            double to[2], ti[2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const uint32_t v = cg + (uint32_t)(2 * tq + i);
                jc[i] = v < C ? map_candidate<double, DP>(S, nr, v, mc[i]) : -1;
                to[i] = jc[i] >= 0 ? TO[jc[i]] : INFINITY;
                ti[i] = jc[i] >= 0 ? TI[jc[i]] : INFINITY;
            }
#pragma unroll
            for (int rg = 0; rg < 2; ++rg) {
                if (rg >= RG) break;
                const int q = rg * 8 + g;
                double d0 = S.qh[q], d1 = S.qh[q];
#pragma unroll
                for (int ks = 0; ks < KS; ++ks) dmma_8x8x4(d0, d1, afr[rg][ks], bfr[ks]);
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const double a = i ? d1 : d0;
                    int nout = 0;
                    double dist = 0.0;
                    int32_t qid = 0, cid = 0;
                    bool band = false;
                    if (q < Q && jc[i] >= 0 && ge_threshold(a, to[i])) {
                        if (ge_threshold(a, ti[i]) && !EMIT) {
                            nout = mc[i] ? 2 : 1;
                            qid = S.qid[q];
                            cid = P.perm[jc[i]];
                        } else {
                            band = true;  // re-decided (and measured) in binary64
                        }
                    }
                    const bool queued = band_push(P, lane, band, I.q0 + q, jc[i], band && mc[i]);
                    if (band && !queued) {  // queue full: decide here
                        const double s =
                            direct_sq(P.xs + (int64_t)(I.q0 + q) * DP, P.xs + (int64_t)jc[i] * DP, P.d);
                        ++rechecked;
                        if (s <= P.e2) {
                            nout = mc[i] ? 2 : 1;
                            qid = S.qid[q];
                            cid = P.perm[jc[i]];
                            if (EMIT) dist = sqrt(s);
                        }
                    }
                    if (EMIT)
                        stage_emit(st, P, lane, nout, qid, cid, dist);
                    else
                        stage_emit_pairs(st, P, lane, nout, qid, cid);
                }
            }
        }
        __syncthreads();
    }
    stage_flush(st, P, lane);
    for (int o = 16; o > 0; o >>= 1) rechecked += __shfl_down_sync(0xffffffffu, rechecked, o);
    if (lane == 0 && rechecked) atomicAdd(&P.counters[2], rechecked);
}

template <int DP, bool EMIT>
static int launch_dpe(Index* ix, const JoinParams& p) {
    auto kern = k_join_dmma<DP, EMIT>;
    int per_sm = 0;
    SJ_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, 0));
    if (per_sm < 1) per_sm = 1;
    long long blocks = (long long)device_sm_count(ix->device) * per_sm;
    if (blocks > ix->n_items) blocks = ix->n_items > 0 ? ix->n_items : 1;
    kern<<<(unsigned)blocks, kThreads, 0, ix->stream>>>(p);
    note_launch();
    SJ_CK(cudaGetLastError());
    return SJ_OK;
}

template <int DP>
static int launch_dp(Index* ix, const JoinParams& p) {
    return p.emit_dist ? launch_dpe<DP, true>(ix, p) : launch_dpe<DP, false>(ix, p);
}

int launch_join_dmma(Index* ix, const JoinOut& out, int emit_dist) {
    const JoinParams p = make_join_params(ix, out, emit_dist);
    switch (ix->dp) {
        case 4: return launch_dp<4>(ix, p);
        case 8: return launch_dp<8>(ix, p);
        case 16: return launch_dp<16>(ix, p);
        case 32: return launch_dp<32>(ix, p);
        case 64: return launch_dp<64>(ix, p);
        case 128: return launch_dp<128>(ix, p);
        default:
            set_error("no DMMA kernel for padded dimension %d", ix->dp);
            return SJ_ERR_UNSUPPORTED;
    }
}

}  // namespace sj
