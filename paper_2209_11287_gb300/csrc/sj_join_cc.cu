// Distance tiles on CUDA cores, fused with the eps threshold and the
// compaction into result pages.
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
// contraction), so the returned set equals the rule's.
//
// T = double is the plain FP64 join (Eq. 3/4 evaluated on FP64 CUDA cores);
// T = float is the certified FP32 filter.
#include "sj_join_common.cuh"

namespace sj {

template <typename T, int DP, int TC>
__global__ void __launch_bounds__(kThreads) k_join_cc(JoinParams P) {
    constexpr int KC = DP < 8 ? DP : 8;  // dims per register chunk
    __shared__ ItemSmem<T, DP> S;
    __shared__ int2 s_stage[kThreads / 32][kStage];
    __shared__ double s_sdist[kThreads / 32][kStage];
    __shared__ long long s_item;

    const T* __restrict__ Y = static_cast<const T*>(P.y);
    const T* __restrict__ TO = static_cast<const T*>(P.thr_out);
    const T* __restrict__ TI = static_cast<const T*>(P.thr_in);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    WarpStage st{s_stage[wid], s_sdist[wid], 0};
    unsigned long long rechecked = 0;

    for (;;) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(&P.counters[0], 1ull);
        __syncthreads();
        const long long it = s_item;
        if (it >= P.n_items) break;
        const Item I = P.items[it];
        const int Q = I.q1 - I.q0;
        const int nr = I.r1 - I.r0;
        const uint32_t C = load_item<T, DP>(S, P, I);

        for (uint32_t base = 0; base < C; base += (uint32_t)(kThreads * TC)) {
            int32_t j[TC];
            bool mir[TC], valid[TC];
            T to[TC];
#pragma unroll
            for (int t = 0; t < TC; ++t) {
                const uint32_t v = base + (uint32_t)(t * kThreads) + threadIdx.x;
                valid[t] = v < C;
                j[t] = 0;
                mir[t] = false;
                to[t] = T(0);
                if (valid[t]) {
                    j[t] = map_candidate<T, DP>(S, nr, v, mir[t]);
                    to[t] = TO[j[t]];
                }
            }
            T acc[TC][kQMax];
#pragma unroll
            for (int q = 0; q < kQMax; ++q)
#pragma unroll
                for (int t = 0; t < TC; ++t) acc[t][q] = S.qh[q];
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
                        for (int t = 0; t < TC; ++t) acc[t][q] = fma(qv, c[t][kk], acc[t][q]);
                    }
                }
            }
#pragma unroll
            for (int t = 0; t < TC; ++t) {
                uint32_t bits = 0;
#pragma unroll
                for (int q = 0; q < kQMax; ++q)
                    if (q < Q && acc[t][q] >= to[t]) bits |= 1u << q;
                if (!valid[t]) bits = 0;
                // emission: one maybe-in pair per lane per round
                while (__any_sync(0xffffffffu, bits != 0)) {
                    int nout = 0;
                    double dist = 0.0;
                    int32_t qid = 0, cid = 0;
                    if (bits) {
                        const int q = __ffs(bits) - 1;
                        bits &= bits - 1u;
                        const int64_t jj = j[t];
                        // the same fma chain as above, so the same value
                        T a = S.qh[q];
#pragma unroll
                        for (int k = 0; k < DP; ++k) a = fma(S.qy[q][k], Y[jj * DP + k], a);
                        bool in = a >= TI[jj];
                        double s = 0.0;
                        if (!in || P.emit_dist) s = direct_sq(P.xs + (int64_t)(I.q0 + q) * DP, P.xs + jj * DP, P.d);
                        if (!in) {
                            in = s <= P.e2;
                            ++rechecked;
                        }
                        if (in) {
                            nout = mir[t] ? 2 : 1;
                            dist = P.emit_dist ? sqrt(s) : 0.0;
                            qid = S.qid[q];
                            cid = P.perm[jj];
                        }
                    }
                    stage_emit(st, P, lane, nout, qid, cid, dist);
                }
            }
        }
        __syncthreads();
    }
    stage_flush(st, P, lane);
    for (int o = 16; o > 0; o >>= 1) rechecked += __shfl_down_sync(0xffffffffu, rechecked, o);
    if (lane == 0 && rechecked) atomicAdd(&P.counters[2], rechecked);
}

template <typename T, int DP>
static int launch_dp(Index* ix, const JoinParams& p) {
    constexpr int TC = 2;
    auto kern = k_join_cc<T, DP, TC>;
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

template <typename T>
static int launch_t(Index* ix, const JoinParams& p) {
    switch (ix->dp) {
        case 2: return launch_dp<T, 2>(ix, p);
        case 4: return launch_dp<T, 4>(ix, p);
        case 8: return launch_dp<T, 8>(ix, p);
        case 16: return launch_dp<T, 16>(ix, p);
        case 32: return launch_dp<T, 32>(ix, p);
        case 64: return launch_dp<T, 64>(ix, p);
        case 128: return launch_dp<T, 128>(ix, p);
        default:
            set_error("no CUDA-core kernel for padded dimension %d", ix->dp);
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
    p.counters = ix->counters;
    p.pages = out.pages;
    p.dpages = out.dpages;
    p.page_log2 = out.page_log2;
    p.capacity = out.capacity;
    p.e2 = ix->e2;
    p.d = ix->d;
    p.emit_dist = emit_dist;
    return p;
}

int launch_join_cc(Index* ix, const JoinOut& out, int emit_dist) {
    const JoinParams p = make_join_params(ix, out, emit_dist);
    if (ix->kernel == SJ_KERNEL_FILTER_F32) return launch_t<float>(ix, p);
    return launch_t<double>(ix, p);
}

}  // namespace sj
