// Certified low-precision filter on the 5th-generation tensor cores
// (tcgen05.mma kind::f16, bf16 operands, FP32 accumulation in TMEM).
//
// The dot products of Eq. 3 (the tensor-core part of Eq. 4) are formed from a
// 3-term bf16 split of every FP32 kernel coordinate, y = y1 + y2 + y3 exactly
// (8 significant bits each), keeping the six products whose term indices sum
// to at most 4: for dim k the candidate row holds (c1, c2, c1, c3, c2, c1)
// and the query row (q1, q1, q2, q1, q2, q3).  Three more K slots carry the
// query's -||y_q||^2 / 2, split the same way, against ones, so the
// accumulator ends as a = -||y_q||^2/2 + y_q . y_c, the quantity every other
// kernel computes.  Each value is compared with per-candidate thresholds
// widened for this arithmetic (dropped split products and the tensor core's
// FP32 accumulation, see pack_coefficients' caller); pairs inside the bound
// are re-decided in binary64 by k_recheck.
//
// Tile: M = 128 candidates (TMEM lanes) x N = 64 queries (TMEM columns) x K;
// operands K-major in shared memory without swizzle (core matrices of 8 rows
// x 16 bytes; leading-dimension offset 128 bytes between K chunks, stride
// offset 16 K bytes between 8-row groups).  One elected thread issues the
// K / 16 MMAs and commits them to an mbarrier; each warp then reads its 32
// TMEM lanes (tcgen05.ld 32x32b) and runs the same compaction / emission as
// the CUDA-core kernels.  Every wait is bounded; on expiry the kernel records
// an error the host reports as SJ_ERR_TIMEOUT.
#include <cuda_bf16.h>

#include "sj_join_common.cuh"

namespace sj {

constexpr int kTcM = 128;
constexpr long long kTcSpin = 4000000;  // bound on mbarrier polls per wait

struct TcParams {
    const __nv_bfloat16* rows_a;  // n x kp, candidate role
    const __nv_bfloat16* rows_b;  // n x kp, query role
    int* error;                   // set to 1 when a bounded wait expires
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: K-major, no swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version bits 46-48 = 0b001
    return d;
}

// Instruction descriptor of kind::f16: D f32, A and B bf16, both K-major.
__host__ __device__ constexpr uint32_t umma_idesc(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

template <int KP>
struct TcSmem {
    uint64_t mbar;
    uint32_t tmem;
    int32_t pad0;
    long long item;
    int32_t rstart[kMaxRuns];
    uint32_t rpre[kMaxRuns + 1];
    uint8_t rmir[kMaxRuns];
    int32_t qid[kTcN];
    int32_t cj[kTcM];
    int32_t cperm[kTcM];
    uint8_t cmir[kTcM];
    uint16_t list[4][32 * kTcN];  // per warp: certain << 15 | lane << 7 | query
    int2 stage[4][kStage];
    double sdist[4][kStage];
};

template <int KP>
constexpr size_t tc_smem_bytes() {
    return 1024 /* alignment slack */ + (size_t)kTcM * KP * 2 + (size_t)kTcN * KP * 2 + sizeof(TcSmem<KP>);
}

// Copies `rows` rows of KP bf16 into the interleaved core-matrix layout at
// dst; row r comes from src + idx(r) * KP, or is zero when idx(r) < 0.
template <int KP, typename F>
__device__ __forceinline__ void stage_rows(unsigned char* dst, const __nv_bfloat16* __restrict__ src, int rows,
                                           F&& idx) {
    constexpr int CH = KP / 8;  // 16-byte chunks per row
    for (int c = threadIdx.x; c < rows * CH; c += blockDim.x) {
        const int r = c / CH, j = c - r * CH;
        unsigned char* d = dst + ((r >> 3) * CH + j) * 128 + (r & 7) * 16;
        const int64_t s = idx(r);
        if (s >= 0) {
            const __nv_bfloat16* g = src + s * KP + j * 8;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(d)), "l"(g));
        } else {
            *reinterpret_cast<uint4*>(d) = make_uint4(0, 0, 0, 0);
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
}

__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t phase) {
    uint32_t done = 0;
    for (long long it = 0; it < kTcSpin; ++it) {
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(smem_u32(mbar)), "r"(phase));
        if (done) return true;
    }
    return false;
}

template <int KP, bool EMIT>
__global__ void __launch_bounds__(128, 1) k_join_tc(JoinParams P, TcParams T) {
    extern __shared__ unsigned char dsm_raw[];
    unsigned char* dsm = reinterpret_cast<unsigned char*>(((uintptr_t)dsm_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* sA = dsm;
    unsigned char* sB = dsm + (size_t)kTcM * KP * 2;
    TcSmem<KP>& S = *reinterpret_cast<TcSmem<KP>*>(sB + (size_t)kTcN * KP * 2);
    const float* __restrict__ TO = static_cast<const float*>(P.thr_out);
    const float* __restrict__ TI = static_cast<const float*>(P.thr_in);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    WarpStage st{S.stage[warp], EMIT ? S.sdist[warp] : nullptr, 0, 0};
    unsigned long long rechecked = 0;

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem)),
                     "r"((uint32_t)kTcN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = S.tmem;
    constexpr uint32_t idesc = umma_idesc(kTcM, kTcN);
    uint32_t phase = 0;
    bool failed = false;

    for (;;) {
        if (tid == 0) S.item = (long long)atomicAdd(&P.counters[0], 1ull);
        __syncthreads();
        const long long it = S.item;
        if (it >= P.n_items) break;
        const Item I = P.items[it];
        const int Q = I.q1 - I.q0;
        const int nr = I.r1 - I.r0;
        // runs and query ids
        for (int r = tid; r < nr; r += blockDim.x) {
            const Run R = P.runs[I.r0 + r];
            S.rstart[r] = R.start;
            S.rpre[r + 1] = (uint32_t)((int32_t)(R.end_flags & ~kMirrorBit) - R.start);
            S.rmir[r] = (uint8_t)(R.end_flags >> 31);
        }
        if (tid < kTcN) S.qid[tid] = tid < Q ? P.perm[I.q0 + tid] : 0;
        __syncthreads();
        if (warp == 0) {
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
        // the queries' operand rows (rows past Q are zero)
        stage_rows<KP>(sB, T.rows_b, kTcN, [&](int r) -> int64_t { return r < Q ? (int64_t)(I.q0 + r) : -1; });
        __syncthreads();
        const uint32_t C = S.rpre[nr];

        for (uint32_t base = 0; base < C; base += kTcM) {
            // this thread's candidate row
            const uint32_t v = base + (uint32_t)tid;
            float to = INFINITY, ti = INFINITY;
            int32_t j = -1;
            if (v < C) {
                bool mir;
                j = map_candidate_tc(S.rstart, S.rpre, S.rmir, nr, v, mir);
                to = TO[j];
                ti = TI[j];
                S.cmir[tid] = mir ? 1 : 0;
                S.cperm[tid] = P.perm[j];
            }
            S.cj[tid] = j;
            __syncthreads();
            stage_rows<KP>(sA, T.rows_a, kTcM, [&](int r) -> int64_t { return (int64_t)S.cj[r]; });
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll 1
                for (int s = 0; s < KP / 16; ++s) {
                    const uint64_t ad = umma_desc(smem_u32(sA) + s * 256, 128, (KP / 8) * 128);
                    const uint64_t bd = umma_desc(smem_u32(sB) + s * 256, 128, (KP / 8) * 128);
                    asm volatile(
                        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                        "l"(ad), "l"(bd), "r"(idesc), "r"((uint32_t)(s > 0)));
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(&S.mbar)));
            }
            const bool ok = mbar_wait(&S.mbar, phase);
            phase ^= 1u;
            if (__syncthreads_or(!ok)) {  // every thread leaves together
                failed = true;
                if (tid == 0) atomicExch(T.error, 1);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            // epilogue: this warp's 32 lanes (candidates) x kTcN queries
            uint32_t bits[kTcN / 32] = {}, cbits[kTcN / 32] = {};
#pragma unroll
            for (int c0 = 0; c0 < kTcN; c0 += 16) {
                uint32_t r[16];
                const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                    "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                      "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                      "=r"(r[14]), "=r"(r[15])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int q = c0 + k;
                    const float a = __uint_as_float(r[k]);
                    if (q < Q && a >= to) bits[q >> 5] |= 1u << (q & 31);
                    if (q < Q && a >= ti) cbits[q >> 5] |= 1u << (q & 31);
                }
            }
            // compact the maybe-in pairs of this warp
            int cnt = 0;
#pragma unroll
            for (int h = 0; h < kTcN / 32; ++h) cnt += __popc(bits[h]);
            int total;
            int off = warp_excl_scan(cnt, lane, &total);
#pragma unroll
            for (int h = 0; h < kTcN / 32; ++h) {
                uint32_t b = bits[h];
                while (b) {
                    const int q = h * 32 + __ffs(b) - 1;
                    b &= b - 1u;
                    const int certain = (cbits[h] >> (q & 31)) & 1u;
                    S.list[warp][off++] = (uint16_t)((certain << 15) | (lane << 7) | q);
                }
            }
            __syncwarp();
            for (int e0 = 0; e0 < total; e0 += 32) {
                const int e = e0 + lane;
                int nout = 0;
                int32_t qid = 0, cid = 0, qs = 0, cs = 0;
                double dist = 0.0;
                bool band = false, mir = false;
                if (e < total) {
                    const int ent = S.list[warp][e];
                    const int row = warp * 32 + ((ent >> 7) & 31);
                    const int q = ent & 127;
                    mir = S.cmir[row] != 0;
                    qs = I.q0 + q;
                    cs = S.cj[row];
                    if ((ent >> 15) && !EMIT) {
                        nout = mir ? 2 : 1;
                        qid = S.qid[q];
                        cid = S.cperm[row];
                    } else {
                        band = true;
                    }
                }
                const bool queued = band_push(P, lane, band, qs, cs, mir);
                if (band && !queued) {  // queue full: decide here
                    const double s = direct_sq(P.xs + (int64_t)qs * P.dp, P.xs + (int64_t)cs * P.dp, P.d);
                    ++rechecked;
                    if (s <= P.e2) {
                        nout = mir ? 2 : 1;
                        qid = P.perm[qs];
                        cid = P.perm[cs];
                        if (EMIT) dist = sqrt(s);
                    }
                }
                if (EMIT)
                    stage_emit(st, P, lane, nout, qid, cid, dist);
                else
                    stage_emit_pairs(st, P, lane, nout, qid, cid);
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
        }
        if (failed) break;
    }
    stage_flush(st, P, lane);
    for (int o = 16; o > 0; o >>= 1) rechecked += __shfl_down_sync(0xffffffffu, rechecked, o);
    if (lane == 0 && rechecked) atomicAdd(&P.counters[2], rechecked);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)kTcN));
    }
}

template <int KP, bool EMIT>
static int launch_kp(Index* ix, const JoinParams& p, const TcParams& t) {
    auto kern = k_join_tc<KP, EMIT>;
    const size_t smem = tc_smem_bytes<KP>();
    SJ_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    SJ_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, smem));
    if (per_sm < 1) {
        set_error("tensor-core tile does not fit on an SM (K = %d)", KP);
        return SJ_ERR_UNSUPPORTED;
    }
    // TMEM: kTcN columns per CTA out of 512 per SM
    per_sm = std::min(per_sm, 512 / kTcN);
    long long blocks = (long long)device_sm_count(ix->device) * per_sm;
    if (blocks > ix->n_items) blocks = ix->n_items > 0 ? ix->n_items : 1;
    kern<<<(unsigned)blocks, 128, smem, ix->stream>>>(p, t);
    note_launch();
    SJ_CK(cudaGetLastError());
    return SJ_OK;
}

template <int KP>
static int launch_k(Index* ix, const JoinParams& p, const TcParams& t) {
    return p.emit_dist ? launch_kp<KP, true>(ix, p, t) : launch_kp<KP, false>(ix, p, t);
}

int launch_join_tc(Index* ix, const JoinOut& out, int emit_dist) {
    const JoinParams p = make_join_params(ix, out, emit_dist);
    TcParams t;
    t.rows_a = static_cast<const __nv_bfloat16*>(ix->rows_a);
    t.rows_b = static_cast<const __nv_bfloat16*>(ix->rows_b);
    t.error = reinterpret_cast<int*>(ix->counters + 4);
    switch (ix->kp) {
        case 16: return launch_k<16>(ix, p, t);
        case 32: return launch_k<32>(ix, p, t);
        case 64: return launch_k<64>(ix, p, t);
        case 112: return launch_k<112>(ix, p, t);
        case 208: return launch_k<208>(ix, p, t);
        case 400: return launch_k<400>(ix, p, t);
        default:
            set_error("no tensor-core kernel for K = %d", ix->kp);
            return SJ_ERR_UNSUPPORTED;
    }
}

}  // namespace sj
