// Certified low-precision filter on the 5th-generation tensor cores
// (tcgen05.mma kind::f16, bf16 or fp16 operands, FP32 accumulation in TMEM).
//
// The dot products of Eq. 3 (the tensor-core part of Eq. 4) are formed from a
// bf16 split of every FP32 kernel coordinate, y = y1 + y2 + y3 exactly (8
// significant bits each).  BF16x3 keeps the six products whose term indices
// sum to at most 4: for dim k the candidate row holds (c1, c2, c1, c3, c2, c1)
// and the query row (q1, q1, q2, q1, q2, q3); BF16x2 keeps three, (c1, c2, c1)
// against (q1, q1, q2), for half the K; FP16x2 keeps the same three products
// of fp16 terms (11 significant bits) of the coordinates scaled by a power of
// two into fp16's range, for a narrower band.  Three more K slots carry the
// query's -||y_q||^2 / 2, split the same way, against ones, so the
// accumulator ends as a = -||y_q||^2/2 + y_q . y_c, the quantity every other
// kernel computes.  Each value is compared with per-candidate thresholds
// widened for this arithmetic (dropped split products and the tensor core's
// FP32 accumulation); pairs inside the bound are re-decided in binary64 by
// k_recheck.
//
// One persistent CTA per SM, warp-specialised:
//   warp 0      producer: takes work items from the queue, loads the item's
//               query tile (MMA B, N <= 256 queries, 8-row groups from an
//               8-aligned start) and streams the candidate tiles (MMA A,
//               128 rows = 16 groups covering the item's runs) in K-slices
//               of 64 with bulk copies completing on mbarriers;
//   warp 1      MMA issuer (one thread): K/16 MMAs per tile into one of two
//               TMEM accumulators (128 lanes x N columns), committed to the
//               stage and accumulator barriers;
//   warps 2..   epilogue (8 to 16 warps): each thread owns one candidate row
//               (its TMEM lane) and a share of its N accumulators (2 to 4
//               warps per lane quarter, interleaved 32-column chunks),
//               compares them with the
//               candidate's two thresholds (a max over 32 columns first; hits
//               are rare), then runs the warp-aggregated emission of the
//               CUDA-core kernels.
// A symmetric join evaluates only the triangle of each self cell: the self
// run starts at the item's first query and pairs below the diagonal are
// masked.  Every wait is bounded; on expiry the CTA stops issuing work,
// drains its copies and MMAs (again bounded), frees TMEM and records an error
// the host reports as SJ_ERR_TIMEOUT.
#include <cuda_bf16.h>

#include "sj_join_common.cuh"

namespace sj {

constexpr int kTcM = 128;             // candidate rows per tile (TMEM lanes)
constexpr int kTcG = kTcM / 8;        // 8-row groups per tile
constexpr int kKS = 64;               // K per pipeline slice
constexpr int kMetaDepth = 4;         // tiles of row metadata in flight
// Epilogue warps: EPI / 4 per TMEM lane quarter, splitting the columns; as
// many as shared memory allows next to the query tile (the epilogue's
// latency is what bounds the tile rate when hits are frequent).
constexpr int tc_epi(int kp, bool emit) { return kp <= 112 ? 16 : (emit ? 8 : 12); }
constexpr int tc_threads(int kp, bool emit) { return 64 + 32 * tc_epi(kp, emit); }  // producer, MMA, epilogue
constexpr long long kTcSpin = 1 << 22;  // bound on barrier polls per wait

struct TcParams {
    const __nv_bfloat16* rows_a;  // candidate role, slice-major 8-row groups (16-bit terms)
    const __nv_bfloat16* rows_b;  // query role, same layout
    long long nrows;              // rows per slice (packed points, padded)
    int* error;                   // set to 1 when a bounded wait expires
    uint32_t ab_bf16;             // 1: A and B are bf16, 0: both fp16
};

template <int KP>
struct TcShape {
    static constexpr int NMAX = tc_nmax(KP);
    static constexpr int SLICES = (KP + kKS - 1) / kKS;
    static constexpr int A_STAGE = kTcM * kKS * 2;  // bytes
    static constexpr int B_BYTES = NMAX * KP * 2;
};

// Per-item information shared by the roles (a ring of two).
struct TcItem {
    long long it;      // work item, or -1: no more work
    int q0, q1;        // queries [q0, q1)
    int qa;            // 8-aligned first row of the query tile
    int ncol;          // MMA N: query-tile rows, a multiple of 16
    int ntiles;        // candidate tiles
};

// Per-tile row metadata: each 8-row group's first row (-1: none), the run's
// valid position range and its flag (0 plain, 1 mirror, 2 self triangle).
struct TcMeta {
    int32_t g[kTcG];
    int32_t lo[kTcG];
    int32_t hi[kTcG];
    uint8_t fl[kTcG];
};

template <int KP, bool EMIT>
struct TcSmem {
    static constexpr int EPI = tc_epi(KP, EMIT);
    static_assert(EPI % 4 == 0, "epilogue warps come in whole warpgroups");
    static constexpr int MAX_STAGES = 6;
    uint64_t a_full[MAX_STAGES], a_empty[MAX_STAGES];
    uint64_t b_full, b_empty;
    uint64_t item_full[2], item_empty[2];
    uint64_t meta_full[kMetaDepth], meta_empty[kMetaDepth];
    uint64_t acc_full[2], acc_empty[2];
    uint64_t drain;
    uint32_t tmem;
    int abort;
    TcItem items[2];
    int32_t qperm[2][256];  // input index of each query-tile row of the items in the ring
    TcMeta meta[kMetaDepth];
    int32_t rgp[kMaxRuns];  // producer: per run of the item, its first group's number in the item
    int32_t rlo[kMaxRuns], rhi[kMaxRuns];
    uint8_t rfl[kMaxRuns];
    int2 stage[EPI][kStage];
    double sdist[EPI][EMIT ? kStage : 1];
    uint16_t hits[EPI][32][32];  // per epilogue warp: maybe-in entries of a 32-column chunk, per lane
};

// Operand stages: as many as fit (up to 6) in the 227 KB of shared memory a
// CTA may use next to the query tile and the rest.
constexpr size_t kSmemMax = 232448;
template <int KP, bool EMIT>
__host__ __device__ constexpr int tc_stages() {
    const long long left = (long long)kSmemMax - 1024 - TcShape<KP>::B_BYTES - (long long)sizeof(TcSmem<KP, EMIT>);
    const long long st = left / TcShape<KP>::A_STAGE;
    return st > TcSmem<KP, EMIT>::MAX_STAGES ? TcSmem<KP, EMIT>::MAX_STAGES : (int)st;
}
template <int KP, bool EMIT>
constexpr size_t tc_smem_bytes() {
    return 1024 /* alignment slack */ + (size_t)TcShape<KP>::B_BYTES +
           (size_t)tc_stages<KP, EMIT>() * TcShape<KP>::A_STAGE + sizeof(TcSmem<KP, EMIT>);
}

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

// Instruction descriptor of kind::f16: D f32, A and B of one type (bf16 when
// ab_bf16 = 1, else fp16), both K-major.
__host__ __device__ constexpr uint32_t umma_idesc(int m, int n, uint32_t ab_bf16) {
    return (1u << 4) | ((ab_bf16 & 1u) << 7) | ((ab_bf16 & 1u) << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void bar_init(uint64_t* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count));
}
__device__ __forceinline__ void bar_arrive(uint64_t* b) {
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ void bar_arrive_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}" ::"r"(smem_u32(b)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool bar_test(uint64_t* b, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return done != 0;
}
// Waits for the phase of the given parity; false when the CTA aborts or the
// bound (polls) expires, which raises the abort.
__device__ __forceinline__ bool bar_wait_n(uint64_t* b, uint32_t parity, volatile int* abort, long long polls) {
    for (long long i = 0; i < polls; ++i) {
        if (bar_test(b, parity)) return true;
        if (*abort) return false;
    }
    *abort = 1;
    return false;
}
__device__ __forceinline__ bool bar_wait(uint64_t* b, uint32_t parity, volatile int* abort) {
    return bar_wait_n(b, parity, abort, kTcSpin);
}
// Bulk copy global -> shared completing on an mbarrier.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 16 consecutive TMEM columns of this thread's lane (no wait).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* v) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}

// Three-input maximum (one instruction on this architecture).
__device__ __forceinline__ float max3f(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// 32 consecutive TMEM columns of this thread's lane (no wait).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* v) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
}

// DBG: the recording instantiation of the filter dump (a test aid; the join
// kernels proper carry none of its code).
template <int KP, bool EMIT, bool DBG>
__global__ void __launch_bounds__(tc_threads(KP, EMIT), 1) k_join_tc(JoinParams P, TcParams T) {
    using SH = TcShape<KP>;
    using SM = TcSmem<KP, EMIT>;
    constexpr int STAGES = tc_stages<KP, EMIT>();
    static_assert(STAGES >= 2, "at least two operand stages");
    constexpr int NMAX = SH::NMAX;
    extern __shared__ unsigned char dsm_raw[];
    unsigned char* dsm = reinterpret_cast<unsigned char*>(((uintptr_t)dsm_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* sB = dsm;
    unsigned char* sA = dsm + SH::B_BYTES;
    SM& S = *reinterpret_cast<SM*>(sA + (size_t)STAGES * SH::A_STAGE);
    volatile int* abort = &S.abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int i = 0; i < STAGES; ++i) {
            bar_init(&S.a_full[i], 1);
            bar_init(&S.a_empty[i], 1);
        }
        bar_init(&S.b_full, 1);
        bar_init(&S.b_empty, 1);
        for (int i = 0; i < 2; ++i) {
            bar_init(&S.item_full[i], 1);
            bar_init(&S.item_empty[i], 1 + SM::EPI);  // the MMA thread and the epilogue warps
            bar_init(&S.acc_full[i], 1);
            bar_init(&S.acc_empty[i], SM::EPI);
        }
        for (int i = 0; i < kMetaDepth; ++i) {
            bar_init(&S.meta_full[i], 1);
            bar_init(&S.meta_empty[i], SM::EPI);
        }
        bar_init(&S.drain, 1);
        S.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem)),
                     "r"((uint32_t)(2 * NMAX)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = S.tmem;

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        // The whole warp: lane i of a tile resolves the tile's 8-row group i
        // (a binary search over the item's per-run group prefix), runs of
        // consecutive groups become one bulk copy per K-slice, issued by the
        // run's first lane.
        uint32_t a_i = 0, a_ph = 0, m_i = 0, m_ph = 0, it_i = 0, it_ph = 0, b_ph = 0;
        uint32_t armed_a[STAGES];  // parity of each stage's last arming + 1 (0: never armed)
        for (int i = 0; i < STAGES; ++i) armed_a[i] = 0;
        uint32_t armed_b = 0;
        int bail = 0;
        while (!bail) {
            long long it = 0;
            if (lane == 0) it = (long long)atomicAdd(&P.counters[0], 1ull);
            it = __shfl_sync(0xffffffffu, it, 0);
            Item I{0, 0, 0, 0};
            if (it < P.n_items) I = P.items[it];
            const int nr = it < P.n_items ? I.r1 - I.r0 : 0;
            // per run: first group, valid range, flag and the exclusive group prefix
            int carry = 0;
            for (int r0 = 0; r0 < nr; r0 += 32) {
                const int r = r0 + lane;
                int cnt = 0;
                if (r < nr) {
                    const Run R = P.runs[I.r0 + r];
                    const bool mir = (R.end_flags & kMirrorBit) != 0;
                    const bool self = P.tri && !mir;
                    const int32_t lo = self ? I.q0 : R.start;
                    const int32_t hi = (int32_t)(R.end_flags & ~kMirrorBit);
                    cnt = hi > lo ? ((hi - 1) >> 3) - (lo >> 3) + 1 : 0;
                    S.rlo[r] = lo;
                    S.rhi[r] = hi;
                    S.rfl[r] = (uint8_t)(mir ? 1 : (self ? 2 : 0));
                }
                int x = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, x, o);
                    if (lane >= o) x += y;
                }
                if (r < nr) S.rgp[r] = carry + x - cnt;
                carry += __shfl_sync(0xffffffffu, x, 31);
            }
            const int ngroups = carry;
            __syncwarp();
            const int ntiles = (ngroups + kTcG - 1) / kTcG;
            const int qa = I.q0 & ~7;
            const int ncol = ((I.q1 - qa) + 15) & ~15;
            // the ring slot is free once its previous item is done; then its query ids
            int freed = 1;
            if (lane == 0) freed = bar_wait(&S.item_empty[it_i], it_ph ^ 1u, abort) ? 1 : 0;
            freed = __shfl_sync(0xffffffffu, freed, 0);
            if (freed && it < P.n_items)
                for (int c = lane; c < ncol; c += 32) {
                    const int q = qa + c;
                    S.qperm[it_i][c] = (q >= I.q0 && q < I.q1) ? P.perm[q] : 0;
                }
            __syncwarp();
            if (lane == 0) {
                if (!freed) {
                    bail = 1;
                } else if (it >= P.n_items) {
                    S.items[it_i].it = -1;
                    bar_arrive(&S.item_full[it_i]);
                    bail = 2;
                } else {
                    TcItem& X = S.items[it_i];
                    X.it = it;
                    X.q0 = I.q0;
                    X.q1 = I.q1;
                    X.qa = qa;
                    X.ncol = ncol;
                    X.ntiles = ntiles;
                    bar_arrive(&S.item_full[it_i]);
                    // the query tile, one copy per K-slice
                    if (!bar_wait(&S.b_empty, b_ph ^ 1u, abort)) {
                        bail = 1;
                    } else {
                        const uint32_t gq = (uint32_t)(ncol >> 3);
                        bar_arrive_tx(&S.b_full, gq * KP * 16u);
                        armed_b = b_ph + 1;
                        for (int sl = 0; sl < SH::SLICES; ++sl) {
                            const int ks = KP - sl * kKS < kKS ? KP - sl * kKS : kKS;
                            const __nv_bfloat16* src =
                                T.rows_b + (long long)sl * kKS * T.nrows + (long long)(qa >> 3) * ks * 8;
                            bulk_g2s(sB + (size_t)NMAX * 2 * kKS * sl, src, gq * (uint32_t)ks * 16u, &S.b_full);
                        }
                        b_ph ^= 1u;
                    }
                }
            }
            bail = __shfl_sync(0xffffffffu, bail, 0);
            if (freed && it < P.n_items && ++it_i == 2) it_i = 0, it_ph ^= 1u;  // (the whole warp)
            // candidate tiles
            for (int t = 0; t < ntiles && !bail; ++t) {
                int w = 1;
                if (lane == 0) w = bar_wait(&S.meta_empty[m_i], m_ph ^ 1u, abort) ? 1 : 0;
                if (!__shfl_sync(0xffffffffu, w, 0)) {
                    bail = 1;
                    break;
                }
                TcMeta& M = S.meta[m_i];
                // this lane's group of the tile
                const int j = t * kTcG + lane;
                int32_t g = -1;
                if (lane < kTcG) {
                    if (j < ngroups) {
                        int lo = 0, hi = nr - 1;  // last run whose prefix is <= j
                        while (lo < hi) {
                            const int mid = (lo + hi + 1) >> 1;
                            if (S.rgp[mid] <= j)
                                lo = mid;
                            else
                                hi = mid - 1;
                        }
                        g = (S.rlo[lo] >> 3) + (j - S.rgp[lo]);
                        M.lo[lane] = S.rlo[lo];
                        M.hi[lane] = S.rhi[lo];
                        M.fl[lane] = S.rfl[lo];
                    }
                    M.g[lane] = g;
                }
                const int cnt = ngroups - t * kTcG < kTcG ? ngroups - t * kTcG : kTcG;
                // runs of consecutive groups: their first lanes
                const int32_t gprev = __shfl_up_sync(0xffffffffu, g, 1);
                const bool first = lane < cnt && (lane == 0 || g != gprev + 1);
                const uint32_t firsts = __ballot_sync(0xffffffffu, first);
                const uint32_t later = firsts & ~((2u << lane) - 1u);
                const int seg_end = later ? __ffs(later) - 1 : cnt;
                __syncwarp();
                if (lane == 0) bar_arrive(&S.meta_full[m_i]);
                if (++m_i == kMetaDepth) m_i = 0, m_ph ^= 1u;
                for (int sl = 0; sl < SH::SLICES; ++sl) {
                    const int ks = KP - sl * kKS < kKS ? KP - sl * kKS : kKS;
                    if (lane == 0) {
                        w = bar_wait(&S.a_empty[a_i], a_ph ^ 1u, abort) ? 1 : 0;
                        if (w) bar_arrive_tx(&S.a_full[a_i], (uint32_t)cnt * ks * 16u);
                    }
                    if (!__shfl_sync(0xffffffffu, w, 0)) {
                        bail = 1;
                        break;
                    }
                    armed_a[a_i] = a_ph + 1;
                    if (first) {
                        unsigned char* dst = sA + (size_t)a_i * SH::A_STAGE + (size_t)lane * ks * 16;
                        const __nv_bfloat16* src = T.rows_a + (long long)sl * kKS * T.nrows + (long long)g * ks * 8;
                        bulk_g2s(dst, src, (uint32_t)(seg_end - lane) * ks * 16u, &S.a_full[a_i]);
                    }
                    if (++a_i == STAGES) a_i = 0, a_ph ^= 1u;
                }
            }
        }
        if (*abort && lane == 0) {
            // drain the copies this CTA armed (bounded), so none lands after exit
            for (int i = 0; i < STAGES; ++i)
                if (armed_a[i])
                    for (long long k = 0; k < kTcSpin && !bar_test(&S.a_full[i], armed_a[i] - 1); ++k) {
                    }
            if (armed_b)
                for (long long k = 0; k < kTcSpin && !bar_test(&S.b_full, armed_b - 1); ++k) {
                }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            uint32_t a_i = 0, a_ph = 0, it_i = 0, it_ph = 0, b_ph = 0, acc = 0, acc_ph = 0;
            bool issued = false;
            for (;;) {
                if (!bar_wait(&S.item_full[it_i], it_ph, abort)) break;
                const TcItem X = S.items[it_i];
                if (X.it < 0) break;
                if (!bar_wait(&S.b_full, b_ph, abort)) break;
                b_ph ^= 1u;
                const uint32_t idesc = umma_idesc(kTcM, X.ncol, T.ab_bf16);
                bool fail = false;
                for (int t = 0; t < X.ntiles && !fail; ++t) {
                    if (!bar_wait(&S.acc_empty[acc], acc_ph ^ 1u, abort)) {
                        fail = true;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const uint32_t dt = tmem + acc * NMAX;
                    for (int sl = 0; sl < SH::SLICES; ++sl) {
                        const int ks = KP - sl * kKS < kKS ? KP - sl * kKS : kKS;
                        if (!bar_wait(&S.a_full[a_i], a_ph, abort)) {
                            fail = true;
                            break;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;");
                        const uint32_t a0 = smem_u32(sA + (size_t)a_i * SH::A_STAGE);
                        const uint32_t b0 = smem_u32(sB + (size_t)NMAX * 2 * kKS * sl);
                        for (int kk = 0; kk < ks / 16; ++kk) {
                            const uint64_t ad = umma_desc(a0 + kk * 256, 128, (uint32_t)ks * 16u);
                            const uint64_t bd = umma_desc(b0 + kk * 256, 128, (uint32_t)ks * 16u);
                            const uint32_t accum = (sl > 0 || kk > 0) ? 1u : 0u;
                            asm volatile(
                                "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(dt),
                                "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
                        }
                        issued = true;
                        umma_commit(&S.a_empty[a_i]);  // the stage is free once these MMAs are done
                        if (++a_i == STAGES) a_i = 0, a_ph ^= 1u;
                    }
                    if (fail) break;
                    umma_commit(&S.acc_full[acc]);
                    if (++acc == 2) acc = 0, acc_ph ^= 1u;
                }
                if (fail) break;
                umma_commit(&S.b_empty);  // the query tile is free once this item's MMAs are done
                bar_arrive(&S.item_empty[it_i]);
                if (++it_i == 2) it_i = 0, it_ph ^= 1u;
            }
            if (issued) {
                // every MMA of this CTA has completed before TMEM is freed
                umma_commit(&S.drain);
                for (long long k = 0; k < kTcSpin && !bar_test(&S.drain, 0); ++k) {
                }
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int ew = warp - 2;       // stage slot
        const int quarter = warp & 3;  // TMEM lanes 32 quarter .. + 31
        const int part = ew >> 2;      // 32-column chunks part, part + EPI / 4, ...
        const int row = quarter * 32 + lane;
        const float* __restrict__ TO = static_cast<const float*>(P.thr_out);
        const float* __restrict__ TI = static_cast<const float*>(P.thr_in);
        WarpStage st{S.stage[ew], EMIT ? S.sdist[ew] : nullptr, 0, 0};
        BandQ bq{0, 0};
        unsigned long long rechecked = 0;
        uint32_t it_i = 0, it_ph = 0, m_i = 0, m_ph = 0, acc = 0, acc_ph = 0;
        for (;;) {
            if (!bar_wait(&S.item_full[it_i], it_ph, abort)) break;
            const TcItem X = S.items[it_i];
            if (X.it < 0) break;
            const ItemRoute R = item_route(st, P, X.it, lane);
            bool fail = false;
            // this thread's candidate row, read one tile ahead so its
            // threshold loads overlap the previous tile
            int32_t p = 0, pid = 0;
            bool valid = false;
            int fl = 0;
            float to = INFINITY, ti = INFINITY;
            const int32_t* qperm = S.qperm[it_i];
            auto read_meta = [&]() -> bool {
                if (!bar_wait(&S.meta_full[m_i], m_ph, abort)) return false;
                const TcMeta& M = S.meta[m_i];
                const int gi = row >> 3;
                const int32_t g = M.g[gi];
                p = g * 8 + (row & 7);
                if (g >= 0 && !SJ_BOUND(P, p < P.n_points + kTcPadRows, 31)) p = 0;
                valid = g >= 0 && p >= M.lo[gi] && p < M.hi[gi];
                fl = M.fl[gi];
                __syncwarp();
                if (lane == 0) bar_arrive(&S.meta_empty[m_i]);
                if (++m_i == kMetaDepth) m_i = 0, m_ph ^= 1u;
                // unconditional loads from an in-bounds row (selecting the
                // loaded values here would wait for them; every use below
                // is guarded by `valid`), so their latency overlaps the
                // current tile's chunks
                const int32_t pl = valid ? p : 0;
                to = TO[pl];
                ti = TI[pl];
                pid = P.perm[pl];
                return true;
            };
            if (X.ntiles > 0 && !read_meta()) fail = true;
            const int cq0 = X.q0 - X.qa, cq1 = X.q1 - X.qa;  // the item's query columns
            for (int t = 0; t < X.ntiles && !fail; ++t) {
                const int32_t cp = p, cpid = pid;
                const bool cvalid = valid;
                const int cfl = fl;
                const float cto = to, cti = ti;
                // this row's valid query columns: the item's, and in a self-cell
                // triangle those at or below the candidate (one unsigned compare)
                const int col_lo = cq0;
                const int col_hi = cfl == 2 ? min(cq1 - 1, cp - X.qa) : cq1 - 1;
                const bool has_cols = col_hi >= col_lo;
                const uint32_t col_span = has_cols ? (uint32_t)(col_hi - col_lo) : 0u;
                if (!bar_wait(&S.acc_full[acc], acc_ph, abort)) {
                    fail = true;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                if (t + 1 < X.ntiles && !read_meta()) {
                    fail = true;
                    break;
                }
                // this lane's maybe-in columns of a 32-column chunk (column | certain << 8),
                // emitted afterwards a warp-wide round at a time
                uint16_t(*hits)[32] = S.hits[ew];
                const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + acc * NMAX;
                for (int c0 = 32 * part; c0 < X.ncol; c0 += 32 * (SM::EPI / 4)) {
                    // only the N accumulated columns are read (a 16-column tail
                    // leaves the upper half at -inf)
                    uint32_t v[32];
                    if (X.ncol - c0 == 16) {
                        tmem_ld16(taddr + (uint32_t)c0, v);
#pragma unroll
                        for (int k = 16; k < 32; ++k) v[k] = 0xFF800000u;
                    } else {
                        tmem_ld32(taddr + (uint32_t)c0, v);
                    }
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    if (DBG && cvalid && has_cols) {  // the filter dump (test aid)
                        // (constant indices: v stays in registers)
#pragma unroll
                        for (int k = 0; k < 32; ++k) {
                            const int col = c0 + k;
                            if (col < X.ncol && (uint32_t)(col - col_lo) <= col_span)
                                dbg_record(P, X.qa + col, cp, __uint_as_float(v[k]));
                        }
                    }
                    // maxima of 8-column groups, then of all 32 (three-input max)
                    float m8[4];
#pragma unroll
                    for (int g8 = 0; g8 < 4; ++g8) {
                        const float* f = reinterpret_cast<const float*>(v + 8 * g8);
                        m8[g8] = max3f(max3f(f[0], f[1], f[2]), max3f(f[3], f[4], f[5]), fmaxf(f[6], f[7]));
                    }
                    const float mall = max3f(m8[0], m8[1], fmaxf(m8[2], m8[3]));
                    if (!__any_sync(0xffffffffu, cvalid && mall >= cto)) continue;
                    int hn = 0;
#pragma unroll
                    for (int g8 = 0; g8 < 4; ++g8) {
                        const bool h = cvalid && m8[g8] >= cto;
                        if (!__any_sync(0xffffffffu, h)) continue;
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            const int col = c0 + 8 * g8 + k;
                            const float a = __uint_as_float(v[8 * g8 + k]);
                            const bool ok = h && has_cols && a >= cto && (uint32_t)(col - col_lo) <= col_span;
                            if (ok) hits[hn++][lane] = (uint16_t)((uint32_t)col | (a >= cti ? 256u : 0u));
                        }
                    }
                    for (int i = 0; __any_sync(0xffffffffu, i < hn); ++i) {
                        int nout = 0;
                        int32_t qid = 0, cid = 0, qs = 0;
                        double dist = 0.0;
                        bool band = false, mir = false;
                        if (i < hn) {
                            const uint32_t e = hits[i][lane];
                            qs = X.qa + (int)(e & 255u);
                            mir = cfl == 1 || (cfl == 2 && cp != qs);
                            if ((e >> 8) && !EMIT) {
                                nout = mir ? 2 : 1;
                                qid = (int32_t)(qperm[qs - X.qa] - R.off);
                                cid = (int32_t)(cpid - R.off);
                            } else {
                                band = true;
                            }
                        }
                        const bool queued = band_push_q(bq, P, lane, band, qs, cp, mir);
                        if (band && !queued) {  // queue full: decide here
                            const double s2 = direct_sq(P.xs + (int64_t)qs * P.dp, P.xs + (int64_t)cp * P.dp, P.d);
                            ++rechecked;
                            if (s2 <= R.e2) {
                                nout = mir ? 2 : 1;
                                qid = (int32_t)(qperm[qs - X.qa] - R.off);
                                cid = (int32_t)(cpid - R.off);
                                if (EMIT) dist = sqrt(s2);
                            }
                        }
                        if (EMIT)
                            stage_emit(st, P, lane, nout, qid, cid, dist);
                        else
                            stage_emit_pairs(st, P, lane, nout, qid, cid);
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;");
                __syncwarp();
                if (lane == 0) bar_arrive(&S.acc_empty[acc]);
                if (++acc == 2) acc = 0, acc_ph ^= 1u;
            }
            if (fail) break;
            __syncwarp();
            if (lane == 0) bar_arrive(&S.item_empty[it_i]);
            if (++it_i == 2) it_i = 0, it_ph ^= 1u;
        }
        band_q_close(bq, P, lane);
        stage_flush(st, P, lane);
        for (int o = 16; o > 0; o >>= 1) rechecked += __shfl_down_sync(0xffffffffu, rechecked, o);
        if (lane == 0 && rechecked) atomicAdd(&P.counters[2], rechecked);
    }

    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (tid == 0 && S.abort) atomicExch(T.error, 1);
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)(2 * NMAX)));
    }
}

// Self-test of the bounded waits: one thread waits on an mbarrier that
// nothing arrives on; the wait must give up after its bound and raise the
// abort flag.  out[0] = 1 when the wait gave up, out[1] = the abort flag.
__global__ void k_wait_selftest(int* out, long long polls) {
    __shared__ uint64_t bar;
    __shared__ int abort;
    if (threadIdx.x == 0) {
        bar_init(&bar, 1);
        abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const bool done = bar_wait_n(&bar, 0, &abort, polls);
        out[0] = done ? 0 : 1;
        out[1] = abort;
    }
}

int selftest_bounded_wait(cudaStream_t s) {
    int* d = nullptr;
    SJ_TRY(dev_alloc_t(&d, 2, s));
    SJ_CK(cudaMemsetAsync(d, 0, 2 * sizeof(int), s));
    k_wait_selftest<<<1, 32, 0, s>>>(d, 1 << 16);
    note_launch();
    SJ_CK(cudaGetLastError());
    int h[2] = {0, 0};
    SJ_CK(cudaMemcpyAsync(h, d, sizeof h, cudaMemcpyDeviceToHost, s));
    SJ_CK(cudaStreamSynchronize(s));
    dev_free(d, s);
    if (h[0] == 1 && h[1] == 1) {
        set_error("the bounded wait gave up as designed");
        return SJ_ERR_TIMEOUT;
    }
    set_error("the bounded wait did not give up (%d, %d)", h[0], h[1]);
    return SJ_ERR_CUDA;
}

template <int KP, bool EMIT, bool DBG = false>
static int launch_kp(Index* ix, const JoinParams& p, const TcParams& t) {
    auto kern = k_join_tc<KP, EMIT, DBG>;
    const size_t smem = tc_smem_bytes<KP, EMIT>();
    if (smem > kSmemMax) {
        set_error("tensor-core tile does not fit in shared memory (K = %d)", KP);
        return SJ_ERR_UNSUPPORTED;
    }
    SJ_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    constexpr int threads = tc_threads(KP, EMIT);
    SJ_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    if (per_sm < 1) {
        set_error("tensor-core tile does not fit on an SM (K = %d)", KP);
        return SJ_ERR_UNSUPPORTED;
    }
    // one CTA per SM: it holds up to all 512 TMEM columns
    long long blocks = (long long)device_sm_count(ix->device);
    if (blocks > ix->n_items) blocks = ix->n_items > 0 ? ix->n_items : 1;
    kern<<<(unsigned)blocks, threads, smem, ix->stream>>>(p, t);
    note_launch();
    SJ_CK(cudaGetLastError());
    return SJ_OK;
}

template <int KP>
static int launch_k(Index* ix, const JoinParams& p, const TcParams& t) {
    if (p.dbg) return launch_kp<KP, false, true>(ix, p, t);  // the filter dump (no distances)
    return p.emit_dist ? launch_kp<KP, true>(ix, p, t) : launch_kp<KP, false>(ix, p, t);
}

int launch_join_tc(Index* ix, const JoinOut& out, int emit_dist) {
    const JoinParams p = make_join_params(ix, out, emit_dist);
    TcParams t;
    t.rows_a = static_cast<const __nv_bfloat16*>(ix->rows_a);
    t.rows_b = static_cast<const __nv_bfloat16*>(ix->rows_b);
    t.nrows = ((ix->n + 7) & ~int64_t(7)) + kTcPadRows;
    t.error = reinterpret_cast<int*>(ix->counters + 4);
    t.ab_bf16 = ix->kernel == SJ_KERNEL_FILTER_FP16X2 ? 0u : 1u;
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
