// Internal declarations of libsj (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <memory>
#include <string>
#include <vector>

#include "simjoin.h"

namespace sj {

// ---- limits ---------------------------------------------------------------
constexpr int kMaxM = 6;                         // indexed dims (3^(m-1) runs per cell)
constexpr int kMaxRuns = 243 + 1;                // 3^(kMaxM-1) + the split self run
constexpr int kQMax = 16;                        // queries per work item (bitmask width)
constexpr int kThreads = 128;                    // CTA size of the distance kernels
constexpr int kStage = 256;                      // per-warp staging slots for emitted pairs
constexpr int64_t kDefaultPagePairs = int64_t(1) << 22;

// ---- error reporting ----------------------------------------------------------
void set_error(const char* fmt, ...);
void clear_error();

#define SJ_CK(call)                                                                              \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) {                                                                 \
            ::sj::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
            return SJ_ERR_CUDA;                                                                  \
        }                                                                                        \
    } while (0)

#define SJ_TRY(expr)            \
    do {                        \
        int st_ = (expr);       \
        if (st_ != SJ_OK) return st_; \
    } while (0)

// ---- device memory (stream-ordered pool, cached across calls) -----------------
int dev_alloc(void** p, size_t bytes, cudaStream_t s);
void dev_free(void* p, cudaStream_t s);

template <typename T>
int dev_alloc_t(T** p, size_t count, cudaStream_t s) {
    return dev_alloc(reinterpret_cast<void**>(p), count * sizeof(T), s);
}

bool is_device_pointer(const void* p);

// Device temporaries of one host routine: every block taken through it is
// freed (stream-ordered) when it goes out of scope, on success and on every
// error return alike.
// A pinned host buffer of at least `bytes` for small device-to-host reads
// (sizes, totals, counts) of the calling thread, kept for the thread's life;
// null when pinned memory cannot be had (the caller reads into its own
// memory then).
void* host_staging(size_t bytes);

struct Scratch {
    cudaStream_t s;
    std::vector<void*> ptrs;
    explicit Scratch(cudaStream_t st) : s(st) {}
    Scratch(const Scratch&) = delete;
    Scratch& operator=(const Scratch&) = delete;
    ~Scratch() { release(); }
    // frees every temporary now (stream-ordered: after the work already
    // enqueued on s that uses them)
    void release() {
        for (void* p : ptrs) dev_free(p, s);
        ptrs.clear();
    }
    template <typename T>
    int alloc(T** p, size_t count) {
        const int st = dev_alloc_t(p, count, s);
        if (st == SJ_OK) ptrs.push_back(*p);
        return st;
    }
};

// ---- work item and candidate run ---------------------------------------------
// A work item: queries [q0, q1) of one cell (sorted positions) and the cell's
// candidate runs [r0, r1) in the run array.
struct Item {
    int32_t q0, q1, r0, r1;
};
// A candidate run: sorted positions [start, end); bit 31 of `end_flags` set
// means "mirror": the run lies in another cell than the queries and every
// hit is emitted in both orders.
struct Run {
    int32_t start;
    uint32_t end_flags;
};
constexpr uint32_t kMirrorBit = 0x80000000u;

// ---- index handle ---------------------------------------------------------------
struct Index {
    int device = 0;
    cudaStream_t stream = nullptr;
    sj_options opt{};
    int kernel = SJ_KERNEL_FP64_FMA;
    int64_t n = 0;
    int32_t d = 0, dp = 0;      // dims and padded dims (multiple of 4)
    double eps = 0, e2 = 0, w = 0;
    int32_t m = 0;
    int32_t dims[kMaxM] = {};
    int64_t ncell[kMaxM] = {};
    uint64_t stride[kMaxM] = {};
    int key_bits = 0;
    int key_bits_cap = 62;      // cell keys use at most this many bits
    bool trim_dims = false;     // batched instances: drop indexed dims by a uniform-density cost model
    std::vector<double> lo, hi;

    // device arrays (cell order)
    double* xs = nullptr;       // n x dp original coordinates, zero padded
    void* y = nullptr;          // n x dp kernel coordinates y = x - lo (double or float)
    void* h = nullptr;          // n: -||y||^2 / 2
    void* thr_out = nullptr;    // n: maybe-in threshold on (y_q.y_c - ||y_q||^2/2)
    void* thr_in = nullptr;     // n: certain-in threshold
    double* sc_w = nullptr;     // short-circuit (FP64 FMA, sj_options.short_circuit):
                                // n half remaining norms (after sc_b dims) plus margin
    int sc_b = 0;               // the checkpoint: after this many kernel dims (0: off)
    std::vector<int> dim_order; // kernel coordinate k is input dim dim_order[k]
    void* aux = nullptr;        // FP32 filter, padded d <= 8: n float4 records
                                // (thr_out, thr_in, input index bits, 0)
    int32_t* perm = nullptr;    // sorted position -> input index
    void* rows_a = nullptr;     // tensor-core filter: n x kp bf16 split rows, candidate role
    void* rows_b = nullptr;     // n x kp bf16 split rows, query role
    int kp = 0;                 // their padded K
    unsigned long long* cell_key = nullptr;
    int32_t* cell_start = nullptr;  // M + 1
    Run* runs = nullptr;
    Item* items = nullptr;
    int64_t n_cells = 0, n_runs = 0, n_items = 0, n_candidates = 0, n_evaluated = 0;
    double filter_band_rel = 0;  // predicted certified band (relative to eps^2)
    double bound_c1 = 0, bound_p = 0;  // certified bound E = c1 (P + pc) of the filter
    double kscale = 1.0;        // kernel coordinates = (x - centre) * kscale (a power of two)
    // binary32 kernels: (eps (1 + g) + eta)^2 in kernel units rounded up; a
    // squared distance of kernel coordinates above it is certified out (the
    // radius of the thresholds, see pack_coefficients)
    float prune_r2 = INFINITY;
    unsigned long long last_pruned = 0;  // pair evaluations the last join's prune removed

    // per-join scratch: counters (item queue, result cursor, recheck count,
    // recheck queue fill)
    unsigned long long* counters = nullptr;
    // events around the distance-tile kernel and its last duration
    cudaEvent_t ev_tile[2] = {nullptr, nullptr};
    cudaEvent_t ev_side[2] = {nullptr, nullptr};  // fork / join of the build's side-stream work
    double last_tile_ms = 0.0;
    // build phases (sj_set_tracing): device and host milliseconds of
    // extent + grid, sort, packing, runs + items; -1 when not traced
    double phase_dev_ms[4] = {-1, -1, -1, -1};
    double phase_host_ms[4] = {-1, -1, -1, -1};
};

// Tracing of the build phases (process-wide switch, sj_set_tracing).
bool tracing_on();
// Marks of a traced build: an event on the stream and the host clock at
// each phase boundary; finish() fills the index's phase times.
struct PhaseClock {
    bool on = false;
    int n = 0;
    cudaStream_t s = nullptr;
    cudaEvent_t ev[5] = {};
    double host[5] = {};
    explicit PhaseClock(cudaStream_t st);
    ~PhaseClock();
    void mark();
    void finish(Index* ix);
};

// Result internals.
struct ResultImpl {
    cudaStream_t stream = nullptr;
    int32_t* block = nullptr;   // the page pool: pages are slices of it
    double* dblock = nullptr;
    int64_t pages_alloc = 0;    // pages the pool holds (single joins; the tables list the used ones)
    std::vector<int32_t*> pair_pages;
    std::vector<double*> dist_pages;
    std::shared_ptr<void> shared_pool;  // batched results: the pool shared by all instances
};

// One group of a batched join: instances of the same padded dimension in
// one index whose cell keys carry the instance number above the local key.
struct BatchGroup {
    Index ix;                       // the group's index (n = the group's points)
    int n_inst = 0;
    std::vector<int> gids;          // instance numbers in the batch
    std::vector<long long> off;     // n_inst + 1 point offsets
    std::vector<double> eps;
    std::vector<int64_t> eval, cand;  // per instance: evaluations, canonical candidates
    long long* d_off = nullptr;
    int32_t* d_gid = nullptr;
    double* d_e2 = nullptr;
    float* d_r2 = nullptr;          // per instance: the bounding-box prune radius^2
    int32_t* d_inst_of_sorted = nullptr;
    int32_t* d_item_inst = nullptr;
};
// Routing of a batched join (sj_join_batch): items and sorted points belong
// to instances; every pair goes, in instance-local indices, to its instance's
// pages, which the device takes from a shared pool on first use.
struct BatchJoin {
    const int32_t* item_inst;       // per work item: group-local instance
    const int32_t* inst_of_sorted;  // per packed point: group-local instance
    const long long* inst_off;      // group-local instance -> its first point in the group
    const int32_t* inst_gid;        // group-local instance -> instance number in the batch
    const double* inst_e2;          // group-local instance -> eps^2
    const float* inst_r2;           // group-local instance -> the small-d FP32 filter's
                                    // bounding-box prune radius^2 (kernel units), or null
    // output (indexed by instance number)
    int2* pool;                     // n_pages pages of 2^page_log2 pairs
    double* dpool;                  // matching distances, or null
    int page_log2;
    long long n_pages;
    unsigned long long* pool_next;  // next free page
    int32_t* page_table;            // per instance: its pages in order (-1 free, -2 being taken,
                                    // -3 pool exhausted)
    const long long* table_off;     // instance -> first slot of its page table
    const int32_t* max_pages;       // instance -> slots of its page table
    unsigned long long* cursor;     // instance -> pairs emitted (exact, even past the pool)
    unsigned long long* error;      // set when a wait for a page claim expired
};

int build_batch_group(BatchGroup* g, const double* const* src_dev_ptrs, const int32_t* d_of_host);

// Whether the join evaluates only the triangle of each self cell (symmetric
// joins on the CUDA-core and tensor-core filter kernels): a work item's
// self-cell candidates start at its own first query and pairs below the
// diagonal are skipped.
inline bool is_tensor_kernel(int k) {
    return k == SJ_KERNEL_FILTER_BF16X3 || k == SJ_KERNEL_FILTER_BF16X2 || k == SJ_KERNEL_FILTER_FP16X2;
}
inline bool uses_triangle(const Index* ix) {
    return ix->opt.symmetric &&
           (ix->kernel == SJ_KERNEL_FILTER_F32 || ix->kernel == SJ_KERNEL_FP64_FMA || is_tensor_kernel(ix->kernel));
}

// ---- index build (sj_index.cu) ------------------------------------------------
int build_index(Index* ix, const double* pts_dev);

// ---- join kernels (sj_join_cc.cu) ----------------------------------------------
struct JoinOut {
    int2* out_pairs = nullptr;     // the result pool (one allocation)
    double* out_dist = nullptr;    // distances (or null)
    uint64_t capacity = 0;         // pairs the pool can hold
    int2* band = nullptr;          // deferred-recheck queue
    unsigned long long band_cap = 0;
    const void* batch = nullptr;   // device BatchJoin of a batched join, or null
    int4* dbg = nullptr;           // filter dump (sj_debug_filter_dump), or null
    unsigned long long dbg_cap = 0;
};
int launch_join_cc(Index* ix, const JoinOut& out, int emit_dist);
// The small-d FP32 filter without distances (sj_join_f32s.cu).
bool f32s_supported(const Index* ix, int emit_dist);
int launch_join_f32s(Index* ix, const JoinOut& out);
// Whether an index gets the per-point records of that kernel.
inline bool wants_aux(const Index* ix) { return ix->kernel == SJ_KERNEL_FILTER_F32 && ix->dp <= 8; }
int build_aux(Index* ix);
// Pair evaluations of each work item of a built index (n_items values), as
// the tile kernels perform them (self-cell runs from the item's first query
// in joins that evaluate triangles).
int launch_item_work(Index* ix, long long* work);
int launch_join_tc(Index* ix, const JoinOut& out, int emit_dist);
int selftest_bounded_wait(cudaStream_t s);
int launch_recheck(Index* ix, const JoinOut& out, int emit_dist);

// Split products per dim of a tensor-core filter: BF16x3 keeps 6, BF16x2 and
// FP16x2 3.
constexpr int tc_products(int kernel) { return kernel == SJ_KERNEL_FILTER_BF16X3 ? 6 : 3; }
// Padded K of the tensor-core filter for padded dimension dp: the products
// per dim plus 3 slots for the query term, rounded up to the MMA K of 16.
constexpr int tc_kp(int dp, int kernel) { return (tc_products(kernel) * dp + 3 + 15) / 16 * 16; }
// Relative coefficient c1 of the tensor-core filter's certified bound
// E = c1 (P + pc) (sj_index.cu).
double tc_c1(int dp, int kernel);
// Queries per work item of the tensor-core filter: the MMA N (the query tile,
// a whole number of 8-row groups from an 8-aligned start) is at most 256
// (128 when K > 208, for shared memory), so an item holds one group less.
constexpr int tc_nmax(int kp) { return kp <= 208 ? 256 : 128; }
constexpr int tc_qmax(int kp) { return tc_nmax(kp) - 8; }
// Zero rows after the last packed point in the split-row arrays, so 8-row
// groups and query tiles past the end read zeros.
constexpr int kTcPadRows = 256;
// Number of counters of a join (item queue, result cursor, rechecked,
// recheck-queue fill, error flag, spare).
constexpr int kCounters = 8;
int launch_join_dmma(Index* ix, const JoinOut& out, int emit_dist);

// Queries per work item of an index: the caller's queries_per_item when set
// (clamped to the kernel's capacity), else the capacity: the query bitmask
// width of the CUDA-core kernels, the query tile of the tensor-core filter.
inline int item_qmax(const Index* ix) {
    const int cap = is_tensor_kernel(ix->kernel) ? tc_qmax(tc_kp(ix->dp, ix->kernel)) : kQMax;
    return ix->opt.queries_per_item > 0 ? (ix->opt.queries_per_item < cap ? ix->opt.queries_per_item : cap) : cap;
}

// ---- tuning cache (sj_tune.cu) -------------------------------------------------
// One tuned configuration: for single joins keyed by (d, round(log2 n)), for
// the groups of batched joins by the padded dimension.
struct TuneEntry {
    int batch = 0;       // 0 single join, 1 batched group
    int d = 0;           // d (single) or padded d (batched group)
    int nlog2 = 0;       // single joins: round(log2 n)
    int kernel = SJ_KERNEL_AUTO;
    int qpi = 0;         // queries per item, 0 = the kernel's capacity
    int m = 0;           // indexed dims, 0 = automatic (single joins only)
    double ms = 0;       // the time it was tuned at
};
// Reads a tuning cache (a missing file is an empty cache); later lines win.
int tune_load(const char* path, std::vector<TuneEntry>* out);
// The entry for a single join of n points in d dims: same d, nearest
// round(log2 n) within 1; null if none.
const TuneEntry* tune_find_single(const std::vector<TuneEntry>& t, int d, int64_t n);
// The entry for a batched group of padded dimension dp; null if none.
const TuneEntry* tune_find_group(const std::vector<TuneEntry>& t, int dp);
// A batched join with per-group overrides: `forced` (tuning runs; kernel
// AUTO in an entry means no override) and the options' tuning cache.
int join_batch_impl(const double* const* pts, const int64_t* n, const int32_t* d, const double* eps, int32_t count,
                    const sj_options* opt, void* stream, sj_result* per_instance_out,
                    const std::vector<TuneEntry>* forced);
int round_dim(int d);

// ---- radix sort / scan (sj_index.cu) ------------------------------------------
int radix_sort_pairs(uint64_t* keys, int32_t* vals, int64_t n, int key_bits, cudaStream_t s);
int scan_exclusive_u32(const uint32_t* in, uint32_t* out, int64_t n, cudaStream_t s);
// As scan_exclusive_u32, also writing the total to out[n].
int scan_exclusive_u32_total(const uint32_t* in, uint32_t* out, int64_t n, cudaStream_t s);

int device_sm_count(int device);
// A second stream per device owned by the library (created on first use,
// non-blocking), for build work that can overlap the caller's stream.
int side_stream(int device, cudaStream_t* out);

// Kernels launched by the library in this process (reported by
// sj_kernel_launches); every launch site calls note_launch().
void note_launch();

}  // namespace sj
