// C ABI of libsj: argument checks, handle and result lifetime, the paged
// result pool and the device memory pool.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <mutex>
#include <new>

#include "sj_internal.cuh"

namespace sj {

// ---- errors ----------------------------------------------------------------------
static thread_local char g_msg[512];

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof g_msg, fmt, ap);
    va_end(ap);
}
void clear_error() { g_msg[0] = 0; }

static std::atomic<long long> g_launches{0};
static std::atomic<bool> g_tracing{false};
bool tracing_on() { return g_tracing.load(std::memory_order_relaxed); }

static double host_ms_now() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

PhaseClock::PhaseClock(cudaStream_t st) : on(tracing_on()), s(st) {}
PhaseClock::~PhaseClock() {
    for (int i = 0; i < n; ++i) cudaEventDestroy(ev[i]);
}
void PhaseClock::mark() {
    if (!on || n >= 5) return;
    if (cudaEventCreate(&ev[n]) != cudaSuccess) {
        on = false;
        return;
    }
    cudaEventRecord(ev[n], s);
    host[n] = host_ms_now();
    ++n;
}
void PhaseClock::finish(Index* ix) {
    if (!on || n < 5) return;
    cudaEventSynchronize(ev[4]);
    for (int k = 0; k < 4; ++k) {
        float ms = 0.f;
        ix->phase_dev_ms[k] = cudaEventElapsedTime(&ms, ev[k], ev[k + 1]) == cudaSuccess ? ms : -1.0;
        ix->phase_host_ms[k] = host[k + 1] - host[k];
    }
}
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// ---- device memory pool -------------------------------------------------------------
// One stream-ordered pool per device whose release threshold keeps freed
// blocks cached, so repeated joins do not return memory to the driver.
static std::mutex g_pool_mu;
static cudaMemPool_t g_pools[64];
static bool g_pool_init[64];

static int pool_for(int dev, cudaMemPool_t* out) {
    if (dev < 0 || dev >= 64) {
        set_error("device ordinal %d out of range", dev);
        return SJ_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool_init[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p;
        SJ_CK(cudaMemPoolCreate(&p, &props));
        unsigned long long thr = ~0ull;
        SJ_CK(cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &thr));
        g_pools[dev] = p;
        g_pool_init[dev] = true;
    }
    *out = g_pools[dev];
    return SJ_OK;
}

// Test aid: allocations still allowed before injected failures start (-1:
// no injection), and the device blocks currently held.
static std::atomic<long long> g_fail_after{-1};
static std::atomic<long long> g_live_blocks{0};

void* host_staging(size_t bytes) {
    struct Buf {
        void* p = nullptr;
        size_t n = 0;
        ~Buf() {
            if (p) cudaFreeHost(p);
        }
    };
    thread_local Buf b;
    if (b.n < bytes) {
        if (b.p) cudaFreeHost(b.p);
        b.p = nullptr;
        b.n = 0;
        const size_t want = bytes < 4096 ? 4096 : bytes;
        if (cudaMallocHost(&b.p, want) != cudaSuccess) {
            cudaGetLastError();
            b.p = nullptr;
            return nullptr;
        }
        b.n = want;
    }
    return b.p;
}

int dev_alloc(void** p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    if (g_fail_after.load(std::memory_order_relaxed) >= 0 &&
        g_fail_after.fetch_sub(1, std::memory_order_relaxed) <= 0) {
        g_fail_after.store(0, std::memory_order_relaxed);
        set_error("device allocation of %zu bytes failed (injected)", bytes);
        return SJ_ERR_OOM;
    }
    int dev = 0;
    SJ_CK(cudaGetDevice(&dev));
    cudaMemPool_t pool;
    SJ_TRY(pool_for(dev, &pool));
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, s);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        *p = nullptr;
        set_error("device allocation of %zu bytes failed", bytes);
        return SJ_ERR_OOM;
    }
    SJ_CK(e);
    g_live_blocks.fetch_add(1, std::memory_order_relaxed);
    return SJ_OK;
}

void dev_free(void* p, cudaStream_t s) {
    if (p) {
        cudaFreeAsync(p, s);
        g_live_blocks.fetch_sub(1, std::memory_order_relaxed);
    }
}

bool is_device_pointer(const void* p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int side_stream(int device, cudaStream_t* out) {
    static std::mutex mu;
    static cudaStream_t streams[64];
    if (device < 0 || device >= 64) {
        set_error("device ordinal %d out of range", device);
        return SJ_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(mu);
    if (!streams[device]) SJ_CK(cudaStreamCreateWithFlags(&streams[device], cudaStreamNonBlocking));
    *out = streams[device];
    return SJ_OK;
}

int device_sm_count(int device) {
    static int cache[64];
    if (device < 0 || device >= 64) return 1;
    if (cache[device] == 0) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
        cache[device] = v > 0 ? v : 1;
    }
    return cache[device];
}

static void release_index(Index* ix) {
    if (!ix) return;
    cudaStream_t s = ix->stream;
    dev_free(ix->xs, s);
    dev_free(ix->y, s);
    dev_free(ix->h, s);
    dev_free(ix->thr_out, s);
    dev_free(ix->thr_in, s);
    dev_free(ix->aux, s);
    dev_free(ix->sc_w, s);
    dev_free(ix->perm, s);
    dev_free(ix->rows_a, s);
    dev_free(ix->rows_b, s);
    dev_free(ix->cell_key, s);
    dev_free(ix->cell_start, s);
    dev_free(ix->runs, s);
    dev_free(ix->items, s);
    dev_free(ix->counters, s);
    if (ix->ev_tile[0]) cudaEventDestroy(ix->ev_tile[0]);
    if (ix->ev_tile[1]) cudaEventDestroy(ix->ev_tile[1]);
    if (ix->ev_side[0]) cudaEventDestroy(ix->ev_side[0]);
    if (ix->ev_side[1]) cudaEventDestroy(ix->ev_side[1]);
}

// AUTO: the certified filters always beat the plain FP64 kernels on this part
// (FP64 runs at ~1/60 of FP32); the tensor-core filter wins from padded
// dimension 16 on (measured, 1M points, step times FP32 filter / FP16x2:
// d = 12 clustered 37.1 / 19.4 ms, uniform 1128 / 109 ms; d = 16 clustered
// 39.6 / 19.1 ms), the FP32 CUDA-core filter below (d = 6: 7.1 / 33.8 ms
// clustered; d = 8 depends on the data: clustered 10.3 / 22.2, uniform
// 36.5 / 14.9 ms).
// Of the tensor-core filters FP16x2 (the K of BF16x2, a narrower band: fewer
// binary64 rechecks) is never slower (measured on the 16-D and 64-D
// workloads).  (build_index turns AUTO into the FP64 tile for an extent that
// scaled binary32 coordinates cannot hold.)
static int pick_kernel(const Index* ix) {
    int k = ix->opt.kernel;
    if (k != SJ_KERNEL_AUTO) return k;
    return (ix->d >= 9 && ix->d <= 64) ? SJ_KERNEL_FILTER_FP16X2 : SJ_KERNEL_FILTER_F32;
}

int round_dim(int d) {
    int p = 2;
    while (p < d) p <<= 1;
    return p;
}

}  // namespace sj

using namespace sj;

struct sj_index : public sj::Index {};

extern "C" {

void sj_default_options(sj_options* o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->kernel = SJ_KERNEL_AUTO;
    o->emit_distances = 0;
    o->indexed_dims = 0;
    o->symmetric = 1;
    o->queries_per_item = 0;
    o->page_pairs = 0;
    o->max_pairs_hint = 0;
}

const char* sj_error_string(int status) {
    switch (status) {
        case SJ_OK: return "ok";
        case SJ_ERR_ARG: return "invalid argument";
        case SJ_ERR_OOM: return "out of memory";
        case SJ_ERR_RESULT_OVERFLOW: return "result larger than the page pool";
        case SJ_ERR_TIMEOUT: return "bounded device wait timed out";
        case SJ_ERR_CUDA: return "CUDA error";
        case SJ_ERR_UNSUPPORTED: return "unsupported kernel or shape";
        default: return "unknown status";
    }
}

const char* sj_last_error_message(void) { return g_msg; }

const char* sj_version(void) { return "libsj 0.1 sm_103a"; }

int64_t sj_kernel_launches(void) { return (int64_t)g_launches.load(std::memory_order_relaxed); }

void sj_set_tracing(int32_t on) { g_tracing.store(on != 0, std::memory_order_relaxed); }

int sj_index_phase_ms(sj_handle h, double* device_ms, double* host_ms) {
    clear_error();
    if (!h) {
        set_error("NULL handle");
        return SJ_ERR_ARG;
    }
    for (int k = 0; k < 4; ++k) {
        if (device_ms) device_ms[k] = h->phase_dev_ms[k];
        if (host_ms) host_ms[k] = h->phase_host_ms[k];
    }
    return SJ_OK;
}

void sj_debug_fail_allocations(int64_t after) { g_fail_after.store(after < 0 ? -1 : after, std::memory_order_relaxed); }

int64_t sj_debug_live_allocations(void) { return (int64_t)g_live_blocks.load(std::memory_order_relaxed); }

int sj_index_perm(sj_handle h, int32_t* perm_out) {
    clear_error();
    if (!h || !perm_out) {
        set_error("NULL argument");
        return SJ_ERR_ARG;
    }
    SJ_CK(cudaMemcpyAsync(perm_out, h->perm, (size_t)h->n * sizeof(int32_t), cudaMemcpyDefault, h->stream));
    SJ_CK(cudaStreamSynchronize(h->stream));
    return SJ_OK;
}

int sj_selftest_bounded_wait(void* stream) {
    clear_error();
    return selftest_bounded_wait(static_cast<cudaStream_t>(stream));
}

int sj_build_index(const double* pts, int64_t n, int32_t d, double eps, const sj_options* opt, void* stream,
                   sj_handle* out) {
    clear_error();
    if (!out) {
        set_error("out is NULL");
        return SJ_ERR_ARG;
    }
    *out = nullptr;
    if (!pts || n < 1 || n > 0x7FFFFFFFll || d < 1 || d > SJ_MAX_D || !(eps > 0) || !isfinite(eps)) {
        set_error("invalid argument: pts=%p n=%lld d=%d eps=%g", (const void*)pts, (long long)n, (int)d, eps);
        return SJ_ERR_ARG;
    }
    sj_options o;
    sj_default_options(&o);
    if (opt) o = *opt;
    if (o.kernel < SJ_KERNEL_AUTO || o.kernel > SJ_KERNEL_FILTER_FP16X2 || o.indexed_dims < SJ_NO_INDEX ||
        o.queries_per_item < 0 || o.page_pairs < 0 || o.max_pairs_hint < 0) {
        set_error("invalid options");
        return SJ_ERR_ARG;
    }
    // AUTO with a tuning cache: a tuned entry for this d and size supplies the
    // kernel and whichever of items / indexed dims the caller left automatic
    if (o.kernel == SJ_KERNEL_AUTO && o.tune_cache && o.tune_cache[0]) {
        std::vector<TuneEntry> table;
        int ts = tune_load(o.tune_cache, &table);
        if (ts != SJ_OK) return ts;
        if (const TuneEntry* te = tune_find_single(table, d, n)) {
            o.kernel = te->kernel;
            if (o.queries_per_item == 0) o.queries_per_item = te->qpi;
            if (o.indexed_dims == 0) o.indexed_dims = te->m;
        }
    }
    sj_index* ix = new (std::nothrow) sj_index();
    if (!ix) return SJ_ERR_OOM;
    cudaError_t e = cudaGetDevice(&ix->device);
    if (e != cudaSuccess) {
        set_error("cudaGetDevice: %s", cudaGetErrorString(e));
        delete ix;
        return SJ_ERR_CUDA;
    }
    ix->stream = static_cast<cudaStream_t>(stream);
    ix->opt = o;
    ix->n = n;
    ix->d = d;
    ix->dp = round_dim(d);
    ix->eps = eps;
    ix->e2 = eps * eps;
    ix->kernel = pick_kernel(ix);
    if (is_tensor_kernel(ix->kernel) && ix->dp > 64) {
        set_error("the tensor-core filter supports d <= 64 (got d = %d)", (int)d);
        delete ix;
        return SJ_ERR_UNSUPPORTED;
    }
    if (ix->kernel == SJ_KERNEL_FP64_DMMA && ix->dp < 4) ix->dp = 4;
    // points: use device memory in place, or stage host memory
    const double* dpts = pts;
    double* staged = nullptr;
    int st = SJ_OK;
    if (!is_device_pointer(pts)) {
        st = dev_alloc_t(&staged, (size_t)n * d, ix->stream);
        if (st == SJ_OK) {
            e = cudaMemcpyAsync(staged, pts, (size_t)n * d * sizeof(double), cudaMemcpyHostToDevice, ix->stream);
            if (e != cudaSuccess) {
                set_error("host-to-device copy: %s", cudaGetErrorString(e));
                st = SJ_ERR_CUDA;
            }
        }
        dpts = staged;
    }
    if (st == SJ_OK) st = build_index(ix, dpts);
    if (staged) dev_free(staged, ix->stream);
    if (st != SJ_OK) {
        release_index(ix);
        cudaStreamSynchronize(ix->stream);
        delete ix;
        return st;
    }
    *out = ix;
    return SJ_OK;
}

void sj_destroy(sj_handle h) {
    if (!h) return;
    release_index(h);
    cudaStreamSynchronize(h->stream);
    delete h;
}

int sj_index_info(sj_handle h, int64_t* n_cells, int64_t* n_items, int32_t* m, int64_t* n_candidates,
                  int64_t* n_evaluated) {
    if (!h) {
        set_error("NULL handle");
        return SJ_ERR_ARG;
    }
    if (n_cells) *n_cells = h->n_cells;
    if (n_items) *n_items = h->n_items;
    if (m) *m = h->m;
    if (n_candidates) *n_candidates = h->n_candidates;
    if (n_evaluated) *n_evaluated = h->n_evaluated;
    return SJ_OK;
}

// The page pool is one allocation sliced into pages (one pool call per join
// instead of one per page); growing it replaces the allocation.
// The pool of a single join's result: one block of pages_needed pages (the
// page tables are filled after the join, with the pages that hold pairs).
static int alloc_pages(ResultImpl* ri, int64_t pages_needed, int64_t page_pairs, bool dist, cudaStream_t s) {
    if (ri->pages_alloc >= pages_needed) return SJ_OK;
    dev_free(ri->block, s);
    dev_free(ri->dblock, s);
    ri->block = nullptr;
    ri->dblock = nullptr;
    ri->pages_alloc = 0;
    SJ_TRY(dev_alloc_t(&ri->block, (size_t)pages_needed * page_pairs * 2, s));
    if (dist) SJ_TRY(dev_alloc_t(&ri->dblock, (size_t)pages_needed * page_pairs, s));
    ri->pages_alloc = pages_needed;
    return SJ_OK;
}

// Free device memory of `dev`, queried at most every 64 calls (a query
// costs ~10 us on the join's critical path); `fresh` forces a query.
static size_t free_memory(int dev, bool fresh) {
    static std::mutex mu;
    static size_t cached[64] = {};
    static int age[64] = {};
    std::lock_guard<std::mutex> lock(mu);
    const int i = dev & 63;
    if (fresh || cached[i] == 0 || ++age[i] >= 64) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            cudaGetLastError();
            fr = 0;
        }
        cached[i] = fr;
        age[i] = 0;
    }
    return cached[i];
}

// The page pool shared by the results of one batched join, freed with the
// last of them.
struct PoolHolder {
    cudaStream_t stream = nullptr;
    int32_t* block = nullptr;
    double* dblock = nullptr;
    ~PoolHolder() {
        dev_free(block, stream);
        dev_free(dblock, stream);
    }
};

static void free_result_impl(ResultImpl* ri) {
    if (!ri) return;
    dev_free(ri->block, ri->stream);
    dev_free(ri->dblock, ri->stream);
    delete ri;
}

static int run_join(sj_index* ix, ResultImpl* ri, int64_t page_pairs, bool dist, unsigned long long* count_out,
                    unsigned long long* rechecked_out, int4* dbg = nullptr, unsigned long long dbg_cap = 0,
                    unsigned long long* dbg_count = nullptr, int64_t item_begin = 0, int64_t item_end = -1) {
    cudaStream_t s = ix->stream;
    const int64_t np = ri->pages_alloc;
    SJ_CK(cudaMemsetAsync(ix->counters, 0, kCounters * sizeof(unsigned long long), s));
    const int64_t all_items = ix->n_items;
    if (item_end < 0 || item_end > all_items) item_end = all_items;
    if (item_begin > 0) {  // the item queue starts at the range
        const unsigned long long b0 = (unsigned long long)item_begin;
        SJ_CK(cudaMemcpyAsync(ix->counters, &b0, sizeof b0, cudaMemcpyHostToDevice, s));
    }
    // deferred-recheck queue: band pairs (and, with distances, every
    // maybe-in pair); pairs past its end are re-decided in place
    const unsigned long long ev = (unsigned long long)std::max<int64_t>(ix->n_evaluated, 1);
    unsigned long long band_cap = dist ? std::max<unsigned long long>(1ull << 20, ev / 8) : std::max<unsigned long long>(1ull << 20, ev / 64);
    band_cap = std::min<unsigned long long>(band_cap, ev);
    Scratch tmp(s);
    int2* band = nullptr;
    SJ_TRY(tmp.alloc(&band, (size_t)band_cap));
    JoinOut jo;
    jo.out_pairs = reinterpret_cast<int2*>(ri->block);
    jo.out_dist = ri->dblock;
    jo.capacity = (unsigned long long)np * (unsigned long long)page_pairs;
    jo.band = band;
    jo.band_cap = band_cap;
    jo.dbg = dbg;
    jo.dbg_cap = dbg_cap;
    int st = SJ_OK;
    if (!ix->ev_tile[0]) {
        SJ_CK(cudaEventCreate(&ix->ev_tile[0]));
        SJ_CK(cudaEventCreate(&ix->ev_tile[1]));
    }
    const bool any = item_end > item_begin;
    if (any) {
        SJ_CK(cudaEventRecord(ix->ev_tile[0], s));
        ix->n_items = item_end;  // the kernels stop at the range's end
        if (ix->kernel == SJ_KERNEL_FP64_DMMA)
            st = launch_join_dmma(ix, jo, dist ? 1 : 0);
        else if (is_tensor_kernel(ix->kernel))
            st = launch_join_tc(ix, jo, dist ? 1 : 0);
        else
            st = launch_join_cc(ix, jo, dist ? 1 : 0);
        ix->n_items = all_items;
        if (st == SJ_OK) SJ_CK(cudaEventRecord(ix->ev_tile[1], s));
        if (st == SJ_OK) st = launch_recheck(ix, jo, dist ? 1 : 0);
    }
    unsigned long long c[kCounters] = {};
    if (st == SJ_OK) {
        tmp.release();  // (stream-ordered: after the kernels that use the queue)
        void* hs = host_staging(sizeof c);  // pinned: a direct copy
        cudaError_t e = cudaMemcpyAsync(hs ? hs : c, ix->counters, sizeof c, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess && hs) memcpy(c, hs, sizeof c);
        if (e != cudaSuccess) {
            set_error("join: %s", cudaGetErrorString(e));
            st = SJ_ERR_CUDA;
        } else if ((int)c[4] != 0) {
            set_error("a bounded wait in the tensor-core kernel expired");
            st = SJ_ERR_TIMEOUT;
        } else if (c[7] != 0) {
            set_error("bounds check at site %llu failed (debug build)", c[7]);
            st = SJ_ERR_CUDA;
        }
    }
    ix->last_tile_ms = 0.0;
    if (st == SJ_OK && any) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ix->ev_tile[0], ix->ev_tile[1]) == cudaSuccess) ix->last_tile_ms = ms;
    }
    *count_out = c[1];
    *rechecked_out = c[2];
    ix->last_pruned = c[6];
    if (dbg_count) *dbg_count = c[5];
    return st;
}

int sj_self_join_to_host(sj_handle h, int32_t* host_pairs, int64_t host_capacity, int64_t device_pairs,
                         int64_t* count_out, int32_t* rounds_out) {
    clear_error();
    if (!h || !count_out || host_capacity < 0 || (host_capacity > 0 && !host_pairs) || device_pairs < 1024) {
        set_error("invalid arguments (device_pairs must be at least 1024)");
        return SJ_ERR_ARG;
    }
    if (host_pairs && is_device_pointer(host_pairs)) {
        set_error("host_pairs must be host memory");
        return SJ_ERR_ARG;
    }
    *count_out = 0;
    if (rounds_out) *rounds_out = 0;
    sj_index* ix = h;
    cudaStream_t s = ix->stream;
    const int64_t n_items = ix->n_items;
    const unsigned long long ev = (unsigned long long)std::max<int64_t>(ix->n_evaluated, 1);
    unsigned long long band_cap = std::min<unsigned long long>(std::max<unsigned long long>(1ull << 20, ev / 64), ev);
    int2* pool[2] = {nullptr, nullptr};
    int2* band = nullptr;
    cudaStream_t cs = nullptr;
    cudaEvent_t done[2] = {nullptr, nullptr}, copied[2] = {nullptr, nullptr};
    int st = SJ_OK;
    if ((st = dev_alloc_t(&pool[0], (size_t)device_pairs, s)) == SJ_OK &&
        (st = dev_alloc_t(&pool[1], (size_t)device_pairs, s)) == SJ_OK)
        st = dev_alloc_t(&band, (size_t)band_cap, s);
    if (st == SJ_OK) {
        cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
            e = cudaEventCreateWithFlags(&done[b], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&copied[b], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) {
            set_error("set-up: %s", cudaGetErrorString(e));
            st = SJ_ERR_CUDA;
        }
    }
    // rounds over consecutive work-item ranges [i0, i0 + L); a round whose
    // pairs exceed the buffer is run again on half the range
    unsigned long long total = 0, rechecked = 0;
    int64_t i0 = 0, L = std::max<int64_t>(1, n_items / 16);
    int rounds = 0, b = 0;
    bool copied_pending[2] = {false, false};
    const int64_t keep_items = ix->n_items;
    while (st == SJ_OK && i0 < n_items) {
        const int64_t i1 = std::min<int64_t>(n_items, i0 + L);
        if (copied_pending[b] && cudaStreamWaitEvent(s, copied[b], 0) != cudaSuccess) st = SJ_ERR_CUDA;
        unsigned long long c[kCounters] = {};
        c[0] = (unsigned long long)i0;  // the item queue starts at the range
        cudaError_t e = st == SJ_OK ? cudaMemcpyAsync(ix->counters, c, sizeof c, cudaMemcpyHostToDevice, s)
                                    : cudaErrorUnknown;
        if (e != cudaSuccess) {
            if (st == SJ_OK) set_error("round set-up: %s", cudaGetErrorString(e));
            st = SJ_ERR_CUDA;
            break;
        }
        JoinOut jo;
        jo.out_pairs = pool[b];
        jo.capacity = (unsigned long long)device_pairs;
        jo.band = band;
        jo.band_cap = band_cap;
        ix->n_items = i1;  // the kernels stop at the range's end
        if (ix->kernel == SJ_KERNEL_FP64_DMMA)
            st = launch_join_dmma(ix, jo, 0);
        else if (is_tensor_kernel(ix->kernel))
            st = launch_join_tc(ix, jo, 0);
        else
            st = launch_join_cc(ix, jo, 0);
        if (st == SJ_OK) st = launch_recheck(ix, jo, 0);
        ix->n_items = keep_items;
        if (st != SJ_OK) break;
        e = cudaMemcpyAsync(c, ix->counters, sizeof c, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            set_error("round: %s", cudaGetErrorString(e));
            st = SJ_ERR_CUDA;
            break;
        }
        if ((int)c[4] != 0) {
            set_error("a bounded wait in the tensor-core kernel expired");
            st = SJ_ERR_TIMEOUT;
            break;
        }
        const unsigned long long got = c[1];
        if (got > (unsigned long long)device_pairs) {  // did not fit: half the range again
            if (L == 1) {
                set_error("work item %lld alone yields %llu pairs, more than device_pairs = %lld", (long long)i0,
                          got, (long long)device_pairs);
                st = SJ_ERR_RESULT_OVERFLOW;
                break;
            }
            L = std::max<int64_t>(1, L / 2);
            continue;
        }
        // copy this round's pairs out on the copy stream while the next round runs
        if (host_pairs && total < (unsigned long long)host_capacity && got > 0) {
            const unsigned long long room = (unsigned long long)host_capacity - total;
            const unsigned long long cnt = got < room ? got : room;
            e = cudaEventRecord(done[b], s);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, done[b], 0);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(host_pairs + 2 * total, pool[b], cnt * sizeof(int2), cudaMemcpyDeviceToHost, cs);
            if (e == cudaSuccess) e = cudaEventRecord(copied[b], cs);
            if (e != cudaSuccess) {
                set_error("result copy: %s", cudaGetErrorString(e));
                st = SJ_ERR_CUDA;
                break;
            }
            copied_pending[b] = true;
        }
        total += got;
        rechecked += c[2];
        ++rounds;
        // next range: aim at 3/4 of the buffer from this round's pairs per item
        const double per_item = (double)got / (double)(i1 - i0);
        const int64_t next = per_item > 0 ? (int64_t)(0.75 * (double)device_pairs / per_item) : 4 * L;
        L = std::max<int64_t>(1, std::min<int64_t>(next, 4 * L));
        i0 = i1;
        b ^= 1;
    }
    if (cs) cudaStreamSynchronize(cs);
    for (int k = 0; k < 2; ++k) {
        if (done[k]) cudaEventDestroy(done[k]);
        if (copied[k]) cudaEventDestroy(copied[k]);
        dev_free(pool[k], s);
    }
    dev_free(band, s);
    if (cs) cudaStreamDestroy(cs);
    cudaStreamSynchronize(s);
    if (st != SJ_OK) return st;
    *count_out = (int64_t)total;
    if (rounds_out) *rounds_out = rounds;
    if (total > (unsigned long long)host_capacity) {
        set_error("result of %llu pairs exceeds host_capacity = %lld (the first pairs were copied)", total,
                  (long long)host_capacity);
        return SJ_ERR_RESULT_OVERFLOW;
    }
    return SJ_OK;
}

static int self_join_impl(sj_handle h, int64_t item_begin, int64_t item_end, sj_result* out) {
    clear_error();
    if (!h || !out) {
        set_error("NULL argument");
        return SJ_ERR_ARG;
    }
    memset(out, 0, sizeof *out);
    int64_t page_pairs = h->opt.page_pairs > 0 ? h->opt.page_pairs : kDefaultPagePairs;
    int page_log2 = 6;  // at least 64 pairs a page (one claiming lane per page in a warp's flush)
    while ((int64_t(1) << page_log2) < page_pairs) ++page_log2;
    page_pairs = int64_t(1) << page_log2;
    const bool dist = h->opt.emit_distances != 0;
    // initial pool: the hint, else the candidate count capped by a share of
    // free memory (the result never exceeds the candidate count)
    int64_t want = h->opt.max_pairs_hint;
    const bool from_free = want <= 0;
    auto budget_pairs = [&](bool fresh) {
        const int64_t per_pair = dist ? 16 : 8;
        const int64_t budget = (int64_t)(free_memory(h->device, fresh) / 4) / per_pair;
        return std::min<int64_t>(h->n_candidates, std::max<int64_t>(budget, 16 * h->n));
    };
    if (from_free) want = budget_pairs(false);
    ResultImpl* ri = new (std::nothrow) ResultImpl();
    if (!ri) return SJ_ERR_OOM;
    ri->stream = h->stream;
    int64_t np = (want + page_pairs - 1) / page_pairs;
    if (np < 1) np = 1;
    int st = alloc_pages(ri, np, page_pairs, dist, h->stream);
    if (st == SJ_ERR_OOM && from_free) {  // the remembered free memory was stale: ask again
        np = std::max<int64_t>(1, (budget_pairs(true) + page_pairs - 1) / page_pairs);
        clear_error();
        st = alloc_pages(ri, np, page_pairs, dist, h->stream);
    }
    unsigned long long count = 0, rechecked = 0;
    int reruns = 0;
    if (st == SJ_OK) st = run_join(h, ri, page_pairs, dist, &count, &rechecked, nullptr, 0, nullptr, item_begin, item_end);
    if (st == SJ_OK && count > (unsigned long long)ri->pages_alloc * (unsigned long long)page_pairs) {
        // overflow: grow the pool to the exact count and run again
        int64_t need = (int64_t)((count + page_pairs - 1) / page_pairs);
        st = alloc_pages(ri, need, page_pairs, dist, h->stream);
        if (st == SJ_OK) {
            reruns = 1;
            st = run_join(h, ri, page_pairs, dist, &count, &rechecked, nullptr, 0, nullptr, item_begin, item_end);
        }
        if (st == SJ_OK && count > (unsigned long long)ri->pages_alloc * (unsigned long long)page_pairs) {
            set_error("result of %llu pairs still exceeds the page pool", count);
            st = SJ_ERR_RESULT_OVERFLOW;
        }
    }
    if (st != SJ_OK && st != SJ_ERR_RESULT_OVERFLOW) {
        free_result_impl(ri);
        return st;
    }
    // report only the pages that hold pairs (the allocation stays whole)
    int64_t used = (int64_t)((count + page_pairs - 1) / page_pairs);
    used = std::min<int64_t>(used, ri->pages_alloc);
    ri->pair_pages.resize((size_t)used);
    if (dist) ri->dist_pages.resize((size_t)used);
    for (int64_t p = 0; p < used; ++p) {
        ri->pair_pages[(size_t)p] = ri->block + p * page_pairs * 2;
        if (dist) ri->dist_pages[(size_t)p] = ri->dblock + p * page_pairs;
    }
    out->count = (int64_t)count;
    out->page_pairs = page_pairs;
    out->n_pages = (int32_t)ri->pair_pages.size();
    out->has_distances = dist ? 1 : 0;
    out->pair_pages = ri->pair_pages.data();
    out->dist_pages = dist ? ri->dist_pages.data() : nullptr;
    out->n_candidates = h->n_candidates;
    out->n_evaluated = h->n_evaluated - (int64_t)h->last_pruned;
    out->n_rechecked = (int64_t)rechecked;
    out->reruns = reruns;
    out->kernel = h->kernel;
    out->ms_tile = h->last_tile_ms;
    out->internal = ri;
    return st;
}

int sj_debug_filter_dump(sj_handle h, int32_t* perm, float* y, float* hnorm, float* thr_out, float* thr_in,
                         int32_t* records, int64_t capacity, sj_filter_dump* info) {
    clear_error();
    if (!h || !info || capacity < 0 || (capacity > 0 && !records)) {
        set_error("invalid argument");
        return SJ_ERR_ARG;
    }
    const bool f32s = h->kernel == SJ_KERNEL_FILTER_F32 && h->dp <= 8;
    if (!f32s && !is_tensor_kernel(h->kernel)) {
        set_error("the filter dump covers the FP32 filter (padded d <= 8) and the tensor-core filters");
        return SJ_ERR_UNSUPPORTED;
    }
    info->n = h->n;
    info->dp = h->dp;
    info->kernel = h->kernel;
    info->c1 = h->bound_c1;
    info->pbound = h->bound_p;
    info->e2 = h->e2;
    info->prune_r2 = f32s ? (double)h->prune_r2 : INFINITY;
    info->records = -1;
    info->count = -1;
    if (!perm && !y && !hnorm && !thr_out && !thr_in && capacity == 0) return SJ_OK;  // sizes only
    cudaStream_t s = h->stream;
    const int64_t n = h->n;
    if (perm) SJ_CK(cudaMemcpyAsync(perm, h->perm, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    if (y) SJ_CK(cudaMemcpyAsync(y, h->y, n * h->dp * sizeof(float), cudaMemcpyDeviceToHost, s));
    if (hnorm) SJ_CK(cudaMemcpyAsync(hnorm, h->h, n * sizeof(float), cudaMemcpyDeviceToHost, s));
    if (thr_out) SJ_CK(cudaMemcpyAsync(thr_out, h->thr_out, n * sizeof(float), cudaMemcpyDeviceToHost, s));
    if (thr_in) SJ_CK(cudaMemcpyAsync(thr_in, h->thr_in, n * sizeof(float), cudaMemcpyDeviceToHost, s));
    int4* dbg = nullptr;
    SJ_TRY(dev_alloc_t(&dbg, (size_t)std::max<int64_t>(capacity, 1), s));
    ResultImpl* ri = new (std::nothrow) ResultImpl();
    if (!ri) {
        dev_free(dbg, s);
        return SJ_ERR_OOM;
    }
    ri->stream = s;
    const int64_t page_pairs = kDefaultPagePairs;
    int st = alloc_pages(ri, std::max<int64_t>(1, (h->n_candidates + page_pairs - 1) / page_pairs), page_pairs,
                         false, s);
    unsigned long long count = 0, rechecked = 0, recorded = 0;
    if (st == SJ_OK) st = run_join(h, ri, page_pairs, false, &count, &rechecked, dbg, (unsigned long long)capacity,
                                   &recorded);
    if (st == SJ_OK && capacity > 0) {
        const int64_t k = std::min<int64_t>((int64_t)recorded, capacity);
        cudaError_t e = cudaMemcpyAsync(records, dbg, k * sizeof(int4), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            set_error("filter dump copy: %s", cudaGetErrorString(e));
            st = SJ_ERR_CUDA;
        }
    }
    free_result_impl(ri);
    dev_free(dbg, s);
    if (st != SJ_OK) return st;
    info->records = (int64_t)recorded;
    info->count = (int64_t)count;
    return SJ_OK;
}

int sj_self_join(sj_handle h, sj_result* out) { return self_join_impl(h, 0, -1, out); }

int sj_self_join_range(sj_handle h, int64_t item_begin, int64_t item_end, sj_result* out) {
    if (!h || item_begin < 0 || item_end < item_begin || item_end > h->n_items) {
        set_error("invalid item range [%lld, %lld) of %lld items", (long long)item_begin, (long long)item_end,
                  h ? (long long)h->n_items : -1ll);
        return SJ_ERR_ARG;
    }
    return self_join_impl(h, item_begin, item_end, out);
}

int sj_index_item_work(sj_handle h, int64_t* work_out) {
    clear_error();
    if (!h || !work_out) {
        set_error("NULL argument");
        return SJ_ERR_ARG;
    }
    if (h->n_items == 0) return SJ_OK;
    Scratch tmp(h->stream);
    long long* dw = nullptr;
    SJ_TRY(tmp.alloc(&dw, (size_t)h->n_items));
    SJ_TRY(launch_item_work(h, dw));
    SJ_CK(cudaMemcpyAsync(work_out, dw, (size_t)h->n_items * sizeof(long long), cudaMemcpyDeviceToHost, h->stream));
    SJ_CK(cudaStreamSynchronize(h->stream));
    return SJ_OK;
}

int sj_shard_bounds(const int64_t* item_work, int64_t n_items, int32_t n_shards, int64_t* bounds) {
    clear_error();
    if (n_items < 0 || n_shards < 1 || !bounds || (n_items > 0 && !item_work)) {
        set_error("invalid argument");
        return SJ_ERR_ARG;
    }
    long double total = 0;
    for (int64_t i = 0; i < n_items; ++i) {
        if (item_work[i] < 0) {
            set_error("negative work for item %lld", (long long)i);
            return SJ_ERR_ARG;
        }
        total += (long double)item_work[i];
    }
    // boundary k: the item boundary whose work prefix is nearest to k / N of
    // the total (ties to the earlier one); prefixes only grow, so the bounds
    // are monotone
    bounds[0] = 0;
    long double pre = 0;
    int64_t i = 0;
    for (int32_t k = 1; k < n_shards; ++k) {
        const long double target = total * (long double)k / (long double)n_shards;
        while (i < n_items && pre + (long double)item_work[i] <= target) pre += (long double)item_work[i++];
        // pre <= target < pre + work[i]: take the nearer boundary
        if (i < n_items && (pre + (long double)item_work[i]) - target < target - pre) pre += (long double)item_work[i++];
        // a boundary never falls before an item of no work (an item that
        // continues its cell: the cell's work sits at its first item)
        while (i < n_items && item_work[i] == 0) ++i;
        bounds[k] = i;
    }
    bounds[n_shards] = n_items;
    return SJ_OK;
}

int sj_result_copy(const sj_result* r, int32_t* pairs_out, double* dist_out) {
    clear_error();
    if (!r) {
        set_error("NULL result");
        return SJ_ERR_ARG;
    }
    if (r->count == 0) return SJ_OK;
    if (!pairs_out && !dist_out) return SJ_OK;
    const ResultImpl* ri = static_cast<const ResultImpl*>(r->internal);
    if (!ri) {
        set_error("result has no pages");
        return SJ_ERR_ARG;
    }
    int64_t left = std::min<int64_t>(r->count, (int64_t)r->n_pages * r->page_pairs);
    for (int p = 0; p < r->n_pages && left > 0; ++p) {
        const int64_t cnt = std::min<int64_t>(left, r->page_pairs);
        const int64_t off = (int64_t)p * r->page_pairs;
        if (pairs_out)
            SJ_CK(cudaMemcpyAsync(pairs_out + 2 * off, r->pair_pages[p], (size_t)cnt * 2 * sizeof(int32_t),
                                  cudaMemcpyDefault, ri->stream));
        if (dist_out && r->has_distances && r->dist_pages)
            SJ_CK(cudaMemcpyAsync(dist_out + off, r->dist_pages[p], (size_t)cnt * sizeof(double), cudaMemcpyDefault,
                                  ri->stream));
        left -= cnt;
    }
    SJ_CK(cudaStreamSynchronize(ri->stream));
    return SJ_OK;
}

void sj_result_free(sj_result* r) {
    if (!r) return;
    free_result_impl(static_cast<ResultImpl*>(r->internal));
    memset(r, 0, sizeof *r);
}

void sj_results_free(sj_result* results, int32_t count) {
    if (!results) return;
    for (int32_t k = 0; k < count; ++k) sj_result_free(&results[k]);
}

int sj_join(const double* pts, int64_t n, int32_t d, double eps, const sj_options* opt, void* stream,
            sj_result* out) {
    sj_handle h = nullptr;
    int st = sj_build_index(pts, n, d, eps, opt, stream, &h);
    if (st != SJ_OK) return st;
    st = sj_self_join(h, out);
    sj_destroy(h);
    return st;
}

int sj_join_batch(const double* const* pts, const int64_t* n, const int32_t* d, const double* eps, int32_t count,
                  const sj_options* opt, void* stream, sj_result* per_instance_out) {
    clear_error();
    return join_batch_impl(pts, n, d, eps, count, opt, stream, per_instance_out, nullptr);
}

}  // extern "C"

namespace sj {

// The join phase of a batched join: per group the counter reset, the
// distance-tile launch between its two timing events and the recheck launch.
// With `graph`, the phase is captured on a private stream into one CUDA graph
// (the tensor-core groups on one branch, the CUDA-core groups on another, so
// a group's tail overlaps the other branch) and launched on `s`; otherwise the
// launches go to `s` in group order.
static int batch_join_phase(std::vector<std::unique_ptr<BatchGroup>>& groups, const std::vector<JoinOut>& jos,
                            int32_t* table, long long table_slots, unsigned long long* cursor, int count, bool dist,
                            bool graph, cudaStream_t s) {
    auto launch_group = [&](size_t gi, cudaStream_t gs) -> int {
        BatchGroup& g = *groups[gi];
        Index* ix = &g.ix;
        if (ix->n_items == 0) return SJ_OK;
        const cudaStream_t keep = ix->stream;
        ix->stream = gs;
        int st = SJ_OK;
        // inside a capture, only an external record becomes a timing node of the graph
        const unsigned rec = graph ? cudaEventRecordExternal : cudaEventRecordDefault;
        cudaError_t e = cudaMemsetAsync(ix->counters, 0, kCounters * sizeof(unsigned long long), gs);
        if (e == cudaSuccess) e = cudaEventRecordWithFlags(ix->ev_tile[0], gs, rec);
        if (e != cudaSuccess) {
            set_error("batch group launch: %s", cudaGetErrorString(e));
            st = SJ_ERR_CUDA;
        }
        if (st == SJ_OK)
            st = is_tensor_kernel(ix->kernel) ? launch_join_tc(ix, jos[gi], dist ? 1 : 0)
                                              : launch_join_cc(ix, jos[gi], dist ? 1 : 0);
        if (st == SJ_OK && cudaEventRecordWithFlags(ix->ev_tile[1], gs, rec) != cudaSuccess) st = SJ_ERR_CUDA;
        if (st == SJ_OK) st = launch_recheck(ix, jos[gi], dist ? 1 : 0);
        ix->stream = keep;
        return st;
    };
    auto reset = [&](cudaStream_t rs) -> int {
        SJ_CK(cudaMemsetAsync(table, 0xFF, table_slots * sizeof(int32_t), rs));
        SJ_CK(cudaMemsetAsync(cursor, 0, (count + 2) * sizeof(unsigned long long), rs));
        return SJ_OK;
    };
    if (!graph) {
        SJ_TRY(reset(s));
        for (size_t gi = 0; gi < groups.size(); ++gi) SJ_TRY(launch_group(gi, s));
        return SJ_OK;
    }
    cudaStream_t cs = nullptr, br[2] = {nullptr, nullptr};
    cudaEvent_t fork = nullptr, join[2] = {nullptr, nullptr};
    cudaGraph_t gr = nullptr;
    cudaGraphExec_t ex = nullptr;
    int st = SJ_OK;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = cudaStreamCreateWithFlags(&br[b], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = cudaEventCreateWithFlags(&join[b], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        set_error("batch graph set-up: %s", cudaGetErrorString(e));
        st = SJ_ERR_CUDA;
    }
    bool capturing = false;
    if (st == SJ_OK) {
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            set_error("batch graph capture: %s", cudaGetErrorString(e));
            st = SJ_ERR_CUDA;
        } else {
            capturing = true;
        }
    }
    if (st == SJ_OK) st = reset(cs);
    if (st == SJ_OK) {
        e = cudaEventRecord(fork, cs);
        for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = cudaStreamWaitEvent(br[b], fork, 0);
        if (e != cudaSuccess) st = SJ_ERR_CUDA;
    }
    for (size_t gi = 0; gi < groups.size() && st == SJ_OK; ++gi)
        st = launch_group(gi, br[is_tensor_kernel(groups[gi]->ix.kernel) ? 0 : 1]);
    if (st == SJ_OK) {
        for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
            e = cudaEventRecord(join[b], br[b]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, join[b], 0);
        }
        if (e != cudaSuccess) st = SJ_ERR_CUDA;
    }
    if (capturing) {
        e = cudaStreamEndCapture(cs, &gr);
        if (st == SJ_OK && e != cudaSuccess) {
            set_error("batch graph capture: %s", cudaGetErrorString(e));
            st = SJ_ERR_CUDA;
        }
    }
    if (st == SJ_OK) {
        e = cudaGraphInstantiate(&ex, gr, 0);
        if (e == cudaSuccess) e = cudaGraphLaunch(ex, s);
        if (e != cudaSuccess) {
            set_error("batch graph launch: %s", cudaGetErrorString(e));
            st = SJ_ERR_CUDA;
        }
    }
    if (st != SJ_OK) cudaGetLastError();
    // the executable graph may be destroyed while its launch is in flight
    if (ex) cudaGraphExecDestroy(ex);
    if (gr) cudaGraphDestroy(gr);
    for (int b = 0; b < 2; ++b) {
        if (join[b]) cudaEventDestroy(join[b]);
        if (br[b]) cudaStreamDestroy(br[b]);
    }
    if (fork) cudaEventDestroy(fork);
    if (cs) cudaStreamDestroy(cs);
    return st;
}

int join_batch_impl(const double* const* pts, const int64_t* n, const int32_t* d, const double* eps, int32_t count,
                    const sj_options* opt, void* stream, sj_result* per_instance_out,
                    const std::vector<TuneEntry>* forced) {
    if (!pts || !n || !d || !eps || !per_instance_out || count < 1) {
        set_error("invalid batch arguments");
        return SJ_ERR_ARG;
    }
    for (int32_t k = 0; k < count; ++k) {
        if (!pts[k] || n[k] < 1 || n[k] > 0x7FFFFFFFll || d[k] < 1 || d[k] > SJ_MAX_D || !(eps[k] > 0) ||
            !isfinite(eps[k])) {
            set_error("invalid batch instance %d: n=%lld d=%d eps=%g", (int)k, (long long)n[k], (int)d[k], eps[k]);
            return SJ_ERR_ARG;
        }
        memset(&per_instance_out[k], 0, sizeof(sj_result));
    }
    sj_options o;
    sj_default_options(&o);
    if (opt) o = *opt;
    if (o.kernel != SJ_KERNEL_AUTO && o.kernel != SJ_KERNEL_FILTER_F32 && o.kernel != SJ_KERNEL_FP64_FMA &&
        o.kernel != SJ_KERNEL_FILTER_BF16X3 && o.kernel != SJ_KERNEL_FILTER_BF16X2 &&
        o.kernel != SJ_KERNEL_FILTER_FP16X2) {
        set_error("batched joins run the FP32 filter, the tensor-core filter or the FP64 CUDA-core kernel (got "
                  "kernel %d)", o.kernel);
        return SJ_ERR_UNSUPPORTED;
    }
    // AUTO: the tensor-core filter (FP16x2: each instance's coordinates are
    // scaled by its own power of two) for padded dimensions 8 .. 64
    // (measured on uniform instances with the batched grid choice: d 8 1.7x,
    // d 16 4x, d 32 12x faster than the FP32 filter), else the FP32 CUDA-core
    // filter
    std::vector<TuneEntry> tuned;
    if (o.kernel == SJ_KERNEL_AUTO && o.tune_cache && o.tune_cache[0]) {
        const int ts = tune_load(o.tune_cache, &tuned);
        if (ts != SJ_OK) return ts;
    }
    // a group's configuration: a forced entry (tuning runs), else a tuned
    // entry of the cache (AUTO), else the options
    auto group_entry = [&](int dp) -> const TuneEntry* {
        const TuneEntry* e = forced ? tune_find_group(*forced, dp) : nullptr;
        if (!e && !tuned.empty()) e = tune_find_group(tuned, dp);
        if (!e || e->kernel == SJ_KERNEL_AUTO || e->kernel == SJ_KERNEL_FP64_DMMA) return nullptr;
        if (is_tensor_kernel(e->kernel) && dp > 64) return nullptr;
        return e;
    };
    auto group_kernel = [&](int dp) {
        if (const TuneEntry* e = group_entry(dp)) return e->kernel;
        if (o.kernel != SJ_KERNEL_AUTO) return o.kernel;
        return (dp >= 8 && dp <= 64) ? SJ_KERNEL_FILTER_FP16X2 : SJ_KERNEL_FILTER_F32;
    };
    for (int32_t k = 0; k < count; ++k)
        if (is_tensor_kernel(group_kernel(round_dim(d[k]))) && round_dim(d[k]) > 64) {
            set_error("the tensor-core filter supports d <= 64 (instance %d has d = %d)", (int)k, (int)d[k]);
            return SJ_ERR_UNSUPPORTED;
        }
    std::vector<int> inst_kernel(count), inst_group(count);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0;
    SJ_CK(cudaGetDevice(&dev));
    const bool dist = o.emit_distances != 0;

    // ---- groups by padded dimension; host inputs are staged on the device ----
    std::vector<double*> staged;
    std::vector<std::unique_ptr<BatchGroup>> groups;
    int st = SJ_OK;
    auto cleanup = [&]() {
        for (auto& g : groups) {
            release_index(&g->ix);
            dev_free(g->d_off, s);
            dev_free(g->d_gid, s);
            dev_free(g->d_e2, s);
            dev_free(g->d_r2, s);
            dev_free(g->d_inst_of_sorted, s);
            dev_free(g->d_item_inst, s);
        }
        for (double* p : staged) dev_free(p, s);
        cudaStreamSynchronize(s);
    };
    {
        std::vector<int> order(count);
        for (int k = 0; k < count; ++k) order[k] = k;
        std::stable_sort(order.begin(), order.end(),
                         [&](int a, int b) { return round_dim(d[a]) < round_dim(d[b]); });
        size_t i = 0;
        while (i < order.size() && st == SJ_OK) {
            const int dp = round_dim(d[order[i]]);
            auto g = std::make_unique<BatchGroup>();
            g->ix.device = dev;
            g->ix.stream = s;
            g->ix.opt = o;
            if (const TuneEntry* te = group_entry(dp)) g->ix.opt.queries_per_item = te->qpi;
            g->ix.kernel = group_kernel(dp);
            g->ix.d = dp;
            g->ix.dp = dp;
            g->off.push_back(0);
            std::vector<const double*> src;
            std::vector<int32_t> dof;
            for (; i < order.size() && round_dim(d[order[i]]) == dp; ++i) {
                const int k = order[i];
                const double* p = pts[k];
                if (!is_device_pointer(p)) {
                    double* c = nullptr;
                    st = dev_alloc_t(&c, (size_t)n[k] * d[k], s);
                    if (st != SJ_OK) break;
                    staged.push_back(c);
                    cudaError_t e = cudaMemcpyAsync(c, p, (size_t)n[k] * d[k] * sizeof(double),
                                                    cudaMemcpyHostToDevice, s);
                    if (e != cudaSuccess) {
                        set_error("host-to-device copy: %s", cudaGetErrorString(e));
                        st = SJ_ERR_CUDA;
                        break;
                    }
                    p = c;
                }
                src.push_back(p);
                dof.push_back(d[k]);
                g->gids.push_back(k);
                inst_kernel[k] = group_kernel(dp);
                inst_group[k] = (int)groups.size();
                g->eps.push_back(eps[k]);
                g->off.push_back(g->off.back() + n[k]);
            }
            if (st != SJ_OK) break;
            g->n_inst = (int)g->gids.size();
            g->ix.n = g->off.back();
            if (g->ix.n > 0x7FFFFFFFll) {
                set_error("a batch group holds more than 2^31 - 1 points");
                st = SJ_ERR_ARG;
                break;
            }
            st = build_batch_group(g.get(), src.data(), dof.data());
            if (st == SJ_OK) st = dev_alloc_t(&g->d_gid, (size_t)g->n_inst, s);
            if (st == SJ_OK) {
                cudaError_t e = cudaMemcpyAsync(g->d_gid, g->gids.data(), g->n_inst * sizeof(int32_t),
                                                cudaMemcpyHostToDevice, s);
                if (e != cudaSuccess) st = SJ_ERR_CUDA;
            }
            groups.push_back(std::move(g));
        }
    }
    if (st != SJ_OK) {
        cleanup();
        return st;
    }

    // ---- output: per-instance page tables over one shared pool ----
    int64_t page_pairs = o.page_pairs > 0 ? o.page_pairs : (int64_t(1) << 16);
    int page_log2 = 6;  // at least 64 pairs a page (one claiming lane per page in a warp's flush)
    while ((int64_t(1) << page_log2) < page_pairs) ++page_log2;
    page_pairs = int64_t(1) << page_log2;
    std::vector<int64_t> cand(count, 0), eval(count, 0);
    for (auto& g : groups)
        for (int i = 0; i < g->n_inst; ++i) {
            cand[g->gids[i]] = g->cand[i];
            eval[g->gids[i]] = g->eval[i];
        }
    std::vector<long long> toff(count + 1, 0);
    std::vector<int32_t> maxp(count);
    for (int k = 0; k < count; ++k) {
        const long long bound = std::min<long long>(cand[k], (long long)n[k] * n[k]);
        maxp[k] = (int32_t)((bound + page_pairs - 1) / page_pairs);
        toff[k + 1] = toff[k] + maxp[k];
    }
    // every page is claimed once, so the exact counts fill exactly this many
    auto pool_pages_for = [&](const std::vector<long long>& want) {
        long long pages = 0;
        for (int k = 0; k < count; ++k) pages += (want[k] + page_pairs - 1) / page_pairs;
        return std::max<long long>(pages, 1);
    };
    std::vector<long long> want(count);
    for (int k = 0; k < count; ++k)
        want[k] = o.max_pairs_hint > 0 ? o.max_pairs_hint / count : std::min<long long>(cand[k], 64ll * n[k]);
    long long n_pages = pool_pages_for(want);

    int32_t* table = nullptr;
    long long* dtoff = nullptr;
    int32_t* dmaxp = nullptr;
    unsigned long long* cursor = nullptr;  // count cursors, pool_next, error flag
    BatchJoin* dbj = nullptr;
    std::shared_ptr<PoolHolder> pool;
    auto free_meta = [&]() {
        dev_free(table, s);
        dev_free(dtoff, s);
        dev_free(dmaxp, s);
        dev_free(cursor, s);
        dev_free(dbj, s);
    };
    if ((st = dev_alloc_t(&table, (size_t)std::max<long long>(toff[count], 1), s)) == SJ_OK &&
        (st = dev_alloc_t(&dtoff, (size_t)count, s)) == SJ_OK && (st = dev_alloc_t(&dmaxp, (size_t)count, s)) == SJ_OK &&
        (st = dev_alloc_t(&cursor, (size_t)count + 2, s)) == SJ_OK &&
        (st = dev_alloc_t(&dbj, groups.size(), s)) == SJ_OK) {
        cudaError_t e = cudaMemcpyAsync(dtoff, toff.data(), count * sizeof(long long), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dmaxp, maxp.data(), count * sizeof(int32_t), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) st = SJ_ERR_CUDA;
    }
    std::vector<unsigned long long> cur(count + 2, 0);
    int reruns = 0;
    std::vector<double> group_ms;
    for (int attempt = 0; attempt < 3 && st == SJ_OK; ++attempt) {
        pool = std::make_shared<PoolHolder>();
        pool->stream = s;
        st = dev_alloc_t(&pool->block, (size_t)n_pages * page_pairs * 2, s);
        if (st == SJ_OK && dist) st = dev_alloc_t(&pool->dblock, (size_t)n_pages * page_pairs, s);
        if (st != SJ_OK) break;
        cudaError_t e = cudaSuccess;
        std::vector<BatchJoin> hbj(groups.size());
        std::vector<JoinOut> jos(groups.size());
        std::vector<int2*> bands(groups.size(), nullptr);
        for (size_t gi = 0; gi < groups.size() && st == SJ_OK; ++gi) {
            BatchGroup& g = *groups[gi];
            BatchJoin bj{};
            bj.item_inst = g.d_item_inst;
            bj.inst_of_sorted = g.d_inst_of_sorted;
            bj.inst_off = g.d_off;
            bj.inst_gid = g.d_gid;
            bj.inst_e2 = g.d_e2;
            bj.inst_r2 = g.d_r2;
            bj.pool = reinterpret_cast<int2*>(pool->block);
            bj.dpool = pool->dblock;
            bj.page_log2 = page_log2;
            bj.n_pages = n_pages;
            bj.pool_next = cursor + count;
            bj.page_table = table;
            bj.table_off = dtoff;
            bj.max_pages = dmaxp;
            bj.cursor = cursor;
            bj.error = cursor + count + 1;
            hbj[gi] = bj;
            Index* ix = &g.ix;
            if (ix->n_items == 0) continue;
            const unsigned long long ev = (unsigned long long)std::max<int64_t>(ix->n_evaluated, 1);
            unsigned long long band_cap =
                std::min<unsigned long long>(ev, std::max<unsigned long long>(1ull << 20, dist ? ev / 8 : ev / 64));
            if ((st = dev_alloc_t(&bands[gi], (size_t)band_cap, s)) != SJ_OK) break;
            jos[gi].band = bands[gi];
            jos[gi].band_cap = band_cap;
            jos[gi].batch = dbj + gi;
            if (!ix->ev_tile[0]) {
                e = cudaEventCreate(&ix->ev_tile[0]);
                if (e == cudaSuccess) e = cudaEventCreate(&ix->ev_tile[1]);
                if (e != cudaSuccess) {
                    set_error("batch events: %s", cudaGetErrorString(e));
                    st = SJ_ERR_CUDA;
                }
            }
        }
        if (st == SJ_OK) {
            e = cudaMemcpyAsync(dbj, hbj.data(), hbj.size() * sizeof(BatchJoin), cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) {
                set_error("batch routing copy: %s", cudaGetErrorString(e));
                st = SJ_ERR_CUDA;
            }
        }
        if (st == SJ_OK)
            st = batch_join_phase(groups, jos, table, std::max<long long>(toff[count], 1), cursor, count, dist,
                                  o.graph != 0, s);
        for (int2* b : bands) dev_free(b, s);
        if (st != SJ_OK) break;
        e = cudaMemcpyAsync(cur.data(), cursor, (count + 2) * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            set_error("batch join: %s", cudaGetErrorString(e));
            st = SJ_ERR_CUDA;
            break;
        }
        bool timed_out = false;
        group_ms.assign(groups.size(), 0.0);
        for (size_t gi = 0; gi < groups.size(); ++gi) {
            auto& g = groups[gi];
            float ms = 0.f;
            if (g->ix.n_items > 0) {
                if (cudaEventElapsedTime(&ms, g->ix.ev_tile[0], g->ix.ev_tile[1]) == cudaSuccess)
                    group_ms[gi] = ms;
                else
                    cudaGetLastError();  // no timing: not an error of the join
            }
            if (is_tensor_kernel(g->ix.kernel) && g->ix.n_items > 0) {
                unsigned long long flag = 0;  // the tensor-core kernel's bounded-wait flag
                if (cudaMemcpy(&flag, g->ix.counters + 4, sizeof flag, cudaMemcpyDeviceToHost) != cudaSuccess ||
                    flag != 0)
                    timed_out = true;
            }
        }
        if (timed_out) {
            set_error("a bounded wait of the tensor-core filter expired");
            st = SJ_ERR_TIMEOUT;
            break;
        }
        if (cur[count + 1] != 0) {
            set_error("a wait for a result page claim expired");
            st = SJ_ERR_TIMEOUT;
            break;
        }
        bool overflow = cur[count] > (unsigned long long)n_pages;
        int bad = -1;
        for (int k = 0; k < count && bad < 0; ++k)
            if (cur[k] > (unsigned long long)maxp[k] * (unsigned long long)page_pairs) bad = k;
        if (bad >= 0) {  // a count above the instance's candidate count: cannot happen
            set_error("instance %d emitted %llu pairs, above its %lld candidates", bad, cur[bad],
                      (long long)cand[bad]);
            st = SJ_ERR_CUDA;
            break;
        }
        if (!overflow) break;
        if (attempt == 2) {
            set_error("batched result larger than its page pool (%llu pages wanted, %lld held)", cur[count],
                      n_pages);
            st = SJ_ERR_RESULT_OVERFLOW;
            break;
        }
        // regrow to the exact counts and run the joins once more
        for (int k = 0; k < count; ++k) want[k] = (long long)cur[k];
        n_pages = pool_pages_for(want);
        reruns = attempt + 1;
    }
    if (st != SJ_OK) {
        free_meta();
        pool.reset();
        cleanup();
        return st;
    }
    std::vector<int32_t> htable((size_t)std::max<long long>(toff[count], 1));
    if (cudaMemcpyAsync(htable.data(), table, htable.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        set_error("batch page table read-back failed");
        free_meta();
        pool.reset();
        cleanup();
        return SJ_ERR_CUDA;
    }
    for (int k = 0; k < count; ++k) {
        ResultImpl* ri = new (std::nothrow) ResultImpl();
        if (!ri) {
            for (int j = 0; j < k; ++j) sj_result_free(&per_instance_out[j]);
            free_meta();
            pool.reset();
            cleanup();
            return SJ_ERR_OOM;
        }
        ri->stream = s;
        ri->shared_pool = pool;
        const long long cnt = (long long)cur[k];
        const long long used = std::min<long long>((cnt + page_pairs - 1) / page_pairs, maxp[k]);
        for (long long i = 0; i < used; ++i) {
            const int32_t pg = htable[(size_t)(toff[k] + i)];
            if (pg < 0) break;  // (only after an overflow)
            ri->pair_pages.push_back(pool->block + (size_t)pg * page_pairs * 2);
            if (dist) ri->dist_pages.push_back(pool->dblock + (size_t)pg * page_pairs);
        }
        sj_result& r = per_instance_out[k];
        r.count = cnt;
        r.page_pairs = page_pairs;
        r.n_pages = (int32_t)ri->pair_pages.size();
        r.has_distances = dist ? 1 : 0;
        r.pair_pages = ri->pair_pages.data();
        r.dist_pages = dist ? ri->dist_pages.data() : nullptr;
        r.n_candidates = cand[k];
        r.n_evaluated = eval[k];
        r.n_rechecked = 0;
        r.reruns = reruns;
        r.kernel = inst_kernel[k];
        r.ms_tile = group_ms.empty() ? 0.0 : group_ms[inst_group[k]];
        r.internal = ri;
    }
    free_meta();
    pool.reset();
    cleanup();
    return st;
}

}  // namespace sj
