/*
 * simjoin.h — C ABI of libsj, a GB300 (sm_103a) Euclidean distance
 * similarity self-join.
 *
 * The operation (Sec. II-A, Eq. 1 of "Leveraging GPU Tensor Cores for Double
 * Precision Euclidean Distance Calculations", Gallet and Gowanlock): given a
 * set V of n points in d dimensions and a distance eps, return every ordered
 * pair (i, j) of V x V with dist(x_i, x_j) <= eps, where dist is the
 * Euclidean distance.  Self pairs (i, i) and both orders (i, j), (j, i) are
 * part of the result (the selectivity of Sec. IV-A, (|R| - |V|) / |V|,
 * counts each point finding itself).
 *
 * Decision rule, fixed for every kernel: with e2 = eps * eps rounded once in
 * binary64 and s = sum_k (x_ik - x_jk)^2 evaluated in binary64 in dimension
 * order, each subtraction, product and sum rounded separately, (i, j) belongs
 * to the result iff s <= e2, and its distance is sqrt(s) correctly rounded.
 * Kernels that compute distances another way (the expanded form of Eq. 3,
 * low-precision tensor-core products) certify each decision with an error
 * bound and re-decide every pair inside the bound with exactly this rule, so
 * every kernel returns the same set.
 *
 * Method (Sec. III): points are indexed by a grid of cells of side >= eps
 * (Sec. III-B); queries of one cell share their candidate set, the points of
 * the 3^m adjacent cells; candidate distances are evaluated in tiles as
 * ||a||^2 + ||b||^2 - 2 a.b (Eq. 3, Eq. 4, Fig. 2).
 *
 * Conventions for every entry point:
 *  - Return value: SJ_OK (0) or a negative SJ_ERR_* status.  Nothing is
 *    thrown across the ABI.  sj_error_string() names a status;
 *    sj_last_error_message() gives detail for the calling thread's last error.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  All device work of a handle runs on the stream given at
 *    sj_build_index.
 *  - Pointers documented "host or device" may point to either kind of memory;
 *    the library detects which (unified addressing).
 *  - Indices are int32: n must be below 2^31.
 */
#ifndef SIMJOIN_H
#define SIMJOIN_H

#include <stdint.h>

#if defined(__GNUC__)
#define SJ_API __attribute__((visibility("default")))
#else
#define SJ_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define SJ_OK 0
#define SJ_ERR_ARG (-1)             /* invalid argument: n < 1, n >= 2^31, d < 1,
                                       d > SJ_MAX_D, eps <= 0 / NaN / Inf,
                                       non-finite coordinate, NULL pointer */
#define SJ_ERR_OOM (-2)             /* device or host allocation failed */
#define SJ_ERR_RESULT_OVERFLOW (-3) /* result larger than the page pool even
                                       after the automatic regrowth; count is
                                       still exact */
#define SJ_ERR_TIMEOUT (-4)         /* a bounded device wait ran out */
#define SJ_ERR_CUDA (-5)            /* a CUDA runtime or driver call failed */
#define SJ_ERR_UNSUPPORTED (-6)     /* kernel / shape combination not built */

#define SJ_MAX_D 128

/* ---- distance kernels -------------------------------------------------- */
#define SJ_KERNEL_AUTO 0        /* single joins: SJ_KERNEL_FILTER_FP16X2 for
                                   9 <= d <= 64, else SJ_KERNEL_FILTER_F32
                                   (SJ_KERNEL_FP64_FMA for an extent that
                                   scaled binary32 coordinates cannot hold)
                                   (batched joins: see sj_join_batch) */
#define SJ_KERNEL_FP64_FMA 1    /* FP64 CUDA-core FMA tiles (expanded form,
                                   Eq. 3) + direct-form recheck of the band */
#define SJ_KERNEL_FP64_DMMA 2   /* FP64 tensor-core tiles, mma.sync m8n8k4
                                   f64 (the paper's FP64 MMA, Fig. 2) */
#define SJ_KERNEL_FILTER_F32 3  /* FP32 CUDA-core filter with certified bound,
                                   FP64 direct recheck of the band.  The
                                   binary32 filters (this and the tensor-core
                                   ones) work on coordinates scaled by a power
                                   of two into binary32's range; an extent
                                   outside it (squared half-extent below about
                                   2^-970) gives SJ_ERR_UNSUPPORTED */
#define SJ_KERNEL_FILTER_BF16X3 4 /* tcgen05 kind::f16 with 3-term bf16 split
                                     operands (6 products per dim), FP32
                                     accumulation in TMEM, certified bound,
                                     FP64 recheck; d <= 64 */
#define SJ_KERNEL_FILTER_BF16X2 5 /* as BF16X3 with a 2-term split (3 products
                                     per dim: half the K, a slightly wider
                                     certified band); d <= 64 */
#define SJ_KERNEL_FILTER_FP16X2 6 /* as BF16X2 with fp16 terms (11 significant
                                     bits each) of the kernel coordinates
                                     scaled by a power of two into fp16's
                                     range: the same K, a narrower certified
                                     band; d <= 64 */

/* ---- options ----------------------------------------------------------- */
#define SJ_NO_INDEX (-1)        /* sj_options.indexed_dims: brute force */
typedef struct sj_options {
    int32_t kernel;           /* SJ_KERNEL_* */
    int32_t emit_distances;   /* 1: also return the FP64 distance of every
                                 pair (direct form, bit-identical to the
                                 decision rule's sqrt(s)) */
    int32_t indexed_dims;     /* m, the number of dims the grid indexes
                                 (Sec. II-D: an index on fewer dims than d);
                                 0 = automatic; SJ_NO_INDEX = no index: all
                                 points form one cell and every pair is
                                 evaluated by the same tile kernels (the
                                 brute-force comparison of Sec. IV, Fig. 3) */
    int32_t symmetric;        /* 1: evaluate each unordered pair of adjacent
                                 cells once and emit both orders (halves the
                                 distance work); 0: every query cell scans its
                                 full 3^m neighbourhood as in Sec. III-B */
    int32_t queries_per_item; /* queries per work item (a cell's queries are
                                 split into items of at most this many; the
                                 query tile of the tensor-core filter);
                                 0 = automatic (the kernel's maximum: 16 for
                                 the CUDA-core kernels, 248 or 120 for the
                                 tensor-core filter) */
    int32_t graph;            /* batched joins: 1 = the join phase (every
                                 group's tile and recheck launches) runs as one
                                 CUDA graph, captured per call on a private
                                 stream with the tensor-core groups and the
                                 CUDA-core groups on two parallel branches, and
                                 launched on the caller's stream; 0 = plain
                                 launches on the stream, group after group.
                                 Ignored by single joins. */
    int64_t page_pairs;       /* pairs per result page; 0 = 1 << 22 */
    int64_t max_pairs_hint;   /* expected result size; 0 = automatic */
    const char* tune_cache;   /* NULL, or the path of a tuning cache written by
                                 sj_autotune / sj_autotune_batch.  With kernel
                                 AUTO, a matching entry supplies the kernel and
                                 (where the options leave them 0) the queries
                                 per item and the indexed dims: for a single
                                 join the entry of the same d whose
                                 round(log2 n) is nearest, within 1; for a
                                 batched join, per group, the entry of the
                                 group's padded dimension.  A missing file is
                                 an empty cache. */
    int32_t short_circuit;    /* SJ_KERNEL_FP64_FMA with d > 8: 1 = order the
                                 kernel coordinates' dims by decreasing variance
                                 (Sec. II-D) and stop a warp's distance tile
                                 after a block of 8 dims once every pair of it
                                 is certainly out (Sec. III-B); the result set
                                 is unchanged.  0 (default) = every tile runs
                                 all dims.  Ignored by the other kernels. */
} sj_options;

/* Fills *opt with the defaults (kernel AUTO, no distances, automatic m,
 * symmetric, automatic item size and pool, no graph, no tuning cache). */
SJ_API void sj_default_options(sj_options* opt);

/* ---- index ------------------------------------------------------------- */
typedef struct sj_index* sj_handle;

/*
 * Builds the grid index of Sec. III-B for `n` points of dimension `d`
 * (row-major, binary64, `pts` host or device, owned by the caller and not
 * retained) and distance `eps`: per-dim extent, cell keys of the m indexed
 * dims, radix sort by key, cell table, points packed in cell order with their
 * norms, and the list of work items (query ranges with their candidate
 * ranges).  `opt` may be NULL (defaults).  On success *out is a new handle,
 * to be released with sj_destroy.  Errors: SJ_ERR_ARG (see above, including a
 * non-finite coordinate), SJ_ERR_OOM, SJ_ERR_CUDA.
 */
SJ_API int sj_build_index(const double* pts, int64_t n, int32_t d, double eps, const sj_options* opt,
                   void* stream, sj_handle* out);

/* Releases a handle and its device memory (after its stream's work). */
SJ_API void sj_destroy(sj_handle h);

/* Sizes of a built index: non-empty cells, work items, indexed dims m,
 * candidate pairs of the full neighbourhoods (ordered, self included),
 * pair evaluations the join performs.  Any output pointer may be NULL. */
SJ_API int sj_index_info(sj_handle h, int64_t* n_cells, int64_t* n_items, int32_t* m, int64_t* n_candidates,
                  int64_t* n_evaluated);

/* ---- join -------------------------------------------------------------- */
typedef struct sj_result {
    int64_t count;            /* |R|, exact */
    int64_t page_pairs;       /* pairs per page */
    int32_t n_pages;          /* pages holding pairs [0, count) */
    int32_t has_distances;
    int32_t* const* pair_pages; /* host array of n_pages device pointers; page p
                                   holds pairs p*page_pairs .. as (i, j) int32
                                   in original input indices */
    double* const* dist_pages;  /* NULL, or host array of n_pages device
                                   pointers to the matching FP64 distances */
    int64_t n_candidates;     /* candidate pairs of the full neighbourhoods */
    int64_t n_evaluated;      /* pair evaluations performed by the kernel: the
                                 index's scheduled evaluations less those the
                                 FP32 filter's bounding-box prune (padded
                                 d <= 8) removed; batched results report the
                                 scheduled evaluations */
    int64_t n_rechecked;      /* pairs re-decided by the FP64 direct form */
    int32_t reruns;           /* reruns after the page pool overflowed */
    int32_t kernel;           /* SJ_KERNEL_* actually used */
    double ms_tile;           /* device time of the distance-tile kernel of the
                                 (last) run, from CUDA events recorded on the
                                 handle's stream around its launch */
    void* internal;           /* library-owned */
} sj_result;

/*
 * Runs the self-join on a built index (Sec. III: for every work item, the
 * distance tile between its queries and candidates, the eps threshold and a
 * warp-aggregated compaction into the paged result buffer).  Work is queued
 * on the handle's stream; the call returns once the result count is known
 * (one device-to-host read of the count).  Pages stay on the device until
 * sj_result_copy.  When the pool is too small the join is rerun once with a
 * pool of the exact size (result->reruns).  *out must be released with
 * sj_result_free.  Errors: SJ_ERR_OOM, SJ_ERR_CUDA, SJ_ERR_UNSUPPORTED,
 * SJ_ERR_RESULT_OVERFLOW (count valid, pages hold a prefix).
 */
SJ_API int sj_self_join(sj_handle h, sj_result* out);

/*
 * Copies the pairs (2 * count int32, (i, j) interleaved) to `pairs_out` and,
 * when the result has them and `dist_out` is not NULL, the distances
 * (count doubles) to `dist_out`; both host or device.  The order of pairs is
 * unspecified.  Synchronous with respect to the host.
 */
SJ_API int sj_result_copy(const sj_result* r, int32_t* pairs_out, double* dist_out);

/* Releases a result's pages (NULL-safe, idempotent). */
SJ_API void sj_result_free(sj_result* r);

/* Releases `count` results in one call (e.g. the results of sj_join_batch). */
SJ_API void sj_results_free(sj_result* results, int32_t count);

/*
 * Results larger than device memory.  Runs the self-join of a built index
 * (the kernel and decision rule of sj_self_join, without distances) in
 * rounds over consecutive ranges of work items; each round's pairs land in
 * one of two device buffers of `device_pairs` pairs (at least 1024) and are
 * copied to `host_pairs` on a second stream while the next round runs
 * (overlapped when host_pairs is pinned).  The range of the next round is
 * sized from the last round's pairs per work item to fill about 3/4 of a
 * buffer; a round whose pairs do not fit is run again on half its range.
 * The paper batches its result transfers for the same reason (Sec. III-B).
 *
 *   host_pairs     host memory with room for host_capacity pairs, (i, j) int32
 *                  interleaved, input indices, unspecified order
 *   count_out      |R|, exact even when it exceeds host_capacity (then
 *                  SJ_ERR_RESULT_OVERFLOW is returned and host_pairs holds
 *                  host_capacity of the pairs)
 *   rounds_out     rounds run (may be NULL)
 *
 * Device memory used beyond the index: 2 x device_pairs x 8 bytes plus the
 * recheck queue.  Synchronous with respect to the host.  Errors: SJ_ERR_ARG
 * (NULL handle or count_out, device memory for host_pairs, device_pairs <
 * 1024), SJ_ERR_RESULT_OVERFLOW (also when a single work item yields more
 * than device_pairs pairs; count_out is then 0), SJ_ERR_OOM, SJ_ERR_CUDA,
 * SJ_ERR_TIMEOUT.
 */
SJ_API int sj_self_join_to_host(sj_handle h, int32_t* host_pairs, int64_t host_capacity, int64_t device_pairs,
                                int64_t* count_out, int32_t* rounds_out);

/* ---- sharding one join over several GPUs (Sec. III-B) -------------------- */
/*
 * The queries of one grid cell, with the candidate runs of its
 * neighbourhood, are an independent unit: every GPU can build the index from
 * the same points and run a contiguous range of whole cells; the union of
 * the ranges' results is the join.  The cells, their order and the work
 * items' positions are the same in every build; the order of the points
 * inside a cell is not, so a cell split into several work items must not be
 * split across GPUs: shards are ranges of whole cells.
 *
 * sj_index_item_work: per work item (n_items int64, host memory; n_items
 * from sj_index_info), the pair evaluations of its whole cell (as the tile
 * kernels perform them) at the cell's first item, 0 at the cell's other
 * items.  The sum is the index's n_evaluated.
 *
 * sj_shard_bounds: host only (no GPU needed).  Splits items [0, n_items)
 * into n_shards contiguous ranges [bounds[k], bounds[k + 1]) of about equal
 * total work: boundary k is the item boundary whose work prefix is nearest
 * to k / n_shards of the total, moved past items of no work (so with the
 * work of sj_index_item_work every boundary is the first item of a cell).
 * bounds: n_shards + 1 int64; bounds[0] = 0, bounds[n_shards] = n_items,
 * non-decreasing.  A pure function of its inputs, so every rank computes
 * the same partition.  Errors: SJ_ERR_ARG.
 *
 * sj_self_join_range: sj_self_join restricted to work items [item_begin,
 * item_end) (pairs of the items' queries, both orders of mirrored pairs, as
 * in the full join); n_candidates and n_evaluated of the result are those of
 * the whole index.  Errors: those of sj_self_join, SJ_ERR_ARG for a range
 * outside [0, n_items].
 */
SJ_API int sj_index_item_work(sj_handle h, int64_t* work_out);
SJ_API int sj_shard_bounds(const int64_t* item_work, int64_t n_items, int32_t n_shards, int64_t* bounds);
SJ_API int sj_self_join_range(sj_handle h, int64_t item_begin, int64_t item_end, sj_result* out);

/* Convenience: build + join + destroy in one call. */
SJ_API int sj_join(const double* pts, int64_t n, int32_t d, double eps, const sj_options* opt, void* stream,
            sj_result* out);

/*
 * Failure-detection self-test (no counterpart in the paper): launches a
 * kernel whose thread waits on a shared-memory mbarrier that nothing arrives
 * on, with the same bounded wait the tensor-core filter uses (here 2^16
 * polls).  The wait must give up, raise the kernel's abort flag and return,
 * leaving the context usable.  Returns SJ_ERR_TIMEOUT when it did (the
 * expected outcome), SJ_ERR_CUDA otherwise.  Synchronous on `stream`.
 */
SJ_API int sj_selftest_bounded_wait(void* stream);

/* ---- batched joins ----------------------------------------------------- */
/*
 * Runs `count` independent self-joins (instance k: pts[k], n[k] row-major
 * points of dimension d[k], distance eps[k]; pts[k] host or device memory,
 * read only during the call).  This is the batched form of the paper's
 * Sec. III join for many small problems: instances of the same padded
 * dimension (the next power of two >= d, at least 2) form one group; a
 * group's index is built by segmented kernels over composite cell keys
 * (instance << S | cell key of the instance's own grid, Sec. III-A) and all
 * of the group's work items run in one persistent distance-tile launch
 * (kernels SJ_KERNEL_FILTER_F32, SJ_KERNEL_FILTER_BF16X3 / _BF16X2 / _FP16X2
 * (padded d <= 64) or SJ_KERNEL_FP64_FMA; AUTO takes SJ_KERNEL_FILTER_FP16X2 for
 * groups of padded dimension 8 .. 64 and the FP32 filter for the others;
 * SJ_KERNEL_FP64_DMMA gives SJ_ERR_UNSUPPORTED).  Pairs carry instance-local indices and
 * satisfy the same decision rule as sj_self_join.  The device takes each
 * instance's result pages from one shared pool (opt->page_pairs rounded up
 * to a power of two of at least 64, default 65536 pairs a page); when the
 * pool runs out the joins are rerun with pools sized from the exact counts
 * (reruns in every result).  per_instance_out[k] gets instance k's result (n_candidates and
 * n_evaluated per instance, n_rechecked 0, ms_tile the tile-kernel time of
 * the instance's group, kernel the group's kernel); release each with sj_result_free (the pool is freed
 * with the last of them).  Errors: SJ_ERR_ARG (a bad instance, named in
 * sj_last_error_message), SJ_ERR_OOM, SJ_ERR_CUDA, SJ_ERR_UNSUPPORTED,
 * SJ_ERR_RESULT_OVERFLOW; on error no result needs freeing.
 */
SJ_API int sj_join_batch(const double* const* pts, const int64_t* n, const int32_t* d, const double* eps,
                  int32_t count, const sj_options* opt, void* stream, sj_result* per_instance_out);

/* ---- autotuner --------------------------------------------------------- */
/*
 * No counterpart in the paper, which fixes one kernel design for its GPU.
 * The tunable choices of a join here are the distance kernel (which also
 * fixes the split count of the tensor-core operands: none for the FP32
 * filter, 2 terms for BF16X2 and FP16X2, 3 for BF16X3), the queries per work item (the
 * query tile of a work item, Sec. III-B's shared candidate set) and the
 * number of indexed dims (Sec. II-D).  The autotuner times each candidate
 * configuration on the caller's data with CUDA events on `stream` and keeps
 * the fastest.
 *
 * Tuning cache file: plain text, one entry per line, '#' starts a comment,
 * later lines override earlier ones with the same key:
 *   single d=<d> nlog2=<round(log2 n)> kernel=<k> qpi=<q> m=<m> ms=<t>
 *   batch dp=<padded d> kernel=<k> qpi=<q> ms=<t>
 * (kernel: an SJ_KERNEL_* number; qpi, m: 0 = automatic; ms: the time the
 * entry was tuned at).  Entries are appended to the file.
 */

/*
 * Tunes a single join of (pts, n, d, eps) (pts host or device, as for
 * sj_build_index).  Candidates: kernel in {FILTER_F32, FILTER_FP16X2 and
 * FILTER_BF16X3 when d <= 64} x queries per item in {the kernel's maximum,
 * half of it, a quarter} (at least 4) x indexed dims in {automatic, one less
 * than the automatic choice}; the FP64 kernels are never candidates (FP64 runs
 * at a small fraction of the FP32 and tensor rates on this part).  Each
 * candidate's time is the whole path, sj_build_index to the count of
 * sj_self_join, on `stream`: one untimed warm-up run, then the median of
 * `reps` timed runs (reps < 1 means 3); a candidate whose warm-up takes more
 * than twice the best median so far is not timed further.  `base` (may be
 * NULL) supplies every other option; its kernel, queries_per_item and
 * indexed_dims are ignored.  On success *best is `base` with the winning
 * kernel, queries_per_item and indexed_dims (tune_cache untouched) and
 * *best_ms (may be NULL) its median time; when `cache_path` is not NULL the
 * winner is appended to that file.  Errors: those of sj_build_index /
 * sj_self_join for the first candidate, SJ_ERR_ARG for a NULL `best` or a
 * cache file that cannot be written.
 */
SJ_API int sj_autotune(const double* pts, int64_t n, int32_t d, double eps, const sj_options* base, void* stream,
                       int32_t reps, const char* cache_path, sj_options* best, double* best_ms);

/*
 * Tunes a batched join (arguments as for sj_join_batch) per group of padded
 * dimension.  Candidates, each applied to every group it supports: FILTER_F32
 * with 16 and 8 queries per item; FILTER_FP16X2 with its maximum, half and a
 * quarter; FILTER_BF16X3 with its maximum (tensor-core candidates only for
 * padded d <= 64).  Each candidate runs the whole batch once untimed and
 * `reps` times timed (reps < 1 means 2); a group's time for a candidate is the
 * median of its distance-tile kernel time (sj_result.ms_tile).  Per group the
 * fastest candidate is written to group_dp[g], group_kernel[g], group_qpi[g]
 * and group_ms[g] (g < *n_groups <= max_groups; any of these arrays may be
 * NULL) and appended to `cache_path` when not NULL.  Errors: those of
 * sj_join_batch, SJ_ERR_ARG for an unwritable cache file.
 */
SJ_API int sj_autotune_batch(const double* const* pts, const int64_t* n, const int32_t* d, const double* eps,
                             int32_t count, const sj_options* base, void* stream, int32_t reps,
                             const char* cache_path, int32_t max_groups, int32_t* n_groups, int32_t* group_dp,
                             int32_t* group_kernel, int32_t* group_qpi, double* group_ms);

/*
 * Looks up the tuning cache at `path` without touching a GPU: for batch = 0
 * the entry a single join of n points in d dims would use, for batch = 1 the
 * entry of a batched group of padded dimension d (n ignored).  Returns 1 and
 * fills kernel / qpi / m (any may be NULL; m is 0 for batched entries) when
 * an entry matches, 0 when none does, SJ_ERR_ARG for a NULL path or a
 * malformed line (named in sj_last_error_message).
 */
SJ_API int sj_tune_lookup(const char* path, int32_t batch, int32_t d, int64_t n, int32_t* kernel, int32_t* qpi,
                          int32_t* m);

/* ---- self-join without allocation -------------------------------------- */
/*
 * No counterpart in the paper: an entry point for callers that must not
 * allocate device memory while they run, for instance a process whose device
 * memory another allocator has reserved up front (a serving runtime that
 * takes a fixed budget at start-up and owns every later allocation), or an
 * embedding runtime that forbids cudaMalloc / cudaFree once it has started.
 *
 * Computes the same set as sj_join with SJ_KERNEL_FP64_FMA (the decision rule
 * above) by brute force: all n points form one cell, so every pair is tiled.
 * Every working array lives in one static device array of about 6 MB
 * compiled into the library, which each GPU that loads the library keeps
 * until the process exits; the call makes no cudaMalloc / cudaFree and no
 * other allocation.
 *
 *   pts        device pointer, n x d row-major binary64, caller-owned
 *   n, d       1 <= n <= SJ_NOALLOC_MAX_N, 1 <= d <= SJ_NOALLOC_MAX_D;
 *              larger sizes are rejected with SJ_ERR_ARG
 *   eps        > 0 and finite
 *   pairs_out  device pointer to room for `capacity` pairs (2 * capacity
 *              int32, (i, j) interleaved, input indices, unspecified order)
 *   count_out  host pointer; receives |R| (exact even when it exceeds
 *              capacity, in which case SJ_ERR_RESULT_OVERFLOW is returned and
 *              pairs_out holds `capacity` of the pairs)
 *   stream     cudaStream_t as void*; the call synchronizes this stream: it
 *              reads the extent of the points and the count back to the host
 *              and returns after its work on `stream` has finished
 *
 * The first call on a device looks up the device address of the static
 * array (cudaGetSymbolAddress) and caches it; make that first call before
 * any stream capture.  All calls on a device share the one array and each
 * call resets what it needs, so calls that overlap on the GPU (from several
 * streams or threads at once) race and must be serialised by the caller.
 * Errors: SJ_ERR_ARG (sizes, NULL or host pointers, non-finite coordinate),
 * SJ_ERR_RESULT_OVERFLOW, SJ_ERR_CUDA.
 */
#define SJ_NOALLOC_MAX_N 32768
#define SJ_NOALLOC_MAX_D 8
SJ_API int sj_self_join_noalloc(const double* pts, int64_t n, int32_t d, double eps, int32_t* pairs_out,
                                int64_t capacity, int64_t* count_out, void* stream);

/* ---- test aid: the certified filter's own values -------------------------- */
/*
 * The low-precision filters certify each decision with an error bound
 * (simjoin.h: decision rule).  For a built index whose kernel is
 * SJ_KERNEL_FILTER_F32 (padded d <= 8) or a tensor-core filter, this runs
 * the join once (the result is discarded) with a recording mode of the same
 * kernel that writes, for every evaluated (query, candidate) pair, the
 * filter's value a = -||y_q||^2 / 2 + y_q . y_c exactly as the kernel holds
 * it (FP32 accumulator of the fma chain or of the tensor-core MMA), and
 * copies the index arrays needed to check it.  The kernel's bound says
 * |s_y - (pc - 2 a)| <= E = c1 (P + pc), with s_y = ||y_q - y_c||^2 of the
 * stored kernel coordinates and pc = -2 h_c; a >= thr_in certifies "in" and
 * a < thr_out certifies "out" under the decision rule.  No counterpart in the
 * paper; a measurement aid for tests (slow: one atomic per pair).
 *
 *   perm, y, hnorm, thr_out, thr_in   host arrays of n (y: n x dp) entries in
 *                                     cell order, or NULL: input index, kernel
 *                                     coordinates, -||y||^2 / 2, thresholds
 *   records    host array of 4 * capacity int32: per evaluated pair (query
 *              position, candidate position, bits of a as float, 0), positions
 *              in cell order; the FP32 filter also records each pair its
 *              bounding-box prune decided out unevaluated as (query position,
 *              candidate position, 0, 1); pairs past capacity are counted, not
 *              stored
 *   info       sizes and the bound: n, dp, kernel, c1, P, e2, records (pairs
 *              recorded, exact), count (|R| of the join), prune_r2 (the FP32
 *              filter's prune radius^2 in kernel units: a recorded pruned pair
 *              has s_y above it; +inf for the tensor-core filters); with every
 *              array NULL and capacity 0 only the sizes and the bound are
 *              filled (records = count = -1) and nothing runs
 * Errors: SJ_ERR_ARG, SJ_ERR_UNSUPPORTED (another kernel), SJ_ERR_OOM,
 * SJ_ERR_CUDA.
 */
typedef struct sj_filter_dump {
    int64_t n;
    int32_t dp;
    int32_t kernel;
    double c1;
    double pbound;
    double e2;
    int64_t records;
    int64_t count;
    double prune_r2;
} sj_filter_dump;
SJ_API int sj_debug_filter_dump(sj_handle h, int32_t* perm, float* y, float* hnorm, float* thr_out, float* thr_in,
                                int32_t* records, int64_t capacity, sj_filter_dump* info);

/*
 * The cell order of a built index: perm_out[p] is the input index of the
 * point at sorted position p (points sorted by grid cell key, Sec. III-B;
 * inside a cell the order is unspecified).  perm_out: n int32, host or
 * device.  Synchronous.  Errors: SJ_ERR_ARG, SJ_ERR_CUDA.
 */
SJ_API int sj_index_perm(sj_handle h, int32_t* perm_out);

/* ---- reuse of the join: DBSCAN ----------------------------------------- */
/*
 * Density-based clustering on a join's eps-neighbourhoods (the paper names
 * this reuse of its join as future work, Sec. V; DBSCAN: Ester et al.
 * 1996).  `r` is the result of sj_self_join / sj_join over `n` points with
 * the clustering's eps (pages still on the device); a point is core iff its
 * neighbourhood, itself included, holds at least min_pts points; clusters
 * are the connected components of the core points under the core-core
 * pairs, numbered 0, 1, ... in the order of their smallest core point; a
 * non-core point with a core neighbour (border point) gets the smallest of
 * its core neighbours' cluster numbers, every other point -1 (noise).  The
 * labels are deterministic.
 *
 *   labels_out  n int32, host or device
 *   n_clusters  host pointer (may be NULL)
 * Synchronous.  Errors: SJ_ERR_ARG (a batched result, n, min_pts < 1),
 * SJ_ERR_RESULT_OVERFLOW (a result that holds only part of its pairs),
 * SJ_ERR_OOM, SJ_ERR_CUDA, SJ_ERR_TIMEOUT (a union-find update ran out of
 * its bounded retries).
 */
SJ_API int sj_dbscan(const sj_result* r, int64_t n, int32_t min_pts, int32_t* labels_out, int64_t* n_clusters);

/* ---- the distance tile alone; kNN from the join ------------------------- */
/*
 * sj_sqdist_tile: out[i * nb + j] = the squared distance of A's row i and
 * B's row j, for all i < m, j < nb (the brute-force distance tile of the
 * paper's Fig. 3 experiment, Sec. IV, as an operation of its own), in the
 * decision rule's arithmetic (binary64, dimension order, subtraction, product
 * and sum each rounded): exactly the s the join decides with.  A: m x d, B:
 * nb x d row-major binary64, out: m x nb binary64, all device pointers owned
 * by the caller; m <= 65535 * 64.  Asynchronous on `stream`.  Errors:
 * SJ_ERR_ARG, SJ_ERR_CUDA.
 *
 * sj_knn_from_join: for every point of a single join's result with
 * distances (sj_options.emit_distances = 1) over n points, its k nearest
 * eps-neighbours other than itself, by (distance, index) ascending (the reuse
 * of the join for kNN the paper names as future work, Sec. V): idx_out and
 * dist_out n x k (row-major; -1 and +inf past the found ones), found_out n
 * (neighbours found, at most k: fewer when the point has fewer than k other
 * points within eps); host or device memory.  Synchronous.  Errors:
 * SJ_ERR_ARG (no distances, a batched result, k outside 1 .. 1024),
 * SJ_ERR_RESULT_OVERFLOW, SJ_ERR_OOM, SJ_ERR_CUDA.
 */
SJ_API int sj_sqdist_tile(const double* A, int64_t m, const double* B, int64_t nb, int32_t d, double* out,
                          void* stream);
SJ_API int sj_knn_from_join(const sj_result* r, int64_t n, int32_t k, int32_t* idx_out, double* dist_out,
                            int32_t* found_out);

/* ---- tracing ------------------------------------------------------------ */
/*
 * No counterpart in the paper (which reports response times only).
 * sj_set_tracing(1) makes every later sj_build_index of the process record a
 * CUDA event and the host clock at its phase boundaries (0 switches it off).
 * sj_index_phase_ms gives, for a handle built with tracing on, the device
 * and host milliseconds of its four build phases: extent + grid choice, sort
 * by cell key, packing (coordinates, norms, thresholds; the tensor-core
 * filter's operand rows), neighbour runs + work items (each array of 4 may
 * be NULL; -1 where not traced).  The join's
 * tile time is sj_result.ms_tile.
 */
SJ_API void sj_set_tracing(int32_t on);
SJ_API int sj_index_phase_ms(sj_handle h, double* device_ms, double* host_ms);

/* ---- test aids: allocation failures ------------------------------------ */
/*
 * No counterpart in the paper.  sj_debug_fail_allocations(k): the library's
 * next k device allocations succeed and every later one fails with
 * SJ_ERR_OOM until the injection is switched off with a negative k
 * (process-wide, all threads).  sj_debug_live_allocations(): device blocks
 * the library holds at the moment (allocated and not yet released); a call
 * that fails must leave it where it was.
 */
SJ_API void sj_debug_fail_allocations(int64_t after);
SJ_API int64_t sj_debug_live_allocations(void);

/* ---- status ------------------------------------------------------------ */
SJ_API const char* sj_error_string(int status);
/* Detail of the calling thread's last error (empty string if none). */
SJ_API const char* sj_last_error_message(void);
/* Library version and the compute capability it was built for. */
SJ_API const char* sj_version(void);
/* Number of CUDA kernels this library has launched in the calling process
 * (all threads, all devices); a measurement aid, no paper counterpart. */
SJ_API int64_t sj_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* SIMJOIN_H */
