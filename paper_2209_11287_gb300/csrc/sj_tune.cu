// Autotuner and tuning cache (no counterpart in the paper, which fixes one
// kernel design for its GPU).  The tunable choices of a join are the distance
// kernel (and with it the split count of the tensor-core operands), the
// queries per work item (the query tile of the queries that share a candidate
// set, Sec. III-B) and, for single joins, the number of indexed dims
// (Sec. II-D).  Candidates are timed on the caller's data with CUDA events on
// the caller's stream; the winners go to a plain-text cache that
// sj_build_index and sj_join_batch consult when the kernel is AUTO.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <sys/stat.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "sj_internal.cuh"

namespace sj {

namespace {

struct CachedFile {
    long long mtime_ns = -1;
    long long size = -1;
    std::vector<TuneEntry> entries;
};
std::mutex g_tune_mu;
std::map<std::string, CachedFile> g_tune_files;

bool valid_kernel(long k) { return k >= SJ_KERNEL_AUTO && k <= SJ_KERNEL_FILTER_FP16X2; }

// Parses one line; *has gets whether it held an entry (blank and comment
// lines hold none).  Returns false for a malformed line.
bool parse_line(const char* line, TuneEntry* e, bool* has) {
    *has = false;
    char buf[512];
    snprintf(buf, sizeof buf, "%s", line);
    if (char* hash = strchr(buf, '#')) *hash = 0;
    char* save = nullptr;
    char* tok = strtok_r(buf, " \t\r\n", &save);
    if (!tok) return true;
    TuneEntry t;
    if (strcmp(tok, "single") == 0)
        t.batch = 0;
    else if (strcmp(tok, "batch") == 0)
        t.batch = 1;
    else
        return false;
    bool have_d = false, have_n = false, have_k = false;
    while ((tok = strtok_r(nullptr, " \t\r\n", &save))) {
        char* eq = strchr(tok, '=');
        if (!eq) return false;
        *eq = 0;
        const char* key = tok;
        const char* val = eq + 1;
        char* end = nullptr;
        if (strcmp(key, "ms") == 0) {
            t.ms = strtod(val, &end);
            if (end == val || *end) return false;
            continue;
        }
        const long v = strtol(val, &end, 10);
        if (end == val || *end) return false;
        if ((strcmp(key, "d") == 0 && !t.batch) || (strcmp(key, "dp") == 0 && t.batch)) {
            if (v < 1 || v > SJ_MAX_D) return false;
            t.d = (int)v;
            have_d = true;
        } else if (strcmp(key, "nlog2") == 0 && !t.batch) {
            if (v < 0 || v > 62) return false;
            t.nlog2 = (int)v;
            have_n = true;
        } else if (strcmp(key, "kernel") == 0) {
            if (!valid_kernel(v)) return false;
            t.kernel = (int)v;
            have_k = true;
        } else if (strcmp(key, "qpi") == 0) {
            if (v < 0 || v > 4096) return false;
            t.qpi = (int)v;
        } else if (strcmp(key, "m") == 0 && !t.batch) {
            if (v < 0 || v > SJ_MAX_D) return false;
            t.m = (int)v;
        } else {
            return false;
        }
    }
    if (!have_d || !have_k || (!t.batch && !have_n)) return false;
    *e = t;
    *has = true;
    return true;
}

int tune_append(const char* path, const TuneEntry& e) {
    FILE* f = fopen(path, "a");
    if (!f) {
        set_error("cannot open the tuning cache %s for appending", path);
        return SJ_ERR_ARG;
    }
    int r;
    if (e.batch)
        r = fprintf(f, "batch dp=%d kernel=%d qpi=%d ms=%.6f\n", e.d, e.kernel, e.qpi, e.ms);
    else
        r = fprintf(f, "single d=%d nlog2=%d kernel=%d qpi=%d m=%d ms=%.6f\n", e.d, e.nlog2, e.kernel, e.qpi, e.m,
                    e.ms);
    const bool ok = r > 0 && fclose(f) == 0;
    if (!ok) {
        set_error("cannot write the tuning cache %s", path);
        return SJ_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_files.erase(path);
    return SJ_OK;
}

int nlog2_of(int64_t n) { return (int)lround(log2((double)std::max<int64_t>(n, 1))); }

double median(std::vector<double> v) {
    std::sort(v.begin(), v.end());
    return v.empty() ? 0.0 : v[v.size() / 2];
}

// The capacity of a work item of `kernel` at padded dimension dp.
int qpi_cap(int kernel, int dp) { return is_tensor_kernel(kernel) ? tc_qmax(tc_kp(dp, kernel)) : kQMax; }

}  // namespace

int tune_load(const char* path, std::vector<TuneEntry>* out) {
    out->clear();
    struct stat sb;
    if (stat(path, &sb) != 0) return SJ_OK;  // no file: an empty cache
    const long long mt = (long long)sb.st_mtim.tv_sec * 1000000000ll + sb.st_mtim.tv_nsec;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_files.find(path);
        if (it != g_tune_files.end() && it->second.mtime_ns == mt && it->second.size == (long long)sb.st_size) {
            *out = it->second.entries;
            return SJ_OK;
        }
    }
    FILE* f = fopen(path, "r");
    if (!f) return SJ_OK;
    char line[512];
    int ln = 0;
    std::vector<TuneEntry> v;
    while (fgets(line, sizeof line, f)) {
        ++ln;
        TuneEntry e;
        bool has = false;
        if (!parse_line(line, &e, &has)) {
            fclose(f);
            set_error("tuning cache %s: malformed line %d", path, ln);
            return SJ_ERR_ARG;
        }
        if (has) v.push_back(e);
    }
    fclose(f);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    CachedFile& c = g_tune_files[path];
    c.mtime_ns = mt;
    c.size = (long long)sb.st_size;
    c.entries = v;
    *out = std::move(v);
    return SJ_OK;
}

const TuneEntry* tune_find_single(const std::vector<TuneEntry>& t, int d, int64_t n) {
    const int nl = nlog2_of(n);
    const TuneEntry* best = nullptr;
    int best_gap = 2;
    for (const TuneEntry& e : t) {
        if (e.batch || e.d != d) continue;
        const int gap = std::abs(e.nlog2 - nl);
        if (gap <= best_gap) {  // later lines win ties
            best = &e;
            best_gap = gap;
        }
    }
    return best_gap <= 1 ? best : nullptr;
}

const TuneEntry* tune_find_group(const std::vector<TuneEntry>& t, int dp) {
    const TuneEntry* best = nullptr;
    for (const TuneEntry& e : t)
        if (e.batch && e.d == dp) best = &e;
    return best;
}

}  // namespace sj

using namespace sj;

extern "C" {

int sj_tune_lookup(const char* path, int32_t batch, int32_t d, int64_t n, int32_t* kernel, int32_t* qpi,
                   int32_t* m) {
    clear_error();
    if (!path) {
        set_error("path is NULL");
        return SJ_ERR_ARG;
    }
    std::vector<TuneEntry> t;
    SJ_TRY(tune_load(path, &t));
    const TuneEntry* e = batch ? tune_find_group(t, d) : tune_find_single(t, d, n);
    if (!e) return 0;
    if (kernel) *kernel = e->kernel;
    if (qpi) *qpi = e->qpi;
    if (m) *m = e->m;
    return 1;
}

int sj_autotune(const double* pts, int64_t n, int32_t d, double eps, const sj_options* base, void* stream,
                int32_t reps, const char* cache_path, sj_options* best, double* best_ms) {
    clear_error();
    if (!best || !pts || n < 1 || n > 0x7FFFFFFFll || d < 1 || d > SJ_MAX_D || !(eps > 0) || !isfinite(eps)) {
        set_error("invalid autotune arguments");
        return SJ_ERR_ARG;
    }
    if (reps < 1) reps = 3;
    sj_options b0;
    sj_default_options(&b0);
    if (base) b0 = *base;
    b0.tune_cache = nullptr;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int dp = round_dim(d);

    // host points are staged once, so every candidate reads device memory
    const double* dpts = pts;
    double* staged = nullptr;
    if (!is_device_pointer(pts)) {
        SJ_TRY(dev_alloc_t(&staged, (size_t)n * d, s));
        cudaError_t e = cudaMemcpyAsync(staged, pts, (size_t)n * d * sizeof(double), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) {
            dev_free(staged, s);
            set_error("host-to-device copy: %s", cudaGetErrorString(e));
            return SJ_ERR_CUDA;
        }
        dpts = staged;
    }
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess) {
        if (ev[0]) cudaEventDestroy(ev[0]);
        dev_free(staged, s);
        set_error("autotune events");
        return SJ_ERR_CUDA;
    }
    // one whole-path run: build + join + count, timed on the stream
    auto run_once = [&](const sj_options& o, double* ms, int32_t* m_used) -> int {
        if (cudaEventRecord(ev[0], s) != cudaSuccess) return SJ_ERR_CUDA;
        sj_handle h = nullptr;
        int st = sj_build_index(dpts, n, d, eps, &o, stream, &h);
        if (st != SJ_OK) return st;
        if (m_used) sj_index_info(h, nullptr, nullptr, m_used, nullptr, nullptr);
        sj_result r;
        memset(&r, 0, sizeof r);
        st = sj_self_join(h, &r);
        if (st == SJ_OK && (cudaEventRecord(ev[1], s) != cudaSuccess || cudaEventSynchronize(ev[1]) != cudaSuccess))
            st = SJ_ERR_CUDA;
        float f = 0.f;
        if (st == SJ_OK && cudaEventElapsedTime(&f, ev[0], ev[1]) != cudaSuccess) st = SJ_ERR_CUDA;
        sj_result_free(&r);
        sj_destroy(h);
        *ms = f;
        return st;
    };

    struct Cand {
        int kernel, qpi, m;
    };
    std::vector<int> kernels;
    // the automatic choice first, so slow candidates meet a good time early
    const int auto_k = (d >= 9 && d <= 64) ? SJ_KERNEL_FILTER_FP16X2 : SJ_KERNEL_FILTER_F32;
    kernels.push_back(auto_k);
    for (int k : {SJ_KERNEL_FILTER_F32, SJ_KERNEL_FILTER_FP16X2, SJ_KERNEL_FILTER_BF16X3})
        if (k != auto_k && (!is_tensor_kernel(k) || dp <= 64)) kernels.push_back(k);

    int first_err = SJ_OK;
    bool have = false;
    Cand win{auto_k, 0, 0};
    double win_ms = 0;
    int32_t m_auto = -1;
    for (int k : kernels) {
        const int cap = qpi_cap(k, dp);
        std::vector<int> qpis{0};
        for (int div : {2, 4})
            if (cap / div >= 4 && std::find(qpis.begin(), qpis.end(), cap / div) == qpis.end()) qpis.push_back(cap / div);
        for (int q : qpis) {
            std::vector<int> ms_list{0};
            if (m_auto > 1) ms_list.push_back(m_auto - 1);
            for (size_t mi = 0; mi < ms_list.size(); ++mi) {
                sj_options o = b0;
                o.kernel = k;
                o.queries_per_item = q;
                o.indexed_dims = ms_list[mi];
                double warm = 0;
                int32_t mu = 0;
                int st = run_once(o, &warm, &mu);
                if (st != SJ_OK) {
                    if (first_err == SJ_OK) first_err = st;
                    cudaGetLastError();
                    continue;
                }
                if (m_auto < 0 && ms_list[mi] == 0) {
                    m_auto = mu;  // the automatic grid of this data
                    if (m_auto > 1 && ms_list.size() == 1) ms_list.push_back(m_auto - 1);
                }
                if (have && warm > 2.0 * win_ms) continue;
                std::vector<double> t;
                for (int r = 0; r < reps && st == SJ_OK; ++r) {
                    double ms = 0;
                    st = run_once(o, &ms, nullptr);
                    t.push_back(ms);
                }
                if (st != SJ_OK) {
                    if (first_err == SJ_OK) first_err = st;
                    continue;
                }
                const double med = median(t);
                if (!have || med < win_ms) {
                    have = true;
                    win = Cand{k, q, ms_list[mi]};
                    win_ms = med;
                }
            }
        }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    dev_free(staged, s);
    cudaStreamSynchronize(s);
    if (!have) return first_err != SJ_OK ? first_err : SJ_ERR_UNSUPPORTED;
    clear_error();
    *best = b0;
    best->kernel = win.kernel;
    best->queries_per_item = win.qpi;
    best->indexed_dims = win.m;
    best->tune_cache = base ? base->tune_cache : nullptr;
    if (best_ms) *best_ms = win_ms;
    if (cache_path) {
        TuneEntry e;
        e.batch = 0;
        e.d = d;
        e.nlog2 = nlog2_of(n);
        e.kernel = win.kernel;
        e.qpi = win.qpi;
        e.m = win.m;
        e.ms = win_ms;
        SJ_TRY(tune_append(cache_path, e));
    }
    return SJ_OK;
}

int sj_autotune_batch(const double* const* pts, const int64_t* n, const int32_t* d, const double* eps,
                      int32_t count, const sj_options* base, void* stream, int32_t reps, const char* cache_path,
                      int32_t max_groups, int32_t* n_groups, int32_t* group_dp, int32_t* group_kernel,
                      int32_t* group_qpi, double* group_ms) {
    clear_error();
    if (!pts || !n || !d || !eps || count < 1) {
        set_error("invalid batch arguments");
        return SJ_ERR_ARG;
    }
    for (int32_t k = 0; k < count; ++k)
        if (d[k] < 1 || d[k] > SJ_MAX_D) {
            set_error("invalid batch instance %d: d=%d", (int)k, (int)d[k]);
            return SJ_ERR_ARG;
        }
    if (reps < 1) reps = 2;
    sj_options b0;
    sj_default_options(&b0);
    if (base) b0 = *base;
    b0.kernel = SJ_KERNEL_AUTO;
    b0.tune_cache = nullptr;
    b0.graph = 0;  // per-group tile times need the groups to run one after another
    std::vector<int> dps;
    for (int32_t k = 0; k < count; ++k) dps.push_back(round_dim(d[k]));
    std::sort(dps.begin(), dps.end());
    dps.erase(std::unique(dps.begin(), dps.end()), dps.end());
    const int G = (int)dps.size();

    struct Cand {
        int kernel, div;  // div: queries per item = capacity / div (1: the capacity, written as 0)
    };
    const Cand cands[] = {{SJ_KERNEL_FILTER_FP16X2, 1}, {SJ_KERNEL_FILTER_F32, 1}, {SJ_KERNEL_FILTER_F32, 2},
                          {SJ_KERNEL_FILTER_FP16X2, 2}, {SJ_KERNEL_FILTER_FP16X2, 4}, {SJ_KERNEL_FILTER_BF16X3, 1}};
    std::vector<double> best(G, 0.0);
    std::vector<int> best_k(G, SJ_KERNEL_AUTO), best_q(G, 0);
    std::vector<bool> have(G, false);
    std::vector<sj_result> res(count);
    int first_err = SJ_OK;
    for (const Cand& c : cands) {
        std::vector<TuneEntry> forced;
        std::vector<bool> applies(G, false);
        for (int g = 0; g < G; ++g) {
            TuneEntry e;
            e.batch = 1;
            e.d = dps[g];
            if (!is_tensor_kernel(c.kernel) || dps[g] <= 64) {
                e.kernel = c.kernel;
                e.qpi = c.div == 1 ? 0 : qpi_cap(c.kernel, dps[g]) / c.div;
                applies[g] = true;
            }  // else AUTO: the group keeps its default and is not scored
            forced.push_back(e);
        }
        std::vector<std::vector<double>> t(G);
        int st = SJ_OK;
        for (int r = 0; r <= reps && st == SJ_OK; ++r) {
            st = join_batch_impl(pts, n, d, eps, count, &b0, stream, res.data(), &forced);
            if (st != SJ_OK) break;
            std::vector<double> gms(G, -1.0);
            for (int32_t k = 0; k < count; ++k) {
                const int g = (int)(std::lower_bound(dps.begin(), dps.end(), round_dim(d[k])) - dps.begin());
                if (applies[g] && res[k].kernel == c.kernel) gms[g] = res[k].ms_tile;
            }
            sj_results_free(res.data(), count);
            if (r == 0) {  // warm-up: stop early when no group can win
                bool hopeful = false;
                for (int g = 0; g < G; ++g)
                    if (gms[g] >= 0 && (!have[g] || gms[g] <= 2.0 * best[g])) hopeful = true;
                if (!hopeful) break;
                continue;
            }
            for (int g = 0; g < G; ++g)
                if (gms[g] >= 0) t[g].push_back(gms[g]);
        }
        if (st != SJ_OK) {
            if (first_err == SJ_OK) first_err = st;
            cudaGetLastError();
            continue;
        }
        for (int g = 0; g < G; ++g) {
            if (t[g].empty()) continue;
            const double med = median(t[g]);
            if (!have[g] || med < best[g]) {
                have[g] = true;
                best[g] = med;
                best_k[g] = c.kernel;
                best_q[g] = c.div == 1 ? 0 : qpi_cap(c.kernel, dps[g]) / c.div;
            }
        }
    }
    bool any = false;
    for (int g = 0; g < G; ++g) any = any || have[g];
    if (!any) return first_err != SJ_OK ? first_err : SJ_ERR_UNSUPPORTED;
    clear_error();
    int out = 0;
    for (int g = 0; g < G; ++g) {
        if (!have[g]) continue;
        if (out < max_groups) {
            if (group_dp) group_dp[out] = dps[g];
            if (group_kernel) group_kernel[out] = best_k[g];
            if (group_qpi) group_qpi[out] = best_q[g];
            if (group_ms) group_ms[out] = best[g];
        }
        ++out;
        if (cache_path) {
            TuneEntry e;
            e.batch = 1;
            e.d = dps[g];
            e.kernel = best_k[g];
            e.qpi = best_q[g];
            e.ms = best[g];
            SJ_TRY(tune_append(cache_path, e));
        }
    }
    if (n_groups) *n_groups = std::min(out, std::max(max_groups, 0));
    return SJ_OK;
}

}  // extern "C"
