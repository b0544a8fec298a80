// abi.cu -- the extern "C" boundary declared in include/l1line.h.
//
// Host code only: validates arguments, carves the caller's workspace and
// enqueues the kernels on the caller's stream.  It never allocates memory and
// never synchronises, except in l1line_status().
#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <memory>
#include <mutex>
#include <numeric>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/l1line.h"
#include "batch_split.h"
#include "checks.cuh"
#include "common.cuh"
#include "launch.h"

using namespace l1l;

namespace {

// NVTX range over a scope (a no-op unless a profiler is attached): every
// entry point that enqueues work and each stage of a fit (staging, pair
// kernel with its exact path and sums, argmin) is one range on the calling
// thread, so ncu/nsys timelines show which library call a kernel came from.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
#define L1L_RANGE_CAT2(a, b) a##b
#define L1L_RANGE_CAT(a, b) L1L_RANGE_CAT2(a, b)
#define L1L_RANGE(name) NvtxRange L1L_RANGE_CAT(nvtx_range_, __LINE__)(name)

// An entry point's range.  It also clears a non-sticky CUDA error that an
// earlier, unrelated runtime call left behind (an invalidated stream capture,
// say): the launch checks below read cudaGetLastError and must see only this
// call's own failures.  A sticky error (a lost context) stays and is reported.
struct EntryRange : NvtxRange {
    explicit EntryRange(const char *name) : NvtxRange(name) { (void)cudaGetLastError(); }
};
#define L1L_ENTRY(name) EntryRange L1L_RANGE_CAT(nvtx_entry_, __LINE__)(name)

thread_local int g_last_launches = 0;
thread_local Tune g_tune;  // l1line_set_tuning
thread_local cudaEvent_t g_ev_start = nullptr, g_ev_stop = nullptr;

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

// The status word at the start of a workspace, decoded (the stream is
// synchronised first).
int status_of(void *workspace, void *stream);

bool mul_ok(int64_t a, int64_t b, int64_t &out) {
    if (a < 0 || b < 0) return false;
    if (a != 0 && b > INT64_MAX / a) return false;
    out = a * b;
    return true;
}

struct Layout {
    size_t status, slow_count, colinfo, Xt, Xf, v_all, s_all, z_all, slow;
    size_t feat_raw, feat_std, score, idx;  // learned proposer: [m][4], [m][4], [m], [m]
    size_t total;
    int64_t ldn;
};

// Returns false on overflow / bad shape.
bool make_layout(int dtype, int64_t n, int64_t m, int64_t nl, Layout &L) {
    if (n < 1 || m < 1 || nl < 1) return false;
    const int64_t es = dtype == L1L_DTYPE_F32 ? 4 : 8;
    const int64_t ldn = (n + ROW_PAD - 1) & ~int64_t(ROW_PAD - 1);
    int64_t mm, pairs, xt, chunk_pairs;
    if (!mul_ok(m, m, mm) || !mul_ok(mm, nl, pairs) || !mul_ok(m, ldn, xt)) return false;
    const int64_t nlc = nl < MAX_LAMBDA_PER_LAUNCH ? nl : MAX_LAMBDA_PER_LAUNCH;
    if (!mul_ok(mm, nlc, chunk_pairs)) return false;
    if (pairs > INT64_MAX / 16 || xt > INT64_MAX / 16) return false;
    // the exact path's list of one launch is counted by a uint32 (slow_count)
    // and walked with a uint32 index: keep it far from wrapping
    if (chunk_pairs > ((int64_t)1 << 31)) return false;
    size_t off = 0;
    L.status = off;
    off += 256;
    L.slow_count = off;
    off += 256;
    L.colinfo = off;
    off = al256(off + (size_t)m * sizeof(ColInfo));
    L.Xt = off;
    off = al256(off + (size_t)xt * es);
    L.Xf = L.Xt;  // double input: a float copy for the approximate keys and
    if (es == 8) {  // the remainders x - fl(x) for the float-float residual
        L.Xf = off;
        off = al256(off + (size_t)xt * 8);
    }
    L.v_all = off;
    off = al256(off + (size_t)pairs * es);
    L.s_all = off;
    off = al256(off + (size_t)pairs * 8);
    L.z_all = off;
    off = al256(off + (size_t)(m * nl) * 8);
    L.slow = off;
    off = al256(off + (size_t)chunk_pairs * sizeof(SlowEntry));
    L.feat_raw = off;
    off = al256(off + (size_t)m * 4 * L1L_MLP_FEATURES);
    L.feat_std = off;
    off = al256(off + (size_t)m * 4 * L1L_MLP_FEATURES);
    L.score = off;
    off = al256(off + (size_t)m * 4);
    L.idx = off;
    off = al256(off + (size_t)m * 4);
    L.total = off;
    L.ldn = ldn;
    return true;
}

// Rows of the restricted fit behind the proposer's fourth feature.
int64_t proposer_rows(int64_t n) {
    if (n < 1) return 0;
    const int64_t r = std::max<int64_t>(256, (n + 7) / 8);
    return std::min<int64_t>(n, r);
}

// Workspace of the proposer calls: the fit's layout, then the restricted
// fit's row norms, row list, row copy and its own fit workspace.
struct ProposedLayout {
    Layout L;
    int64_t R;
    size_t rho, rows, xr, pws, pws_bytes, total;
};
bool make_proposed_layout(int dtype, int64_t n, int64_t m, int64_t nl, ProposedLayout &P) {
    // the column-feature kernel holds a column's n keys in shared memory
    if (n > (dtype == L1L_DTYPE_F32 ? max_rows_pairs<float>() : max_rows_pairs<double>()))
        return false;
    if (!make_layout(dtype, n, m, nl, P.L)) return false;
    P.R = proposer_rows(n);
    Layout LR;
    if (!make_layout(dtype, P.R, m, 1, LR)) return false;
    const size_t es = dtype == L1L_DTYPE_F32 ? 4 : 8;
    size_t off = al256(P.L.total);
    P.rho = off;
    off = al256(off + (size_t)n * 4);
    P.rows = off;
    off = al256(off + (size_t)P.R * 4);
    P.xr = off;
    off = al256(off + (size_t)P.R * (size_t)m * es);
    P.pws = off;
    P.pws_bytes = LR.total;
    off = al256(off + LR.total);
    P.total = off;
    return true;
}

int num_sms() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return sms;
}

template <typename T> int dtype_of();
template <> int dtype_of<float>() { return L1L_DTYPE_F32; }
template <> int dtype_of<double>() { return L1L_DTYPE_F64; }

// One scan or fit in stages: setup (validation, workspace carving), prep
// (transpose, column info), pairs (steps A2-A5 for the listed jhat), argmin.
template <typename T> struct Scan {
    ScanArgs<T> a;
    Layout L;
    int sms = 0;
    double *z = nullptr;
    unsigned char *base = nullptr;
    cudaStream_t st = nullptr;
    int launches = 0;
};

template <typename T>
int scan_setup(const T *X, int64_t n, int64_t m, const double *lambdas, int64_t nl, T *v_all,
               double *s_all, double *z_all, void *ws, size_t ws_bytes, void *stream,
               uint32_t flags, Scan<T> &c) {
    g_last_launches = 0;
    if (!X || !lambdas || n < 1 || m < 1 || nl < 1) return L1L_ERR_ARG;
    if (m > 0x7FFFFFFF || nl > 65535) return L1L_ERR_UNSUPPORTED;
    for (int64_t t = 0; t < nl; ++t)
        if (!(lambdas[t] >= 0.0) || std::isinf(lambdas[t])) return L1L_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(X) % sizeof(T)) != 0) return L1L_ERR_ARG;
    if (n > large_max_rows()) return L1L_ERR_UNSUPPORTED;
    Layout &L = c.L;
    if (!make_layout(dtype_of<T>(), n, m, nl, L)) return L1L_ERR_UNSUPPORTED;
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255) != 0 || ws_bytes < L.total)
        return L1L_ERR_WORKSPACE;
    c.sms = num_sms();
    if (c.sms <= 0) return L1L_ERR_CUDA;
    c.base = static_cast<unsigned char *>(ws);
    c.st = static_cast<cudaStream_t>(stream);
    ScanArgs<T> &a = c.a;
    a.Xt = reinterpret_cast<T *>(c.base + L.Xt);
    a.Xf = reinterpret_cast<float *>(c.base + L.Xf);
    a.ci = reinterpret_cast<ColInfo *>(c.base + L.colinfo);
    a.n = n;
    a.m = m;
    a.ldn = L.ldn;
    a.n_lambda = (int32_t)nl;
    a.v_all = v_all ? v_all : reinterpret_cast<T *>(c.base + L.v_all);
    a.s_all = s_all ? s_all : reinterpret_cast<double *>(c.base + L.s_all);
    a.status = reinterpret_cast<uint32_t *>(c.base + L.status);
    a.slow_count = reinterpret_cast<uint32_t *>(c.base + L.slow_count);
    a.slow = reinterpret_cast<SlowEntry *>(c.base + L.slow);
    a.force_exact = (flags & L1L_FLAG_FORCE_EXACT) ? 1 : 0;
    a.inst = 0;
    a.jlist = nullptr;
    a.nj = m;
    a.d0 = D0_DEFAULT;
    c.z = z_all ? z_all : reinterpret_cast<double *>(c.base + L.z_all);
    return L1L_OK;
}

template <typename T> int scan_prep(const T *X, Scan<T> &c) {
    L1L_RANGE("l1l::stage");
    ScanArgs<T> &a = c.a;
    if (cudaMemsetAsync(a.status, 0, sizeof(uint32_t), c.st) != cudaSuccess) return L1L_ERR_CUDA;
    if (launch_prep<T>(X, const_cast<T *>(a.Xt), const_cast<float *>(a.Xf),
                       const_cast<ColInfo *>(a.ci), a.n, a.m, a.ldn,
                       a.status, c.st, c.launches) != cudaSuccess)
        return L1L_ERR_CUDA;
    return L1L_OK;
}

// Steps A2-A5 for n beyond the pair kernel's shared memory: the cluster
// kernel streaming both columns from the staged copy, then the exact path.
template <typename T>
int scan_pairs_large(Scan<T> &c, const double *lambdas, int64_t nl, const int32_t *jlist,
                     int64_t nj) {
    L1L_RANGE("l1l::pairs_global_memory");
    ScanArgs<T> &a = c.a;
    const bool prof = g_ev_start && g_ev_stop;
    for (int64_t t0 = 0; t0 < nl; t0 += MAX_LAMBDA_PER_LAUNCH) {
        const int nlc = (int)((nl - t0) < MAX_LAMBDA_PER_LAUNCH ? (nl - t0) : MAX_LAMBDA_PER_LAUNCH);
        const bool last = t0 + MAX_LAMBDA_PER_LAUNCH >= nl;
        if (cudaMemsetAsync(a.slow_count, 0, sizeof(uint32_t), c.st) != cudaSuccess)
            return L1L_ERR_CUDA;
        if (prof && t0 == 0 && cudaEventRecord(g_ev_start, c.st) != cudaSuccess)
            return L1L_ERR_CUDA;
        if (launch_large<T>(a, lambdas, (int)t0, nlc, c.st, c.launches) != cudaSuccess)
            return L1L_ERR_CUDA;
        if (prof && last && cudaEventRecord(g_ev_stop, c.st) != cudaSuccess) return L1L_ERR_CUDA;
        if (launch_exact<T>(a, lambdas, (int)t0, nlc, c.sms, c.st, c.launches) != cudaSuccess)
            return L1L_ERR_CUDA;
    }
    if (launch_zreduce(a.s_all, c.z, a.m, nl, jlist, nj, c.st, c.launches) != cudaSuccess)
        return L1L_ERR_CUDA;
    return L1L_OK;
}

// Steps A2-A5 for the jhat in jlist[0..nj) (jlist == nullptr: all m).
template <typename T>
int scan_pairs(Scan<T> &c, const double *lambdas, int64_t nl, const int32_t *jlist, int64_t nj) {
    L1L_RANGE("l1l::pairs");
    ScanArgs<T> &a = c.a;
    a.jlist = jlist;
    a.nj = nj;
    if (a.n > max_rows_pairs<T>()) return scan_pairs_large<T>(c, lambdas, nl, jlist, nj);
    const PairPlan plan = plan_pairs<T>(a.n, a.m, c.sms, nj, g_tune);
    if (plan.warps == 0) return L1L_ERR_UNSUPPORTED;
    a.d0 = plan.d0;
    const bool prof = g_ev_start && g_ev_stop;
    for (int64_t t0 = 0; t0 < nl; t0 += MAX_LAMBDA_PER_LAUNCH) {
        const int nlc = (int)((nl - t0) < MAX_LAMBDA_PER_LAUNCH ? (nl - t0) : MAX_LAMBDA_PER_LAUNCH);
        const bool last = t0 + MAX_LAMBDA_PER_LAUNCH >= nl;
        if (cudaMemsetAsync(a.slow_count, 0, sizeof(uint32_t), c.st) != cudaSuccess)
            return L1L_ERR_CUDA;
        if (prof && t0 == 0 && cudaEventRecord(g_ev_start, c.st) != cudaSuccess)
            return L1L_ERR_CUDA;
        if (launch_pairs<T>(a, lambdas, (int)t0, nlc, plan, c.st, c.launches) != cudaSuccess)
            return L1L_ERR_CUDA;
        if (prof && last && cudaEventRecord(g_ev_stop, c.st) != cudaSuccess) return L1L_ERR_CUDA;
        if (launch_exact<T>(a, lambdas, (int)t0, nlc, c.sms, c.st, c.launches) != cudaSuccess)
            return L1L_ERR_CUDA;
    }
    if (launch_zreduce(a.s_all, c.z, a.m, nl, jlist, nj, c.st, c.launches) != cudaSuccess)
        return L1L_ERR_CUDA;
    return L1L_OK;
}

template <typename T>
int scan_argmin(Scan<T> &c, int64_t nl, T *out_v, double *out_obj, int32_t *out_jstar) {
    L1L_RANGE("l1l::argmin");
    if (launch_argmin<T>(c.z, c.a.v_all, c.a.m, nl, c.a.jlist, c.a.nj, out_v, out_obj, out_jstar,
                         c.st, c.launches) != cudaSuccess)
        return L1L_ERR_CUDA;
    return L1L_OK;
}

#define L1L_TRY(expr)                                                                             \
    do {                                                                                          \
        const int rc_ = (expr);                                                                   \
        if (rc_ != L1L_OK) return rc_;                                                            \
    } while (0)

template <typename T>
int scan_impl(const T *X, int64_t n, int64_t m, const double *lambdas, int64_t nl, T *v_all,
              double *s_all, double *z_all, void *ws, size_t ws_bytes, void *stream,
              uint32_t flags) {
    Scan<T> c;
    L1L_TRY(scan_setup<T>(X, n, m, lambdas, nl, v_all, s_all, z_all, ws, ws_bytes, stream, flags,
                          c));
    L1L_TRY(scan_prep<T>(X, c));
    L1L_TRY(scan_pairs<T>(c, lambdas, nl, nullptr, m));
    g_last_launches = c.launches;
    return L1L_OK;
}

// Full fit (jlist == nullptr) or subset fit of jlist[0..nj).
template <typename T>
int fit_impl(const T *X, int64_t n, int64_t m, const double *lambdas, int64_t nl,
             const int32_t *jlist, int64_t nj, T *out_v, double *out_obj, int32_t *out_jstar,
             void *ws, size_t ws_bytes, void *stream) {
    if (!out_v || !out_obj || !out_jstar) return L1L_ERR_ARG;
    // at most m entries: the exact path's pair list of a launch holds m * m
    // pairs per lambda, one per listed (jhat, k) at most
    if (jlist && (nj < 1 || nj > m)) return L1L_ERR_ARG;
    Scan<T> c;
    L1L_TRY(scan_setup<T>(X, n, m, lambdas, nl, nullptr, nullptr, nullptr, ws, ws_bytes, stream,
                          0u, c));
    L1L_TRY(scan_prep<T>(X, c));
    L1L_TRY(scan_pairs<T>(c, lambdas, nl, jlist, jlist ? nj : m));
    L1L_TRY(scan_argmin<T>(c, nl, out_v, out_obj, out_jstar));
    g_last_launches = c.launches;
    return L1L_OK;
}

const double k_zero_lambda = 0.0;

// Workspace of the lambda-path calls: the fit layout for one lambda, then the
// scan scratch, the big-pair list and counters, and the big-pair slices.
struct PathLayout {
    Layout L;
    size_t scan_tmp, big, big_count, scratch, total;
};

bool make_path_layout(int dtype, int64_t n, int64_t m, PathLayout &P) {
    if (n > (dtype == L1L_DTYPE_F32 ? path_max_rows<float>() : path_max_rows<double>()))
        return false;
    if (!make_layout(dtype, n, m, 1, P.L)) return false;
    int64_t mm;
    if (!mul_ok(m, m, mm) || mm > ((int64_t)1 << 40)) return false;
    size_t off = P.L.total;
    P.scan_tmp = off;
    off = al256(off + path_scan_scratch(mm));
    P.big = off;
    off = al256(off + (size_t)mm * 4);
    P.big_count = off;
    off += 256;
    P.scratch = off;
    const size_t sl = dtype == L1L_DTYPE_F32 ? path_slice_bytes<float>(n) : path_slice_bytes<double>(n);
    off = al256(off + (size_t)path_big_workers() * sl);
    P.total = off;
    return true;
}

template <typename T>
int path_count_impl(const T *X, int64_t n, int64_t m, int64_t *offsets, void *ws, size_t ws_bytes,
                    void *stream) {
    g_last_launches = 0;
    if (!offsets) return L1L_ERR_ARG;
    PathLayout P;
    if (X && n >= 1 && m >= 1 && !make_path_layout(dtype_of<T>(), n, m, P))
        return L1L_ERR_UNSUPPORTED;
    if (X && n >= 1 && m >= 1 && (!ws || ws_bytes < P.total)) return L1L_ERR_WORKSPACE;
    Scan<T> c;
    L1L_TRY(scan_setup<T>(X, n, m, &k_zero_lambda, 1, nullptr, nullptr, nullptr, ws, ws_bytes,
                          stream, 0u, c));
    L1L_TRY(scan_prep<T>(X, c));
    L1L_TRY(scan_pairs<T>(c, &k_zero_lambda, 1, nullptr, m));  // lambda = 0 medians
    if (launch_path<T>(true, c.a.Xt, c.a.Xf, c.a.ci, n, m, c.a.ldn, c.a.v_all, offsets,
                       reinterpret_cast<int64_t *>(c.base + P.scan_tmp), nullptr, nullptr, nullptr,
                       nullptr, nullptr, nullptr, nullptr, c.a.status, c.sms, c.st,
                       c.launches) !=
        cudaSuccess)
        return L1L_ERR_CUDA;
    g_last_launches = c.launches;
    return L1L_OK;
}

template <typename T>
int path_write_impl(const T *X, int64_t n, int64_t m, const int64_t *offsets, double *out_lam,
                    T *out_v, double *out_res, int32_t *out_len, void *ws, size_t ws_bytes,
                    void *stream) {
    g_last_launches = 0;
    if (!X || !offsets || !out_lam || !out_v || !out_len || n < 1 || m < 1) return L1L_ERR_ARG;
    if (n > max_rows_pairs<T>() || m > 0x7FFFFFFF) return L1L_ERR_UNSUPPORTED;
    PathLayout P;
    if (!make_path_layout(dtype_of<T>(), n, m, P)) return L1L_ERR_UNSUPPORTED;
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255) != 0 || ws_bytes < P.total)
        return L1L_ERR_WORKSPACE;
    const int sms = num_sms();
    if (sms <= 0) return L1L_ERR_CUDA;
    unsigned char *base = static_cast<unsigned char *>(ws);
    int launches = 0;
    if (launch_path<T>(false, reinterpret_cast<const T *>(base + P.L.Xt),
                       reinterpret_cast<const float *>(base + P.L.Xf),
                       reinterpret_cast<const ColInfo *>(base + P.L.colinfo), n, m, P.L.ldn,
                       reinterpret_cast<const T *>(base + P.L.v_all),
                       const_cast<int64_t *>(offsets), nullptr, out_lam, out_v, out_res, out_len,
                       reinterpret_cast<int32_t *>(base + P.big),
                       reinterpret_cast<uint32_t *>(base + P.big_count), base + P.scratch,
                       reinterpret_cast<uint32_t *>(base + P.L.status), sms,
                       static_cast<cudaStream_t>(stream), launches) != cudaSuccess)
        return L1L_ERR_CUDA;
    g_last_launches = launches;
    return L1L_OK;
}

// Every feature of the proposer into raw / stdz: the column features of the
// staged copy, then the restricted objective: row norms, the R heaviest rows
// copied out, and this library's own fit of them (z only, at lambda) in the
// workspace region after the main one; its device status joins the main
// status word.
template <typename T>
int proposer_features(const T *X, int64_t n, int64_t m, double lambda, Scan<T> &c,
                      const ProposedLayout &P, float *raw, float *stdz) {
    if (launch_colfeat<T>(c.a.Xt, c.a.ldn, n, m, raw, c.st, c.launches) != cudaSuccess)
        return L1L_ERR_CUDA;
    float *rho = reinterpret_cast<float *>(c.base + P.rho);
    int32_t *rows = reinterpret_cast<int32_t *>(c.base + P.rows);
    T *xr = reinterpret_cast<T *>(c.base + P.xr);
    if (launch_heavy_rows<T>(X, n, m, P.R, rho, rows, xr, c.st, c.launches) != cudaSuccess)
        return L1L_ERR_CUDA;
    Scan<T> p;
    L1L_TRY(scan_setup<T>(xr, P.R, m, &lambda, 1, nullptr, nullptr, nullptr, c.base + P.pws,
                          P.pws_bytes, c.st, 0u, p));
    L1L_TRY(scan_prep<T>(xr, p));
    L1L_TRY(scan_pairs<T>(p, &lambda, 1, nullptr, m));
    c.launches += p.launches;
    if (launch_setfeat(p.z, m, 3, raw, c.st, c.launches) != cudaSuccess ||
        launch_status_or(c.a.status, p.a.status, c.st, c.launches) != cudaSuccess ||
        launch_featstd(raw, m, stdz, c.st, c.launches) != cudaSuccess)
        return L1L_ERR_CUDA;
    return L1L_OK;
}

template <typename T>
int features_impl(const T *X, int64_t n, int64_t m, double lambda, float *out_raw,
                  float *out_std, void *ws, size_t ws_bytes, void *stream) {
    g_last_launches = 0;
    if (!X || !out_std || n < 1 || m < 1) return L1L_ERR_ARG;
    ProposedLayout P;
    if (!make_proposed_layout(dtype_of<T>(), n, m, 1, P)) return L1L_ERR_UNSUPPORTED;
    if (ws_bytes < P.total) return L1L_ERR_WORKSPACE;
    Scan<T> c;
    L1L_TRY(scan_setup<T>(X, n, m, &lambda, 1, nullptr, nullptr, nullptr, ws, ws_bytes, stream,
                          0u, c));
    L1L_TRY(scan_prep<T>(X, c));
    float *raw = out_raw ? out_raw : reinterpret_cast<float *>(c.base + c.L.feat_raw);
    L1L_TRY(proposer_features<T>(X, n, m, lambda, c, P, raw, out_std));
    g_last_launches = c.launches;
    return L1L_OK;
}

template <typename T>
int proposed_impl(const T *X, int64_t n, int64_t m, const double *lambdas, int64_t nl,
                  const l1line_mlp *mlp, int64_t K, int32_t *out_idx, T *out_v, double *out_obj,
                  int32_t *out_jstar, void *ws, size_t ws_bytes, void *stream) {
    g_last_launches = 0;
    if (!X || !lambdas || !mlp || !out_v || !out_obj || !out_jstar || n < 1 || m < 1 || nl < 1)
        return L1L_ERR_ARG;
    if (K < 1 || K > m) return L1L_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(mlp) & 15) != 0) return L1L_ERR_ARG;
    ProposedLayout P;
    if (!make_proposed_layout(dtype_of<T>(), n, m, nl, P)) return L1L_ERR_UNSUPPORTED;
    if (ws_bytes < P.total) return L1L_ERR_WORKSPACE;
    Scan<T> c;
    L1L_TRY(scan_setup<T>(X, n, m, lambdas, nl, nullptr, nullptr, nullptr, ws, ws_bytes, stream,
                          0u, c));
    L1L_TRY(scan_prep<T>(X, c));
    float *raw = reinterpret_cast<float *>(c.base + c.L.feat_raw);
    float *stdz = reinterpret_cast<float *>(c.base + c.L.feat_std);
    float *score = reinterpret_cast<float *>(c.base + c.L.score);
    int32_t *idx = out_idx ? out_idx : reinterpret_cast<int32_t *>(c.base + c.L.idx);
    L1L_TRY(proposer_features<T>(X, n, m, lambdas[0], c, P, raw, stdz));
    if (launch_mlp_forward(stdz, nullptr, m, mlp, score, c.st, c.launches) != cudaSuccess ||
        launch_topk(score, m, (int)K, idx, c.st, c.launches) != cudaSuccess)
        return L1L_ERR_CUDA;
    L1L_TRY(scan_pairs<T>(c, lambdas, nl, idx, K));
    L1L_TRY(scan_argmin<T>(c, nl, out_v, out_obj, out_jstar));
    g_last_launches = c.launches;
    return L1L_OK;
}

}  // namespace

extern "C" {

int64_t l1line_max_rows(int dtype) {
    if (dtype == L1L_DTYPE_F32) return max_rows_pairs<float>();
    if (dtype == L1L_DTYPE_F64) return max_rows_pairs<double>();
    return 0;
}

size_t l1line_workspace_bytes(int dtype, int64_t n, int64_t m, int64_t n_lambda) {
    if (dtype != L1L_DTYPE_F32 && dtype != L1L_DTYPE_F64) return 0;
    Layout L;
    if (!make_layout(dtype, n, m, n_lambda, L)) return 0;
    return L.total;
}

int l1line_scan_ex_f32(const float *X, int64_t n, int64_t m, const double *lambdas,
                       int64_t n_lambda, float *v_all, double *s_all, double *z_all,
                       void *workspace, size_t workspace_bytes, void *stream, uint32_t flags) {
    L1L_ENTRY("l1line_scan_ex_f32");
    return scan_impl<float>(X, n, m, lambdas, n_lambda, v_all, s_all, z_all, workspace,
                            workspace_bytes, stream, flags);
}

int l1line_scan_ex_f64(const double *X, int64_t n, int64_t m, const double *lambdas,
                       int64_t n_lambda, double *v_all, double *s_all, double *z_all,
                       void *workspace, size_t workspace_bytes, void *stream, uint32_t flags) {
    L1L_ENTRY("l1line_scan_ex_f64");
    return scan_impl<double>(X, n, m, lambdas, n_lambda, v_all, s_all, z_all, workspace,
                             workspace_bytes, stream, flags);
}

int l1line_scan_f32(const float *X, int64_t n, int64_t m, const double *lambdas,
                    int64_t n_lambda, float *v_all, double *s_all, double *z_all,
                    void *workspace, size_t workspace_bytes, void *stream) {
    L1L_ENTRY("l1line_scan_f32");
    return l1line_scan_ex_f32(X, n, m, lambdas, n_lambda, v_all, s_all, z_all, workspace,
                              workspace_bytes, stream, 0u);
}

int l1line_scan_f64(const double *X, int64_t n, int64_t m, const double *lambdas,
                    int64_t n_lambda, double *v_all, double *s_all, double *z_all,
                    void *workspace, size_t workspace_bytes, void *stream) {
    L1L_ENTRY("l1line_scan_f64");
    return l1line_scan_ex_f64(X, n, m, lambdas, n_lambda, v_all, s_all, z_all, workspace,
                              workspace_bytes, stream, 0u);
}

int l1line_fit_f32(const float *X, int64_t n, int64_t m, const double *lambdas,
                   int64_t n_lambda, float *out_v, double *out_obj, int32_t *out_jstar,
                   void *workspace, size_t workspace_bytes, void *stream) {
    L1L_ENTRY("l1line_fit_f32");
    return fit_impl<float>(X, n, m, lambdas, n_lambda, nullptr, 0, out_v, out_obj, out_jstar,
                           workspace, workspace_bytes, stream);
}

int l1line_fit_f64(const double *X, int64_t n, int64_t m, const double *lambdas,
                   int64_t n_lambda, double *out_v, double *out_obj, int32_t *out_jstar,
                   void *workspace, size_t workspace_bytes, void *stream) {
    L1L_ENTRY("l1line_fit_f64");
    return fit_impl<double>(X, n, m, lambdas, n_lambda, nullptr, 0, out_v, out_obj, out_jstar,
                            workspace, workspace_bytes, stream);
}

int l1line_fit_subset_f32(const float *X, int64_t n, int64_t m, const double *lambdas,
                          int64_t n_lambda, const int32_t *jhat_list, int64_t K, float *out_v,
                          double *out_obj, int32_t *out_jstar, void *workspace,
                          size_t workspace_bytes, void *stream) {
    L1L_ENTRY("l1line_fit_subset_f32");
    if (!jhat_list) return L1L_ERR_ARG;
    return fit_impl<float>(X, n, m, lambdas, n_lambda, jhat_list, K, out_v, out_obj, out_jstar,
                           workspace, workspace_bytes, stream);
}

int l1line_fit_subset_f64(const double *X, int64_t n, int64_t m, const double *lambdas,
                          int64_t n_lambda, const int32_t *jhat_list, int64_t K, double *out_v,
                          double *out_obj, int32_t *out_jstar, void *workspace,
                          size_t workspace_bytes, void *stream) {
    L1L_ENTRY("l1line_fit_subset_f64");
    if (!jhat_list) return L1L_ERR_ARG;
    return fit_impl<double>(X, n, m, lambdas, n_lambda, jhat_list, K, out_v, out_obj, out_jstar,
                            workspace, workspace_bytes, stream);
}

int64_t l1line_proposer_rows(int64_t n) { return proposer_rows(n); }

size_t l1line_proposed_workspace_bytes(int dtype, int64_t n, int64_t m, int64_t n_lambda) {
    if (dtype != L1L_DTYPE_F32 && dtype != L1L_DTYPE_F64) return 0;
    ProposedLayout P;
    if (!make_proposed_layout(dtype, n, m, n_lambda, P)) return 0;
    return P.total;
}

int l1line_features_f32(const float *X, int64_t n, int64_t m, double lambda, float *out_raw,
                        float *out_std, void *workspace, size_t workspace_bytes, void *stream) {
    L1L_ENTRY("l1line_features_f32");
    return features_impl<float>(X, n, m, lambda, out_raw, out_std, workspace, workspace_bytes,
                                stream);
}

int l1line_features_f64(const double *X, int64_t n, int64_t m, double lambda, float *out_raw,
                        float *out_std, void *workspace, size_t workspace_bytes, void *stream) {
    L1L_ENTRY("l1line_features_f64");
    return features_impl<double>(X, n, m, lambda, out_raw, out_std, workspace, workspace_bytes,
                                 stream);
}

int l1line_mlp_forward(const float *feat, const int32_t *rows, int64_t N, const l1line_mlp *mlp,
                       float *scores, void *stream) {
    L1L_ENTRY("l1line_mlp_forward");
    g_last_launches = 0;
    if (!feat || !mlp || !scores || N < 1) return L1L_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(mlp) & 15) != 0) return L1L_ERR_ARG;
    if ((N + MLP_TILE - 1) / MLP_TILE > 0x7FFFFFFF) return L1L_ERR_UNSUPPORTED;
    int launches = 0;
    if (launch_mlp_forward(feat, rows, N, mlp, scores, static_cast<cudaStream_t>(stream),
                           launches) != cudaSuccess)
        return L1L_ERR_CUDA;
    g_last_launches = launches;
    return L1L_OK;
}

size_t l1line_mlp_workspace_bytes(int64_t N) {
    if (N < 1 || N > ((int64_t)1 << 34)) return 0;
    return al256((size_t)((N + MLP_TILE - 1) / MLP_TILE) * L1L_MLP_PARAMS * sizeof(float));
}

int l1line_mlp_backward(const float *feat, const int32_t *rows, int64_t N, const l1line_mlp *mlp,
                        const float *dscores, float *grad, void *workspace,
                        size_t workspace_bytes, void *stream) {
    L1L_ENTRY("l1line_mlp_backward");
    g_last_launches = 0;
    if (!feat || !mlp || !dscores || !grad || N < 1) return L1L_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(mlp) & 15) != 0) return L1L_ERR_ARG;
    const size_t need = l1line_mlp_workspace_bytes(N);
    if (need == 0) return L1L_ERR_UNSUPPORTED;
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) != 0 ||
        workspace_bytes < need)
        return L1L_ERR_WORKSPACE;
    int launches = 0;
    if (launch_mlp_backward(feat, rows, N, mlp, dscores, static_cast<float *>(workspace), grad,
                            static_cast<cudaStream_t>(stream), launches) != cudaSuccess)
        return L1L_ERR_CUDA;
    g_last_launches = launches;
    return L1L_OK;
}

int l1line_rank_loss(const float *scores, const float *targets, const int32_t *rows,
                     const int64_t *offsets, int64_t n_inst, float *dscores, float *loss,
                     void *stream) {
    L1L_ENTRY("l1line_rank_loss");
    g_last_launches = 0;
    if (!scores || !targets || !offsets || !dscores || !loss || n_inst < 1) return L1L_ERR_ARG;
    if (n_inst > 0x7FFFFFFF) return L1L_ERR_UNSUPPORTED;
    int launches = 0;
    if (launch_rank_loss(scores, targets, rows, offsets, n_inst, dscores, loss,
                         static_cast<cudaStream_t>(stream), launches) != cudaSuccess)
        return L1L_ERR_CUDA;
    g_last_launches = launches;
    return L1L_OK;
}

int l1line_adam_step(float *theta, const float *grad, float *m1, float *m2, int64_t step,
                     float lr, float beta1, float beta2, float eps, l1line_mlp *mlp,
                     void *stream) {
    L1L_ENTRY("l1line_adam_step");
    g_last_launches = 0;
    if (!theta || !grad || !m1 || !m2 || step < 1) return L1L_ERR_ARG;
    if (!(lr >= 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) ||
        !(eps >= 0.0f) || std::isinf(lr) || std::isinf(eps))
        return L1L_ERR_ARG;
    if (mlp && (reinterpret_cast<uintptr_t>(mlp) & 15) != 0) return L1L_ERR_ARG;
    // bias corrections 1 / (1 - beta^step), formed in double on the host
    const double c1 = 1.0 / (1.0 - std::pow((double)beta1, (double)step));
    const double c2 = 1.0 / (1.0 - std::pow((double)beta2, (double)step));
    int launches = 0;
    if (launch_adam(theta, grad, m1, m2, lr, beta1, beta2, eps, (float)c1, (float)c2, mlp,
                    static_cast<cudaStream_t>(stream), launches) != cudaSuccess)
        return L1L_ERR_CUDA;
    g_last_launches = launches;
    return L1L_OK;
}

int l1line_mlp_pack(const float *theta, l1line_mlp *mlp, void *stream) {
    L1L_ENTRY("l1line_mlp_pack");
    g_last_launches = 0;
    if (!theta || !mlp || (reinterpret_cast<uintptr_t>(mlp) & 15) != 0) return L1L_ERR_ARG;
    int launches = 0;
    if (launch_mlp_pack(theta, mlp, static_cast<cudaStream_t>(stream), launches) != cudaSuccess)
        return L1L_ERR_CUDA;
    g_last_launches = launches;
    return L1L_OK;
}

int l1line_topk(const float *scores, int64_t m, int64_t K, int32_t *out_idx, void *stream) {
    L1L_ENTRY("l1line_topk");
    g_last_launches = 0;
    if (!scores || !out_idx || m < 1 || K < 1 || K > m) return L1L_ERR_ARG;
    if (m > 0x7FFFFFFF) return L1L_ERR_UNSUPPORTED;
    int launches = 0;
    if (launch_topk(scores, m, (int)K, out_idx, static_cast<cudaStream_t>(stream), launches) !=
        cudaSuccess)
        return L1L_ERR_CUDA;
    g_last_launches = launches;
    return L1L_OK;
}

int l1line_fit_proposed_f32(const float *X, int64_t n, int64_t m, const double *lambdas,
                            int64_t n_lambda, const l1line_mlp *mlp, int64_t K, int32_t *out_idx,
                            float *out_v, double *out_obj, int32_t *out_jstar, void *workspace,
                            size_t workspace_bytes, void *stream) {
    L1L_ENTRY("l1line_fit_proposed_f32");
    return proposed_impl<float>(X, n, m, lambdas, n_lambda, mlp, K, out_idx, out_v, out_obj,
                                out_jstar, workspace, workspace_bytes, stream);
}

int l1line_fit_proposed_f64(const double *X, int64_t n, int64_t m, const double *lambdas,
                            int64_t n_lambda, const l1line_mlp *mlp, int64_t K,
                            int32_t *out_idx, double *out_v, double *out_obj,
                            int32_t *out_jstar, void *workspace, size_t workspace_bytes,
                            void *stream) {
    L1L_ENTRY("l1line_fit_proposed_f64");
    return proposed_impl<double>(X, n, m, lambdas, n_lambda, mlp, K, out_idx, out_v, out_obj,
                                 out_jstar, workspace, workspace_bytes, stream);
}

int64_t l1line_path_max_rows(int dtype) {
    if (dtype == L1L_DTYPE_F32) return path_max_rows<float>();
    if (dtype == L1L_DTYPE_F64) return path_max_rows<double>();
    return 0;
}

size_t l1line_path_workspace_bytes(int dtype, int64_t n, int64_t m) {
    if (dtype != L1L_DTYPE_F32 && dtype != L1L_DTYPE_F64) return 0;
    PathLayout P;
    if (!make_path_layout(dtype, n, m, P)) return 0;
    return P.total;
}

int l1line_path_count_f32(const float *X, int64_t n, int64_t m, int64_t *offsets,
                          void *workspace, size_t workspace_bytes, void *stream) {
    L1L_ENTRY("l1line_path_count_f32");
    return path_count_impl<float>(X, n, m, offsets, workspace, workspace_bytes, stream);
}

int l1line_path_count_f64(const double *X, int64_t n, int64_t m, int64_t *offsets,
                          void *workspace, size_t workspace_bytes, void *stream) {
    L1L_ENTRY("l1line_path_count_f64");
    return path_count_impl<double>(X, n, m, offsets, workspace, workspace_bytes, stream);
}

int l1line_path_write_f32(const float *X, int64_t n, int64_t m, const int64_t *offsets,
                          double *out_lambda, float *out_v, double *out_resid, int32_t *out_len,
                          void *workspace, size_t workspace_bytes, void *stream) {
    L1L_ENTRY("l1line_path_write_f32");
    return path_write_impl<float>(X, n, m, offsets, out_lambda, out_v, out_resid, out_len,
                                  workspace, workspace_bytes, stream);
}

int l1line_path_write_f64(const double *X, int64_t n, int64_t m, const int64_t *offsets,
                          double *out_lambda, double *out_v, double *out_resid, int32_t *out_len,
                          void *workspace, size_t workspace_bytes, void *stream) {
    L1L_ENTRY("l1line_path_write_f64");
    return path_write_impl<double>(X, n, m, offsets, out_lambda, out_v, out_resid, out_len,
                                   workspace, workspace_bytes, stream);
}

size_t l1line_solution_path_workspace_bytes(int64_t m, int64_t entries) {
    if (m < 1 || entries < 1 || m > 0x7FFFFFFF || entries > ((int64_t)1 << 40)) return 0;
    if ((double)m * (double)(m + 2) > 1e12) return 0;
    return solpath_bytes(m, entries);
}

}  // extern "C"

namespace {
template <typename T>
int solution_path_impl(int64_t m, const int64_t *offsets, const double *lam, const T *v,
                       const double *resid, const int32_t *len, int64_t entries,
                       double *out_start, int32_t *out_jhat, double *out_intercept,
                       double *out_slope, T *out_v, int64_t *out_count, int64_t cap, void *ws,
                       size_t ws_bytes, void *stream) {
    g_last_launches = 0;
    if (!offsets || !lam || !v || !resid || !len || !out_start || !out_jhat || !out_intercept ||
        !out_slope || !out_count || m < 1 || entries < 1 || cap < 1)
        return L1L_ERR_ARG;
    const size_t need = l1line_solution_path_workspace_bytes(m, entries);
    if (need == 0) return L1L_ERR_UNSUPPORTED;
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255) != 0 || ws_bytes < need)
        return L1L_ERR_WORKSPACE;
    int launches = 0;
    if (launch_solpath<T>(m, offsets, len, lam, v, resid, static_cast<unsigned char *>(ws),
                          entries, out_start, out_jhat, out_intercept, out_slope, out_v,
                          out_count, cap, static_cast<cudaStream_t>(stream), launches) !=
        cudaSuccess)
        return L1L_ERR_CUDA;
    g_last_launches = launches;
    return L1L_OK;
}
}  // namespace

extern "C" {

int l1line_solution_path_f32(int64_t m, const int64_t *offsets, const double *lambda,
                             const float *v, const double *resid, const int32_t *len,
                             int64_t entries, double *out_start, int32_t *out_jhat,
                             double *out_intercept, double *out_slope, float *out_v,
                             int64_t *out_count, int64_t cap, void *workspace,
                             size_t workspace_bytes, void *stream) {
    L1L_ENTRY("l1line_solution_path_f32");
    return solution_path_impl<float>(m, offsets, lambda, v, resid, len, entries, out_start,
                                     out_jhat, out_intercept, out_slope, out_v, out_count, cap,
                                     workspace, workspace_bytes, stream);
}

int l1line_solution_path_f64(int64_t m, const int64_t *offsets, const double *lambda,
                             const double *v, const double *resid, const int32_t *len,
                             int64_t entries, double *out_start, int32_t *out_jhat,
                             double *out_intercept, double *out_slope, double *out_v,
                             int64_t *out_count, int64_t cap, void *workspace,
                             size_t workspace_bytes, void *stream) {
    L1L_ENTRY("l1line_solution_path_f64");
    return solution_path_impl<double>(m, offsets, lambda, v, resid, len, entries, out_start,
                                      out_jhat, out_intercept, out_slope, out_v, out_count, cap,
                                      workspace, workspace_bytes, stream);
}

size_t l1line_components_workspace_bytes(int dtype, int64_t n, int64_t m) {
    const size_t fw = l1line_workspace_bytes(dtype, n, m, 1);
    if (fw == 0) return 0;
    const size_t es = dtype == L1L_DTYPE_F32 ? 4 : 8;
    return fw + 2 * al256((size_t)n * (size_t)m * es);
}

}  // extern "C"

namespace {
template <typename T>
int components_impl(const T *X, int64_t n, int64_t m, double lambda, int64_t ncomp, T *out_v,
                    double *out_obj, int32_t *out_jstar, void *ws, size_t ws_bytes,
                    void *stream) {
    if (!X || !out_v || !out_obj || !out_jstar || n < 1 || m < 1 || ncomp < 1)
        return L1L_ERR_ARG;
    if (!(lambda >= 0.0) || std::isinf(lambda)) return L1L_ERR_ARG;
    const size_t fw = l1line_workspace_bytes(dtype_of<T>(), n, m, 1);
    const size_t need = l1line_components_workspace_bytes(dtype_of<T>(), n, m);
    if (fw == 0 || need == 0) return L1L_ERR_UNSUPPORTED;
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255) != 0 || ws_bytes < need)
        return L1L_ERR_WORKSPACE;
    const int sms = num_sms();
    if (sms <= 0) return L1L_ERR_CUDA;
    unsigned char *base = static_cast<unsigned char *>(ws);
    T *buf[2] = {reinterpret_cast<T *>(base + fw),
                 reinterpret_cast<T *>(base + fw + al256((size_t)n * (size_t)m * sizeof(T)))};
    const T *cur = X;
    int launches = 0;
    for (int64_t c = 0; c < ncomp; ++c) {
        L1L_TRY(fit_impl<T>(cur, n, m, &lambda, 1, nullptr, 0, out_v + c * m, out_obj + c,
                            out_jstar + c, ws, fw, stream));
        launches += g_last_launches;
        if (c + 1 < ncomp) {
            T *next = buf[c & 1];
            if (launch_deflate<T>(cur, next, n, m, out_jstar + c, out_v + c * m, sms,
                                  static_cast<cudaStream_t>(stream), launches) != cudaSuccess)
                return L1L_ERR_CUDA;
            cur = next;
        }
    }
    g_last_launches = launches;
    return L1L_OK;
}
}  // namespace

extern "C" {

int l1line_components_f32(const float *X, int64_t n, int64_t m, double lambda, int64_t ncomp,
                          float *out_v, double *out_obj, int32_t *out_jstar, void *workspace,
                          size_t workspace_bytes, void *stream) {
    L1L_ENTRY("l1line_components_f32");
    return components_impl<float>(X, n, m, lambda, ncomp, out_v, out_obj, out_jstar, workspace,
                                  workspace_bytes, stream);
}

int l1line_components_f64(const double *X, int64_t n, int64_t m, double lambda, int64_t ncomp,
                          double *out_v, double *out_obj, int32_t *out_jstar, void *workspace,
                          size_t workspace_bytes, void *stream) {
    L1L_ENTRY("l1line_components_f64");
    return components_impl<double>(X, n, m, lambda, ncomp, out_v, out_obj, out_jstar, workspace,
                                   workspace_bytes, stream);
}

int l1line_status(void *workspace, void *stream) {
    L1L_ENTRY("l1line_status");
    return status_of(workspace, stream);
}

}  // extern "C"

namespace {
int status_of(void *workspace, void *stream) {
    if (!workspace) return L1L_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(st) != cudaSuccess) return L1L_ERR_CUDA;
    uint32_t w = 0;
    if (cudaMemcpy(&w, workspace, sizeof(w), cudaMemcpyDeviceToHost) != cudaSuccess)
        return L1L_ERR_CUDA;
    if (w & ST_NONFINITE) return L1L_ERR_NONFINITE;
    if (w & ST_TIMEOUT) return L1L_ERR_TIMEOUT;
    if (w & ST_INTERNAL) return L1L_ERR_INTERNAL;
    if (w & ST_BADINDEX) return L1L_ERR_ARG;
    return L1L_OK;
}
}  // namespace

extern "C" {

const char *l1line_status_string(int status) {
    switch (status) {
    case L1L_OK: return "ok";
    case L1L_ERR_ARG: return "invalid argument";
    case L1L_ERR_NONFINITE: return "input holds NaN or infinity";
    case L1L_ERR_CUDA: return "CUDA runtime error";
    case L1L_ERR_WORKSPACE: return "workspace missing, too small or misaligned";
    case L1L_ERR_TIMEOUT: return "bounded device-side wait ran out";
    case L1L_ERR_UNSUPPORTED: return "size not supported by the kernels";
    case L1L_ERR_INTERNAL: return "device-side invariant failed";
    default: return "unknown status";
    }
}

int l1line_last_launch_count(void) { return g_last_launches; }

#if L1L_CHECKS
extern "C" long long l1l_checks_shape_0_0(int, int *);
extern "C" long long l1l_checks_shape_1_0(int, int *);
extern "C" long long l1l_checks_shape_2_0(int, int *);
extern "C" long long l1l_checks_shape_0_1(int, int *);
extern "C" long long l1l_checks_shape_1_1(int, int *);
extern "C" long long l1l_checks_shape_2_1(int, int *);
extern "C" long long l1l_checks_batch(int, int *);
extern "C" long long l1l_checks_exact(int, int *);
extern "C" long long l1l_checks_path(int, int *);
extern "C" long long l1l_checks_solpath(int, int *);
extern "C" long long l1l_checks_propose(int, int *);
extern "C" long long l1l_checks_large(int, int *);
#endif

int64_t l1line_check_hits(int reset, int *line) {
#if L1L_CHECKS
    if (cudaDeviceSynchronize() != cudaSuccess) return -2;
    long long (*readers[])(int, int *) = {l1l_checks_shape_0_0, l1l_checks_shape_1_0,
                                          l1l_checks_shape_2_0, l1l_checks_shape_0_1,
                                          l1l_checks_shape_1_1, l1l_checks_shape_2_1,
                                          l1l_checks_batch, l1l_checks_exact,
                                          l1l_checks_path, l1l_checks_solpath,
                                          l1l_checks_propose, l1l_checks_large};
    long long total = 0;
    for (auto r : readers) {
        const long long h = r(reset, line);
        if (h < 0) return -2;
        total += h;
    }
    return total;
#else
    (void)reset;
    (void)line;
    return -1;
#endif
}

int l1line_set_tuning(const l1line_tuning *t) {
    if (!t) {
        g_tune = Tune();
        return L1L_OK;
    }
    if (t->warps < 0 || t->warps > 16 || t->ctas_per_sm < 0 || t->ctas_per_sm > 3 ||
        t->kchunk < 0 || t->d0 < 0 || t->d0 > 24 || t->batch_classes < 0 ||
        t->batch_classes > MAX_BATCH_CLASSES || t->column < 0 || t->column > 2)
        return L1L_ERR_ARG;
    g_tune.warps = t->warps;
    g_tune.ctas = t->ctas_per_sm;
    g_tune.kchunk = t->kchunk;
    g_tune.d0 = t->d0;
    g_tune.batch_classes = t->batch_classes;
    g_tune.column = t->column;
    return L1L_OK;
}

int l1line_plan(int dtype, int64_t n, int64_t m, int64_t nj, l1line_tuning *out) {
    if (!out || n < 1 || m < 1 || nj < 1) return L1L_ERR_ARG;
    if (dtype != L1L_DTYPE_F32 && dtype != L1L_DTYPE_F64) return L1L_ERR_ARG;
    const int sms = num_sms();
    if (sms <= 0) return L1L_ERR_CUDA;
    return l1line_plan_for(dtype, n, m, nj, sms, out);
}

int l1line_plan_for(int dtype, int64_t n, int64_t m, int64_t nj, int sms, l1line_tuning *out) {
    if (!out || n < 1 || m < 1 || nj < 1 || sms < 1) return L1L_ERR_ARG;
    if (dtype != L1L_DTYPE_F32 && dtype != L1L_DTYPE_F64) return L1L_ERR_ARG;
    const PairPlan p = dtype == L1L_DTYPE_F32 ? plan_pairs<float>(n, m, sms, nj, g_tune)
                                              : plan_pairs<double>(n, m, sms, nj, g_tune);
    if (p.warps == 0) return L1L_ERR_UNSUPPORTED;
    out->warps = p.warps;
    out->ctas_per_sm = p.ctas;
    out->kchunk = p.kchunk;
    out->d0 = p.d0;
    out->batch_classes = g_tune.batch_classes;
    out->column = p.cs ? 1 : 2;
    return L1L_OK;
}

int l1line_probe(int kind, const void *buf, size_t bytes, int reps, void *sink, void *stream,
                 double *bytes_read) {
    L1L_ENTRY("l1line_probe");
    g_last_launches = 0;
    if (!sink || !bytes_read || reps < 1 || (reinterpret_cast<uintptr_t>(sink) & 3) != 0)
        return L1L_ERR_ARG;
    if (kind != L1L_PROBE_L2 && kind != L1L_PROBE_SMEM) return L1L_ERR_ARG;
    if (kind == L1L_PROBE_L2 &&
        (!buf || bytes < 16 || (reinterpret_cast<uintptr_t>(buf) & 15) != 0))
        return L1L_ERR_ARG;
    const int sms = num_sms();
    if (sms <= 0) return L1L_ERR_CUDA;
    int launches = 0;
    if (launch_probe(kind == L1L_PROBE_L2 ? PROBE_L2 : PROBE_SMEM, buf, bytes, reps,
                     static_cast<unsigned *>(sink), sms, static_cast<cudaStream_t>(stream),
                     bytes_read, launches) != cudaSuccess)
        return L1L_ERR_CUDA;
    g_last_launches = launches;
    return L1L_OK;
}

int l1line_profile_events(void *start, void *stop) {
    if (start && stop) {
        g_ev_start = static_cast<cudaEvent_t>(start);
        g_ev_stop = static_cast<cudaEvent_t>(stop);
    } else {
        g_ev_start = g_ev_stop = nullptr;
    }
    return L1L_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched fit
// ---------------------------------------------------------------------------
namespace {

struct BatchShape {
    std::vector<int> order;  // processing order (size class, then largest work first) -> caller index
    size_t ws_total = 0;
    int64_t max_n = 0;
    bool multi = false;
};

// Splits the batch into at most MAX_BATCH_CLASSES size classes by n, each run
// as its own persistent pair launch with shared memory laid out for the
// class's largest n: a few large instances otherwise set the occupancy of
// every small one.  Cost model: a class takes (its pair-rows, the sum of
// n m^2 nl) / (resident warps of its plan).  Classes are runs of the instances
// ordered by n (cuts only where n changes); best_split (batch_split.h) finds
// the best split into k classes by dynamic programming for each k.  Unless
// the tuning fixes k, the planner adds a class while the model puts it at
// least 5% below the best with one class fewer.  Reorders `order`
// (stably, so largest work first within a class) and returns the instance
// count of each class, largest n first.
template <typename T>
std::vector<int64_t> batch_classes(int64_t batch, const int64_t *ns, const int64_t *ms,
                                   const int64_t *loff, int sms, const Tune &tb,
                                   std::vector<int> &order) {
    const size_t B = (size_t)batch;
    std::vector<int> byn(order);
    std::stable_sort(byn.begin(), byn.end(), [&](int x, int y) { return ns[x] > ns[y]; });
    std::vector<double> S(B + 1, 0.0), rate(B, 0.0);
    for (size_t p = 0; p < B; ++p) {
        const int b = byn[p];
        S[p + 1] = S[p] + (double)ns[b] * ms[b] * ms[b] * (loff[b + 1] - loff[b]);
        if (p == 0 || ns[b] != ns[byn[p - 1]]) {
            const PairPlan pl = plan_pairs<T>(ns[b], 1, sms, 1, tb, false);
            rate[p] = (double)pl.warps * (double)pl.ctas;  // 0 marks no cut here
        }
    }
    const std::vector<size_t> starts =
        best_split(S, rate, MAX_BATCH_CLASSES, tb.batch_classes, 0.05);
    std::vector<int64_t> counts;
    std::vector<int> cls((size_t)batch, 0);
    for (size_t i = 0; i < starts.size(); ++i) {
        const size_t p = starts[i], q = i + 1 < starts.size() ? starts[i + 1] : B;
        for (size_t r = p; r < q; ++r) cls[(size_t)byn[r]] = (int)i;
        counts.push_back((int64_t)(q - p));
    }
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return cls[(size_t)x] < cls[(size_t)y]; });
    return counts;
}

// Validates the shapes and lambda offsets; fills `sh`.  Returns an l1l_status.
int batch_shape(int dtype, int64_t batch, const int64_t *ns, const int64_t *ms,
                const int64_t *loff, BatchShape &sh) {
    if (batch < 1 || !ns || !ms || !loff) return L1L_ERR_ARG;
    if (batch > MAX_BATCH) return L1L_ERR_UNSUPPORTED;
    if (loff[0] != 0) return L1L_ERR_ARG;
    const int64_t es = dtype == L1L_DTYPE_F32 ? 4 : 8;
    const int64_t maxr = dtype == L1L_DTYPE_F32 ? max_rows_pairs<float>() : max_rows_pairs<double>();
    int64_t units = 0, ztasks = 0, pairs = 0;
    size_t regions = 0;
    for (int64_t b = 0; b < batch; ++b) {
        const int64_t nl = loff[b + 1] - loff[b];
        if (ns[b] < 1 || ms[b] < 1 || nl < 1) return L1L_ERR_ARG;
        if (ns[b] > maxr || ms[b] > (1 << 20)) return L1L_ERR_UNSUPPORTED;
        const int64_t ldn = (ns[b] + ROW_PAD - 1) & ~int64_t(ROW_PAD - 1);
        units += ms[b];
        ztasks += nl * ms[b];
        pairs += nl * ms[b] * ms[b];
        regions += inst_layout(ms[b], ldn, nl, (size_t)es).total;
        sh.max_n = std::max(sh.max_n, ns[b]);
        sh.multi = sh.multi || nl >= 3;
    }
    if (loff[batch] > MAX_BATCH_LAMBDAS) return L1L_ERR_UNSUPPORTED;
    // pairs bounds the exact path's list, counted by a uint32
    if (units > 0x7FFFFFFF || ztasks > 0x7FFFFFFF || pairs > ((int64_t)1 << 31))
        return L1L_ERR_UNSUPPORTED;
    sh.ws_total = BATCH_HEAD + al256((size_t)pairs * sizeof(SlowEntry)) + regions;
    sh.order.resize((size_t)batch);
    std::iota(sh.order.begin(), sh.order.end(), 0);
    std::stable_sort(sh.order.begin(), sh.order.end(), [&](int x, int y) {
        const double cx = (double)ns[x] * ms[x] * ms[x] * (loff[x + 1] - loff[x]);
        const double cy = (double)ns[y] * ms[y] * ms[y] * (loff[y + 1] - loff[y]);
        return cx > cy;
    });
    return L1L_OK;
}

template <typename T>
int fit_batched_impl(int64_t batch, const T *const *Xs, const int64_t *ns, const int64_t *ms,
                     const double *lambdas, const int64_t *loff, T *out_v, double *out_obj,
                     int32_t *out_jstar, void *ws, size_t ws_bytes, void *stream, uint32_t flags) {
    g_last_launches = 0;
    if (!Xs || !lambdas || !out_v || !out_obj || !out_jstar) return L1L_ERR_ARG;
    BatchShape sh;
    int rc = batch_shape(dtype_of<T>(), batch, ns, ms, loff, sh);
    if (rc != L1L_OK) return rc;
    for (int64_t t = 0; t < loff[batch]; ++t)
        if (!(lambdas[t] >= 0.0) || std::isinf(lambdas[t])) return L1L_ERR_ARG;
    for (int64_t b = 0; b < batch; ++b)
        if (!Xs[b] || (reinterpret_cast<uintptr_t>(Xs[b]) % sizeof(T)) != 0) return L1L_ERR_ARG;
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255) != 0 || ws_bytes < sh.ws_total)
        return L1L_ERR_WORKSPACE;
    const int sms = num_sms();
    if (sms <= 0) return L1L_ERR_CUDA;
    Tune tb = g_tune;
    tb.kchunk = 0;  // the persistent kernel's unit is a whole column jhat
    // the processing order holds the size classes one after another
    const std::vector<int64_t> counts = batch_classes<T>(batch, ns, ms, loff, sms, tb, sh.order);
    BatchClass cls[MAX_BATCH_CLASSES];
    int nclasses = 0;
    for (int64_t p0 = 0; p0 < batch;) {
        const int64_t p1 = p0 + counts[(size_t)nclasses];
        int64_t mx = 0;
        for (int64_t p = p0; p < p1; ++p) mx = std::max(mx, ns[sh.order[(size_t)p]]);
        BatchClass &c = cls[nclasses++];
        c.plan = plan_pairs<T>(mx, 1, sms, 1, tb, false);
        if (c.plan.warps == 0) return L1L_ERR_UNSUPPORTED;
        c.lay_npad = (int)((mx + ROW_PAD - 1) & ~int64_t(ROW_PAD - 1));
        c.u0 = p0;  // instance range for now; converted to units below
        c.u1 = p1;
        p0 = p1;
    }

    std::unique_ptr<BatchDesc<T>> bd(new BatchDesc<T>());
    std::memset(bd.get(), 0, sizeof(BatchDesc<T>));
    // caller-order output offsets
    std::vector<int64_t> vo((size_t)batch), to((size_t)batch);
    int64_t acc_v = 0, acc_t = 0;
    for (int64_t b = 0; b < batch; ++b) {
        vo[(size_t)b] = acc_v;
        to[(size_t)b] = acc_t;
        const int64_t nl = loff[b + 1] - loff[b];
        acc_v += nl * ms[b];
        acc_t += nl;
    }
    size_t off = BATCH_HEAD;
    int64_t pairs = 0;
    for (int64_t b = 0; b < batch; ++b) pairs += (loff[b + 1] - loff[b]) * ms[b] * ms[b];
    off += al256((size_t)pairs * sizeof(SlowEntry));
    bd->count = (int32_t)batch;
    bd->force_exact = (flags & L1L_FLAG_FORCE_EXACT) ? 1 : 0;
    bd->d0 = cls[0].plan.d0;
    int64_t units = 0, tiles = 0, ztasks = 0, lams = 0;
    for (int64_t p = 0; p < batch; ++p) {
        const int b = sh.order[(size_t)p];
        const int64_t n = ns[b], m = ms[b], nl = loff[b + 1] - loff[b];
        const int64_t ldn = (n + ROW_PAD - 1) & ~int64_t(ROW_PAD - 1);
        BatchInst<T> &in = bd->inst[p];
        in.X = Xs[b];
        in.ws_off = (int64_t)off;
        in.out_v_off = vo[(size_t)b];
        in.out_t_off = (int32_t)to[(size_t)b];
        in.n = (int32_t)n;
        in.m = (int32_t)m;
        in.ldn = (int32_t)ldn;
        in.nl = (int32_t)nl;
        int tmin = 0, tmax = 0;
        for (int64_t t = 0; t < nl; ++t) {
            const double l = lambdas[loff[b] + t];
            bd->lam[lams + t] = l;
            if (l < lambdas[loff[b] + tmin]) tmin = (int)t;
            if (l > lambdas[loff[b] + tmax]) tmax = (int)t;
        }
        in.tl_min = (int16_t)tmin;
        in.tl_max = (int16_t)tmax;
        bd->unit_begin[p] = units;
        bd->tile_begin[p] = (int32_t)tiles;
        bd->ztask_begin[p] = (int32_t)ztasks;
        bd->lam_begin[p] = (int32_t)lams;
        units += m;
        tiles += ((m + 31) / 32) * (ldn / 32);
        ztasks += nl * m;
        lams += nl;
        off += inst_layout(m, ldn, nl, sizeof(T)).total;
    }
    if (tiles > 0x7FFFFFFF) return L1L_ERR_UNSUPPORTED;
    bd->unit_begin[batch] = units;
    bd->tile_begin[batch] = (int32_t)tiles;
    bd->ztask_begin[batch] = (int32_t)ztasks;
    bd->lam_begin[batch] = (int32_t)lams;
    bd->units = units;
    bd->tiles = (int32_t)tiles;
    bd->ztasks = (int32_t)ztasks;
    bd->lams = (int32_t)lams;
    for (int c = 0; c < nclasses; ++c) {
        cls[c].u0 = bd->unit_begin[cls[c].u0];
        cls[c].u1 = bd->unit_begin[cls[c].u1];
    }
    int launches = 0;
    if (launch_batch<T>(*bd, static_cast<unsigned char *>(ws), out_v, out_obj, out_jstar, cls,
                        nclasses, sh.multi, sms, static_cast<cudaStream_t>(stream),
                        launches) != cudaSuccess)
        return L1L_ERR_CUDA;
    g_last_launches = launches;
    return L1L_OK;
}

}  // namespace

extern "C" {

size_t l1line_batched_workspace_bytes(int dtype, int64_t batch, const int64_t *ns,
                                      const int64_t *ms, const int64_t *lambda_offsets) {
    if (dtype != L1L_DTYPE_F32 && dtype != L1L_DTYPE_F64) return 0;
    BatchShape sh;
    if (batch_shape(dtype, batch, ns, ms, lambda_offsets, sh) != L1L_OK) return 0;
    return sh.ws_total;
}

int l1line_fit_batched_f32(int64_t batch, const float *const *Xs, const int64_t *ns,
                           const int64_t *ms, const double *lambdas,
                           const int64_t *lambda_offsets, float *out_v, double *out_obj,
                           int32_t *out_jstar, void *workspace, size_t workspace_bytes,
                           void *stream) {
    L1L_ENTRY("l1line_fit_batched_f32");
    return fit_batched_impl<float>(batch, Xs, ns, ms, lambdas, lambda_offsets, out_v, out_obj,
                                   out_jstar, workspace, workspace_bytes, stream, 0u);
}

int l1line_fit_batched_f64(int64_t batch, const double *const *Xs, const int64_t *ns,
                           const int64_t *ms, const double *lambdas,
                           const int64_t *lambda_offsets, double *out_v, double *out_obj,
                           int32_t *out_jstar, void *workspace, size_t workspace_bytes,
                           void *stream) {
    L1L_ENTRY("l1line_fit_batched_f64");
    return fit_batched_impl<double>(batch, Xs, ns, ms, lambdas, lambda_offsets, out_v, out_obj,
                                    out_jstar, workspace, workspace_bytes, stream, 0u);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// No-allocation fit: the workspace is a fixed array in device memory declared
// by this file.  Host code never uses the array's name as an address (on the
// host it is only a stand-in for the symbol); the device address is looked up
// once per device with cudaGetSymbolAddress while that device is current.
// ---------------------------------------------------------------------------
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[L1L_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 128;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[kMaxDevices] = {};

int noalloc_scratch_address(void **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return L1L_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return L1L_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return L1L_ERR_CUDA;
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return L1L_OK;
}

}  // namespace

extern "C" int l1line_noalloc_status(void *stream) {
    L1L_ENTRY("l1line_noalloc_status");
    void *ws = nullptr;
    const int rc = noalloc_scratch_address(&ws);
    if (rc != L1L_OK) return rc;
    return status_of(ws, stream);
}

extern "C" int l1line_fit_noalloc_f32(const float *X, int64_t n, int64_t m,
                                      const double *lambdas, int64_t n_lambda, float *out_v,
                                      double *out_obj, int32_t *out_jstar, void *stream) {
    L1L_ENTRY("l1line_fit_noalloc_f32");
    if (!X || !lambdas || !out_v || !out_obj || !out_jstar || n < 1 || m < 1 || n_lambda < 1)
        return L1L_ERR_ARG;
    const size_t need = l1line_workspace_bytes(L1L_DTYPE_F32, n, m, n_lambda);
    if (need == 0 || need > L1L_NOALLOC_SCRATCH_BYTES) return L1L_ERR_UNSUPPORTED;
    void *ws = nullptr;
    const int rc = noalloc_scratch_address(&ws);
    if (rc != L1L_OK) return rc;
    // the status word and the exact-path counter are zeroed by the fit itself;
    // every other region of the workspace is fully overwritten before it is read
    return fit_impl<float>(X, n, m, lambdas, n_lambda, nullptr, 0, out_v, out_obj, out_jstar, ws,
                           L1L_NOALLOC_SCRATCH_BYTES, stream);
}
