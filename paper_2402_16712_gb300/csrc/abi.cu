// abi.cu -- the extern "C" boundary declared in include/l1line.h.
//
// Host code only: validates arguments, carves the caller's workspace and
// enqueues the kernels on the caller's stream.  It never allocates memory and
// never synchronises, except in l1line_status().
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/l1line.h"
#include "common.cuh"
#include "launch.h"

using namespace l1l;

namespace {

thread_local int g_last_launches = 0;
thread_local cudaEvent_t g_ev_start = nullptr, g_ev_stop = nullptr;

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

bool mul_ok(int64_t a, int64_t b, int64_t &out) {
    if (a < 0 || b < 0) return false;
    if (a != 0 && b > INT64_MAX / a) return false;
    out = a * b;
    return true;
}

struct Layout {
    size_t status, slow_count, colinfo, Xt, v_all, s_all, z_all, slow, total;
    int64_t ldn;
};

// Returns false on overflow / bad shape.
bool make_layout(int dtype, int64_t n, int64_t m, int64_t nl, Layout &L) {
    if (n < 1 || m < 1 || nl < 1) return false;
    const int64_t es = dtype == L1L_DTYPE_F32 ? 4 : 8;
    const int64_t ldn = (n + 31) & ~int64_t(31);
    int64_t mm, pairs, xt, chunk_pairs;
    if (!mul_ok(m, m, mm) || !mul_ok(mm, nl, pairs) || !mul_ok(m, ldn, xt)) return false;
    const int64_t nlc = nl < MAX_LAMBDA_PER_LAUNCH ? nl : MAX_LAMBDA_PER_LAUNCH;
    if (!mul_ok(mm, nlc, chunk_pairs)) return false;
    if (pairs > INT64_MAX / 16 || xt > INT64_MAX / 16 || chunk_pairs > INT64_MAX / 32) return false;
    size_t off = 0;
    L.status = off;
    off += 256;
    L.slow_count = off;
    off += 256;
    L.colinfo = off;
    off = al256(off + (size_t)m * sizeof(ColInfo));
    L.Xt = off;
    off = al256(off + (size_t)xt * es);
    L.v_all = off;
    off = al256(off + (size_t)pairs * es);
    L.s_all = off;
    off = al256(off + (size_t)pairs * 8);
    L.z_all = off;
    off = al256(off + (size_t)(m * nl) * 8);
    L.slow = off;
    off = al256(off + (size_t)chunk_pairs * sizeof(SlowEntry));
    L.total = off;
    L.ldn = ldn;
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

template <typename T>
int scan_impl(const T *X, int64_t n, int64_t m, const double *lambdas, int64_t nl, T *v_all,
              double *s_all, double *z_all, void *ws, size_t ws_bytes, void *stream,
              uint32_t flags, Layout &L) {
    g_last_launches = 0;
    if (!X || !lambdas || n < 1 || m < 1 || nl < 1) return L1L_ERR_ARG;
    if (m > 0x7FFFFFFF || nl > 65535) return L1L_ERR_UNSUPPORTED;
    for (int64_t t = 0; t < nl; ++t)
        if (!(lambdas[t] >= 0.0) || std::isinf(lambdas[t])) return L1L_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(X) % sizeof(T)) != 0) return L1L_ERR_ARG;
    if (n > max_rows_pairs<T>()) return L1L_ERR_UNSUPPORTED;
    if (!make_layout(dtype_of<T>(), n, m, nl, L)) return L1L_ERR_UNSUPPORTED;
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255) != 0 || ws_bytes < L.total)
        return L1L_ERR_WORKSPACE;
    const int sms = num_sms();
    if (sms <= 0) return L1L_ERR_CUDA;
    const PairPlan plan = plan_pairs<T>(n, m, sms);
    if (plan.warps == 0) return L1L_ERR_UNSUPPORTED;

    unsigned char *base = static_cast<unsigned char *>(ws);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    ScanArgs<T> a;
    a.Xt = reinterpret_cast<T *>(base + L.Xt);
    a.ci = reinterpret_cast<ColInfo *>(base + L.colinfo);
    a.n = n;
    a.m = m;
    a.ldn = L.ldn;
    a.n_lambda = (int32_t)nl;
    a.v_all = v_all ? v_all : reinterpret_cast<T *>(base + L.v_all);
    a.s_all = s_all ? s_all : reinterpret_cast<double *>(base + L.s_all);
    a.status = reinterpret_cast<uint32_t *>(base + L.status);
    a.slow_count = reinterpret_cast<uint32_t *>(base + L.slow_count);
    a.slow = reinterpret_cast<SlowEntry *>(base + L.slow);
    a.force_exact = (flags & L1L_FLAG_FORCE_EXACT) ? 1 : 0;
    double *z = z_all ? z_all : reinterpret_cast<double *>(base + L.z_all);

    int launches = 0;
    if (cudaMemsetAsync(a.status, 0, sizeof(uint32_t), st) != cudaSuccess) return L1L_ERR_CUDA;
    if (launch_prep<T>(X, const_cast<T *>(a.Xt), const_cast<ColInfo *>(a.ci), n, m, L.ldn,
                       a.status, st, launches) != cudaSuccess)
        return L1L_ERR_CUDA;
    const bool prof = g_ev_start && g_ev_stop;
    for (int64_t t0 = 0; t0 < nl; t0 += MAX_LAMBDA_PER_LAUNCH) {
        const int nlc = (int)((nl - t0) < MAX_LAMBDA_PER_LAUNCH ? (nl - t0) : MAX_LAMBDA_PER_LAUNCH);
        const bool last = t0 + MAX_LAMBDA_PER_LAUNCH >= nl;
        if (cudaMemsetAsync(a.slow_count, 0, sizeof(uint32_t), st) != cudaSuccess)
            return L1L_ERR_CUDA;
        if (prof && t0 == 0 && cudaEventRecord(g_ev_start, st) != cudaSuccess) return L1L_ERR_CUDA;
        if (launch_pairs<T>(a, lambdas, (int)t0, nlc, plan, st, launches) != cudaSuccess)
            return L1L_ERR_CUDA;
        if (prof && last && cudaEventRecord(g_ev_stop, st) != cudaSuccess) return L1L_ERR_CUDA;
        if (launch_exact<T>(a, lambdas, (int)t0, nlc, sms, st, launches) != cudaSuccess)
            return L1L_ERR_CUDA;
    }
    if (launch_zreduce(a.s_all, z, m, nl, st, launches) != cudaSuccess) return L1L_ERR_CUDA;
    g_last_launches = launches;
    return L1L_OK;
}

template <typename T>
int fit_impl(const T *X, int64_t n, int64_t m, const double *lambdas, int64_t nl, T *out_v,
             double *out_obj, int32_t *out_jstar, void *ws, size_t ws_bytes, void *stream) {
    if (!out_v || !out_obj || !out_jstar) return L1L_ERR_ARG;
    Layout L;
    int rc = scan_impl<T>(X, n, m, lambdas, nl, nullptr, nullptr, nullptr, ws, ws_bytes, stream,
                          0u, L);
    if (rc != L1L_OK) return rc;
    unsigned char *base = static_cast<unsigned char *>(ws);
    int launches = g_last_launches;
    if (launch_argmin<T>(reinterpret_cast<double *>(base + L.z_all),
                         reinterpret_cast<T *>(base + L.v_all), m, nl, out_v, out_obj, out_jstar,
                         static_cast<cudaStream_t>(stream), launches) != cudaSuccess)
        return L1L_ERR_CUDA;
    g_last_launches = launches;
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
    Layout L;
    return scan_impl<float>(X, n, m, lambdas, n_lambda, v_all, s_all, z_all, workspace,
                            workspace_bytes, stream, flags, L);
}

int l1line_scan_ex_f64(const double *X, int64_t n, int64_t m, const double *lambdas,
                       int64_t n_lambda, double *v_all, double *s_all, double *z_all,
                       void *workspace, size_t workspace_bytes, void *stream, uint32_t flags) {
    Layout L;
    return scan_impl<double>(X, n, m, lambdas, n_lambda, v_all, s_all, z_all, workspace,
                             workspace_bytes, stream, flags, L);
}

int l1line_scan_f32(const float *X, int64_t n, int64_t m, const double *lambdas,
                    int64_t n_lambda, float *v_all, double *s_all, double *z_all,
                    void *workspace, size_t workspace_bytes, void *stream) {
    return l1line_scan_ex_f32(X, n, m, lambdas, n_lambda, v_all, s_all, z_all, workspace,
                              workspace_bytes, stream, 0u);
}

int l1line_scan_f64(const double *X, int64_t n, int64_t m, const double *lambdas,
                    int64_t n_lambda, double *v_all, double *s_all, double *z_all,
                    void *workspace, size_t workspace_bytes, void *stream) {
    return l1line_scan_ex_f64(X, n, m, lambdas, n_lambda, v_all, s_all, z_all, workspace,
                              workspace_bytes, stream, 0u);
}

int l1line_fit_f32(const float *X, int64_t n, int64_t m, const double *lambdas,
                   int64_t n_lambda, float *out_v, double *out_obj, int32_t *out_jstar,
                   void *workspace, size_t workspace_bytes, void *stream) {
    return fit_impl<float>(X, n, m, lambdas, n_lambda, out_v, out_obj, out_jstar, workspace,
                           workspace_bytes, stream);
}

int l1line_fit_f64(const double *X, int64_t n, int64_t m, const double *lambdas,
                   int64_t n_lambda, double *out_v, double *out_obj, int32_t *out_jstar,
                   void *workspace, size_t workspace_bytes, void *stream) {
    return fit_impl<double>(X, n, m, lambdas, n_lambda, out_v, out_obj, out_jstar, workspace,
                            workspace_bytes, stream);
}

int l1line_status(void *workspace, void *stream) {
    if (!workspace) return L1L_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(st) != cudaSuccess) return L1L_ERR_CUDA;
    uint32_t w = 0;
    if (cudaMemcpy(&w, workspace, sizeof(w), cudaMemcpyDeviceToHost) != cudaSuccess)
        return L1L_ERR_CUDA;
    if (w & ST_NONFINITE) return L1L_ERR_NONFINITE;
    if (w & ST_TIMEOUT) return L1L_ERR_TIMEOUT;
    if (w & ST_INTERNAL) return L1L_ERR_INTERNAL;
    return L1L_OK;
}

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

extern "C" int l1line_fit_noalloc_f32(const float *X, int64_t n, int64_t m,
                                      const double *lambdas, int64_t n_lambda, float *out_v,
                                      double *out_obj, int32_t *out_jstar, void *stream) {
    if (!X || !lambdas || !out_v || !out_obj || !out_jstar || n < 1 || m < 1 || n_lambda < 1)
        return L1L_ERR_ARG;
    const size_t need = l1line_workspace_bytes(L1L_DTYPE_F32, n, m, n_lambda);
    if (need == 0 || need > L1L_NOALLOC_SCRATCH_BYTES) return L1L_ERR_UNSUPPORTED;
    void *ws = nullptr;
    const int rc = noalloc_scratch_address(&ws);
    if (rc != L1L_OK) return rc;
    // the status word and the exact-path counter are zeroed by the fit itself;
    // every other region of the workspace is fully overwritten before it is read
    return fit_impl<float>(X, n, m, lambdas, n_lambda, out_v, out_obj, out_jstar, ws,
                           L1L_NOALLOC_SCRATCH_BYTES, stream);
}
