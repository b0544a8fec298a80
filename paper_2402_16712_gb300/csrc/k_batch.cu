// k_batch.cu -- a batch of independent instances (uneven n, m and lambdas)
// in a handful of launches: batched staging, ONE persistent pair kernel whose
// CTAs pull (instance, jhat) units from an atomic counter, largest instances
// first, then the exact path, the objective sums and the argmin.  The
// per-instance descriptors travel in the launch parameters, so the whole
// sequence can be captured in a CUDA graph.
#include <algorithm>

#include "common.cuh"
#include "exact.cuh"
#include "launch.h"
#include "pairs.cuh"
#include "prep.cuh"

namespace l1l {

// Largest b with begin[b] <= x (begin is a non-decreasing prefix, begin[0] = 0).
template <typename I>
__device__ __forceinline__ int find_inst(const I *begin, int count, I x) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (begin[mid] <= x)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

template <typename T>
__device__ __forceinline__ ScanArgs<T> inst_args(const BatchDesc<T> &bd, int b,
                                                 unsigned char *ws) {
    const BatchInst<T> &in = bd.inst[b];
    const InstLayout L = inst_layout(in.m, in.ldn, in.nl, sizeof(T));
    unsigned char *base = ws + in.ws_off;
    ScanArgs<T> a;
    a.Xt = reinterpret_cast<const T *>(base + L.Xt);
    a.Xf = reinterpret_cast<const float *>(base + L.Xf);
    a.ci = reinterpret_cast<const ColInfo *>(base + L.ci);
    a.n = in.n;
    a.m = in.m;
    a.ldn = in.ldn;
    a.n_lambda = in.nl;
    a.v_all = reinterpret_cast<T *>(base + L.v_all);
    a.s_all = reinterpret_cast<double *>(base + L.s_all);
    a.status = reinterpret_cast<uint32_t *>(ws);
    a.slow_count = reinterpret_cast<uint32_t *>(ws + 256);
    a.slow = reinterpret_cast<SlowEntry *>(ws + BATCH_HEAD);
    a.force_exact = bd.force_exact;
    a.inst = b;
    a.jlist = nullptr;
    a.nj = a.m;
    a.d0 = bd.d0;
    return a;
}

template <typename T>
__global__ void __launch_bounds__(256) k_transpose_b(const __grid_constant__ BatchDesc<T> bd,
                                                     unsigned char *ws) {
    const int b = find_inst<int32_t>(bd.tile_begin, bd.count, (int32_t)blockIdx.x);
    const BatchInst<T> &in = bd.inst[b];
    const int t = (int)blockIdx.x - bd.tile_begin[b];
    const int tiles_c = (in.m + 31) / 32;
    const InstLayout L = inst_layout(in.m, in.ldn, in.nl, sizeof(T));
    T *Xt = reinterpret_cast<T *>(ws + in.ws_off + L.Xt);
    float *Xf = reinterpret_cast<float *>(ws + in.ws_off + L.Xf);
    transpose_tile<T>(in.X, Xt, Xf, in.n, in.m, in.ldn, reinterpret_cast<uint32_t *>(ws), t % tiles_c,
                      t / tiles_c);
}

template <typename T>
__global__ void __launch_bounds__(256) k_colprep_b(const __grid_constant__ BatchDesc<T> bd,
                                                   unsigned char *ws) {
    const int b = find_inst<int64_t>(bd.unit_begin, bd.count, (int64_t)blockIdx.x);
    const BatchInst<T> &in = bd.inst[b];
    const int j = (int)((int64_t)blockIdx.x - bd.unit_begin[b]);
    const InstLayout L = inst_layout(in.m, in.ldn, in.nl, sizeof(T));
    const T *Xt = reinterpret_cast<const T *>(ws + in.ws_off + L.Xt);
    ColInfo *ci = reinterpret_cast<ColInfo *>(ws + in.ws_off + L.ci);
    colprep_column<T>(Xt + (int64_t)j * in.ldn, ci + j, in.n);
}

// Persistent: every CTA loops, taking the next (instance, jhat) unit of units
// [u0, u1) (one size class of the batch) from that class's counter; units are
// numbered largest instance first.  No CTA waits on another.
template <typename T, bool MULTI, bool CS>
__global__ void __launch_bounds__(256, 3)
    k_pairs_persist(const __grid_constant__ BatchDesc<T> bd, unsigned char *ws, int64_t u0,
                    int64_t u1, int slot, int lay_npad, int cap) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ Decide s_dec[NDEC];
    __shared__ long long s_unit;
    unsigned long long *counter = reinterpret_cast<unsigned long long *>(ws + 512) + slot;
    for (;;) {
        if (threadIdx.x == 0) s_unit = (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        const int64_t u = u0 + s_unit;
        __syncthreads();
        if (u >= u1) break;
        const int b = find_inst<int64_t>(bd.unit_begin, bd.count, u);
        const BatchInst<T> &in = bd.inst[b];
        const ScanArgs<T> a = inst_args<T>(bd, b, ws);
        const LamView lv{bd.lam + bd.lam_begin[b], in.tl_min, in.tl_max};
        pairs_unit<T, MULTI, CS>(a, lv, 0, in.nl, (int)(u - bd.unit_begin[b]), 0, in.m, cap,
                             lay_npad, smem, s_dec);
    }
}

template <typename T>
__global__ void __launch_bounds__(128) k_exact_b(const __grid_constant__ BatchDesc<T> bd,
                                                 unsigned char *ws) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t count = *(volatile uint32_t *)(ws + 256);
    const SlowEntry *slow = reinterpret_cast<const SlowEntry *>(ws + BATCH_HEAD);
    uint32_t acc[WL];
    uint32_t S[WL], W[WL];
    for (uint32_t e = gw; e < count; e += nwarps) {
        const SlowEntry en = slow[e];
        const ScanArgs<T> a = inst_args<T>(bd, en.inst, ws);
        exact_entry<T>(a, en, bd.lam[bd.lam_begin[en.inst] + en.t], acc, S, W, lane);
    }
}

template <typename T>
__global__ void __launch_bounds__(32) k_zreduce_b(const __grid_constant__ BatchDesc<T> bd,
                                                  unsigned char *ws) {
    const int b = find_inst<int32_t>(bd.ztask_begin, bd.count, (int32_t)blockIdx.x);
    const BatchInst<T> &in = bd.inst[b];
    const int local = (int)blockIdx.x - bd.ztask_begin[b];
    const int64_t m = in.m;
    const InstLayout L = inst_layout(in.m, in.ldn, in.nl, sizeof(T));
    const double *s = reinterpret_cast<const double *>(ws + in.ws_off + L.s_all) + (int64_t)local * m;
    double acc = 0.0;
    for (int64_t k = threadIdx.x; k < m; k += 32) acc += s[k];
    acc = warp_sum_f64(acc);
    if (threadIdx.x == 0) reinterpret_cast<double *>(ws + in.ws_off + L.z_all)[local] = acc;
}

template <typename T>
__global__ void __launch_bounds__(256) k_argmin_b(const __grid_constant__ BatchDesc<T> bd,
                                                  unsigned char *ws, T *out_v, double *out_obj,
                                                  int32_t *out_jstar) {
    const int b = find_inst<int32_t>(bd.lam_begin, bd.count, (int32_t)blockIdx.x);
    const BatchInst<T> &in = bd.inst[b];
    const int t = (int)blockIdx.x - bd.lam_begin[b];
    const int64_t m = in.m;
    const InstLayout L = inst_layout(in.m, in.ldn, in.nl, sizeof(T));
    const double *z = reinterpret_cast<const double *>(ws + in.ws_off + L.z_all) + t * m;
    const T *v_all = reinterpret_cast<const T *>(ws + in.ws_off + L.v_all);
    double bz = 0.0;
    int64_t bj = -1;
    for (int64_t j = threadIdx.x; j < m; j += blockDim.x) {
        const double zj = z[j];
        if (zj == zj && (bj < 0 || zj < bz)) {
            bz = zj;
            bj = j;
        }
    }
    __shared__ double sz[256];
    __shared__ int64_t sj[256];
    sz[threadIdx.x] = bz;
    sj[threadIdx.x] = bj;
    __syncthreads();
    for (int s2 = blockDim.x >> 1; s2 > 0; s2 >>= 1) {
        if (threadIdx.x < s2) {
            const int64_t oj = sj[threadIdx.x + s2], cj = sj[threadIdx.x];
            const double oz = sz[threadIdx.x + s2], cz = sz[threadIdx.x];
            if (oj >= 0 && (cj < 0 || oz < cz || (oz == cz && oj < cj))) {
                sz[threadIdx.x] = oz;
                sj[threadIdx.x] = oj;
            }
        }
        __syncthreads();
    }
    const int64_t js = sj[0];
    if (threadIdx.x == 0) {
        out_obj[in.out_t_off + t] = js >= 0 ? sz[0] : (double)NAN;
        out_jstar[in.out_t_off + t] = (int32_t)js;
    }
    for (int64_t k = threadIdx.x; k < m; k += blockDim.x)
        out_v[in.out_v_off + t * m + k] = js >= 0 ? v_all[(t * m + js) * m + k] : T(NAN);
}

template <typename T>
cudaError_t launch_batch(const BatchDesc<T> &bd, unsigned char *ws, T *out_v, double *out_obj,
                         int32_t *out_jstar, const BatchClass *classes, int nclasses, bool multi,
                         int num_sms, cudaStream_t st, int &launches) {
    cudaError_t e = cudaMemsetAsync(ws, 0, BATCH_HEAD, st);  // status, exact counter, units
    if (e != cudaSuccess) return e;
    k_transpose_b<T><<<bd.tiles, dim3(32, 8), 0, st>>>(bd, ws);
    k_colprep_b<T><<<(unsigned)bd.units, 256, 0, st>>>(bd, ws);
    launches += 2;
    // one persistent launch per size class, each with shared memory for its largest n
    for (int c = 0; c < nclasses; ++c) {
        const BatchClass &bc = classes[c];
        if (bc.u1 <= bc.u0) continue;
        auto kern = multi ? (bc.plan.cs ? k_pairs_persist<T, true, true>
                                        : k_pairs_persist<T, true, false>)
                          : (bc.plan.cs ? k_pairs_persist<T, false, true>
                                        : k_pairs_persist<T, false, false>);
        e = ensure_smem(reinterpret_cast<const void *>(kern), bc.plan.smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        e = blocks_per_sm(reinterpret_cast<const void *>(kern), bc.plan.warps * 32, bc.plan.smem,
                          &per_sm);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        const int64_t grid = std::min<int64_t>((int64_t)num_sms * per_sm, bc.u1 - bc.u0);
        kern<<<(unsigned)grid, bc.plan.warps * 32, bc.plan.smem, st>>>(
            bd, ws, bc.u0, bc.u1, c, bc.lay_npad, bc.plan.cap);
        launches++;
    }
    k_exact_b<T><<<num_sms * 2, 128, 0, st>>>(bd, ws);
    k_zreduce_b<T><<<bd.ztasks, 32, 0, st>>>(bd, ws);
    k_argmin_b<T><<<bd.lams, 256, 0, st>>>(bd, ws, out_v, out_obj, out_jstar);
    launches += 3;
    return cudaGetLastError();
}

template cudaError_t launch_batch<float>(const BatchDesc<float> &, unsigned char *, float *,
                                         double *, int32_t *, const BatchClass *, int, bool, int,
                                         cudaStream_t, int &);
template cudaError_t launch_batch<double>(const BatchDesc<double> &, unsigned char *, double *,
                                          double *, int32_t *, const BatchClass *, int, bool, int,
                                          cudaStream_t, int &);

L1L_CHECKS_READER(l1l_checks_batch)

}  // namespace l1l
