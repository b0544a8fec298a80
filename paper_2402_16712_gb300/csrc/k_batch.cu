// k_batch.cu -- a batch of independent instances (uneven n, m and lambdas)
// in a handful of launches: batched staging, ONE persistent pair kernel whose
// CTAs pull (instance, jhat) units from an atomic counter, largest instances
// first, then the exact path, the objective sums and the argmin.  The
// per-instance descriptors travel in the launch parameters, so the whole
// sequence can be captured in a CUDA graph.
#include <algorithm>

#include "batch.cuh"
#include "common.cuh"
#include "exact.cuh"
#include "launch.h"
#include "pairs.cuh"
#include "prep.cuh"

namespace l1l {

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
        switch (bc.plan.shape) {
            case SHAPE_R80: e = launch_persist_sh<T, SHAPE_R80>(bd, ws, bc, c, multi, num_sms, st); break;
            case SHAPE_R64: e = launch_persist_sh<T, SHAPE_R64>(bd, ws, bc, c, multi, num_sms, st); break;
            case SHAPE_R128: e = launch_persist_sh<T, SHAPE_R128>(bd, ws, bc, c, multi, num_sms, st); break;
            default: e = cudaErrorInvalidConfiguration;
        }
        if (e != cudaSuccess) return e;
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
