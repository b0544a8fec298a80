// k_reduce.cu -- steps A5 (z_jhat) and A6 (argmin over jhat, gather of v*).
#include <algorithm>

#include "common.cuh"
#include "launch.h"

namespace l1l {

// z[t][jhat] = sum_k s_all[t][jhat][k]  (the diagonal holds lambda * |v_jhat| =
// lambda).  One warp per (t, listed jhat); fixed summation order, so
// deterministic.  jlist == nullptr scores every jhat.
__global__ void __launch_bounds__(32) k_zreduce(const double *__restrict__ s_all,
                                                double *__restrict__ z_all, int64_t m,
                                                const int32_t *__restrict__ jlist) {
    const int64_t t = blockIdx.y;
    const int64_t j = jlist ? (int64_t)jlist[blockIdx.x] : (int64_t)blockIdx.x;
    if (j < 0 || j >= m) return;  // flagged by the pair kernel
    const double *s = s_all + (t * m + j) * m;
    double acc = 0.0;
    for (int64_t k = threadIdx.x; k < m; k += 32) acc += s[k];
    acc = warp_sum_f64(acc);
    if (threadIdx.x == 0) z_all[t * m + j] = acc;
}

// Per lambda: jhat* = smallest index attaining min z (Algorithm 1 keeps the
// first strict improvement in increasing jhat); copy v^{jhat*} out.
template <typename T>
__global__ void __launch_bounds__(256) k_argmin(const double *__restrict__ z_all,
                                                const T *__restrict__ v_all, int64_t m,
                                                const int32_t *__restrict__ jlist, int64_t nj,
                                                T *out_v, double *out_obj, int32_t *out_jstar) {
    const int64_t t = blockIdx.x;
    const double *z = z_all + t * m;
    double bz = 0.0;
    int64_t bj = -1;
    for (int64_t p = threadIdx.x; p < nj; p += blockDim.x) {
        const int64_t j = jlist ? (int64_t)jlist[p] : p;
        if (j < 0 || j >= m) continue;
        double zj = z[j];
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
    for (int s = blockDim.x >> 1; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            int64_t oj = sj[threadIdx.x + s];
            double oz = sz[threadIdx.x + s];
            int64_t cj = sj[threadIdx.x];
            double cz = sz[threadIdx.x];
            bool take = oj >= 0 && (cj < 0 || oz < cz || (oz == cz && oj < cj));
            if (take) {
                sz[threadIdx.x] = oz;
                sj[threadIdx.x] = oj;
            }
        }
        __syncthreads();
    }
    const int64_t js = sj[0];
    if (threadIdx.x == 0) {
        out_obj[t] = js >= 0 ? sz[0] : (double)NAN;
        out_jstar[t] = (int32_t)js;
    }
    for (int64_t k = threadIdx.x; k < m; k += blockDim.x)
        out_v[t * m + k] = js >= 0 ? v_all[(t * m + js) * m + k] : T(NAN);
}

cudaError_t launch_zreduce(const double *s_all, double *z_all, int64_t m, int64_t n_lambda,
                           const int32_t *jlist, int64_t nj, cudaStream_t st, int &launches) {
    dim3 grid((unsigned)nj, (unsigned)n_lambda);
    k_zreduce<<<grid, 32, 0, st>>>(s_all, z_all, m, jlist);
    launches++;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_argmin(const double *z_all, const T *v_all, int64_t m, int64_t n_lambda,
                          const int32_t *jlist, int64_t nj, T *out_v, double *out_obj,
                          int32_t *out_jstar, cudaStream_t st, int &launches) {
    k_argmin<T><<<(unsigned)n_lambda, 256, 0, st>>>(z_all, v_all, m, jlist, nj, out_v, out_obj,
                                                    out_jstar);
    launches++;
    return cudaGetLastError();
}

// Successive components: x'_ik = fl(x_ik - fl(v_k x_ijhat)) (no fused
// multiply-add), with jhat and v the component just fitted (device values).
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }

template <typename T>
__global__ void k_deflate(const T *__restrict__ X, T *__restrict__ Y, int64_t n, int64_t m,
                          const int32_t *__restrict__ jstar, const T *__restrict__ v) {
    const int64_t j = *jstar;
    const int64_t N = n * m;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / m, k = e - i * m;
        Y[e] = j >= 0 ? sub_rn(X[e], mul_rn(v[k], X[i * m + j])) : X[e];
    }
}

template <typename T>
cudaError_t launch_deflate(const T *X, T *Y, int64_t n, int64_t m, const int32_t *jstar,
                           const T *v, int num_sms, cudaStream_t st, int &launches) {
    const int64_t N = n * m;
    const int64_t blocks = std::min<int64_t>((N + 255) / 256, (int64_t)num_sms * 8);
    k_deflate<T><<<(unsigned)std::max<int64_t>(1, blocks), 256, 0, st>>>(X, Y, n, m, jstar, v);
    launches++;
    return cudaGetLastError();
}

template cudaError_t launch_deflate<float>(const float *, float *, int64_t, int64_t,
                                           const int32_t *, const float *, int, cudaStream_t,
                                           int &);
template cudaError_t launch_deflate<double>(const double *, double *, int64_t, int64_t,
                                            const int32_t *, const double *, int, cudaStream_t,
                                            int &);

template cudaError_t launch_argmin<float>(const double *, const float *, int64_t, int64_t,
                                          const int32_t *, int64_t, float *, double *, int32_t *,
                                          cudaStream_t, int &);
template cudaError_t launch_argmin<double>(const double *, const double *, int64_t, int64_t,
                                           const int32_t *, int64_t, double *, double *,
                                           int32_t *, cudaStream_t, int &);

}  // namespace l1l
