// k_prep.cu -- step A1 (staging) kernels for one instance.
#include <algorithm>

#include "common.cuh"
#include "launch.h"
#include "prep.cuh"

namespace l1l {

// grid.x: 32-column tiles; grid.y strides over the 32-row tiles (tall X
// has more of them than a grid dimension holds).
template <typename T>
__global__ void __launch_bounds__(256) k_transpose(const T *__restrict__ X, T *__restrict__ Xt,
                                                   float *__restrict__ Xf,
                                                   int64_t n, int64_t m, int64_t ldn,
                                                   uint32_t *status, int64_t tiles_r) {
    for (int64_t tr = blockIdx.y; tr < tiles_r; tr += gridDim.y) {
        transpose_tile<T>(X, Xt, Xf, n, m, ldn, status, blockIdx.x, tr);
        __syncthreads();  // the next row tile refills the shared tile
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_colprep(const T *__restrict__ Xt, ColInfo *ci,
                                                 int64_t n, int64_t ldn) {
    colprep_column<T>(Xt + (int64_t)blockIdx.x * ldn, ci + blockIdx.x, n);
}

template <typename T>
cudaError_t launch_prep(const T *X, T *Xt, float *Xf, ColInfo *ci, int64_t n, int64_t m,
                        int64_t ldn, uint32_t *status, cudaStream_t st, int &launches) {
    dim3 tb(32, 8);
    const int64_t tiles_r = (ldn + 31) / 32;
    dim3 tg((unsigned)((m + 31) / 32), (unsigned)std::min<int64_t>(tiles_r, 65535));
    k_transpose<T><<<tg, tb, 0, st>>>(X, Xt, Xf, n, m, ldn, status, tiles_r);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_colprep<T><<<(unsigned)m, 256, 0, st>>>(Xt, ci, n, ldn);
    launches += 2;
    return cudaGetLastError();
}

template cudaError_t launch_prep<float>(const float *, float *, float *, ColInfo *, int64_t,
                                        int64_t, int64_t, uint32_t *, cudaStream_t, int &);
template cudaError_t launch_prep<double>(const double *, double *, float *, ColInfo *, int64_t,
                                         int64_t, int64_t, uint32_t *, cudaStream_t, int &);

}  // namespace l1l
