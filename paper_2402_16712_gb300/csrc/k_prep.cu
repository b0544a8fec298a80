// k_prep.cu -- step A1 (staging) kernels for one instance.
#include <cooperative_groups.h>

#include <algorithm>

#include "common.cuh"
#include "launch.h"
#include "prep.cuh"

namespace cg = cooperative_groups;

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

// Block-wide reductions of one value per thread (512 threads); `red` holds
// the warp partials, `out` receives the result for every thread.
enum { RED_SUM, RED_MAX, RED_MIN };
template <int OP>
__device__ __forceinline__ long long block_reduce_ll(long long x, long long *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long y = __shfl_xor_sync(0xFFFFFFFFu, x, o);
        x = OP == RED_SUM ? x + y : (OP == RED_MAX ? (x > y ? x : y) : (x < y ? x : y));
    }
    __syncthreads();  // red may still be read by an earlier reduction
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
    __syncthreads();
    long long r = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
        const long long y = red[w];
        r = OP == RED_SUM ? r + y : (OP == RED_MAX ? (r > y ? r : y) : (r < y ? r : y));
    }
    return r;
}

// Column statistics of tall columns: a cluster of C CTAs per column, each
// over its slice of rows; the three dependent reductions (count and exponent
// range -> sigma; Q and truncations -> the 32-bit shift; Q32 and its
// truncations) are combined across the cluster through distributed shared
// memory.  Integer sums, so the result equals the one-CTA version's.
template <typename T>
__global__ void __launch_bounds__(512) k_colprep_tall(const T *__restrict__ Xt, ColInfo *ci,
                                                      int64_t n, int64_t ldn, int64_t rpc) {
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks(), rank = (int)cl.block_rank();
    const int64_t j = blockIdx.x / C;
    const T *col = Xt + j * ldn;
    const int64_t r0 = std::min<int64_t>(n, (int64_t)rank * rpc);
    const int64_t r1 = std::min<int64_t>(n, r0 + rpc);
    __shared__ long long red[16];
    __shared__ long long p1[3], p2[2], p3[2];  // this CTA's partials, read by the cluster

    int cnt = 0, emax = -100000, emin = 100000;
#pragma unroll 4
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        const T b = col[i];
        if (b != T(0)) {
            cnt++;
            const int e = ilog2_pos(b);
            emax = max(emax, e);
            emin = min(emin, e);
        }
    }
    long long v0 = block_reduce_ll<RED_SUM>(cnt, red);
    long long v1 = block_reduce_ll<RED_MAX>(emax, red);
    long long v2 = block_reduce_ll<RED_MIN>(emin, red);
    if (threadIdx.x == 0) {
        p1[0] = v0;
        p1[1] = v1;
        p1[2] = v2;
    }
    cl.sync();
    long long nvl = 0;
    int E = -100000, Emin = 100000;
    for (int r = 0; r < C; ++r) {
        const long long *q = cl.map_shared_rank(&p1[0], r);
        nvl += q[0];
        E = max(E, (int)q[1]);
        Emin = min(Emin, (int)q[2]);
    }
    const int nv = (int)nvl;
    const int sigma = colprep_sigma(nv, E);

    long long qs = 0;
    int inx = 0;
#pragma unroll 4
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        const T b = col[i];
        if (b != T(0)) {
            int e = 0;
            qs += fixq(absval(b), sigma, e);
            inx += e;
        }
    }
    v0 = block_reduce_ll<RED_SUM>(qs, red);
    v1 = block_reduce_ll<RED_SUM>(inx, red);
    if (threadIdx.x == 0) {
        p2[0] = v0;
        p2[1] = v1;
    }
    cl.sync();
    long long Q = 0, I = 0;
    for (int r = 0; r < C; ++r) {
        const long long *q = cl.map_shared_rank(&p2[0], r);
        Q += q[0];
        I += q[1];
    }
    const int shift = colprep_shift32(Q);
    const uint64_t lowmask = (1ull << shift) - 1ull;

    long long q32 = 0;
    int inx32 = 0;
#pragma unroll 4
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        const T b = col[i];
        if (b != T(0)) {
            int e = 0;
            const uint64_t qi = (uint64_t)fixq(absval(b), sigma, e);
            q32 += (long long)(qi >> shift);
            inx32 += (e || (qi & lowmask) != 0) ? 1 : 0;
        }
    }
    v0 = block_reduce_ll<RED_SUM>(q32, red);
    v1 = block_reduce_ll<RED_SUM>(inx32, red);
    if (threadIdx.x == 0) {
        p3[0] = v0;
        p3[1] = v1;
    }
    cl.sync();
    if (rank == 0 && threadIdx.x == 0) {
        long long Q32 = 0, I32 = 0;
        for (int r = 0; r < C; ++r) {
            const long long *q = cl.map_shared_rank(&p3[0], r);
            Q32 += q[0];
            I32 += q[1];
        }
        ci[j] = colprep_make<T>(Q, sigma, nv, (int)I, Emin, E, Q32, shift, (int)I32);
    }
    cl.sync();  // no CTA leaves while rank 0 may still read its partials
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
    launches++;
    const int C = large_cluster_size(ldn);
    if (C == 1) {
        k_colprep<T><<<(unsigned)m, 256, 0, st>>>(Xt, ci, n, ldn);
        launches++;
        return cudaGetLastError();
    }
    // tall columns: one cluster of C CTAs per column
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(m * C));
    cfg.blockDim = dim3(512);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const int64_t rpc = (n + C - 1) / C;
    e = cudaLaunchKernelEx(&cfg, k_colprep_tall<T>, (const T *)Xt, ci, n, ldn, rpc);
    launches++;
    return e;
}

template cudaError_t launch_prep<float>(const float *, float *, float *, ColInfo *, int64_t,
                                        int64_t, int64_t, uint32_t *, cudaStream_t, int &);
template cudaError_t launch_prep<double>(const double *, double *, float *, ColInfo *, int64_t,
                                         int64_t, int64_t, uint32_t *, cudaStream_t, int &);

}  // namespace l1l
