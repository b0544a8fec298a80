// prep.cuh -- step A1 (staging) bodies shared by the single-instance and
// batched kernels: column-major copy of X with the non-finite check, and the
// per-column fixed-point statistics of the exact weighted-median decisions.
#pragma once
#include "common.cuh"

namespace l1l {

// X (n x m, row-major, rows = points) -> Xt (m x ldn, column-major, rows
// n..ldn-1 zero), and for double input also Xf, the same copy rounded to float
// (the pair kernel's approximate keys read it, so they need no conversion on
// the narrow double pipe), followed by Xlo = Xf + m ldn, the rounding
// remainders (the float-float residual reads both).  32x32 tiles through shared memory so both the read
// and the write are coalesced.  Any NaN/inf sets ST_NONFINITE.
template <typename T>
__device__ __forceinline__ void transpose_tile(const T *__restrict__ X, T *__restrict__ Xt,
                                               float *__restrict__ Xf, int64_t n, int64_t m,
                                               int64_t ldn, uint32_t *status, int64_t tile_c,
                                               int64_t tile_r) {
    __shared__ T tile[32][33];
    const int64_t c0 = tile_c * 32;  // column of X
    const int64_t r0 = tile_r * 32;  // row of X
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    bool bad = false;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        int64_t r = r0 + ty + 8 * q, c = c0 + tx;
        T v = 0;
        if (r < n && c < m) {
            v = X[r * m + c];
            bad |= !isfinite(v);
        }
        tile[ty + 8 * q][tx] = v;
    }
    if (__any_sync(0xFFFFFFFFu, bad) && tx == 0) atomicOr(status, ST_NONFINITE);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        int64_t c = c0 + ty + 8 * q, r = r0 + tx;
        if (c < m && r < ldn) {
            const T v = tile[tx][ty + 8 * q];
            Xt[c * ldn + r] = v;
            if constexpr (sizeof(T) == 8) {
                // the float pair of the double residual: hi, then (at m ldn
                // further) lo = fl(v - hi), where v - hi is exact in double
                const float hi = (float)v;
                Xf[c * ldn + r] = hi;
                Xf[(m + c) * ldn + r] = (float)(v - (double)hi);
            }
        }
    }
}

template <typename T> __device__ __forceinline__ T absval(T x) { return x < T(0) ? -x : x; }

// The column statistics from its reductions (shared by the one-CTA and the
// cluster versions below).  sigma: the scale that keeps every q_i below
// 2^(60 - L) with L the bit length of n_valid (E = floor(log2 max |x|)).
__device__ __forceinline__ int colprep_sigma(int nv, int E) {
    const int Lbits = nv > 0 ? 32 - __clz(nv) : 0;
    return nv > 0 ? 60 - E - Lbits : 0;
}
// 32-bit weights: drop the fewest low bits that bring the total below 2^32
// (floor(floor(x) / 2^s) = floor(x / 2^s), so q32 = q >> s is the weight
// rounded down at scale sigma - s, and sum q32 <= Q / 2^s < 2^32).
__device__ __forceinline__ int colprep_shift32(long long Q) {
    const int qbits = Q > 0 ? 64 - __clzll(Q) : 0;
    return qbits > 32 ? qbits - 32 : 0;
}
template <typename T>
__device__ __forceinline__ ColInfo colprep_make(long long Q, int sigma, int nv, int I, int Emin,
                                                int E, long long Q32, int shift, int I32) {
    ColInfo c;
    c.Q = Q;
    c.sigma = sigma;
    c.n_valid = nv;
    c.n_inexact = I;
    c.flags = (nv > 0 && (Emin < WideRange<T>::lo || E > WideRange<T>::hi)) ? COL_WIDE : 0;
    c.Q32 = (uint32_t)Q32;
    c.shift32 = shift;
    c.n_inexact32 = I32;
    // each q_i = floor(|x_i| 2^sigma) is short of |x_i| 2^sigma by less than
    // one, and only for the n_inexact truncated rows
    c.l1_up = __double2float_ru((double)(Q + I) * ldexp(1.0, -sigma) * (1.0 + 0x1p-50));
    return c;
}

// One block per column jhat: n_valid, sigma (from the largest |x_ijhat|), the
// fixed-point total Q and the number of truncated weights.
template <typename T>
__device__ __forceinline__ void colprep_column(const T *__restrict__ col, ColInfo *out, int64_t n) {
    __shared__ int s_max[8];
    __shared__ int s_min[8];
    __shared__ int s_cnt[8];
    __shared__ long long s_q[8];
    __shared__ int s_inx[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    int emax = -100000, emin = 100000, cnt = 0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        T b = col[i];
        if (b != T(0)) {
            cnt++;
            const int e = ilog2_pos(b);
            emax = max(emax, e);
            emin = min(emin, e);
        }
    }
    cnt = __reduce_add_sync(0xFFFFFFFFu, cnt);
    emax = __reduce_max_sync(0xFFFFFFFFu, emax);
    emin = __reduce_min_sync(0xFFFFFFFFu, emin);
    if (lane == 0) {
        s_max[warp] = emax;
        s_min[warp] = emin;
        s_cnt[warp] = cnt;
    }
    __syncthreads();
    int nv = 0, E = -100000, Emin = 100000;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        nv += s_cnt[w];
        E = max(E, s_max[w]);
        Emin = min(Emin, s_min[w]);
    }
    const int sigma = colprep_sigma(nv, E);

    long long q = 0;
    int inx = 0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        T b = col[i];
        if (b != T(0)) {
            int e = 0;
            q += fixq(absval(b), sigma, e);
            inx += e;
        }
    }
    q = warp_sum_i64(q);
    inx = __reduce_add_sync(0xFFFFFFFFu, inx);
    if (lane == 0) {
        s_q[warp] = q;
        s_inx[warp] = inx;
    }
    __syncthreads();
    long long Q = 0;
    int I = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        Q += s_q[w];
        I += s_inx[w];
    }
    const int shift = colprep_shift32(Q);
    const uint64_t lowmask = (1ull << shift) - 1ull;
    long long q32 = 0;
    int inx32 = 0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        T b = col[i];
        if (b != T(0)) {
            int e = 0;
            const uint64_t qi = (uint64_t)fixq(absval(b), sigma, e);
            q32 += (long long)(qi >> shift);
            inx32 += (e || (qi & lowmask) != 0) ? 1 : 0;
        }
    }
    q32 = warp_sum_i64(q32);
    inx32 = __reduce_add_sync(0xFFFFFFFFu, inx32);
    __syncthreads();  // s_q / s_inx are reused
    if (lane == 0) {
        s_q[warp] = q32;
        s_inx[warp] = inx32;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long Q32 = 0;
        int I32 = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            Q32 += s_q[w];
            I32 += s_inx[w];
        }
        *out = colprep_make<T>(Q, sigma, nv, I, Emin, E, Q32, shift, I32);
    }
}

}  // namespace l1l
