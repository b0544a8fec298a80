// exact.cuh -- exact slow path of step A3 (shared by the single-instance and
// batched kernels).  One warp solves one listed pair by bisection over the
// key space; at each probe the weight of rows at or below it is summed
// exactly in a wide fixed-point integer (unit 2^-1074: every finite double,
// and so every float, is an integer multiple of it), reduced across the warp
// limb by limb and compared with the exact total W = sum w + lambda.
#pragma once
#include "checks.cuh"
#include "common.cuh"
#include "pairs.cuh"

namespace l1l {

constexpr int WL = 68;  // 32-bit limbs: 2176 bits, unit 2^-1074

// acc += x (x >= 0, finite); widens [lmin, lmax] to the limbs touched.
__device__ __forceinline__ void wide_add(uint32_t *acc, double x, int &lmin, int &lmax) {
    uint64_t u = (uint64_t)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
    int be = (int)(u >> 52);
    uint64_t mant = u & 0xFFFFFFFFFFFFFull;
    if (be == 0 && mant == 0) return;
    int shift = 0;
    if (be) {
        mant |= 0x10000000000000ull;
        shift = be - 1;
    }
    int l = shift >> 5, off = shift & 31;
    uint64_t a0 = (mant & 0xFFFFFFFFull) << off;  // < 2^63
    uint64_t a1 = (mant >> 32) << off;            // < 2^52
    uint64_t c = (uint64_t)acc[l] + (a0 & 0xFFFFFFFFull);
    acc[l] = (uint32_t)c;
    c >>= 32;
    c += (uint64_t)acc[l + 1] + (a0 >> 32) + (a1 & 0xFFFFFFFFull);
    acc[l + 1] = (uint32_t)c;
    c >>= 32;
    c += (uint64_t)acc[l + 2] + (a1 >> 32);
    acc[l + 2] = (uint32_t)c;
    c >>= 32;
    int top = l + 2;
    for (int q = l + 3; c && q < WL; ++q) {
        c += acc[q];
        acc[q] = (uint32_t)c;
        c >>= 32;
        top = q;
    }
    lmin = min(lmin, l);
    lmax = max(lmax, top);
}

// Sum the lanes' accumulators over limbs [lmin, lmax] into lane 0's `out`
// (normalised, all limbs written).
__device__ __forceinline__ void wide_warp_reduce(const uint32_t *acc, uint32_t *out, int lmin, int lmax,
                                 int lane) {
    lmin = __reduce_min_sync(0xFFFFFFFFu, lmin);  // signed reductions
    lmax = __reduce_max_sync(0xFFFFFFFFu, lmax);
    if (lane == 0)
        for (int q = 0; q < WL; ++q) out[q] = 0;
    uint64_t carry = 0;
    for (int q = lmin; q <= lmax && q < WL; ++q) {
        uint64_t s = acc[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
        if (lane == 0) {
            carry += s;
            out[q] = (uint32_t)carry;
            carry >>= 32;
        }
    }
    if (lane == 0)
        for (int q = max(lmax + 1, 0); carry && q < WL; ++q) {
            carry += out[q];
            out[q] = (uint32_t)carry;
            carry >>= 32;
        }
}

// 2*S > W for wide non-negative integers (S < 2^(32*WL-1)).
__device__ __forceinline__ bool wide_twice_gt(const uint32_t *S, const uint32_t *W) {
    for (int q = WL - 1; q >= 0; --q) {
        uint32_t s2 = (S[q] << 1) | (q > 0 ? (S[q - 1] >> 31) : 0u);
        if (s2 != W[q]) return s2 > W[q];
    }
    return false;
}

// Solve one listed pair: a = the instance's arguments, en.j / en.k the pair,
// lam its lambda.  acc, S and W are per-thread scratch of WL limbs.
template <typename T>
__device__ void exact_entry(const ScanArgs<T> &a, const SlowEntry &en, double lam, uint32_t *acc,
                            uint32_t *S, uint32_t *W, int lane) {
    using Tr = Traits<T>;
    using K = typename Tr::K;
    const int n = (int)a.n;
    const int64_t m = a.m;
    const T *xk = a.Xt + (int64_t)L1L_CHK(en.k, (int32_t)m) * a.ldn;
    const T *xj = a.Xt + (int64_t)L1L_CHK(en.j, (int32_t)m) * a.ldn;
    K ts = Tr::KEY0;
    if (a.ci[en.j].n_valid > 0) {
        // exact total W = sum_i |x_ijhat| + lambda
        int lmin = WL, lmax = -1;
        for (int q = 0; q < WL; ++q) acc[q] = 0;
        for (int i = lane; i < n; i += 32) {
            T b = xj[i];
            if (b != T(0)) wide_add(acc, (double)fabs(b), lmin, lmax);
        }
        wide_warp_reduce(acc, W, lmin, lmax, lane);
        if (lane == 0) {
            int a0 = WL, a1 = -1;
            wide_add(W, lam, a0, a1);
        }
        K lo = 0, hi = Tr::NONE - 1;
        while (lo < hi) {
            const K mid = lo + (hi - lo) / 2;
            lmin = WL;
            lmax = -1;
            for (int q = 0; q < WL; ++q) acc[q] = 0;
            for (int i = lane; i < n; i += 32) {
                T b = xj[i];
                if (b != T(0) && Tr::key(Tr::div_rn(xk[i], b)) <= mid)
                    wide_add(acc, (double)fabs(b), lmin, lmax);
            }
            wide_warp_reduce(acc, S, lmin, lmax, lane);
            int res = 0;
            if (lane == 0) {
                if (mid >= Tr::KEY0) {
                    int a0 = WL, a1 = -1;
                    wide_add(S, lam, a0, a1);
                }
                res = wide_twice_gt(S, W) ? 1 : 0;
            }
            res = __shfl_sync(0xFFFFFFFFu, res, 0);
            if (res)
                hi = mid;
            else
                lo = mid + 1;
        }
        ts = lo;
    }
    const T v = Tr::value(ts);
    // the pair kernel's residual routine (x_ijhat read from the column copy):
    // the same sum in the same order, so s does not depend on which path a
    // pair took
    const T res = pair_residual<T, false>(a, en.j, en.k, xk, xj, n, v, lane);
    if (lane == 0) {
        const int64_t o =
            L1L_CHK(((int64_t)en.t * m + en.j) * m + en.k, (int64_t)a.n_lambda * m * m);
        a.v_all[o] = v;
        a.s_all[o] = (double)res + lam * (double)fabs(v);
    }
}

}  // namespace l1l
