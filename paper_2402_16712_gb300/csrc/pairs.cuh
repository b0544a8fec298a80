// pairs.cuh -- steps A2-A4 for every (lambda, jhat, k): ratios, exact
// weighted median (Lemma 1) and per-pair residual (Algorithm 1).
//
// Layout: one CTA per (jhat, k-chunk).  Column jhat is staged once in shared
// memory -- x_ijhat, its float reciprocal and its fixed-point weight q_i -- and
// shared by the CTA's warps; each warp owns one k at a time and keeps a short
// candidate list of its own.
//
// Per pair the warp never divides per row.  It orders rows by a COARSE key,
// the 32-bit order-preserving image of the ratio rounded to float, and
// approximates it by one multiply, fl(x_ik * fl(1/x_ijhat)) (both rounded to
// float first for double input).  The approximation is within G keys of the
// coarse key of the correctly rounded ratio (G = 8 float, 16 double; the bound
// is derived in the design notes), so a row whose approximate key is more than
// G away from a pivot is classified exactly without dividing; the few rows
// inside a guard band, and the final <= 31 candidates, are divided exactly.
//
//   level 0  64 sampled rows are keyed and sorted across the warp; two pivots
//            bracketing the estimated crossing of half the weight are taken;
//            one pass over all rows sums the exact fixed-point weight below
//            the lower pivot and compacts the rows between the pivots (guard
//            bands included) into the candidate list;
//   resolve  guard-band candidates are divided exactly; an exact 64-bin
//            weight histogram of [P1, P2] and the exact weight below P1 decide
//            whether the median lies between the pivots (else level 0 repeats
//            on the indicated side) and in which bin; that bin's candidates
//            are kept;
//   levels   while more than 31 candidates remain: the same exact histogram
//            over the surviving key range, keep the crossing bin;
//   final    exact keys (double: 64-bit) of the <= 31 candidates plus the
//            penalty point's key, one per lane; each lane's cumulative weight
//            (a shuffle sum over the keys <= its own) is tested and the
//            smallest passing key is the median (the test of Lemma 1, decided
//            exactly);
//   residual sum_i |x_ik - v x_ijhat| over all rows (Algorithm 1, objective).
//
// A decision the truncated fixed-point weights cannot settle, a column whose
// magnitudes fall outside the approximation's range, or a candidate list that
// cannot be narrowed sends the pair to the exact wide-accumulator kernel.
#pragma once
#include <algorithm>
#include <cmath>

#include "binmap.cuh"
#include "checks.cuh"
#include "common.cuh"

namespace l1l {

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~size_t(15); }

__device__ __forceinline__ uint32_t ckey(float r) { return Traits<float>::key(r); }
// Key of an approximate ratio: -0 is not folded onto +0 (the two keys are
// adjacent, well inside the guard band), which saves two instructions.
__device__ __forceinline__ uint32_t akey(float r) {
    const uint32_t u = __float_as_uint(r);
    return u ^ ((uint32_t)((int32_t)u >> 31) | 0x80000000u);
}

template <typename T> struct Approx;
template <> struct Approx<float> {
    static constexpr uint32_t G = 8;
    static __device__ __forceinline__ float inv_of(float b) { return __frcp_rn(b); }
    static __device__ __forceinline__ uint32_t exact_ck(float a, float b) {
        return ckey(__fdiv_rn(a, b));
    }
};
template <> struct Approx<double> {
    static constexpr uint32_t G = 16;
    static __device__ __forceinline__ float inv_of(double b) {
        return __frcp_rn(__double2float_rn(b));
    }
    static __device__ __forceinline__ uint32_t exact_ck(double a, double b) {
        return ckey(__double2float_rn(__ddiv_rn(a, b)));
    }
};

constexpr int NSAMP = 64;   // weight-proportional sample rows per column
constexpr int HIST_WORDS = 4 * 64;  // per-warp exact histogram (4 chunks x 64 bins)

template <typename T> struct PairSmem {
    // per CTA: x_ijhat (T; only when `cs`, else it is read from the column
    // copy in global memory), 1/x_ijhat (float, NaN marks x_ijhat == 0), the
    // 32-bit weights q32_i, the 64 sample rows (uint16)
    __host__ __device__ static size_t col_bytes(int64_t npad, bool cs) {
        return (cs ? al16(npad * sizeof(T)) : 0) + al16(npad * 4) + al16(npad * 4) +
               al16(NSAMP * 2);
    }
    // per warp, 64-bit selection: candidate keys (uint32), row indices
    // (uint16; bit 15 = exact key) and the histogram (4 x 64 uint32)
    __host__ __device__ static size_t bytes64(int64_t cap) {
        return al16(cap * 4) + al16(cap * 2) + al16(HIST_WORDS * 4);
    }
    // per warp, 32-bit selection: 8-byte entries and a 64-word histogram,
    // overlaid by the arrays of its 64-bit fallback
    __host__ __device__ static size_t bytes32(int64_t cap) { return al16(cap * 8) + al16(64 * 4); }
    __host__ __device__ static size_t warp_bytes(int64_t cap) {
        const size_t a = bytes32(cap), b = bytes64(cap);
        return a > b ? a : b;
    }
    // the largest capacity (a multiple of 32) whose per-warp region fits `bytes`
    __host__ __device__ static int64_t cap_fit(int64_t bytes) {
        const int64_t c64 = (bytes - HIST_WORDS * 4 - 32) / 6;
        const int64_t c32 = (bytes - 64 * 4 - 16) / 8;
        int64_t c = (c64 < c32 ? c64 : c32) & ~int64_t(31);
        while (c > 0 && warp_bytes(c) > (size_t)bytes) c -= 32;
        return c;
    }
};

constexpr uint16_t EXACT_BIT = 0x8000u;
constexpr uint32_t CKMAX = 0xFFFFFFFEu;    // largest usable coarse key
constexpr uint32_t CKNONE = 0xFFFFFFFFu;

// ---------------------------------------------------------------------------
// Warp sorts.
// ---------------------------------------------------------------------------
template <typename K, typename W>
__device__ __forceinline__ void warp_sort32(K &key, W &w, int lane) {
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            K ok = __shfl_xor_sync(0xFFFFFFFFu, key, stride);
            W ow = __shfl_xor_sync(0xFFFFFFFFu, w, stride);
            bool up = (lane & size) == 0 || size == 32;
            bool lower = (lane & stride) == 0;
            bool take = lower == up ? (ok < key) : (ok > key);
            if (take) {
                key = ok;
                w = ow;
            }
        }
    }
}

// 64 keys, element g = e*32 + lane held in slot e; ascending in g.
__device__ __forceinline__ void warp_sort64(uint32_t (&k)[2], int lane) {
#pragma unroll
    for (int size = 2; size <= 64; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride == 32) {  // only in the final merge: ascending
                const uint32_t lo = min(k[0], k[1]), hi = max(k[0], k[1]);
                k[0] = lo;
                k[1] = hi;
            } else {
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const uint32_t ok = __shfl_xor_sync(0xFFFFFFFFu, k[e], stride);
                    const int g = e * 32 + lane;
                    const bool up = (g & size) == 0;
                    const bool lower = (lane & stride) == 0;
                    k[e] = (lower == up) ? min(ok, k[e]) : max(ok, k[e]);
                }
            }
        }
    }
}

template <typename V> __device__ __forceinline__ V warp_scan_add(V x, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        V y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Residual over the padded rows: Xt and the staged column are zero past n, so
// a padding row adds |0 - v 0| = 0.  np is a multiple of ROW_PAD.
//   float:  eight rows per lane per step, all eight global loads issued before
//           any is summed, four accumulators (a load issued a step ahead
//           measured slower at low occupancy);
//   double: four rows per lane per step, the next step's loads issued before
//           this step is summed (eight double loads in flight spill at the
//           kernel's register cap).
template <typename T>
__device__ __forceinline__ T warp_residual_pad(const T *__restrict__ xk, const T *__restrict__ xj,
                                               int n, T v, int lane) {
    const int np = (n + ROW_PAD - 1) & ~(ROW_PAD - 1);
    T acc[4] = {T(0), T(0), T(0), T(0)};
    if constexpr (sizeof(T) == 4) {
        constexpr int U = 8;
        static_assert(32 * U == 2 * ROW_PAD, "a step is two row pads");
        int i0 = 0;
        for (; i0 + 32 * U <= np; i0 += 32 * U) {
            T ac[U];
#pragma unroll
            for (int u = 0; u < U; ++u) ac[u] = xk[i0 + u * 32 + lane];
#pragma unroll
            for (int u = 0; u < U; ++u)
                acc[u & 3] += fabs(fma(-v, xj[i0 + u * 32 + lane], ac[u]));
        }
        if (i0 < np) {  // one row pad left
            T ac[U / 2];
#pragma unroll
            for (int u = 0; u < U / 2; ++u) ac[u] = xk[i0 + u * 32 + lane];
#pragma unroll
            for (int u = 0; u < U / 2; ++u) acc[u] += fabs(fma(-v, xj[i0 + u * 32 + lane], ac[u]));
        }
    } else {
        constexpr int U = 4;
        static_assert(U * 32 == ROW_PAD, "one step = one row pad");
        T an[U];
#pragma unroll
        for (int u = 0; u < U; ++u) an[u] = xk[u * 32 + lane];
        for (int i0 = 0; i0 < np; i0 += 32 * U) {
            T ac[U];
#pragma unroll
            for (int u = 0; u < U; ++u) ac[u] = an[u];
            if (i0 + 32 * U < np) {
#pragma unroll
                for (int u = 0; u < U; ++u) an[u] = xk[i0 + 32 * U + u * 32 + lane];
            }
#pragma unroll
            for (int u = 0; u < U; ++u) acc[u] += fabs(fma(-v, xj[i0 + u * 32 + lane], ac[u]));
        }
    }
    T s = (acc[0] + acc[1]) + (acc[2] + acc[3]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
    return s;
}

// Outcomes of select_v2.  Every code >= SEL_SLOW hands the pair to the exact
// path; the code says why (kept in the slow list for diagnostics).
enum {
    SEL_OK = 0,
    SEL_INTERNAL = 1,
    SEL_SLOW = 2,        // column outside the approximate-key range / forced
    SEL_SLOW_TRIES,      // level 0 kept missing the median
    SEL_SLOW_CAP,        // too many rows between the closest pivots
    SEL_SLOW_BAND,       // truncated weights cannot settle a decision
    SEL_SLOW_LEVELS,     // candidate list did not shrink
    SEL_SLOW_TIE         // double: one coarse key holds distinct exact keys
};

__device__ __forceinline__ uint32_t sat_sub(uint32_t a, uint32_t b) { return a > b ? a - b : 0u; }
__device__ __forceinline__ uint32_t sat_add(uint32_t a, uint32_t b) {
    return a < CKNONE - b ? a + b : CKNONE;
}

// Estimated index (0..ns-1) of the first sorted sample whose scaled cumulative
// weight passes the crossing target; targets are relative to L.
// Pivot estimates are float: they only steer the search (every decision that
// matters is exact, in int64), and this GPU's double pipe is narrow.
__device__ __forceinline__ float target_for(uint32_t key, float hneg, float hpos) {
    return key >= CK0 ? hpos : hneg;
}

// ---------------------------------------------------------------------------
// Exact weight histogram: XB bins, each an int64 sum kept as four 16-bit
// chunks in 32-bit shared-memory counters (exact for up to 65,535 rows per
// bin; 64-bit shared atomics are several times slower on this GPU).
// ---------------------------------------------------------------------------
constexpr int XB = 64;
constexpr uint16_t ROW_MASK = 0x7FFFu;

__device__ __forceinline__ void hist_zero(uint32_t *h, int lane) {
#pragma unroll
    for (int q = 0; q < (4 * XB) / 32; ++q) h[q * 32 + lane] = 0u;
}
__device__ __forceinline__ void hist_add(uint32_t *h, int bin, int64_t q) {
    bin = L1L_CHK(bin, XB);
    const uint64_t u = (uint64_t)q;
    atomicAdd(&h[bin], (uint32_t)(u & 0xFFFFu));
    atomicAdd(&h[XB + bin], (uint32_t)((u >> 16) & 0xFFFFu));
    atomicAdd(&h[2 * XB + bin], (uint32_t)((u >> 32) & 0xFFFFu));
    atomicAdd(&h[3 * XB + bin], (uint32_t)(u >> 48));
}
__device__ __forceinline__ int64_t hist_get(const uint32_t *h, int bin) {
    return (int64_t)h[bin] + ((int64_t)h[XB + bin] << 16) + ((int64_t)h[2 * XB + bin] << 32) +
           ((int64_t)h[3 * XB + bin] << 48);
}

// Among bins 0..nbins-1 of [base, top] (bin b = keys base + [b, b+1) << sh),
// find the first whose upper key passes the exact test with S = Sbase + weight
// of bins <= b.  Returns the bin (-1: none passes, -2: undecidable) and the
// weight below it in *below.
__device__ __forceinline__ int hist_cross(const uint32_t *h, int nbins, uint32_t base,
                                          uint32_t top, int sh, int64_t Sbase,
                                          const Decide &dc, int64_t *below, int lane) {
    const unsigned FULL = 0xFFFFFFFFu;
    const int b0 = 2 * lane, b1 = 2 * lane + 1;
    const int64_t s0 = b0 < nbins ? hist_get(h, b0) : 0;
    const int64_t s1 = b1 < nbins ? hist_get(h, b1) : 0;
    const int64_t incl = warp_scan_add(s0 + s1, lane);
    const int64_t ex = incl - s0 - s1;
    auto bhi = [&](int b) -> uint32_t {
        const uint64_t v = (uint64_t)base + ((uint64_t)(b + 1) << sh) - 1;
        return v > top ? top : (uint32_t)v;
    };
    const int c0 = b0 < nbins ? dc.cond(Sbase + ex + s0, bhi(b0) >= CK0) : 0;
    const int c1 = b1 < nbins ? dc.cond(Sbase + ex + s0 + s1, bhi(b1) >= CK0) : 0;
    const unsigned m0 = __ballot_sync(FULL, c0 != 0), m1 = __ballot_sync(FULL, c1 != 0);
    const unsigned any = m0 | m1;
    if (!any) return -1;
    const int ln = __ffs(any) - 1;
    const bool first_is_b0 = (m0 >> ln) & 1u;
    const int bsel = 2 * ln + (first_is_b0 ? 0 : 1);
    const int csel = __shfl_sync(FULL, first_is_b0 ? c0 : c1, ln);
    const int64_t bel = __shfl_sync(FULL, first_is_b0 ? ex : ex + s0, ln);
    if (csel < 0) return -2;
    *below = Sbase + bel;
    return bsel;
}

// hist_cross over the bins of a BinMap (at most XB of them).
__device__ __forceinline__ int hist_cross_map(const uint32_t *h, const BinMap &bm, int64_t Sbase,
                                              const Decide &dc, int64_t *below, int lane) {
    const unsigned FULL = 0xFFFFFFFFu;
    const int nbins = bm.nbins();
    const int b0 = 2 * lane, b1 = 2 * lane + 1;
    const int64_t s0 = b0 < nbins ? hist_get(h, b0) : 0;
    const int64_t s1 = b1 < nbins ? hist_get(h, b1) : 0;
    const int64_t incl = warp_scan_add(s0 + s1, lane);
    const int64_t ex = incl - s0 - s1;
    const int c0 = b0 < nbins ? dc.cond(Sbase + ex + s0, bm.upper(b0) >= CK0) : 0;
    const int c1 = b1 < nbins ? dc.cond(Sbase + ex + s0 + s1, bm.upper(b1) >= CK0) : 0;
    const unsigned m0 = __ballot_sync(FULL, c0 != 0), m1 = __ballot_sync(FULL, c1 != 0);
    const unsigned any = m0 | m1;
    if (!any) return -1;
    const int ln = __ffs(any) - 1;
    const bool first_is_b0 = (m0 >> ln) & 1u;
    const int bsel = 2 * ln + (first_is_b0 ? 0 : 1);
    const int csel = __shfl_sync(FULL, first_is_b0 ? c0 : c1, ln);
    const int64_t bel = __shfl_sync(FULL, first_is_b0 ? ex : ex + s0, ln);
    if (csel < 0) return -2;
    *below = Sbase + bel;
    return bsel;
}

// The 64-bit fixed-point weight q_i of row i for the 64-bit selection,
// computed from x_ijhat on the spot (the fast path stages 32-bit weights;
// the 64-bit selection is its rare fallback).
template <typename T> struct WqFly {
    const T *colb;
    int sigma;
    __device__ __forceinline__ int64_t operator()(int i) const {
        const T b = colb[i];
        int e = 0;
        return b != T(0) ? fixq(b < T(0) ? -b : b, sigma, e) : 0;
    }
};

}  // namespace l1l

#include "select32.cuh"

namespace l1l {

// ---------------------------------------------------------------------------
// Weighted median of one pair.  Returns SEL_* and the exact key in tstar.
//
// The candidate list is kept as 32 interleaved per-lane segments: lane l's
// j-th candidate sits at slot j*32 + l (bank l, so every access is free of bank
// conflicts) and each lane counts its own candidates against a quota of
// qt = cap/32 slots; only the final <= 31 candidates are gathered across the
// warp.  Row indices carry a flag bit, EXACT: the stored key is exact.  The
// candidate arrays, the histogram and the column arrays never overlap (hence
// __restrict__), so the loops over the list below, unrolled by two, can issue
// the shared-memory loads of one candidate before the atomics of the other.
// ---------------------------------------------------------------------------
template <typename T, typename WQ>
__device__ int select_v2(const T *__restrict__ xk, const float *__restrict__ xf,
                         const T *__restrict__ colb, const float *__restrict__ inv,
                         const WQ colq, const uint16_t *__restrict__ samp,
                         uint32_t *__restrict__ lk, uint16_t *__restrict__ li,
                         uint32_t *__restrict__ hist, int qt, int n, int d0, const Decide &dc,
                         typename Traits<T>::K &tstar, int lane) {
    using Tr = Traits<T>;
    using K = typename Tr::K;
    using A = Approx<T>;
    constexpr uint32_t G = A::G;
    const unsigned FULL = 0xFFFFFFFFu;
    const float Qf = (float)dc.Q;
    const float hneg0 = 0.5f * (Qf + (float)dc.Lf), hpos0 = 0.5f * (Qf - (float)dc.Lc);
    const int nrow = (n + ROW_PAD - 1) & ~(ROW_PAD - 1);  // rows the columns hold
    const int nslot = qt * 32;                             // candidate slots
    (void)nrow;
    (void)nslot;

    // ---------------- level 0 -------------------------------------------
    // 64 rows drawn in proportion to their weight (each stands for Q/64), so the
    // sorted sample keys estimate the weighted quantiles directly.
    uint32_t sk[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int i = L1L_CHK((int)samp[e * 32 + lane], nrow);
        sk[e] = akey(__fmul_rn(xf[i], inv[i]));
    }
    warp_sort64(sk, lane);
    int jx;
    {
        const float unit = Qf * (1.0f / 64.0f);
        const bool c0 = (float)(lane + 1) * unit > target_for(sk[0], hneg0, hpos0);
        const bool c1 = (float)(lane + 33) * unit > target_for(sk[1], hneg0, hpos0);
        const unsigned m0 = __ballot_sync(FULL, c0), m1 = __ballot_sync(FULL, c1);
        jx = m0 ? __ffs(m0) - 1 : (m1 ? 32 + __ffs(m1) - 1 : 63);
    }
    auto sample_key = [&](int g) -> uint32_t {
        const uint32_t a0 = __shfl_sync(FULL, sk[0], g & 31);
        const uint32_t a1 = __shfl_sync(FULL, sk[1], g & 31);
        return g < 32 ? a0 : a1;
    };
    // the median's coarse key is known to lie in [lo0, hi0]; pivots stay inside
    uint32_t lo0 = 0, hi0 = CKMAX;
    auto pick = [&](int g, uint32_t dflt) -> uint32_t {
        uint32_t kk = (g < 0 || g > 63) ? dflt : sample_key(g);
        if (kk > CKMAX) kk = dflt;
        return min(max(kk, lo0), hi0);
    };
    // d0: half-width of the first bracket in sample positions (6 of 64: ~15%
    // of the rows in the bracket, ~1.5% misses)
    // pivots 2G + 1 keys outside the sample keys, so that the sample rows (and
    // rows tied with them) lie clear of the guard bands
    uint32_t P1 = pick(jx - d0, lo0);
    uint32_t P2 = pick(jx + d0, hi0);
    P1 = max(sat_sub(P1, 2 * G + 1), lo0);
    P2 = min(sat_add(P2, 2 * G + 1), hi0);
    if (P1 > P2) P1 = P2;
    bool sampled = true;     // the bracket still comes from the sample
    bool count_pass = false;  // next attempt: narrow by a histogram over all rows

    int64_t L = 0;   // exact weight of rows with coarse key < lo
    uint32_t lo = 0, hi = CKMAX;
    int cnt = 0;     // this lane's candidates
    bool placed = false;
    for (int attempt = 0; attempt < 12 && !placed; ++attempt) {
        if (count_pass) {
            // One pass over all rows straight into the exact histogram of
            // [P1, P2] (rows near a bin edge are divided on the spot); nothing
            // is stored, so it cannot overflow.  The median's bin becomes the
            // next bracket, 1/64 of this one.
            const uint32_t span = P2 - P1;
            const int sh = span >= (uint32_t)XB ? (32 - __clz((int)span)) - 6 : 0;
            const uint32_t bmask = (1u << sh) - 1u;
            const int nbins = (int)(span >> sh) + 1;
            const uint32_t bt = sat_sub(P1, G), at = min(sat_add(P2, G), CKMAX);
            const uint32_t g1 = sat_add(P1, G), g2 = sat_sub(P2, G);
            hist_zero(hist, lane);
            __syncwarp();
            int64_t Sb = 0;
            for (int i = lane; i < n; i += 32) {
                const float iv = inv[i];
                if (isnan(iv)) continue;  // x_ijhat = 0 or a padding row
                uint32_t kk = akey(__fmul_rn(xf[i], iv));
                if (kk < bt) {
                    Sb += colq(i);
                    continue;
                }
                if (kk > at) continue;
                const uint32_t off = (kk - P1) & bmask;
                if (!(kk >= g1 && kk <= g2 && off >= G && off + G <= bmask))
                    kk = A::exact_ck(xk[i], colb[i]);
                if (kk < P1)
                    Sb += colq(i);
                else if (kk <= P2)
                    hist_add(hist, (int)((kk - P1) >> sh), colq(i));
            }
            Sb = warp_sum_i64(Sb);
            __syncwarp();
            const int r1 = P1 == lo0 ? 0 : dc.cond(Sb, (P1 - 1) >= CK0);
            if (r1 < 0) return SEL_SLOW_BAND;
            if (r1 == 1) {
                hi0 = P1 - 1;
                P1 = lo0;
                P2 = hi0;
                continue;
            }
            int64_t below = 0;
            const int bs = hist_cross(hist, nbins, P1, P2, sh, Sb, dc, &below, lane);
            __syncwarp();
            if (bs == -2) return SEL_SLOW_BAND;
            if (bs < 0) {
                if (P2 >= hi0) return SEL_INTERNAL;
                lo0 = P2 + 1;
                P1 = lo0;
                P2 = hi0;
                continue;
            }
            const uint32_t K1 = P1 + ((uint32_t)bs << sh);
            const uint32_t K2 = min(P2, K1 + bmask);
            lo0 = K1;
            hi0 = K2;
            P1 = K1;
            P2 = K2;
            sampled = false;
            count_pass = false;
            if (K1 == K2) {  // one coarse key holds the median
                if (sizeof(T) == 4) {
                    tstar = (K)K1;
                    return SEL_OK;
                }
                return SEL_SLOW_CAP;  // double: its exact keys are not known here
            }
            continue;
        }
        // one pass over all rows: exact weight of rows certainly below P1; rows
        // whose approximate key is within G of [P1, P2] become candidates
        const uint32_t bt = sat_sub(P1, G);  // certain below: key' < bt
        const uint32_t at = min(sat_add(P2, G), CKMAX);  // certain above: key' > at
        int64_t Sb = 0;
        cnt = 0;
        // rows are visited in batches of 4 per lane; the global loads of the next
        // batch are issued before the current one is classified, so the L2
        // latency overlaps the work
        // U * 32 = ROW_PAD rows per batch: every index below the padded row
        // count is readable, and padding rows (reciprocal NaN) are neither
        // below nor candidates
        constexpr int U = 4;
        static_assert(U * 32 == ROW_PAD, "one batch = one row pad");
        float an[U];
#pragma unroll
        for (int u = 0; u < U; ++u) an[u] = xf[u * 32 + lane];
        for (int i0 = 0; i0 < n; i0 += 32 * U) {
            float ac[U];
#pragma unroll
            for (int u = 0; u < U; ++u) ac[u] = an[u];
            if (i0 + 32 * U < n) {
#pragma unroll
                for (int u = 0; u < U; ++u) an[u] = xf[i0 + 32 * U + u * 32 + lane];
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                // branch-free
                const int i = i0 + u * 32 + lane;
                const float iv = inv[i];
                const uint32_t kk = akey(__fmul_rn(ac[u], iv));
                const bool below = kk < bt;
                const bool cand = !below && kk <= at;
                const int64_t q = colq(i);
                Sb += below ? q : 0;
                // speculative store: the slot is only kept when cnt advances
                if (cnt < qt) {
                    lk[L1L_CHK(cnt * 32 + lane, nslot)] = kk;
                    li[cnt * 32 + lane] = (uint16_t)L1L_CHK(i, nrow);
                }
                cnt += cand ? 1 : 0;
            }
        }
        Sb = warp_sum_i64(Sb);
        __syncwarp();
        if (__any_sync(FULL, cnt > qt)) {  // a lane overflowed: narrow by a count pass
            if (P1 == P2) return SEL_SLOW_CAP;
            count_pass = true;
            continue;
        }
        // exact histogram of the candidates over the bins of [P1, P2]; rows
        // within G of P1, P2 or their bin's edges are divided exactly first;
        // Sb2 = exact weight below P1
        BinMap bm;
        bm.init(P1, P2, XB);
        const uint32_t g1 = sat_add(P1, G), g2 = sat_sub(P2, G);
        hist_zero(hist, lane);
        __syncwarp();
        int64_t Sb2 = 0;
#pragma unroll 2
        for (int j = 0; j < cnt; ++j) {
            const int p = L1L_CHK(j * 32 + lane, nslot);
            uint32_t kk = lk[p];
            const uint16_t id = (uint16_t)L1L_CHK((int)li[p], nrow);
            // clear: the keys G either side fall in the same bin
            const bool clear = kk >= g1 && kk <= g2 && bm.bin(kk - G) == bm.bin(kk + G);
            if (!clear) {
                kk = A::exact_ck(xk[id], colb[id]);
                lk[p] = kk;
                li[p] = id | EXACT_BIT;
            }
            const int64_t q = colq(id);
            if (kk < P1)
                Sb2 += q;
            else if (kk <= P2)
                hist_add(hist, bm.bin(kk), q);
        }
        Sb += warp_sum_i64(Sb2);
        __syncwarp();
        const int r1 = P1 == lo0 ? 0 : dc.cond(Sb, (P1 - 1) >= CK0);
        if (r1 < 0) return SEL_SLOW_BAND;
        if (r1 == 1) {  // median below P1: retry under P1
            hi0 = P1 - 1;
            P2 = hi0;
            P1 = sampled ? max(sat_sub(pick(jx - 3 * max(d0, 1) - 1, lo0), 2 * G + 1), lo0) : lo0;
            if (P1 > P2) P1 = lo0;
            continue;
        }
        int64_t below = 0;
        const int bs = hist_cross_map(hist, bm, Sb, dc, &below, lane);
        __syncwarp();
        if (bs == -2) return SEL_SLOW_BAND;
        if (bs < 0) {  // median above P2: retry over P2
            if (P2 >= hi0) return SEL_INTERNAL;
            lo0 = P2 + 1;
            P1 = lo0;
            P2 = sampled ? min(sat_add(pick(jx + 3 * max(d0, 1) + 1, hi0), 2 * G + 1), hi0) : hi0;
            if (P2 < P1) P2 = hi0;
            continue;
        }
        // the median is in bin bs: keep its candidates (lane-local, in place)
        const uint32_t K1 = bm.lower(bs);
        const uint32_t K2 = bm.upper(bs);
        int w = 0;
#pragma unroll 2
        for (int j = 0; j < cnt; ++j) {
            const int p = j * 32 + lane;
            const uint32_t kk = lk[p];
            const uint16_t id = li[p];
            lk[w * 32 + lane] = kk;  // w <= j: kept only if w advances
            li[w * 32 + lane] = id;
            w += (kk >= K1 && kk <= K2) ? 1 : 0;
        }
        __syncwarp();
        cnt = w;
        L = below;
        lo = K1;
        hi = K2;
        placed = true;
    }
    if (!placed) return SEL_SLOW_TRIES;

    // ---------------- levels on the candidate list: exact histograms ------
    int c = __reduce_add_sync(FULL, cnt);
    for (int level = 0; c > 31 && lo < hi; ++level) {
        if (level >= 8) return SEL_SLOW_LEVELS;
        const uint32_t span = hi - lo;
        const int sh = span >= (uint32_t)XB ? (32 - __clz((int)span)) - 6 : 0;
        const uint32_t bmask = (1u << sh) - 1u;
        const int nbins = (int)(span >> sh) + 1;
        hist_zero(hist, lane);
        __syncwarp();
#pragma unroll 2
        for (int j = 0; j < cnt; ++j) {
            const int p = L1L_CHK(j * 32 + lane, nslot);
            uint32_t kk = lk[p];
            uint16_t id = li[p];
            (void)L1L_CHK((int)(id & ROW_MASK), nrow);  // counted in the checked build
            const uint32_t off = (kk - lo) & bmask;
            if (!(id & EXACT_BIT) && (off < G || off + G > bmask)) {
                const int row = id & ROW_MASK;
                kk = A::exact_ck(xk[row], colb[row]);
                lk[p] = kk;
                id = (uint16_t)row | EXACT_BIT;
                li[p] = id;
            }
            hist_add(hist, (int)((kk - lo) >> sh), colq(id & ROW_MASK));
        }
        __syncwarp();
        int64_t below = 0;
        const int bs = hist_cross(hist, nbins, lo, hi, sh, L, dc, &below, lane);
        __syncwarp();
        if (bs == -2) return SEL_SLOW_BAND;
        if (bs < 0) return SEL_INTERNAL;
        const uint32_t K1 = lo + ((uint32_t)bs << sh);
        const uint32_t K2 = min(hi, K1 + bmask);
        int w = 0;
#pragma unroll 2
        for (int j = 0; j < cnt; ++j) {
            const int p = j * 32 + lane;
            const uint32_t kk = lk[p];
            const uint16_t id = li[p];
            lk[w * 32 + lane] = kk;
            li[w * 32 + lane] = id;
            w += (kk >= K1 && kk <= K2) ? 1 : 0;
        }
        __syncwarp();
        cnt = w;
        L = below;
        lo = K1;
        hi = K2;
        c = __reduce_add_sync(FULL, cnt);
    }

    // ---------------- final: exact keys of the candidates ------------------
    if (sizeof(T) == 4 && lo == hi) {  // coarse keys are the exact keys for float
        tstar = (K)lo;
        return SEL_OK;
    }
    if (c > 31) {  // one coarse key left, many rows: all exact keys equal?
        K kmin = Tr::NONE, kmax = 0;
#pragma unroll 2
        for (int j = 0; j < cnt; ++j) {
            const int row = li[j * 32 + lane] & ROW_MASK;
            const K ke = Tr::key(Tr::div_rn(xk[row], colb[row]));
            kmin = min(kmin, ke);
            kmax = max(kmax, ke);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            kmin = min(kmin, __shfl_xor_sync(FULL, kmin, o));
            kmax = max(kmax, __shfl_xor_sync(FULL, kmax, o));
        }
        const bool zero_in = lo <= CK0 && CK0 <= hi;
        if (kmin == kmax && !(zero_in && kmin != Tr::KEY0)) {
            tstar = kmin;
            return SEL_OK;
        }
        return SEL_SLOW_TIE;
    }
    // gather the <= 31 candidate rows into lanes 0..c-1 (via the histogram buffer)
    {
        const int excl = warp_scan_add(cnt, lane) - cnt;
        uint16_t *stage = reinterpret_cast<uint16_t *>(hist);
        for (int j = 0; j < cnt; ++j)
            stage[L1L_CHK(excl + j, 31)] = li[L1L_CHK(j * 32 + lane, nslot)] & ROW_MASK;
    }
    __syncwarp();
    K fk = Tr::NONE;
    int64_t fq = 0;
    if (lane < c) {
        const int row = L1L_CHK((int)reinterpret_cast<const uint16_t *>(hist)[lane], nrow);
        fk = Tr::key(Tr::div_rn(xk[row], colb[row]));
        fq = colq(row);
    } else if (lane == c && lo <= CK0 && CK0 <= hi) {
        fk = Tr::KEY0;
        fq = 0;
    }
    __syncwarp();
    // Rank form of "sort, prefix-sum, take the first key that passes": each
    // candidate sums the weight of the candidates whose key is <= its own
    // (equal keys get equal sums), tests it, and the smallest key that passes
    // (or cannot be settled) is the answer.  A few candidates remain here, so
    // this costs a few shuffles per candidate instead of a 32-lane sort.
    const int nv = c + ((lo <= CK0 && CK0 <= hi) ? 1 : 0);
    int64_t S = 0;
    for (int u = 0; u < nv; ++u) {
        const K ku = __shfl_sync(FULL, fk, u);
        const int64_t qu = __shfl_sync(FULL, fq, u);
        S += ku <= fk ? qu : 0;
    }
    int r = 0;
    if (lane < nv) r = dc.cond(L + S, fk >= Tr::KEY0);
    K kmin = r != 0 ? fk : Tr::NONE;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) kmin = min(kmin, __shfl_xor_sync(FULL, kmin, o));
    if (kmin == Tr::NONE) return SEL_INTERNAL;
    if (__any_sync(FULL, r == -1 && fk == kmin)) return SEL_SLOW_BAND;
    tstar = kmin;
    return SEL_OK;
}

// The lambdas of one launch (or of one instance of a batch).
struct LamView {
    const double *lam;
    int tl_min, tl_max;  // positions of the smallest and largest lambda
};

// Everything one warp needs to solve the pairs of its CTA's column jhat.
// The fast path's weights are the 32-bit q32 (both input types); s_dec and
// decide_for use the same scale.
template <typename T> struct WarpCtx {
    const T *colb;
    const float *inv;
    const uint32_t *q32;
    const uint16_t *samp;
    uint32_t *lk;          // 64-bit fallback's lists and histogram
    uint16_t *li;
    uint32_t *hist;
    uint2 *lst;            // 32-bit selection's list and histogram
    uint32_t *hist32;
    const Decide *s_dec;  // per-lambda thresholds for the first NDEC lambdas
    int qt, n;
    int d0;               // first-bracket half-width in sample positions
    ColInfo cinfo;
    __device__ __forceinline__ int64_t q(int i) const { return (int64_t)q32[i]; }
};
constexpr int NDEC = 32;

// The exact test of lambda tl on the fast path's weight scale (q32).
template <typename T>
__device__ __forceinline__ void decide_init(Decide &dc, const ColInfo &ci, double lam) {
    dc.init32(ci, lam);
}
template <typename T>
__device__ __forceinline__ Decide decide_for(const WarpCtx<T> &w, const LamView &lp, int tl) {
    Decide dc;
    if (tl < NDEC)
        dc = w.s_dec[tl];
    else
        decide_init<T>(dc, w.cinfo, lp.lam[tl]);
    return dc;
}

// The 64-bit selection of a pair that the 32-bit weights could not settle
// (rare): a separate, not inlined function, so that its code stays out of the
// hot loop's instruction stream.  Weights are computed from x_ijhat.
template <typename T>
__device__ __noinline__ int select_fallback64(const T *xk, const float *xf, const T *colb,
                                              const float *inv, const uint16_t *samp,
                                              uint32_t *lk, uint16_t *li, uint32_t *hist,
                                              int qt, int n, int d0, int64_t Q, int sigma,
                                              int inexact, double lam,
                                              typename Traits<T>::K *ts, int lane) {
    Decide d64;
    d64.init_at(Q, sigma, inexact, lam);
    typename Traits<T>::K k = 0;
    const int st = select_v2<T>(xk, xf, colb, inv, WqFly<T>{colb, sigma}, samp, lk, li, hist, qt,
                                n, d0, d64, k, lane);
    *ts = k;
    return st;
}

// The full selection of one (lambda, pair): the 32-bit weights first, and the
// pair again on 64-bit weights (computed from x_ijhat) when those cannot
// settle it.
template <typename T>
__device__ __forceinline__ int select_pair(const T *xk, const float *xf, const WarpCtx<T> &w,
                                           const LamView &lp, int tl,
                                           typename Traits<T>::K &ts, int lane) {
    const Decide dc = decide_for(w, lp, tl);
    typename Traits<T>::K t32 = 0;
    const int st = select_w32<T>(xf, xk, w.colb, w.inv, w.q32, w.samp, w.lst, w.hist32, w.qt,
                                 w.n, w.d0, dc, t32, lane);
    if (st != SEL_W64) {
        ts = t32;
        return st;
    }
    __syncwarp();
    typename Traits<T>::K t64 = 0;
    const int st64 = select_fallback64<T>(xk, xf, w.colb, w.inv, w.samp, w.lk, w.li, w.hist, w.qt,
                                          w.n, w.d0, w.cinfo.Q, w.cinfo.sigma, w.cinfo.n_inexact,
                                          lp.lam[tl], &t64, lane);
    ts = t64;
    return st64;
}

// ---------------------------------------------------------------------------
// Residual of a double pair in float-float arithmetic (the double pipe of
// this GPU runs at 1/64 of the float rate; summed in double, the residual's
// two double operations per row made that pipe the bound of the double fit).  Each double x is held as two floats, x1 = fl(x) and
// x2 = fl(x - x1) (the staged copies Xf and Xlo), so |x - x1 - x2| <= u^2|x|
// with u = 2^-24; v likewise.  Per row, with K = |v||x_ijhat|:
//   p1 = fl(v1 b1), e1 = fma(v1, b1, -p1) (exact), c = fma(v1, b2, fma(v2, b1, e1));
//   (s, t) = TwoSum(a1, -p1) (exact), d = fl(fl(a2 - c) + t);
// then s + d = x_ik - v x_ijhat within u^2 (4.04|x_ik| + 15.12 K) + 8 eta
// (eta = 2^-150, the products' underflow), and |s + d| is the pair negated
// when fl(s + d) < 0.  A lane sums its rows in blocks of 8: (H, e) =
// TwoSum(H, s'), L = fl(L + fl(d' + e)), error <= 9.02 u sum|d| + 72.1 u^2
// T_block with |d| <= u (2.04|x_ik| + 4.06 K); each block goes to a double
// accumulator (two roundings of 2^-53 per block), the lanes' sums are added
// in double.  In all, with C_k = sum_i |x_ik|, W = sum_i |x_ijhat|, T the
// exact residual and ldn the padded rows,
//   |T_ff - T| <= E = u^2 (24 C_k + 56 |v| W + (76 + ldn/4096) T) + ldn 2^-146.
// ff_certified accepts T_ff when E (with 77 T_ff in place of 76 T, and C_k, W
// bounded above from the fixed-point column totals) is at most 2^-40 T_ff,
// i.e. a relative error of at most 9.1e-13; any other pair (a near-exact
// fit, v outside [2^-60, 2^60]) is summed again in double.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void ff_row(float a1, float a2, float b1, float b2, float v1, float v2,
                                       float &H, float &L) {
    const float p1 = __fmul_rn(v1, b1);
    const float e1 = __fmaf_rn(v1, b1, -p1);
    const float c = __fmaf_rn(v1, b2, __fmaf_rn(v2, b1, e1));
    const float s = __fsub_rn(a1, p1);
    const float sb = __fsub_rn(s, a1);
    const float t = __fadd_rn(__fsub_rn(a1, __fsub_rn(s, sb)), __fsub_rn(-p1, sb));
    const float d = __fadd_rn(__fsub_rn(a2, c), t);
    // |s + d|: both halves take the sign of fl(s + d)
    const uint32_t sg = __float_as_uint(__fadd_rn(s, d)) & 0x80000000u;
    const float sp = __uint_as_float(__float_as_uint(s) ^ sg);
    const float dp = __uint_as_float(__float_as_uint(d) ^ sg);
    const float h = __fadd_rn(H, sp);
    const float hb = __fsub_rn(h, H);
    const float e = __fadd_rn(__fsub_rn(H, __fsub_rn(h, hb)), __fsub_rn(sp, hb));
    H = h;
    L = __fadd_rn(L, __fadd_rn(dp, e));
}
__device__ __forceinline__ void ff_group(const float4 &a1, const float4 &a2, const float4 &b1,
                                         const float4 &b2, float v1, float v2, float &H, float &L) {
    ff_row(a1.x, a2.x, b1.x, b2.x, v1, v2, H, L);
    ff_row(a1.y, a2.y, b1.y, b2.y, v1, v2, H, L);
    ff_row(a1.z, a2.z, b1.z, b2.z, v1, v2, H, L);
    ff_row(a1.w, a2.w, b1.w, b2.w, v1, v2, H, L);
}
// The sum over the ldn padded rows (zero in both columns past n); a1p, a2p:
// column k's float pair, b1p, b2p: column jhat's.  Every lane returns it.
__device__ __forceinline__ double residual_ff(const float *__restrict__ a1p,
                                              const float *__restrict__ a2p,
                                              const float *__restrict__ b1p,
                                              const float *__restrict__ b2p, int64_t ldn,
                                              float v1, float v2, int lane) {
    const float4 *A1 = reinterpret_cast<const float4 *>(a1p) + lane;
    const float4 *A2 = reinterpret_cast<const float4 *>(a2p) + lane;
    const float4 *B1 = reinterpret_cast<const float4 *>(b1p) + lane;
    const float4 *B2 = reinterpret_cast<const float4 *>(b2p) + lane;
    const int ng = (int)(ldn >> 7);  // 128-row groups; a lane takes 4 rows of each
    const float4 z4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    double D = 0.0;
    for (int g = 0; g < ng; g += 2) {  // blocks of 8 rows per lane
        // an odd last group is paired with zero rows, which add exactly 0
        const bool two = g + 1 < ng;
        const int o0 = g * 32, o1 = (g + 1) * 32;
        const float4 xa = __ldg(A1 + o0), xb = two ? __ldg(A1 + o1) : z4;
        const float4 la = __ldg(A2 + o0), lb = two ? __ldg(A2 + o1) : z4;
        const float4 ya = __ldg(B1 + o0), yb = two ? __ldg(B1 + o1) : z4;
        const float4 ma = __ldg(B2 + o0), mb = two ? __ldg(B2 + o1) : z4;
        float H = 0.0f, L = 0.0f;
        ff_group(xa, la, ya, ma, v1, v2, H, L);
        ff_group(xb, lb, yb, mb, v1, v2, H, L);
        D = __dadd_rn(D, (double)H);
        D = __dadd_rn(D, (double)L);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) D = __dadd_rn(D, __shfl_xor_sync(0xFFFFFFFFu, D, o));
    return D;
}
// The certificate, divided by 2^-48 and evaluated in float (off the double
// pipe): accept T_ff when
//   24 C_k + 56 |v| W + (77 + ldn/4096) T_ff + ldn 2^-98 <= 256 T_ff,
// with C_k, W rounded up, |v| from its float rounding and both sides given a
// 2^-20 relative margin for the float roundings of this test.  A huge,
// infinite or NaN sum is not accepted.
__device__ __forceinline__ bool ff_certified(double Tff, float Ck, float W, float av,
                                             int64_t ldn) {
    const float T = (float)Tff;
    if (!(T < 0x1p100f)) return false;
    const float ln = (float)ldn;
    const float lhs = 24.0f * Ck + 56.0f * av * W + (77.0f + ln * (1.0f / 4096.0f)) * T +
                      ln * 0x1p-98f;
    return lhs * (1.0f + 0x1p-20f) <= 256.0f * T * (1.0f - 0x1p-20f);
}

// Residual of one pair (CS: x_ijhat staged in shared memory); j, k: the
// pair's columns in a (double input reads their float pairs and totals).
template <typename T, bool CS>
__device__ __forceinline__ T pair_residual(const ScanArgs<T> &a, int64_t j, int64_t k,
                                           const T *xk, const T *colb, int n, T v, int lane) {
    if constexpr (sizeof(T) == 4) {
        (void)a, (void)j, (void)k;
        return warp_residual_f4<CS>(xk, colb, n, v, lane);
    } else {
        // one 128-row group: the double sum's 8 double operations per lane
        // cost less than the float-float sum's fixed part (measured: 100 x 100
        // double fits 30% slower in float-float)
        const ColInfo &ck = a.ci[k], &cj = a.ci[j];
        const float v1 = (float)v;
        const float av = fabsf(v1);
        if (a.ldn > ROW_PAD && ((ck.flags | cj.flags) & COL_WIDE) == 0 &&
            (av == 0.0f || (av >= 0x1p-60f && av <= 0x1p60f))) {
            const float v2 = (float)(v - (double)v1);
            const int64_t ldn = a.ldn, lo = a.m * ldn;  // Xlo follows Xf
            const double Tff = residual_ff(a.Xf + k * ldn, a.Xf + lo + k * ldn, a.Xf + j * ldn,
                                           a.Xf + lo + j * ldn, ldn, v1, v2, lane);
            if (ff_certified(Tff, ck.l1_up, cj.l1_up, av, ldn)) return Tff;
        }
        return warp_residual_pad<T>(xk, colb, n, v, lane);
    }
}

// Writes v and s of (lambda t0+tl, jhat, k), or lists the pair for the exact path.
template <typename T, bool CS>
__device__ void emit_pair(const ScanArgs<T> &a, int t, int64_t j, int64_t k, int st,
                          typename Traits<T>::K ts, const T *xk, const T *colb, int n,
                          double lam, int lane) {
    using Tr = Traits<T>;
    const int64_t m = a.m;
    const int64_t o = L1L_CHK(((int64_t)t * m + j) * m + k, (int64_t)a.n_lambda * m * m);
    if (st >= SEL_SLOW) {
        if (lane == 0) {
            uint32_t slot = atomicAdd(a.slow_count, 1u);
            SlowEntry e;
            e.t = t;
            e.j = (int32_t)j;
            e.k = (int32_t)k;
            e.inst = (int16_t)a.inst;
            e.reason = (int16_t)st;
            a.slow[slot] = e;
        }
        return;
    }
    if (st == SEL_INTERNAL) {
        if (lane == 0) {
            atomicOr(a.status, ST_INTERNAL);
            a.v_all[o] = T(NAN);
            a.s_all[o] = NAN;
        }
        return;
    }
    const T v = Tr::value(ts);
    const T res = pair_residual<T, CS>(a, j, k, xk, colb, n, v, lane);
    if (lane == 0) {
        a.v_all[o] = v;
        a.s_all[o] = (double)res + lam * (double)fabs(v);
    }
}

// One lambda of one pair: the full selection.
template <typename T, bool CS>
__device__ void solve_one(const ScanArgs<T> &a, const LamView &lp, int t0, int tl, int64_t j,
                          int64_t k, const T *xk, const float *xf, const WarpCtx<T> &w,
                          bool slow_pair, int lane) {
    using Tr = Traits<T>;
    typename Tr::K ts = Tr::KEY0;
    int st = SEL_OK;
    if (slow_pair) {
        st = SEL_SLOW;
    } else if (w.cinfo.n_valid > 0) {
        st = select_pair<T>(xk, xf, w, lp, tl, ts, lane);
    }
    emit_pair<T, CS>(a, t0 + tl, j, k, st, ts, xk, w.colb, w.n, lp.lam[tl], lane);
}

// Lambda batch (step A7).  The weighted median moves monotonically toward 0
// as lambda grows (the penalty point only gains weight), so every lambda's
// median lies between those of the smallest and the largest lambda.  Solve
// those two fully, collect the rows whose exact keys lie between them (one
// pass, exact divisions only near the bounds) together with the exact weight
// below, and decide every lambda from one sort and prefix scan of those rows.
// Returns false (nothing written) when more than 31 rows lie between.
template <typename T, bool CS>
__device__ bool lambda_path(const ScanArgs<T> &a, const LamView &lp, int t0, int nlc, int64_t j,
                            int64_t k, const T *__restrict__ xk, const float *__restrict__ xf,
                            const WarpCtx<T> &w, int lane) {
    using Tr = Traits<T>;
    using K = typename Tr::K;
    using A = Approx<T>;
    constexpr uint32_t G = A::G;
    const unsigned FULL = 0xFFFFFFFFu;
    const int n = w.n;
    K Ka = Tr::KEY0, Kb = Tr::KEY0;
    if (select_pair<T>(xk, xf, w, lp, lp.tl_min, Ka, lane) != SEL_OK) return false;
    if (select_pair<T>(xk, xf, w, lp, lp.tl_max, Kb, lane) != SEL_OK) return false;
    const K Klo = min(Ka, Kb), Khi = max(Ka, Kb);
    const uint32_t cl = ckey((float)Tr::value(Klo)), ch = ckey((float)Tr::value(Khi));
    const uint32_t bt = sat_sub(cl, G), at = min(sat_add(ch, G), CKMAX);
    int64_t Sb = 0;  // exact weight of rows with key < Klo
    int cnt = 0;
    uint16_t *stage = reinterpret_cast<uint16_t *>(w.hist);
    int c = 0;
    constexpr int U = 4;  // loads of the next batch in flight while this one is classified
    float an[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int i = u * 32 + lane;
        an[u] = i < n ? xf[i] : 0.0f;
    }
    for (int i0 = 0; i0 < n; i0 += 32 * U) {
        float ac[U];
#pragma unroll
        for (int u = 0; u < U; ++u) ac[u] = an[u];
        if (i0 + 32 * U < n) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int i = i0 + 32 * U + u * 32 + lane;
                an[u] = i < n ? xf[i] : 0.0f;
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * 32 + lane;
            bool take = false;
            if (i < n) {
                const float iv = w.inv[i];
                if (!isnan(iv)) {
                    const uint32_t kk = akey(__fmul_rn(ac[u], iv));
                    if (kk < bt) {
                        Sb += w.q(i);
                    } else if (kk <= at) {
                        const K ke = Tr::key(Tr::div_rn(xk[i], w.colb[i]));
                        if (ke < Klo)
                            Sb += w.q(i);
                        else if (ke <= Khi)
                            take = true;
                    }
                }
            }
            const unsigned msk = __ballot_sync(FULL, take);
            if (take) {
                const int pos = c + __popc(msk & ((1u << lane) - 1u));
                if (pos < 31) stage[pos] = (uint16_t)i;
            }
            c += __popc(msk);
            cnt += take ? 1 : 0;
        }
    }
    (void)cnt;
    Sb = warp_sum_i64(Sb);
    __syncwarp();
    if (c > 31) return false;
    K fk = Tr::NONE;
    int64_t fq = 0;
    if (lane < c) {
        const int row = L1L_CHK((int)stage[lane], (n + ROW_PAD - 1) & ~(ROW_PAD - 1));
        fk = Tr::key(Tr::div_rn(xk[row], w.colb[row]));
        fq = w.q(row);
    } else if (lane == c && Klo <= Tr::KEY0 && Tr::KEY0 <= Khi) {
        fk = Tr::KEY0;
    }
    __syncwarp();
    warp_sort32(fk, fq, lane);
    const int64_t P = warp_scan_add(fq, lane);
    const K nxt = __shfl_down_sync(FULL, fk, 1);
    const bool last = (lane == 31) || (nxt != fk);
    K prev = Tr::NONE;
    T prev_res = T(0);
    for (int tl = 0; tl < nlc; ++tl) {
        const Decide dc = decide_for(w, lp, tl);
        int r = -2;
        if (last && fk != Tr::NONE) r = dc.cond(Sb + P, fk >= Tr::KEY0);
        const unsigned okm = __ballot_sync(FULL, r == 1);
        const unsigned unm = __ballot_sync(FULL, r == -1);
        const unsigned any = okm | unm;
        const int first = any ? __ffs(any) - 1 : 0;
        if (!any || ((unm >> first) & 1u)) {  // undecided here: full selection
            solve_one<T, CS>(a, lp, t0, tl, j, k, xk, xf, w, false, lane);
            prev = Tr::NONE;
            continue;
        }
        const K ts = __shfl_sync(FULL, fk, first);
        const T v = Tr::value(ts);
        if (ts != prev) {
            prev_res = pair_residual<T, CS>(a, j, k, xk, w.colb, n, v, lane);
            prev = ts;
        }
        if (lane == 0) {
            const int64_t o = ((int64_t)(t0 + tl) * a.m + j) * a.m + k;
            a.v_all[o] = v;
            a.s_all[o] = (double)prev_res + lp.lam[tl] * (double)fabs(v);
        }
    }
    return true;
}

// One work unit: column jhat = j of an instance and the k in [k0, k1), all
// lambdas of the launch.  Called by every thread of a CTA; `smem` is laid out
// for lay_npad rows (column arrays, then one candidate list per warp).  CS:
// x_ijhat is staged in shared memory; otherwise the warps read it from the
// column copy in global memory (L2-resident), which frees shared memory for
// more resident warps when n is large.
template <typename T, bool MULTI, bool CS>
__device__ void pairs_unit(const ScanArgs<T> &a, const LamView &lp, int t0, int nlc, int j,
                           int64_t k0, int64_t k1, int cap, int lay_npad, unsigned char *smem,
                           Decide *s_dec) {
    using Tr = Traits<T>;
    using K = typename Tr::K;
    const int n = (int)a.n;
    const int64_t m = a.m, ldn = a.ldn;
    const int npad = lay_npad;  // shared-memory layout stride (>= n rounded up to 32)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;

    const T *xj = a.Xt + (int64_t)j * ldn;
    T *colb_s = reinterpret_cast<T *>(smem);
    const T *colb = CS ? colb_s : xj;
    size_t off = CS ? al16((size_t)npad * sizeof(T)) : 0;
    float *inv = reinterpret_cast<float *>(smem + off);
    off += al16((size_t)npad * 4);
    // fast-path weights: 32-bit q32_i
    uint32_t *q32 = reinterpret_cast<uint32_t *>(smem + off);
    off += al16((size_t)npad * 4);
    uint16_t *samp = reinterpret_cast<uint16_t *>(smem + off);
    unsigned char *wbase =
        smem + PairSmem<T>::col_bytes(npad, CS) + (size_t)warp * PairSmem<T>::warp_bytes(cap);
    uint32_t *lk = reinterpret_cast<uint32_t *>(wbase);
    uint16_t *li = reinterpret_cast<uint16_t *>(wbase + al16((size_t)cap * 4));
    uint32_t *hist = reinterpret_cast<uint32_t *>(wbase + al16((size_t)cap * 4) +
                                                  al16((size_t)cap * 2));
    uint2 *lst = reinterpret_cast<uint2 *>(wbase);
    uint32_t *hist32 = reinterpret_cast<uint32_t *>(wbase + al16((size_t)cap * 8));
    // prologue scratch: the first 256 bytes of warp 0's candidate list
    long long *s_wsum = reinterpret_cast<long long *>(smem + PairSmem<T>::col_bytes(npad, CS));

    const ColInfo cinfo = a.ci[j];
    for (int i = threadIdx.x; i < npad; i += blockDim.x) {
        const T b = i < n ? xj[i] : T(0);
        if (CS) colb_s[i] = b;
        // rows with x_ijhat = 0 (and padding rows) get a NaN reciprocal: their
        // approximate key is the NaN key CKNONE, above every bracket (bounds
        // stop at CKMAX), so the level-0 pass needs no validity test.  Their
        // weight is 0, so even a NaN of the other sign (a key near 0) could
        // only add zero-weight candidates, which never decide the median.
        inv[i] = b != T(0) ? Approx<T>::inv_of(b) : __int_as_float(0x7FFFFFFF);
        int e = 0;
        const int64_t qi = b != T(0) ? fixq(b < T(0) ? -b : b, cinfo.sigma, e) : 0;
        q32[i] = (uint32_t)((uint64_t)qi >> cinfo.shift32);
    }
    for (int q = threadIdx.x; q < NSAMP; q += blockDim.x) samp[q] = 0;  // always a valid row
    __syncthreads();
    // Systematic weight-proportional sample of the rows of column jhat: sample
    // s is the row whose cumulative weight interval contains (s + 1/2) Q / 64.
    if (cinfo.n_valid > 0) {
        const int nt = blockDim.x;
        const int chunk = (n + nt - 1) / nt;
        const int r0 = min(n, threadIdx.x * chunk), r1 = min(n, r0 + chunk);
        auto wq = [&](int r) -> long long { return (long long)q32[r]; };
        long long mine = 0;
        for (int r = r0; r < r1; ++r) mine += wq(r);
        long long incl = warp_scan_add(mine, lane);
        if (lane == 31) s_wsum[warp] = incl;
        __syncthreads();
        long long before = incl - mine;
        for (int w = 0; w < warp; ++w) before += s_wsum[w];
        const double per = (double)NSAMP / (double)cinfo.Q32;
        for (int r = r0; r < r1; ++r) {
            const long long after = before + wq(r);
            const double x0 = (double)before * per - 0.5, x1 = (double)after * per - 0.5;
            int s0 = (int)floor(x0) + 1, s1 = (int)floor(x1);
            s0 = max(s0, 0);
            s1 = min(s1, NSAMP - 1);
            for (int sidx = s0; sidx <= s1; ++sidx) samp[L1L_CHK(sidx, NSAMP)] = (uint16_t)r;
            before = after;
        }
        __syncthreads();
    }
    // per-lambda thresholds of the exact test depend on (jhat, lambda) only
    for (int tl = threadIdx.x; tl < min(nlc, NDEC); tl += blockDim.x)
        decide_init<T>(s_dec[tl], cinfo, lp.lam[tl]);
#if L1L_DYNAMIC_K
    __shared__ int s_knext;  // next k of this unit (offset from k0)
    if (threadIdx.x == 0) s_knext = 0;
#endif
    __syncthreads();
    WarpCtx<T> wc;
    wc.colb = colb;
    wc.inv = inv;
    wc.q32 = q32;
    wc.samp = samp;
    wc.lk = lk;
    wc.li = li;
    wc.hist = hist;
    wc.lst = lst;
    wc.hist32 = hist32;
    wc.s_dec = s_dec;
    wc.qt = cap / 32;
    wc.d0 = a.d0;
    wc.n = n;
    wc.cinfo = cinfo;

    const bool jwide = (cinfo.flags & COL_WIDE) != 0;
#if L1L_DYNAMIC_K
    // a warp takes the next k when it is done with its pair: pairs cost
    // different times (bracket misses, overflows), and a fixed share per warp
    // leaves the CTA waiting for its slowest warp
    (void)nw;
    for (;;) {
        int idx = 0;
        if (lane == 0) idx = atomicAdd(&s_knext, 1);
        const int64_t k = k0 + __shfl_sync(0xFFFFFFFFu, idx, 0);
        if (k >= k1) break;
#else
    for (int64_t k = k0 + warp; k < k1; k += nw) {
#endif
        if (k == j) {  // v_jhat = 1: zero residual, penalty lambda * 1
            for (int tl = lane; tl < nlc; tl += 32) {
                int64_t o = L1L_CHK(((int64_t)(t0 + tl) * m + j) * m + k,
                                    (int64_t)a.n_lambda * m * m);
                a.v_all[o] = T(1);
                a.s_all[o] = lp.lam[tl];
            }
            continue;
        }
        const T *xk = a.Xt + k * ldn;
        const float *xf = a.Xf + k * ldn;
        const bool slow_pair = a.force_exact || jwide ||
                               (sizeof(T) == 8 && (a.ci[k].flags & COL_WIDE));
        if (MULTI && nlc >= 3 && !slow_pair && cinfo.n_valid > 0 &&
            lambda_path<T, CS>(a, lp, t0, nlc, j, k, xk, xf, wc, lane)) {
            __syncwarp();
            continue;
        }
        for (int tl = 0; tl < nlc; ++tl)
            solve_one<T, CS>(a, lp, t0, tl, j, k, xk, xf, wc, slow_pair, lane);
        __syncwarp();
    }
    __syncthreads();  // the CTA may stage another column next
}

}  // namespace l1l
