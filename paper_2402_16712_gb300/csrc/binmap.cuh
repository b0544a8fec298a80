// binmap.cuh -- the bins of the exact histogram over a level-0 bracket of
// coarse keys (host and device code, so that a host test can check the
// layout).
#pragma once
#include <cstdint>

#ifndef __CUDACC__
#define __host__
#define __device__
#define __forceinline__ inline
#endif

namespace l1l {

constexpr uint32_t CK0 = 0x80000000u;  // coarse key of 0

// Bit length of x (0 for 0).
__host__ __device__ __forceinline__ int bitlen32(uint32_t x) {
#ifdef __CUDA_ARCH__
    return 32 - __clz((int)x);
#else
    return x ? 32 - __builtin_clz(x) : 0;
#endif
}

// Bins of the level-0 bracket [p1, p2].  Uniform: equal key ranges.  A
// bracket that crosses 0 spans every binade of tiny magnitudes on both sides,
// where few ratios lie (key space is logarithmic near 0), so equal key ranges
// would crowd its candidates into the one or two bins of the largest
// magnitudes.  Crossing layout instead: on each side, equal bins over the
// 7.75 binades of largest magnitude (the wing, up to 31 bins of a quarter
// binade or less), the innermost of them widened to reach key 0:
//   negative side [p1, CK0): bins 0 .. n0-1, bin b = p1 + [b, b+1) << sh0,
//                            the last one ends at CK0 - 1;
//   positive side [CK0, p2]: bins n0 .. n0+n1-1, bin n0 + j = s1 + [j, j+1) << sh1,
//                            the first one starts at CK0 (the penalty point's key).
// Bin indices are computed without branches on the key (no divergence).
struct BinMap {
    uint32_t p1, p2, s1;
    int sh0, sh1, n0, n1;
    bool cross;

    // fewest shift with at most maxbins bins over len keys
    static __host__ __device__ __forceinline__ int shift_for(uint32_t len, int maxbins) {
        int s = 0;
        while (((len - 1u) >> s) >= (uint32_t)maxbins) ++s;
        return s;
    }
    __host__ __device__ void init(uint32_t P1, uint32_t P2, int xb) {
        p1 = P1;
        p2 = P2;
        constexpr uint32_t WING = 31u << 21;  // 7.75 binades of keys
        cross = P1 < CK0 && CK0 <= P2 && (P2 - P1) > 2u * WING;
        if (!cross) {
            const uint32_t span = P2 - P1;
            sh0 = span >= (uint32_t)xb ? bitlen32(span) - 6 : 0;
            n0 = (int)(span >> sh0) + 1;
            n1 = 0;
            sh1 = 0;
            s1 = P2;
            return;
        }
        const int wb = xb / 2;  // bins per side
        // negative side: the wing starts at p1; its last bin reaches CK0 - 1
        const uint32_t len0 = (CK0 - P1) < WING ? CK0 - P1 : WING;
        sh0 = shift_for(len0, wb);
        n0 = (int)((len0 - 1u) >> sh0) + 1;
        // positive side: the wing ends at p2; its first bin starts at CK0
        const uint32_t len1 = (P2 - CK0 + 1u) < WING ? P2 - CK0 + 1u : WING;
        sh1 = shift_for(len1, wb);
        n1 = (int)((len1 - 1u) >> sh1) + 1;
        s1 = P2 - ((uint32_t)n1 << sh1) + 1u;  // bins n0 + j start at s1 + j << sh1 (j >= 1)
    }
    __host__ __device__ __forceinline__ int nbins() const { return n0 + n1; }
    // kk in [p1, p2]
    __host__ __device__ __forceinline__ int bin(uint32_t kk) const {
        if (!cross) return (int)((kk - p1) >> sh0);
        const int bn = (int)((kk - p1) >> sh0);
        const int bneg = bn < n0 - 1 ? bn : n0 - 1;
        const uint32_t kp = kk > s1 ? kk : s1;
        const int bp = (int)((kp - s1) >> sh1);
        const int bpos = n0 + (bp < n1 - 1 ? bp : n1 - 1);
        return kk < CK0 ? bneg : bpos;
    }
    __host__ __device__ __forceinline__ uint32_t lower(int b) const {
        if (!cross) return p1 + ((uint32_t)b << sh0);
        if (b < n0) return p1 + ((uint32_t)b << sh0);
        if (b == n0) return CK0;
        return s1 + ((uint32_t)(b - n0) << sh1);
    }
    __host__ __device__ __forceinline__ uint32_t upper(int b) const {
        if (!cross || b < n0 - 1 || b >= n0) {
            const uint64_t v = b < n0 ? (uint64_t)p1 + ((uint64_t)(b + 1) << sh0) - 1u
                                      : (uint64_t)s1 + ((uint64_t)(b - n0 + 1) << sh1) - 1u;
            return v > p2 ? p2 : (uint32_t)v;
        }
        return CK0 - 1u;  // the last negative bin
    }
};

// Bins of the 32-bit selection's bracket histogram: the same two layouts, with
// every inner bin edge on a multiple of 2^sh of the key (offset from p1 in the
// uniform layout), so that "the keys G below and above a key fall in one bin"
// is one shift-compare (same()).
//   uniform [p1, p2]: bin b = keys p1 + [b, b+1) << sh, at most 64 bins;
//   crossing (p1 < key 0 <= p2, wider than two wings): quarter-binade bins
//   (2^21 keys, aligned) on each side, the 32 of the negative side from
//   p1 up, the 32 of the positive side down to p2; the innermost bin of each
//   side also takes every smaller magnitude, up to key 0 (negative side) or
//   from key 0 (positive side).  Inner multiples of 2^21 within those two
//   catch-all bins are not edges; same() treats them as edges (a key next to
//   one is divided exactly although it need not be).
struct BinMapA {
    uint32_t p1, p2, base;
    int sh, tp1, tp2, nneg, npos;
    bool cross;
    static constexpr int QSH = 21;  // quarter binade of the key
    __host__ __device__ void init(uint32_t P1, uint32_t P2) {
        p1 = P1;
        p2 = P2;
        constexpr uint32_t WING = 31u << 21;
        cross = P1 < CK0 && CK0 <= P2 && (P2 - P1) > 2u * WING;
        if (!cross) {
            const uint32_t span = P2 - P1;
            sh = span >= 64u ? bitlen32(span) - 6 : 0;
            base = P1;
            nneg = (int)(span >> sh) + 1;
            npos = 0;
            tp1 = tp2 = 0;
            return;
        }
        sh = QSH;
        base = 0;
        tp1 = (int)(P1 >> QSH);
        tp2 = (int)(P2 >> QSH);
        const int t0 = (int)(CK0 >> QSH);
        nneg = (t0 - tp1) < 32 ? t0 - tp1 : 32;
        npos = (tp2 - t0 + 1) < 32 ? tp2 - t0 + 1 : 32;
    }
    __host__ __device__ __forceinline__ int nbins() const { return nneg + npos; }
    // kk in [p1, p2]
    __host__ __device__ __forceinline__ int bin(uint32_t kk) const {
        if (!cross) return (int)((kk - base) >> sh);
        const int t = (int)(kk >> QSH);
        const int dn = t - tp1, dp = tp2 - t;
        const int bneg = dn < nneg - 1 ? dn : nneg - 1;
        const int bpos = nneg + npos - 1 - (dp < npos - 1 ? dp : npos - 1);
        return kk < CK0 ? bneg : bpos;
    }
    // kk - G and kk + G in [p1, p2]: true when both lie in kk's bin (keys
    // next to an inner multiple of 2^21 of a catch-all bin count as not)
    __host__ __device__ __forceinline__ bool same(uint32_t kk, uint32_t G) const {
        return ((kk - G - base) >> sh) == ((kk + G - base) >> sh);
    }
    __host__ __device__ __forceinline__ uint32_t lower(int b) const {
        if (!cross) return p1 + ((uint32_t)b << sh);
        if (b < nneg) return b == 0 ? p1 : (uint32_t)(tp1 + b) << QSH;
        const int bp = b - nneg;
        if (bp == 0) return CK0;
        return (uint32_t)(tp2 - (npos - 1 - bp)) << QSH;
    }
    __host__ __device__ __forceinline__ uint32_t upper(int b) const {
        if (!cross) {
            const uint64_t v = (uint64_t)p1 + ((uint64_t)(b + 1) << sh) - 1u;
            return v > p2 ? p2 : (uint32_t)v;
        }
        if (b < nneg) return b == nneg - 1 ? CK0 - 1u : ((uint32_t)(tp1 + b + 1) << QSH) - 1u;
        const int bp = b - nneg;
        if (bp == npos - 1) return p2;
        return (uint32_t)(((uint64_t)(tp2 - (npos - 1 - bp)) + 1u) << QSH) - 1u;
    }
};

}  // namespace l1l
