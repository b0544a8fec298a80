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

}  // namespace l1l
