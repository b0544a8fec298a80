// checks.cuh -- bounds checks of the bounds-checked build (L1L_CHECKS=1).
//
// L1L_CHK(i, n) is the index i of an array of n elements.  In the normal
// build it is i itself.  In the checked build an index outside [0, n) is
// counted in this translation unit's device counters (hits, and the source
// line of the last one) and replaced by 0, so the access stays inside the
// array and the kernel runs on with its control flow unchanged: no trap, no
// early return (a lane leaving warp-synchronous code early would leave the
// others waiting at their next shuffle).  l1line_check_hits reads and clears
// the counters of every translation unit.
#pragma once
#include <cstdint>

#ifndef L1L_CHECKS
#define L1L_CHECKS 0
#endif

namespace l1l {

#if L1L_CHECKS
namespace {
__device__ unsigned long long g_check_hits;
__device__ int g_check_line;
}  // namespace

template <typename I, typename N>
__device__ __forceinline__ I check_index(I i, N n, int line) {
    if ((unsigned long long)(long long)i >= (unsigned long long)(long long)n) {
        atomicAdd(&g_check_hits, 1ull);
        atomicExch(&g_check_line, line);
        return I(0);
    }
    return i;
}
#define L1L_CHK(i, n) (::l1l::check_index((i), (n), __LINE__))
// Host side: reads (and when `reset`, clears) this translation unit's counters.
#define L1L_CHECKS_READER(name)                                                              \
    extern "C" long long name(int reset, int *line) {                                       \
        unsigned long long h = 0;                                                            \
        int ln = 0;                                                                          \
        if (cudaMemcpyFromSymbol(&h, ::l1l::g_check_hits, sizeof(h)) != cudaSuccess ||       \
            cudaMemcpyFromSymbol(&ln, ::l1l::g_check_line, sizeof(ln)) != cudaSuccess)       \
            return -1;                                                                       \
        if (reset) {                                                                         \
            const unsigned long long z = 0;                                                  \
            const int zl = 0;                                                                \
            cudaMemcpyToSymbol(::l1l::g_check_hits, &z, sizeof(z));                          \
            cudaMemcpyToSymbol(::l1l::g_check_line, &zl, sizeof(zl));                        \
        }                                                                                    \
        if (line && h) *line = ln;                                                           \
        return (long long)h;                                                                 \
    }
#else
#define L1L_CHK(i, n) (i)
#define L1L_CHECKS_READER(name)
#endif

}  // namespace l1l
