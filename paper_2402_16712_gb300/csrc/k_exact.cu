// k_exact.cu -- exact slow path of step A3 for the pairs the fixed-point fast
// path could not settle (a column with weights too small for its scale, tied
// within the truncation band) or for every pair under L1L_FLAG_FORCE_EXACT.
//
// One warp per pair.  The median key is found by bisection over the key
// space: at each probe t the weight of rows with key <= t is summed EXACTLY in
// a wide fixed-point integer whose unit is 2^-1074 (every finite double, and
// so every float, is an integer multiple of it), reduced across the warp limb
// by limb, and compared with the exact total W = sum w + lambda.
#include <algorithm>

#include "common.cuh"
#include "exact.cuh"
#include "launch.h"

namespace l1l {

template <typename T>
__global__ void __launch_bounds__(128) k_exact(ScanArgs<T> a, const __grid_constant__ LambdaPack lp,
                                               int t0) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t count = *(volatile uint32_t *)a.slow_count;
    uint32_t acc[WL];
    uint32_t S[WL], W[WL];  // used by lane 0
    for (uint32_t e = gw; e < count; e += nwarps) {
        const SlowEntry en = a.slow[e];
        exact_entry<T>(a, en, lp.lam[en.t - t0], acc, S, W, lane);
    }
}

template <typename T>
cudaError_t launch_exact(const ScanArgs<T> &a, const double *lambdas, int t0, int nlc,
                         int num_sms, cudaStream_t st, int &launches) {
    LambdaPack lp;
    lp.tl_min = lp.tl_max = 0;
    for (int q = 0; q < nlc; ++q) lp.lam[q] = lambdas[t0 + q];
    k_exact<T><<<num_sms * 2, 128, 0, st>>>(a, lp, t0);
    launches++;
    return cudaGetLastError();
}

template cudaError_t launch_exact<float>(const ScanArgs<float> &, const double *, int, int, int,
                                         cudaStream_t, int &);
template cudaError_t launch_exact<double>(const ScanArgs<double> &, const double *, int, int, int,
                                          cudaStream_t, int &);

L1L_CHECKS_READER(l1l_checks_exact)

}  // namespace l1l
