// batch.cuh -- device helpers of the batched fit shared by its kernels
// (k_batch.cu) and the persistent pair kernel of each launch shape
// (k_pairs_shape.cu).
#pragma once
#include "common.cuh"

namespace l1l {

// Largest b with begin[b] <= x (begin is a non-decreasing prefix, begin[0] = 0).
template <typename I>
__device__ __forceinline__ int find_inst(const I *begin, int count, I x) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (begin[mid] <= x)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

template <typename T>
__device__ __forceinline__ ScanArgs<T> inst_args(const BatchDesc<T> &bd, int b,
                                                 unsigned char *ws) {
    const BatchInst<T> &in = bd.inst[b];
    const InstLayout L = inst_layout(in.m, in.ldn, in.nl, sizeof(T));
    unsigned char *base = ws + in.ws_off;
    ScanArgs<T> a;
    a.Xt = reinterpret_cast<const T *>(base + L.Xt);
    a.Xf = reinterpret_cast<const float *>(base + L.Xf);
    a.ci = reinterpret_cast<const ColInfo *>(base + L.ci);
    a.n = in.n;
    a.m = in.m;
    a.ldn = in.ldn;
    a.n_lambda = in.nl;
    a.v_all = reinterpret_cast<T *>(base + L.v_all);
    a.s_all = reinterpret_cast<double *>(base + L.s_all);
    a.status = reinterpret_cast<uint32_t *>(ws);
    a.slow_count = reinterpret_cast<uint32_t *>(ws + 256);
    a.slow = reinterpret_cast<SlowEntry *>(ws + BATCH_HEAD);
    a.force_exact = bd.force_exact;
    a.inst = b;
    a.jlist = nullptr;
    a.nj = a.m;
    a.d0 = bd.d0;
    return a;
}

}  // namespace l1l
