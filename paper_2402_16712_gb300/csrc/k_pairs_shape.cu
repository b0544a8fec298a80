// k_pairs_shape.cu -- the pair kernels (steps A2-A4; the per-pair algorithm
// is in pairs.cuh) for ONE launch shape, chosen at compile time:
//   -DL1L_SHAPE=0  SHAPE_R80:  <= 8 warps per CTA, up to 3 CTAs per SM (80 registers)
//   -DL1L_SHAPE=1  SHAPE_R64:  <= 16 warps per CTA, up to 32 warps per SM (64 registers)
//   -DL1L_SHAPE=2  SHAPE_R128: <= 16 warps per SM (128 registers, no spills)
// and -DL1L_PERSIST=0 (the single-instance kernel, grid over jhat x k-chunks)
// or 1 (the batched persistent kernel).  The build compiles this file once
// per (shape, kind), so the instantiations compile in parallel.
#ifndef L1L_SHAPE
#error "compile with -DL1L_SHAPE=0|1|2"
#endif
// Loop unrolling of the 32-bit selection per shape (select32.cuh); measured
// on the planner's launches, kernel time: 2000 x 2000 (64 registers)
// level-0 loop unrolled by two 14.18 -> 13.51 ms, 1000 x 500 0.70 -> 0.67 ms;
// 5000 x 1000 (128 registers) level-0 unroll 11.00 -> 11.46 ms (kept at one),
// list loops unrolled by two 11.00 -> 10.88 ms.
#if L1L_SHAPE == 2
#ifndef L1L_L0_UNROLL
#define L1L_L0_UNROLL 1
#endif
#ifndef L1L_LIST_UNROLL
#define L1L_LIST_UNROLL 2
#endif
#else
#ifndef L1L_L0_UNROLL
#define L1L_L0_UNROLL 2
#endif
#ifndef L1L_LIST_UNROLL
#define L1L_LIST_UNROLL 1
#endif
#endif
// Lane balancing of the candidate lists (list32_balance), measured on the
// 2000 x 2000 float fit, kernel time: 8 x 3 warps (80 registers) 14.36 ->
// 13.86 ms, 16 x 2 warps (64 registers) 13.11 -> 13.61 ms, 16 x 1 warps (128
// registers) 16.82 -> 16.80 ms; so only the 80-register shape balances.
#ifndef L1L_BALANCE
#define L1L_BALANCE (L1L_SHAPE == 0)
#endif

#include <algorithm>

#include "batch.cuh"
#include "checks.cuh"
#include "common.cuh"
#include "launch.h"
#include "pairs.cuh"

#ifndef L1L_PERSIST
#error "compile with -DL1L_PERSIST=0|1"
#endif

namespace l1l {

// Threads per CTA and CTAs per SM the compiler budgets registers for.
template <int SH> struct ShapeBounds;
template <> struct ShapeBounds<SHAPE_R80> { static constexpr int threads = 256, blocks = 3; };
template <> struct ShapeBounds<SHAPE_R64> { static constexpr int threads = 512, blocks = 2; };
template <> struct ShapeBounds<SHAPE_R128> { static constexpr int threads = 512, blocks = 1; };

constexpr int SH = L1L_SHAPE;

#if L1L_PERSIST == 0

template <typename T, bool MULTI, bool CS, int S>
__global__ void __launch_bounds__(ShapeBounds<S>::threads, ShapeBounds<S>::blocks)
    k_pairs(ScanArgs<T> a, const __grid_constant__ LambdaPack lp, int t0, int nlc, int kchunk,
            int cap) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ Decide s_dec[NDEC];
    const int64_t k0 = (int64_t)blockIdx.y * kchunk;
    const int64_t k1 = min(a.m, k0 + kchunk);
    const LamView lv{lp.lam, lp.tl_min, lp.tl_max};
    const int64_t j = a.jlist ? (int64_t)a.jlist[blockIdx.x] : (int64_t)blockIdx.x;
    if (j < 0 || j >= a.m) {  // uniform over the CTA
        if (threadIdx.x == 0) atomicOr(a.status, ST_BADINDEX);
        return;
    }
    pairs_unit<T, MULTI, CS>(a, lv, t0, nlc, (int)j, k0, k1, cap,
                             ((int)a.n + ROW_PAD - 1) & ~(ROW_PAD - 1), smem, s_dec);
}

template <typename T, int S>
cudaError_t launch_pairs_sh(const ScanArgs<T> &a, const LambdaPack &lp, int t0, int nlc,
                            const PairPlan &plan, cudaStream_t st) {
    // separate instantiations keep the single-lambda kernel small
    auto kern = nlc >= 3 ? (plan.cs ? k_pairs<T, true, true, S> : k_pairs<T, true, false, S>)
                         : (plan.cs ? k_pairs<T, false, true, S> : k_pairs<T, false, false, S>);
    if (plan.warps * 32 > ShapeBounds<S>::threads) return cudaErrorInvalidConfiguration;
    cudaError_t e = ensure_smem(reinterpret_cast<const void *>(kern), plan.smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)a.nj, (unsigned)plan.kchunks);
    kern<<<grid, plan.warps * 32, plan.smem, st>>>(a, lp, t0, nlc, plan.kchunk, plan.cap);
    return cudaGetLastError();
}

template cudaError_t launch_pairs_sh<float, SH>(const ScanArgs<float> &, const LambdaPack &, int,
                                                int, const PairPlan &, cudaStream_t);
template cudaError_t launch_pairs_sh<double, SH>(const ScanArgs<double> &, const LambdaPack &,
                                                 int, int, const PairPlan &, cudaStream_t);

#else

// Persistent: every CTA loops, taking the next (instance, jhat) unit of units
// [u0, u1) (one size class of the batch) from that class's counter; units are
// numbered largest instance first.  No CTA waits on another.
template <typename T, bool MULTI, bool CS, int S>
__global__ void __launch_bounds__(ShapeBounds<S>::threads, ShapeBounds<S>::blocks)
    k_pairs_persist(const __grid_constant__ BatchDesc<T> bd, unsigned char *ws, int64_t u0,
                    int64_t u1, int slot, int lay_npad, int cap) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ Decide s_dec[NDEC];
    __shared__ long long s_unit;
    unsigned long long *counter = reinterpret_cast<unsigned long long *>(ws + 512) + slot;
    for (;;) {
        if (threadIdx.x == 0) s_unit = (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        const int64_t u = u0 + s_unit;
        __syncthreads();
        if (u >= u1) break;
        const int b = find_inst<int64_t>(bd.unit_begin, bd.count, u);
        const BatchInst<T> &in = bd.inst[b];
        const ScanArgs<T> a = inst_args<T>(bd, b, ws);
        const LamView lv{bd.lam + bd.lam_begin[b], in.tl_min, in.tl_max};
        pairs_unit<T, MULTI, CS>(a, lv, 0, in.nl, (int)(u - bd.unit_begin[b]), 0, in.m, cap,
                                 lay_npad, smem, s_dec);
    }
}

template <typename T, int S>
cudaError_t launch_persist_sh(const BatchDesc<T> &bd, unsigned char *ws, const BatchClass &bc,
                              int slot, bool multi, int num_sms, cudaStream_t st) {
    auto kern = multi ? (bc.plan.cs ? k_pairs_persist<T, true, true, S>
                                    : k_pairs_persist<T, true, false, S>)
                      : (bc.plan.cs ? k_pairs_persist<T, false, true, S>
                                    : k_pairs_persist<T, false, false, S>);
    if (bc.plan.warps * 32 > ShapeBounds<S>::threads) return cudaErrorInvalidConfiguration;
    cudaError_t e = ensure_smem(reinterpret_cast<const void *>(kern), bc.plan.smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = blocks_per_sm(reinterpret_cast<const void *>(kern), bc.plan.warps * 32, bc.plan.smem,
                      &per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int64_t grid = std::min<int64_t>((int64_t)num_sms * per_sm, bc.u1 - bc.u0);
    kern<<<(unsigned)grid, bc.plan.warps * 32, bc.plan.smem, st>>>(bd, ws, bc.u0, bc.u1, slot,
                                                                   bc.lay_npad, bc.plan.cap);
    return cudaGetLastError();
}

template cudaError_t launch_persist_sh<float, SH>(const BatchDesc<float> &, unsigned char *,
                                                  const BatchClass &, int, bool, int,
                                                  cudaStream_t);
template cudaError_t launch_persist_sh<double, SH>(const BatchDesc<double> &, unsigned char *,
                                                   const BatchClass &, int, bool, int,
                                                   cudaStream_t);

#endif

#define L1L_READER_NAME2(s, p) l1l_checks_shape_##s##_##p
#define L1L_READER_NAME(s, p) L1L_READER_NAME2(s, p)
L1L_CHECKS_READER(L1L_READER_NAME(L1L_SHAPE, L1L_PERSIST))

}  // namespace l1l
