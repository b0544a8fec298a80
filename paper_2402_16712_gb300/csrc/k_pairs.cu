// k_pairs.cu -- the shared-memory planner of the pair kernels and the launch
// of the single-instance kernel in the planned shape (the kernels themselves
// are in k_pairs_shape.cu, the per-pair algorithm in pairs.cuh).
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "launch.h"
#include "pairs.cuh"

namespace l1l {

namespace {
struct AttrEntry {
    const void *fn;
    int dev;
    size_t smem;
    int threads;
    int value;
};
std::mutex g_attr_mu;
std::vector<AttrEntry> g_smem_set, g_occ;
}  // namespace

cudaError_t ensure_smem(const void *fn, size_t bytes) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_attr_mu);
    for (auto &x : g_smem_set)
        if (x.fn == fn && x.dev == dev) {
            if (bytes <= x.smem) return cudaSuccess;
            e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
            if (e == cudaSuccess) x.smem = bytes;
            return e;
        }
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) g_smem_set.push_back({fn, dev, bytes, 0, 0});
    return e;
}

cudaError_t blocks_per_sm(const void *fn, int threads, size_t smem, int *out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_attr_mu);
    for (auto &x : g_occ)
        if (x.fn == fn && x.dev == dev && x.smem == smem && x.threads == threads) {
            *out = x.value;
            return cudaSuccess;
        }
    int v = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, fn, threads, smem);
    if (e != cudaSuccess) return e;
    g_occ.push_back({fn, dev, smem, threads, v});
    *out = v;
    return cudaSuccess;
}

// Candidate slots per warp (a multiple of 32: 32 lanes x quota).  About 40% of
// the rows, at least 512 (small n: every row fits).
template <typename T> static int cap_for(int64_t npad) {
    int64_t c = std::max<int64_t>(512, (npad * 2 / 5 + 31) & ~int64_t(31));
    return (int)(std::min<int64_t>(npad, c) & ~int64_t(31));
}

template <typename T> int64_t max_rows_pairs() {
    const size_t budget = 227 * 1024;
    int64_t n = ROW_PAD;
    while (n + ROW_PAD <= (int64_t)ROW_MASK + 1 &&
           PairSmem<T>::col_bytes(n + ROW_PAD, false) +
                   PairSmem<T>::warp_bytes(cap_for<T>(n + ROW_PAD)) <=
               budget)
        n += ROW_PAD;
    return n;
}

// 17-24 resident warps only in CTAs of up to 8 warps (80 registers): larger
// CTAs there would take the 64-register budget, whose spills cost more than
// the extra warps gain (3500 x 1000 float: 11 x 2 warps at 64 registers
// 8.1 ms, 16 x 1 at 128 registers 7.3 ms).
int pair_shape(int warps, int ctas) {
    if (warps < 1 || warps > 16 || ctas < 1 || ctas > 3) return -1;
    const int t = warps * ctas;
    if (t <= 16) return SHAPE_R128;
    if (t <= 24) return warps <= 8 ? SHAPE_R80 : -1;
    if (t <= 32) return SHAPE_R64;
    return -1;
}

// The resident-warp plan for one placement of x_ijhat (cs: shared memory).
template <typename T>
static PairPlan plan_placement(int64_t npad, bool cs, int d0, const Tune &tune) {
    PairPlan p{0, 0, 0, 0, 0, 0, 0, 0, 0};
    const size_t cb = PairSmem<T>::col_bytes(npad, cs);
    // Per-lane candidate quota wanted: the level-0 bracket (+-d0 of 64 weight
    // samples) holds ~2.5% of the rows per sample position, i.e. mu = 0.025 d0
    // n/32 per lane; ask for mu + 3.5 sqrt(mu) + 1 so that the busiest of 32
    // lanes rarely overflows (an overflow costs one more pass).
    const double mu = 0.025 * (double)d0 * (double)npad / 32.0;
    const int64_t qt_need = std::min<int64_t>(npad / 32, (int64_t)ceil(mu + 3.5 * sqrt(mu) + 1.0));
    // Over 1-3 CTAs per SM and 1-16 warps per CTA (or the caller's choice),
    // up to 32 resident warps in one of the launch shapes (pair_shape), keep
    // the plan with the most resident warps whose lists meet the quota in
    // 228 KB of shared memory (1 KB reserved per CTA, static arrays included);
    // on a tie the fewer, larger CTAs (column jhat staged fewer times, so
    // longer lists per warp).  Measured, 2000 x 2000 float: 16 x 2 warps
    // (64 registers) 14.1 ms, 8 x 3 (80 registers) 14.4 ms; 5000 x 1000:
    // 16 x 1 (128 registers, x_ijhat in shared memory) 11.0 ms, 8 x 2 with
    // x_ijhat in global memory 13.6 ms.
    int w = 0, cap = 0, best = 0, nc = 0;
    const int c_hi = tune.ctas > 0 ? tune.ctas : 3, c_lo = tune.ctas > 0 ? tune.ctas : 1;
    const int w_hi = tune.warps > 0 ? tune.warps : 16, w_lo = tune.warps > 0 ? tune.warps : 1;
    for (int ctas = c_lo; ctas <= c_hi; ++ctas) {
        const int64_t per_cta = 233472 / ctas - 1024 - 1024;
        for (int cand = w_hi; cand >= w_lo; --cand) {
            if (ctas * cand <= best || pair_shape(cand, ctas) < 0) continue;
            const int64_t fit = PairSmem<T>::cap_fit((per_cta - (int64_t)cb) / cand);
            const int64_t c32 = std::min<int64_t>(npad, fit) & ~int64_t(31);
            if (fit > 0 && c32 >= 32 * qt_need) {
                w = cand;
                cap = (int)c32;
                best = ctas * cand;
                nc = ctas;
            }
        }
    }
    if (w == 0) return p;
    p.warps = w;
    p.cap = cap;
    p.ctas = nc;
    p.d0 = d0;
    p.cs = cs ? 1 : 0;
    p.shape = pair_shape(w, nc);
    p.smem = cb + (size_t)w * PairSmem<T>::warp_bytes(cap);
    return p;
}

template <typename T>
static PairPlan plan_pairs_for(int64_t n, int64_t m, int num_sms, int64_t nj, const Tune &tune) {
    PairPlan p{0, 0, 0, 0, 0, 0, 0, 0, 0};
    const int64_t npad = (n + ROW_PAD - 1) & ~int64_t(ROW_PAD - 1);
    if (n > max_rows_pairs<T>()) return p;
    const int d0 = tune.d0 > 0 ? tune.d0 : D0_DEFAULT;
    // Where x_ijhat lives.  Shared memory saves the residual pass an L2 read
    // per row; global memory frees n * sizeof(T) bytes per CTA.  Measured:
    // float keeps it in shared memory whenever that plan holds at least 16
    // resident warps or as many as the global one (2000 x 2000: equal plans,
    // shared 2-4% faster; 3500 x 1000: 16 warps in shared memory 7.3 ms, 21
    // with x_ijhat in global memory 7.7 ms); double reads it from global
    // memory (2000 x 2000: 5% faster at equal plans).
    const PairPlan ps = tune.column == 2 ? p : plan_placement<T>(npad, true, d0, tune);
    const PairPlan pg = tune.column == 1 ? p : plan_placement<T>(npad, false, d0, tune);
    const int rs = ps.warps * ps.ctas, rg = pg.warps * pg.ctas;
    if (rs == 0 && rg == 0) return p;
    if (rg == 0)
        p = ps;
    else if (rs == 0)
        p = pg;
    else
        p = (sizeof(T) == 8 || (rg > rs && rs < 16)) ? pg : ps;
    const int w = p.warps, nc = p.ctas;
    int64_t chunks;
    if (tune.kchunk > 0) {
        chunks = (m + std::min<int64_t>(m, tune.kchunk) - 1) / std::min<int64_t>(m, tune.kchunk);
    } else {
        // At least four CTAs per SM over the nj x chunks grid; then the fewest
        // chunks (1-4) whose last wave of resident CTAs is nearly full, so that
        // staging column jhat is amortised over many k without a long tail.
        const int64_t slots = (int64_t)num_sms * nc;
        const int64_t cmax = std::max<int64_t>(1, (m + w - 1) / w);
        chunks = std::max<int64_t>(1, std::min<int64_t>(cmax, (num_sms * 4 + nj - 1) / nj));
        if (chunks == 1) {
            double best_loss = 1e30;
            for (int64_t c = 1; c <= std::min<int64_t>(4, cmax); ++c) {
                const double waves = (double)(nj * c) / (double)slots;
                const double loss = std::ceil(waves) / waves;
                if (loss < best_loss - 0.02) {
                    best_loss = loss;
                    chunks = c;
                }
                if (loss <= 1.05) break;
            }
        }
    }
    p.kchunk = (int)((m + chunks - 1) / chunks);
    p.kchunks = (int)((m + p.kchunk - 1) / p.kchunk);
    return p;
}

template <typename T>
PairPlan plan_pairs(int64_t n, int64_t m, int num_sms, int64_t nj, const Tune &tune, bool single) {
    // A single-instance call whose pairs fit in one wave at 16 warps per SM
    // is bound by the latency of one pair, not by throughput: 8-16 warps per
    // CTA (fewer CTAs stage column jhat fewer times) spreading the pairs over
    // the SMs, in the 80-register shape up to 8 warps (its lists sized for 3
    // CTAs per SM) and the 128-register one above; the throughput plan when
    // those lists do not fit.  Small 200 x 20 double fit, CUDA graph: 16 x 2
    // warps 36.4 us, 3 x 1 and 8 x 1 34.4 us, 8 x 3 32.9 us.
    if (single && tune.warps == 0 && tune.ctas == 0 && nj > 0 &&
        nj * m <= (int64_t)num_sms * 16) {
        const int64_t per_col = std::max<int64_t>(1, num_sms / nj);  // CTAs per column jhat
        const int64_t w = std::max<int64_t>(std::min<int64_t>(m, 8), (m + per_col - 1) / per_col);
        Tune lt = tune;
        lt.warps = (int)std::min<int64_t>(16, std::max<int64_t>(1, w));
        lt.ctas = lt.warps <= 8 ? 3 : 1;
        const PairPlan p = plan_pairs_for<T>(n, m, num_sms, nj, lt);
        if (p.warps > 0) return p;
    }
    return plan_pairs_for<T>(n, m, num_sms, nj, tune);
}

template <typename T>
cudaError_t launch_pairs(const ScanArgs<T> &a, const double *lambdas, int t0, int nlc,
                         const PairPlan &plan, cudaStream_t st, int &launches) {
    LambdaPack lp;
    lp.tl_min = lp.tl_max = 0;
    for (int q = 0; q < nlc; ++q) {
        lp.lam[q] = lambdas[t0 + q];
        if (lp.lam[q] < lp.lam[lp.tl_min]) lp.tl_min = q;
        if (lp.lam[q] > lp.lam[lp.tl_max]) lp.tl_max = q;
    }
    cudaError_t e;
    switch (plan.shape) {
        case SHAPE_R80: e = launch_pairs_sh<T, SHAPE_R80>(a, lp, t0, nlc, plan, st); break;
        case SHAPE_R64: e = launch_pairs_sh<T, SHAPE_R64>(a, lp, t0, nlc, plan, st); break;
        case SHAPE_R128: e = launch_pairs_sh<T, SHAPE_R128>(a, lp, t0, nlc, plan, st); break;
        default: e = cudaErrorInvalidConfiguration;
    }
    launches++;
    return e;
}

template PairPlan plan_pairs<float>(int64_t, int64_t, int, int64_t, const Tune &, bool);
template PairPlan plan_pairs<double>(int64_t, int64_t, int, int64_t, const Tune &, bool);
template int64_t max_rows_pairs<float>();
template int64_t max_rows_pairs<double>();
template cudaError_t launch_pairs<float>(const ScanArgs<float> &, const double *, int, int,
                                         const PairPlan &, cudaStream_t, int &);
template cudaError_t launch_pairs<double>(const ScanArgs<double> &, const double *, int, int,
                                          const PairPlan &, cudaStream_t, int &);


}  // namespace l1l
