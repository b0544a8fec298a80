// k_pairs.cu -- the pair kernel for one instance (grid over jhat x k-chunks)
// and its shared-memory planner; the per-pair algorithm is in pairs.cuh.
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

template <typename T, bool MULTI, bool CS>
__global__ void __launch_bounds__(256, 3)
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

// The resident-warp plan for one placement of x_ijhat (cs: shared memory).
template <typename T>
static PairPlan plan_placement(int64_t npad, bool cs, int d0, const Tune &tune) {
    PairPlan p{0, 0, 0, 0, 0, 0, 0, 0};
    const size_t cb = PairSmem<T>::col_bytes(npad, cs);
    // Per-lane candidate quota wanted: the level-0 bracket (+-d0 of 64 weight
    // samples) holds ~2.5% of the rows per sample position, i.e. mu = 0.025 d0
    // n/32 per lane; ask for mu + 3.5 sqrt(mu) + 1 so that the busiest of 32
    // lanes rarely overflows (an overflow costs one more pass).
    const double mu = 0.025 * (double)d0 * (double)npad / 32.0;
    const int64_t qt_need = std::min<int64_t>(npad / 32, (int64_t)ceil(mu + 3.5 * sqrt(mu) + 1.0));
    // Up to three 8-warp CTAs per SM fit the register budget (80 registers x
    // 256 threads).  Over 1-3 CTAs per SM and 1-8 warps per CTA (or the
    // caller's choice), keep the plan with the most resident warps whose lists
    // meet the quota in 228 KB of shared memory (1 KB reserved per CTA,
    // static arrays included).
    int w = 0, cap = 0, best = 0, nc = 0;
    const int c_hi = tune.ctas > 0 ? tune.ctas : 3, c_lo = tune.ctas > 0 ? tune.ctas : 1;
    const int w_hi = tune.warps > 0 ? tune.warps : 8, w_lo = tune.warps > 0 ? tune.warps : 1;
    for (int ctas = c_hi; ctas >= c_lo; --ctas) {
        const int64_t per_cta = 233472 / ctas - 1024 - 1024;
        for (int cand = w_hi; cand >= w_lo; --cand) {
            if (ctas * cand <= best || ctas * cand > 24) continue;
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
    p.smem = cb + (size_t)w * PairSmem<T>::warp_bytes(cap);
    return p;
}

template <typename T>
PairPlan plan_pairs(int64_t n, int64_t m, int num_sms, int64_t nj, const Tune &tune) {
    PairPlan p{0, 0, 0, 0, 0, 0, 0, 0};
    const int64_t npad = (n + ROW_PAD - 1) & ~int64_t(ROW_PAD - 1);
    if (n > max_rows_pairs<T>()) return p;
    const int d0 = tune.d0 > 0 ? tune.d0 : D0_DEFAULT;
    // Where x_ijhat lives.  Shared memory saves the residual pass an L2 read
    // per row; global memory frees n * sizeof(T) bytes per CTA.  Measured:
    // float keeps it in shared memory unless the smaller footprint admits more
    // resident warps (2000 x 2000: equal plans, shared 3% faster; 5000 x 1000:
    // 8 -> 14 warps per SM, global 11% faster); double reads it from global
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
        p = (sizeof(T) == 8 || rg > rs) ? pg : ps;
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
cudaError_t launch_pairs(const ScanArgs<T> &a, const double *lambdas, int t0, int nlc,
                         const PairPlan &plan, cudaStream_t st, int &launches) {
    // separate instantiations keep the single-lambda kernel small
    auto kern = nlc >= 3 ? (plan.cs ? k_pairs<T, true, true> : k_pairs<T, true, false>)
                         : (plan.cs ? k_pairs<T, false, true> : k_pairs<T, false, false>);
    cudaError_t e = ensure_smem(reinterpret_cast<const void *>(kern), plan.smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)a.nj, (unsigned)plan.kchunks);
    LambdaPack lp;
    lp.tl_min = lp.tl_max = 0;
    for (int q = 0; q < nlc; ++q) {
        lp.lam[q] = lambdas[t0 + q];
        if (lp.lam[q] < lp.lam[lp.tl_min]) lp.tl_min = q;
        if (lp.lam[q] > lp.lam[lp.tl_max]) lp.tl_max = q;
    }
    kern<<<grid, plan.warps * 32, plan.smem, st>>>(a, lp, t0, nlc, plan.kchunk, plan.cap);
    launches++;
    return cudaGetLastError();
}

template PairPlan plan_pairs<float>(int64_t, int64_t, int, int64_t, const Tune &);
template PairPlan plan_pairs<double>(int64_t, int64_t, int, int64_t, const Tune &);
template int64_t max_rows_pairs<float>();
template int64_t max_rows_pairs<double>();
template cudaError_t launch_pairs<float>(const ScanArgs<float> &, const double *, int, int,
                                         const PairPlan &, cudaStream_t, int &);
template cudaError_t launch_pairs<double>(const ScanArgs<double> &, const double *, int, int,
                                          const PairPlan &, cudaStream_t, int &);

L1L_CHECKS_READER(l1l_checks_pairs)

}  // namespace l1l
