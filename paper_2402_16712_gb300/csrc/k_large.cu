// k_large.cu -- steps A2-A4 (ratios, exact weighted median of Lemma 1,
// per-pair residual of Algorithm 1) for n beyond what the pair kernel holds
// in shared memory.
//
// The pair kernel stages column jhat in shared memory, which bounds n.  Here
// every (lambda, jhat, k) is solved by a cluster of C CTAs that stream the two
// columns from the staged column-major copy in global memory (L2-resident for
// moderate m), each CTA over its own slice of the rows:
//
//   descent  a radix descent over the order-preserving key of the correctly
//            rounded ratio r_i = x_ik / x_ijhat, 11 key bits per pass (float:
//            3 passes, double: 6).  A pass histograms the exact fixed-point
//            weights q_i (the pair kernel's q_i and Decide test) of the rows
//            whose key lies in the surviving range by its next digit; the CTAs
//            of the cluster read each other's histograms through distributed
//            shared memory, every CTA takes the same decision from the same
//            totals, and the first bin at which "weight at or below t exceeds
//            W/2" (penalty point (0, lambda) included) becomes true is kept.
//            After the last digit the surviving key is the median itself.
//   residual sum_i |x_ik - v x_ijhat| over the rows (float input: runs of 32
//            terms in float, the runs in double; double input: double), a
//            fixed reduction order per CTA, then rank order over the cluster;
//            C depends on n only, so results do not depend on m or on the
//            number of lambdas.
//
// Ratios are recomputed by division in every pass rather than stored.  A
// decision the truncated weights cannot settle lists the pair for the exact
// wide-accumulator path, as in the pair kernel.  Control flow depends only on
// the pair index and on values every CTA of a cluster computes identically,
// so all CTAs meet every cluster barrier.
#include <cooperative_groups.h>

#include <algorithm>

#include "checks.cuh"
#include "common.cuh"
#include "launch.h"
#include "pairs.cuh"

namespace cg = cooperative_groups;

namespace l1l {

constexpr int LG_NT = 512;                // threads per CTA
constexpr int LG_BITS = 11;               // key bits per pass (at most)
constexpr int LG_NB = 1 << LG_BITS;       // histogram bins
constexpr int LG_BPT = LG_NB / LG_NT;     // bins per thread in the scan
constexpr int LG_COPIES = 4;              // privatised histogram copies per CTA
constexpr int LG_MAXC = 8;                // CTAs per cluster (portable limit)
constexpr int64_t LG_ROWS_PER_CTA = 65536;  // rows of one CTA before the cluster grows

// Shift of the lowest key bit of pass l (digits of 11 bits from the top, the
// last two of 10 bits for double keys, the last one for float keys).
template <typename T> struct LgDigits;
template <> struct LgDigits<float> {
    static constexpr int levels = 3;
    static __device__ __forceinline__ int shift(int l) { return l == 0 ? 21 : (l == 1 ? 10 : 0); }
};
template <> struct LgDigits<double> {
    static constexpr int levels = 6;
    static __device__ __forceinline__ int shift(int l) {
        return l < 4 ? 53 - 11 * l : (l == 4 ? 10 : 0);
    }
};

// Two rows per 8-byte word / four per 16-byte word: the vector of one load.
template <typename T> struct LgVec;
template <> struct LgVec<float> {
    using V = float4;
    static constexpr int W = 4;
    static __device__ __forceinline__ void get(const V &v, float *o) {
        o[0] = v.x;
        o[1] = v.y;
        o[2] = v.z;
        o[3] = v.w;
    }
};
template <> struct LgVec<double> {
    using V = double2;
    static constexpr int W = 2;
    static __device__ __forceinline__ void get(const V &v, double *o) {
        o[0] = v.x;
        o[1] = v.y;
    }
};

enum : int { LG_SEARCH = 0, LG_FOUND = 1, LG_EXACT = 2, LG_NONE = 3, LG_INTERNAL = 4 };

template <typename K> struct LgDecision {
    K prefix;        // key bits decided so far
    int64_t sbelow;  // weight of valid rows whose key lies below the surviving range
    int state;
    int first;       // first bin whose test is not "false" (LG_NB: none)
};

template <typename T> struct LgSmem {
    using K = typename Traits<T>::K;
    unsigned long long copies[LG_COPIES][LG_NB];  // this CTA's histogram copies
    unsigned long long tot[2][LG_NB];             // their sum, read by the cluster
    double part[2];                               // residual partial, read by rank 0
    long long wsum[LG_NT / 32];                   // scan: warp totals
    double wres[LG_NT / 32];                      // residual: warp partials
    LgDecision<K> dec;
};

template <typename T>
__global__ void __launch_bounds__(LG_NT, 2)
    k_large(ScanArgs<T> a, const __grid_constant__ LambdaPack lp, int t0, int nlc,
            int64_t rows_per_cta) {
    using Tr = Traits<T>;
    using K = typename Tr::K;
    using VT = LgVec<T>;
    using V = typename VT::V;
    constexpr int VW = VT::W;
    constexpr int KB = Tr::KEY_BITS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    LgSmem<T> &sm = *reinterpret_cast<LgSmem<T> *>(smem_raw);

    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks();
    const int rank = (int)cl.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t cid = blockIdx.x / C, ncl = gridDim.x / C;
    const int64_t m = a.m, nj = a.nj, ldn = a.ldn;
    const int64_t P = (int64_t)nlc * nj * m;
    // this CTA's rows [r0, r1), whole vectors (ldn and rows_per_cta are multiples of 128)
    const int64_t r0 = std::min<int64_t>(ldn, (int64_t)rank * rows_per_cta);
    const int64_t r1 = std::min<int64_t>(ldn, r0 + rows_per_cta);
    const int64_t v0 = r0 / VW, v1 = r1 / VW;
    int buf = 0;

    for (int64_t p = cid; p < P; p += ncl) {
        const int tl = (int)(p / (nj * m));
        const int64_t rem = p - (int64_t)tl * nj * m;
        const int64_t q = rem / m, k = rem - q * m;
        const int64_t j = a.jlist ? (int64_t)a.jlist[q] : q;
        const bool leader = rank == 0 && tid == 0;
        if (j < 0 || j >= m) {
            if (leader) atomicOr(a.status, ST_BADINDEX);
            continue;
        }
        const int t = t0 + tl;
        const double lam = lp.lam[tl];
        const int64_t o = L1L_CHK(((int64_t)t * m + j) * m + k, (int64_t)a.n_lambda * m * m);
        if (k == j) {  // v_jhat = 1: zero residual, penalty lambda * 1
            if (leader) {
                a.v_all[o] = T(1);
                a.s_all[o] = lam;
            }
            continue;
        }
        const ColInfo ci = a.ci[j];
        if (a.force_exact) {
            if (leader) {
                const uint32_t slot = atomicAdd(a.slow_count, 1u);
                a.slow[slot] = SlowEntry{t, (int32_t)j, (int32_t)k, (int16_t)a.inst,
                                         (int16_t)SEL_SLOW};
            }
            continue;
        }
        const V *xjv = reinterpret_cast<const V *>(a.Xt + j * ldn);
        const V *xkv = reinterpret_cast<const V *>(a.Xt + k * ldn);
        Decide dec;
        dec.init(ci, lam);

        K prefix = 0;
        int64_t sbelow = 0;
        int state = ci.n_valid > 0 ? LG_SEARCH : LG_NONE;  // no valid row: v = 0
        for (int l = 0; state == LG_SEARCH && l < LgDigits<T>::levels; ++l) {
            const int sh = LgDigits<T>::shift(l);
            const int top = l == 0 ? KB : LgDigits<T>::shift(l - 1);
            const int nbl = 1 << (top - sh);
            const K bmask = (K)(nbl - 1);
            const K pmask = top == KB ? (K)0 : ~(((K)1 << top) - 1);
            // ---- one pass: histogram of the surviving rows by this digit ----
            for (int b = tid; b < LG_COPIES * LG_NB; b += LG_NT) (&sm.copies[0][0])[b] = 0ull;
            if (tid == 0) sm.dec.first = LG_NB;
            __syncthreads();
            unsigned long long *cp = sm.copies[warp % LG_COPIES];
            int cur = -1;
            unsigned long long csum = 0;
            // the next vectors are loaded while the current ones are processed
            V nj{}, nk{};
            if (v0 + tid < v1) {
                nj = xjv[v0 + tid];
                nk = xkv[v0 + tid];
            }
            for (int64_t v = v0 + tid; v < v1; v += LG_NT) {
                T xb[VW], xa[VW];
                VT::get(nj, xb);
                VT::get(nk, xa);
                if (v + LG_NT < v1) {
                    nj = xjv[v + LG_NT];
                    nk = xkv[v + LG_NT];
                }
#pragma unroll
                for (int u = 0; u < VW; ++u) {
                    if (xb[u] == T(0)) continue;
                    const K kk = Tr::key(Tr::div_rn(xa[u], xb[u]));
                    if ((kk & pmask) != prefix) continue;
                    const int bin = (int)((kk >> sh) & bmask);
                    int inx = 0;
                    const unsigned long long w =
                        (unsigned long long)fixq(fabs(xb[u]), ci.sigma, inx);
                    if (bin == cur) {
                        csum += w;
                    } else {
                        if (cur >= 0 && csum) atomicAdd(&cp[cur], csum);
                        cur = bin;
                        csum = w;
                    }
                }
            }
            if (cur >= 0 && csum) atomicAdd(&cp[cur], csum);
            __syncthreads();
            for (int b = tid; b < LG_NB; b += LG_NT) {
                unsigned long long s = 0;
#pragma unroll
                for (int c = 0; c < LG_COPIES; ++c) s += sm.copies[c][b];
                sm.tot[buf][b] = s;
            }
            cl.sync();  // every CTA's totals are complete and visible
            // ---- the cluster's totals, scanned in bin order ----
            long long h[LG_BPT];
            long long run = 0;
#pragma unroll
            for (int u = 0; u < LG_BPT; ++u) {
                const int b = tid * LG_BPT + u;
                unsigned long long s = 0;
                for (int r = 0; r < C; ++r) s += cl.map_shared_rank(&sm.tot[buf][0], r)[b];
                h[u] = (long long)s;
                run += h[u];
            }
            long long incl = run;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const long long y = __shfl_up_sync(0xFFFFFFFFu, incl, off);
                if (lane >= off) incl += y;
            }
            if (lane == 31) sm.wsum[warp] = incl;
            __syncthreads();
            long long before = incl - run;  // weight of this CTA's earlier bins
            for (int w = 0; w < warp; ++w) before += sm.wsum[w];
            // first bin whose test is true or undecidable
            int mine = LG_NB, mine_res = 0;
            long long mine_below = 0;
            long long acc = before;
#pragma unroll
            for (int u = 0; u < LG_BPT; ++u) {
                const int b = tid * LG_BPT + u;
                const long long below = acc;
                acc += h[u];
                if (mine == LG_NB && b < nbl) {
                    const K full = prefix | ((K)b << sh);
                    const bool nonneg = ((full >> (KB - 1)) & 1) != 0;
                    const int res = dec.cond(sbelow + acc, nonneg);
                    if (res != 0) {
                        mine = b;
                        mine_res = res;
                        mine_below = below;
                    }
                }
            }
            if (mine < LG_NB) atomicMin(&sm.dec.first, mine);
            __syncthreads();
            if (mine < LG_NB && mine == sm.dec.first) {
                LgDecision<K> d;
                d.first = mine;
                d.prefix = prefix | ((K)mine << sh);
                d.sbelow = sbelow + mine_below;
                d.state = mine_res == 1 ? (l + 1 == LgDigits<T>::levels ? LG_FOUND : LG_SEARCH)
                                        : LG_EXACT;
                sm.dec = d;
            }
            __syncthreads();
            if (sm.dec.first == LG_NB) {
                // "true" at no key: W = 0 at the top level; below it the parent
                // bin's test was true at its last key, so this cannot happen
                state = l == 0 ? LG_NONE : LG_INTERNAL;
            } else {
                prefix = sm.dec.prefix;
                sbelow = sm.dec.sbelow;
                state = sm.dec.state;
            }
            buf ^= 1;
            __syncthreads();  // sm.dec is rewritten by the next pass
        }
        if (state == LG_EXACT) {
            if (leader) {
                const uint32_t slot = atomicAdd(a.slow_count, 1u);
                a.slow[slot] = SlowEntry{t, (int32_t)j, (int32_t)k, (int16_t)a.inst,
                                         (int16_t)SEL_SLOW_BAND};
            }
            continue;
        }
        if (state == LG_INTERNAL) {
            if (leader) {
                atomicOr(a.status, ST_INTERNAL);
                a.v_all[o] = T(NAN);
                a.s_all[o] = NAN;
            }
            continue;
        }
        const T vv = state == LG_FOUND ? Tr::value(prefix) : T(0);
        // ---- residual: sum_i |x_ik - v x_ijhat| ----
        // float input: terms summed in float over runs of 32 rows (a relative
        // error below 2^-19 of the run's sum), runs in double; double input:
        // every term in double
        double racc = 0.0;
        T run = T(0);
        int nrun = 0;
        for (int64_t v = v0 + tid; v < v1; v += LG_NT) {
            T xb[VW], xa[VW];
            VT::get(xjv[v], xb);
            VT::get(xkv[v], xa);
            T t4 = T(0);
#pragma unroll
            for (int u = 0; u < VW; ++u) t4 += fabs(fma(-vv, xb[u], xa[u]));
            run += t4;
            if (++nrun == 32 / VW || sizeof(T) == 8) {
                racc += (double)run;
                run = T(0);
                nrun = 0;
            }
        }
        racc += (double)run;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) racc += __shfl_xor_sync(0xFFFFFFFFu, racc, off);
        if (lane == 0) sm.wres[warp] = racc;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int w = 0; w < LG_NT / 32; ++w) s += sm.wres[w];
            sm.part[buf] = s;
        }
        cl.sync();  // every CTA's partial is visible
        if (leader) {
            double s = 0.0;
            for (int r = 0; r < C; ++r) s += cl.map_shared_rank(&sm.part[0], r)[buf];
            a.v_all[o] = vv;
            a.s_all[o] = s + lam * (double)fabs(vv);
        }
        buf ^= 1;
    }
    cl.sync();  // no CTA leaves while another may still read its shared memory
}

int large_cluster_size(int64_t ldn) {
    const int64_t c = (ldn + LG_ROWS_PER_CTA - 1) / LG_ROWS_PER_CTA;
    return (int)std::max<int64_t>(1, std::min<int64_t>(LG_MAXC, c));
}

template <typename T>
cudaError_t launch_large(const ScanArgs<T> &a, const double *lambdas, int t0, int nlc,
                         cudaStream_t st, int &launches) {
    const int C = large_cluster_size(a.ldn);
    const int64_t rpc = ((a.ldn + C - 1) / C + ROW_PAD - 1) & ~int64_t(ROW_PAD - 1);
    const size_t smem = sizeof(LgSmem<T>);
    auto kern = k_large<T>;
    cudaError_t e = ensure_smem(reinterpret_cast<const void *>(kern), smem);
    if (e != cudaSuccess) return e;
    LambdaPack lp;
    lp.tl_min = lp.tl_max = 0;
    for (int q = 0; q < nlc; ++q) lp.lam[q] = lambdas[t0 + q];
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(LG_NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3((unsigned)C);
    int clusters = 0;
    e = cudaOccupancyMaxActiveClusters(&clusters, reinterpret_cast<const void *>(kern), &cfg);
    if (e != cudaSuccess) return e;
    if (clusters < 1) return cudaErrorInvalidConfiguration;
    const int64_t P = (int64_t)nlc * a.nj * a.m;
    const int64_t ncl = std::max<int64_t>(1, std::min<int64_t>(P, clusters));
    cfg.gridDim = dim3((unsigned)(ncl * C));
    e = cudaLaunchKernelEx(&cfg, kern, a, lp, t0, nlc, rpc);
    launches++;
    return e;
}

template cudaError_t launch_large<float>(const ScanArgs<float> &, const double *, int, int,
                                         cudaStream_t, int &);
template cudaError_t launch_large<double>(const ScanArgs<double> &, const double *, int, int,
                                          cudaStream_t, int &);

L1L_CHECKS_READER(l1l_checks_large)

}  // namespace l1l
