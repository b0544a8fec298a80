// k_pairs.cu -- steps A2-A4 for every (lambda, jhat, k): ratios, exact
// weighted median (Lemma 1) and per-pair residual (Algorithm 1).
//
// Layout: one CTA per (jhat, k-chunk); column jhat (x_ijhat and its
// fixed-point weights q_i) is staged once in shared memory and shared by the
// CTA's warps; each warp owns one k at a time.  Per pair the warp
//   1. forms key_i = key(fl(x_ik / x_ijhat)) for every row (A2) into its
//      shared-memory key array (the penalty point is implicit, see Decide);
//   2. per lambda, finds the weighted median by sample-pivot narrowing (A3):
//      32 candidate keys are sorted across the warp, two pivots bracketing the
//      estimated crossing are taken, the exact fixed-point weight below and
//      between them is summed with warp reductions, the side holding the
//      median is decided exactly and compacted; at <= 31 candidates a final
//      warp sort + prefix scan picks the smallest key whose cumulative weight
//      passes half the total;
//   3. sums the residual |x_ik - v x_ijhat| over all rows (A4).
// A decision that the truncated fixed-point weights cannot settle sends the
// pair to the exact wide-accumulator kernel (k_exact.cu).
#include <algorithm>

#include "common.cuh"
#include "launch.h"

namespace l1l {

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~size_t(15); }

template <typename T> struct PairSmem {
    using K = typename Traits<T>::K;
    __host__ __device__ static size_t col_bytes(int64_t npad) { return al16(npad * sizeof(T)) + al16(npad * 8); }
    __host__ __device__ static size_t warp_bytes(int64_t npad) {
        return 2 * al16(npad * sizeof(K)) + al16(npad * sizeof(uint16_t));
    }
};

template <typename K>
__device__ __forceinline__ void warp_sort32(K &key, int64_t &q, int lane) {
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            K ok = __shfl_xor_sync(0xFFFFFFFFu, key, stride);
            int64_t oq = __shfl_xor_sync(0xFFFFFFFFu, q, stride);
            bool up = (lane & size) == 0 || size == 32;
            bool lower = (lane & stride) == 0;
            bool take = lower == up ? (ok < key) : (ok > key);
            if (take) {
                key = ok;
                q = oq;
            }
        }
    }
}

__device__ __forceinline__ int64_t warp_scan_i64(int64_t x, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

enum { SEL_OK = 0, SEL_SLOW = 1, SEL_INTERNAL = 2 };

// Weighted median over the warp's keys (row-indexed, NONE = row excluded).
template <typename T>
__device__ int warp_select(const typename Traits<T>::K *keys, const int64_t *colq,
                           typename Traits<T>::K *ck, uint16_t *ci, int n, int n_valid,
                           const Decide &dc, typename Traits<T>::K &tstar, int lane) {
    using Tr = Traits<T>;
    using K = typename Tr::K;
    const K KEY0 = Tr::KEY0, NONE = Tr::NONE;
    const unsigned FULL = 0xFFFFFFFFu;
    const unsigned lt_mask = (1u << lane) - 1u;

    K lo = 0, hi = NONE - 1;  // invariant: the median key lies in [lo, hi]
    int64_t L = 0;            // exact weight of valid rows with key < lo
    int64_t Sc = dc.Q;        // weight of the current candidates
    int c = 0;                // candidate count (when !from_full)
    bool from_full = true;
    int d = 3;

    for (int level = 0;; ++level) {
        if (level >= 64) return SEL_SLOW;
        const int ctot = from_full ? n_valid : c;
        if (ctot <= 31) {
            if (from_full) {  // compact every valid row
                int base = 0;
                for (int i0 = 0; i0 < n; i0 += 32) {
                    int i = i0 + lane;
                    K kk = i < n ? keys[i] : NONE;
                    bool keep = kk != NONE;
                    unsigned msk = __ballot_sync(FULL, keep);
                    if (keep) {
                        int pos = base + __popc(msk & lt_mask);
                        ck[pos] = kk;
                        ci[pos] = (uint16_t)i;
                    }
                    base += __popc(msk);
                }
                c = base;
                from_full = false;
                __syncwarp();
            }
            break;
        }
        // ---- sample 32 candidates, sort them, estimate the crossing --------
        K sk;
        int64_t sq;
        if (from_full) {
            int i = (int)(((int64_t)lane * n) >> 5);
            sk = keys[i];
            sq = sk == NONE ? 0 : colq[i];
        } else {
            int p = (int)(((int64_t)lane * c) >> 5);
            sk = ck[p];
            sq = colq[ci[p]];
        }
        warp_sort32<K>(sk, sq, lane);
        int64_t P = warp_scan_i64(sq, lane);
        int64_t P31 = __shfl_sync(FULL, P, 31);
        double scale = P31 > 0 ? (double)Sc / (double)P31 : 0.0;
        double est = (double)P * scale;
        double hneg = 0.5 * ((double)dc.Q + (double)dc.Lf) - (double)L;
        double hpos = 0.5 * ((double)dc.Q - (double)dc.Lc) - (double)L;
        bool crossed = sk != NONE && est > (sk >= KEY0 ? hpos : hneg);
        unsigned cm_ = __ballot_sync(FULL, crossed);
        int jx = cm_ ? __ffs(cm_) - 1 : 31;
        K p1 = __shfl_sync(FULL, sk, max(jx - d, 0));
        K p2 = __shfl_sync(FULL, sk, min(jx + d, 31));
        if (p1 == NONE) p1 = hi;
        if (p2 == NONE) p2 = hi;
        p1 = p1 < lo ? lo : (p1 > hi ? hi : p1);
        p2 = p2 < lo ? lo : (p2 > hi ? hi : p2);
        if (p1 > p2) p1 = p2;

        // ---- exact weight below p1 and within [p1, p2] ---------------------
        int64_t Sb = 0, Sm = 0;
        int cb = 0, cmid = 0;
        if (from_full) {
            for (int i = lane; i < n; i += 32) {
                K kk = keys[i];
                if (kk == NONE) continue;
                int64_t q = colq[i];
                if (kk < p1) {
                    Sb += q;
                    cb++;
                } else if (kk <= p2) {
                    Sm += q;
                    cmid++;
                }
            }
        } else {
            for (int p = lane; p < c; p += 32) {
                K kk = ck[p];
                int64_t q = colq[ci[p]];
                if (kk < p1) {
                    Sb += q;
                    cb++;
                } else if (kk <= p2) {
                    Sm += q;
                    cmid++;
                }
            }
        }
        Sb = warp_sum_i64(Sb);
        Sm = warp_sum_i64(Sm);
        cb = warp_sum_i32(cb);
        cmid = warp_sum_i32(cmid);

        // ---- decide which part holds the median (exact) --------------------
        int part, newc;
        int r1 = (p1 == lo) ? 0 : dc.cond(L + Sb, (K)(p1 - 1) >= KEY0);
        if (r1 < 0) return SEL_SLOW;
        if (r1 == 1) {
            part = 0;
            hi = p1 - 1;
            Sc = Sb;
            newc = cb;
        } else {
            int r2 = dc.cond(L + Sb + Sm, p2 >= KEY0);
            if (r2 < 0) return SEL_SLOW;
            if (r2 == 1) {
                part = 1;
                lo = p1;
                hi = p2;
                L += Sb;
                Sc = Sm;
                newc = cmid;
            } else {
                if (p2 == hi) return SEL_INTERNAL;
                part = 2;
                lo = p2 + 1;
                L += Sb + Sm;
                Sc = Sc - Sb - Sm;
                newc = ctot - cb - cmid;
            }
        }
        if (lo == hi) {
            tstar = lo;
            return SEL_OK;
        }
        d = (newc == ctot) ? 0 : 3;

        // ---- compact the chosen part (stable; in place on the candidates) --
        int base = 0;
        const int lim = from_full ? n : c;
        for (int p0 = 0; p0 < lim; p0 += 32) {
            int p = p0 + lane;
            K kk = NONE;
            uint16_t idx = 0;
            if (p < lim) {
                if (from_full) {
                    kk = keys[p];
                    idx = (uint16_t)p;
                } else {
                    kk = ck[p];
                    idx = ci[p];
                }
            }
            bool keep = kk != NONE &&
                        (part == 0 ? kk < p1 : (part == 1 ? (kk >= p1 && kk <= p2) : kk > p2));
            unsigned msk = __ballot_sync(FULL, keep);
            if (keep) {
                int pos = base + __popc(msk & lt_mask);
                ck[pos] = kk;
                ci[pos] = idx;
            }
            base += __popc(msk);
        }
        __syncwarp();
        c = base;
        from_full = false;
    }

    // ---- final: <= 31 candidates (+ the penalty point's key if in range) ---
    K fk = NONE;
    int64_t fq = 0;
    if (lane < c) {
        fk = ck[lane];
        fq = colq[ci[lane]];
    } else if (lane == c && lo <= KEY0 && KEY0 <= hi) {
        fk = KEY0;
        fq = 0;
    }
    warp_sort32<K>(fk, fq, lane);
    int64_t P = warp_scan_i64(fq, lane);
    K nxt = __shfl_down_sync(FULL, fk, 1);
    bool last = (lane == 31) || (nxt != fk);
    int r = -2;
    if (last && fk != NONE) r = dc.cond(L + P, fk >= KEY0);
    unsigned okm = __ballot_sync(FULL, r == 1);
    unsigned unm = __ballot_sync(FULL, r == -1);
    unsigned any = okm | unm;
    if (!any) return SEL_INTERNAL;
    int first = __ffs(any) - 1;
    if ((unm >> first) & 1u) return SEL_SLOW;
    tstar = __shfl_sync(FULL, fk, first);
    return SEL_OK;
}

template <typename T>
__global__ void __launch_bounds__(256) k_pairs(ScanArgs<T> a, LambdaPack lp, int t0, int nlc,
                                               int kchunk) {
    using Tr = Traits<T>;
    using K = typename Tr::K;
    extern __shared__ __align__(16) unsigned char smem[];
    const int n = (int)a.n;
    const int64_t m = a.m, ldn = a.ldn;
    const int npad = (n + 31) & ~31;
    const int j = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;

    T *colx = reinterpret_cast<T *>(smem);
    int64_t *colq = reinterpret_cast<int64_t *>(smem + al16((size_t)npad * sizeof(T)));
    unsigned char *wbase = smem + PairSmem<T>::col_bytes(npad) +
                           (size_t)warp * PairSmem<T>::warp_bytes(npad);
    K *keys = reinterpret_cast<K *>(wbase);
    K *ck = reinterpret_cast<K *>(wbase + al16((size_t)npad * sizeof(K)));
    uint16_t *ci = reinterpret_cast<uint16_t *>(wbase + 2 * al16((size_t)npad * sizeof(K)));

    const ColInfo cinfo = a.ci[j];
    const T *xj = a.Xt + (int64_t)j * ldn;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        T b = xj[i];
        colx[i] = b;
        int e = 0;
        colq[i] = b != T(0) ? fixq(b < T(0) ? -b : b, cinfo.sigma, e) : 0;
    }
    __syncthreads();

    const int64_t k0 = (int64_t)blockIdx.y * kchunk;
    const int64_t k1 = min(m, k0 + kchunk);
    for (int64_t k = k0 + warp; k < k1; k += nw) {
        if (k == j) {  // v_jhat = 1: zero residual, penalty lambda * 1
            for (int tl = lane; tl < nlc; tl += 32) {
                int64_t o = ((int64_t)(t0 + tl) * m + j) * m + k;
                a.v_all[o] = T(1);
                a.s_all[o] = lp.lam[tl];
            }
            continue;
        }
        const T *xk = a.Xt + k * ldn;
        if (cinfo.n_valid > 0 && !a.force_exact) {
            for (int i = lane; i < n; i += 32) {
                T b = colx[i];
                keys[i] = b != T(0) ? Tr::key(Tr::div_rn(xk[i], b)) : Tr::NONE;
            }
            __syncwarp();
        }
        for (int tl = 0; tl < nlc; ++tl) {
            const int t = t0 + tl;
            const double lam = lp.lam[tl];
            const int64_t o = ((int64_t)t * m + j) * m + k;
            K ts = Tr::KEY0;
            int st = SEL_OK;
            if (a.force_exact) {
                st = SEL_SLOW;
            } else if (cinfo.n_valid > 0) {
                Decide dc;
                dc.init(cinfo, lam);
                st = warp_select<T>(keys, colq, ck, ci, n, cinfo.n_valid, dc, ts, lane);
            }
            if (st == SEL_SLOW) {
                if (lane == 0) {
                    uint32_t slot = atomicAdd(a.slow_count, 1u);
                    SlowEntry e;
                    e.t = t;
                    e.j = j;
                    e.k = (int32_t)k;
                    e.inst = 0;
                    a.slow[slot] = e;
                }
                continue;
            }
            if (st == SEL_INTERNAL) {
                if (lane == 0) {
                    atomicOr(a.status, ST_INTERNAL);
                    a.v_all[o] = T(NAN);
                    a.s_all[o] = NAN;
                }
                continue;
            }
            const T v = Tr::value(ts);
            const T res = warp_residual<T>(xk, colx, n, v, lane);
            if (lane == 0) {
                a.v_all[o] = v;
                a.s_all[o] = (double)res + lam * (double)fabs(v);
            }
        }
        __syncwarp();
    }
}

template <typename T> int64_t max_rows_pairs() {
    // one warp must fit: column (T + int64) + one warp's arrays
    const size_t budget = 227 * 1024;
    int64_t n = 32;
    while (PairSmem<T>::col_bytes(n + 32) + PairSmem<T>::warp_bytes(n + 32) <= budget &&
           n + 32 <= 65535)
        n += 32;
    return n;
}

template <typename T> PairPlan plan_pairs(int64_t n, int64_t m, int num_sms) {
    PairPlan p{0, 0, 0, 0};
    const int64_t npad = (n + 31) & ~int64_t(31);
    if (n > max_rows_pairs<T>()) return p;
    const size_t cb = PairSmem<T>::col_bytes(npad), wb = PairSmem<T>::warp_bytes(npad);
    // prefer two CTAs per SM (<= ~113 KB each) with as many warps as fit, up to 8
    int w = 0;
    for (int cand = 8; cand >= 1; --cand)
        if (cb + cand * wb <= 113 * 1024) {
            w = cand;
            break;
        }
    if (w == 0)
        for (int cand = 8; cand >= 1; --cand)
            if (cb + cand * wb <= 227 * 1024) {
                w = cand;
                break;
            }
    if (w == 0) return p;
    p.warps = w;
    p.smem = cb + (size_t)w * wb;
    // split k so that there are enough CTAs to fill the GPU
    int64_t want_ctas = (int64_t)num_sms * 4;
    int64_t chunks = std::max<int64_t>(1, std::min<int64_t>((m + w - 1) / w, (want_ctas + m - 1) / m));
    p.kchunk = (int)((m + chunks - 1) / chunks);
    p.kchunks = (int)((m + p.kchunk - 1) / p.kchunk);
    return p;
}

template <typename T>
cudaError_t launch_pairs(const ScanArgs<T> &a, const double *lambdas, int t0, int nlc,
                         const PairPlan &plan, cudaStream_t st, int &launches) {
    cudaError_t e = cudaFuncSetAttribute(k_pairs<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)plan.smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)a.m, (unsigned)plan.kchunks);
    LambdaPack lp;
    for (int q = 0; q < nlc; ++q) lp.lam[q] = lambdas[t0 + q];
    k_pairs<T><<<grid, plan.warps * 32, plan.smem, st>>>(a, lp, t0, nlc, plan.kchunk);
    launches++;
    return cudaGetLastError();
}

template PairPlan plan_pairs<float>(int64_t, int64_t, int);
template PairPlan plan_pairs<double>(int64_t, int64_t, int);
template int64_t max_rows_pairs<float>();
template int64_t max_rows_pairs<double>();
template cudaError_t launch_pairs<float>(const ScanArgs<float> &, const double *, int, int,
                                         const PairPlan &, cudaStream_t, int &);
template cudaError_t launch_pairs<double>(const ScanArgs<double> &, const double *, int, int,
                                          const PairPlan &, cudaStream_t, int &);

}  // namespace l1l
