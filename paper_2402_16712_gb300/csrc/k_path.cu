// k_path.cu -- Algorithm 2: the lambda path of every (jhat, k) pair.
//
// As lambda grows the penalty point at 0 gains weight, so the weighted median
// v_k(lambda) moves monotonically from v0 = v_k(0) to 0 through the distinct
// ratios between them.  For v0 > 0, with S(t) the weight of the rows whose
// ratio is <= t and Q the column's total weight, v_k takes the value t just
// above lambda = Q - 2 S(t) (Algorithm 2's lambda_p at the last row of t's
// run) and reaches 0 above Q - 2 S(0) (its lambda_max); for v0 < 0 it leaves
// t at lambda = 2 S(t) - Q.  So a pair's path needs v0 (the exact lambda = 0
// scan), the rows whose ratio lies between v0 and 0, sorted, and prefix sums
// of their exact fixed-point weights.
//
// Count pass: one warp per pair counts the rows in that range (entries <=
// rows + 1).  A device scan turns the counts into offsets.  Write pass: the
// warp collects the rows (exact keys, row index) into its shared-memory list,
// sorts them, and each run of equal keys writes its entry; pairs with more
// rows than the list holds are queued for a second kernel that does the same
// with a list in global scratch.
#include <cmath>

#include "checks.cuh"
#include "common.cuh"
#include "launch.h"
#include "pairs.cuh"

namespace l1l {

namespace {

constexpr int PW = 8;          // warps per CTA
constexpr int PATH_CAP = 256;  // shared-memory list entries per warp

template <typename T> struct PathArgs {
    const T *Xt;
    const float *Xf;
    const ColInfo *ci;
    int64_t n, m, ldn;
    const T *v0;           // [m][m] lambda = 0 medians
    int64_t *bound;        // count pass: [m*m] entries upper bound
    const int64_t *off;    // write pass: [m*m + 1]
    double *lam;           // write pass outputs
    T *val;
    double *res;           // optional: residual sum_i |x_ik - v x_ijhat| of each entry
    int32_t *len;          // [m*m]
    int32_t *big;          // pairs whose rows exceed the warp list
    uint32_t *big_count;
    uint32_t *big_next;    // work counter of the big-pair kernel
    unsigned char *scratch;  // big-pair lists, one slice per worker warp
    int64_t slice;         // entries per slice (power of two >= n)
    uint32_t *status;
};

// Double sums of one pass for the residual R(t) = sum_i |x_ik - t x_ijhat|,
// which for t a ratio value is  Btot - 2 B(t) + t (2 A(t) - Wv) + C0  with
// A(t), B(t) the sums of |x_ijhat| and sgn(x_ijhat) x_ik over valid rows whose
// ratio is <= t, Btot, Wv their totals and C0 the sum of |x_ik| over rows with
// x_ijhat = 0 (|x_ijhat| (r_i - t) = sgn(x_ijhat) x_ik - t |x_ijhat|).
struct RowSums {
    double Btot, Wv, C0, Ab, Bb;  // Ab, Bb: over the rows below the range
};

// Classification of one row against the range between 0 and v0 (exclusive
// of 0): -1 below it (exact weight counts in S), 0 inside, +1 above.
// kexact receives the exact key when it was computed (else NONE).  x_ik is
// read through xkp only when the exact key is needed.
template <typename T>
__device__ __forceinline__ int classify(float xf, float inv, const T *xkp, T xj, bool wide,
                                        bool pos,
                                        uint32_t ck_lo, uint32_t ck_hi,
                                        typename Traits<T>::K kv,
                                        typename Traits<T>::K &kexact) {
    using Tr = Traits<T>;
    using K = typename Tr::K;
    constexpr uint32_t G = Approx<T>::G;
    kexact = Tr::NONE;
    if (!wide) {
        const uint32_t kk = akey(__fmul_rn(xf, inv));
        // certain when the approximate coarse key is more than G from both
        // ends of the coarse range (the coarse image is monotone in the key)
        if (kk > ck_lo + G && kk + G < ck_hi) return 0;
        if (kk + G < ck_lo) return -1;
        if (kk > ck_hi + G) return 1;
    }
    const K ke = Tr::key(Tr::div_rn(*xkp, xj));
    kexact = ke;
    if (pos) {  // range (KEY0, kv]
        if (ke <= Tr::KEY0) return -1;
        return ke <= kv ? 0 : 1;
    }
    // range [kv, KEY0)
    if (ke < kv) return -1;
    return ke < Tr::KEY0 ? 0 : 1;
}

// Coarse-key range of (0, v0] or [v0, 0), and its exact upper/lower key.
template <typename T>
__device__ __forceinline__ void range_of(T v0, bool &pos, uint32_t &ck_lo, uint32_t &ck_hi,
                                         typename Traits<T>::K &kv) {
    pos = v0 > T(0);
    kv = Traits<T>::key(v0);
    const uint32_t cv = ckey((float)v0);
    if (pos) {
        ck_lo = CK0;
        ck_hi = cv;
    } else {
        ck_lo = cv;
        ck_hi = CK0;
    }
}

// Stage column jhat (x, float reciprocal, fixed-point weight) into shared memory.
template <typename T>
__device__ void stage_column(const PathArgs<T> &a, int64_t j, T *colb, float *inv, int64_t *colq,
                             int npad) {
    const ColInfo ci = a.ci[j];
    const T *xj = a.Xt + j * a.ldn;
    for (int i = threadIdx.x; i < npad; i += blockDim.x) {
        const T b = i < a.n ? xj[i] : T(0);
        colb[i] = b;
        inv[i] = b != T(0) ? Approx<T>::inv_of(b) : 0.0f;
        int e = 0;
        colq[i] = b != T(0) ? fixq(b < T(0) ? -b : b, ci.sigma, e) : 0;
    }
}

// Warp bitonic sort of (key, row) over P (power of two) entries of a list;
// entries c..P-1 are first filled with NONE.
template <typename K>
__device__ void warp_list_sort(K *keys, uint32_t *rows, int c, int P, int lane) {
    for (int i = c + lane; i < P; i += 32) {
        keys[i] = (K)~(K)0;
        rows[i] = 0;
    }
    __syncwarp();
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = lane; t < P / 2; t += 32) {
                const int i = 2 * t - (t & (stride - 1));
                const int jx = i + stride;
                const bool up = (i & size) == 0;
                const K ki = keys[i], kj = keys[jx];
                if ((ki > kj) == up) {
                    keys[i] = kj;
                    keys[jx] = ki;
                    const uint32_t r = rows[i];
                    rows[i] = rows[jx];
                    rows[jx] = r;
                }
            }
            __syncwarp();
        }
    }
}

__device__ __forceinline__ double fix_to_double(int64_t D, int sigma) {
    return scalbn((double)D, -sigma);
}

// Entries of one pair from its sorted in-range list (c > 0 rows).
template <typename T>
__device__ void emit_path(const PathArgs<T> &a, int64_t p, T v0, bool pos,
                          const typename Traits<T>::K *keys, const uint32_t *rows, int c,
                          const int64_t *colq, int64_t Q, int64_t Sbelow, int sigma,
                          const T *colb, const T *xk, const RowSums &rs, int lane) {
    using Tr = Traits<T>;
    using K = typename Tr::K;
    const unsigned FULL = 0xFFFFFFFFu;
    const int64_t o = a.off[p];
    const int64_t room = a.off[p + 1] - o;  // entries the count pass reserved
    // number of runs of equal keys
    int groups = 0;
    for (int i0 = 0; i0 < c; i0 += 32) {
        const int i = i0 + lane;
        const bool end = i < c && (i == c - 1 || keys[i] != keys[i + 1]);
        groups += __popc(__ballot_sync(FULL, end));
    }
    // the entries 0 .. groups lie inside the room the count pass reserved
    L1L_CHK((int64_t)groups, room);
    int64_t carry = Sbelow;  // S at the end of the previous chunk
    double cA = rs.Ab, cB = rs.Bb;  // residual sums at the end of the previous chunk
    double cQrun = 0.0;             // corrections of the run open at the chunk's end
    int gbase = 0;           // runs ended before this chunk
    for (int i0 = 0; i0 < c; i0 += 32) {
        const int i = i0 + lane;
        const int64_t q = i < c ? colq[rows[i]] : 0;
        const int64_t S = carry + warp_scan_add(q, lane);  // S(key_i) at a run end
        const bool end = i < c && (i == c - 1 || keys[i] != keys[i + 1]);
        const unsigned em = __ballot_sync(FULL, end);
        const int g = gbase + __popc(em & ((1u << lane) - 1u));  // run index (ascending)
        if (a.res) {
            // A, B: prefix sums through this row.  The formula counts the
            // rows of t's own run as "ratio <= t"; a row whose exact ratio
            // lies above its rounded value t then enters with the wrong sign,
            // so each row of the run adds the correction
            // qc = |x - t b| - (t |b| - sgn(b) x), summed over the run.
            double w = 0.0, sx = 0.0, qc = 0.0, t = 0.0;
            if (i < c) {
                const double b = (double)colb[rows[i]], x = (double)xk[rows[i]];
                t = (double)Tr::value(keys[i]);
                w = fabs(b);
                sx = b < 0.0 ? -x : x;
                qc = fabs(x - t * b) - (t * w - sx);
            }
            const double A = cA + warp_scan_add(w, lane), B = cB + warp_scan_add(sx, lane);
            const double Qi = warp_scan_add(qc, lane);  // inclusive, this chunk only
            // run sums of qc: the run's start holds the prefix before it
            const bool start = i < c && (i == 0 || keys[i - 1] != keys[i]);
            const unsigned smk = __ballot_sync(FULL, start);
            const double Qs = Qi - qc;  // chunk prefix before this row
            const unsigned upto = smk & (lane == 31 ? FULL : ((2u << lane) - 1u));
            const int hs = upto ? 31 - __clz(upto) : -1;
            const double Qstart = __shfl_sync(FULL, Qs, hs < 0 ? 0 : hs);
            // the run began in an earlier chunk: its prefix is cQ - cQrun
            const double run_q = hs >= 0 ? Qi - Qstart : cQrun + Qi;
            if (end) {  // each run writes the residual of its own entry
                const int slot = pos ? groups - 1 - g : g;
                a.res[o + slot] = rs.Btot - 2.0 * B + t * (2.0 * A - rs.Wv) + rs.C0 + run_q;
            }
            // the run still open at the end of this chunk carries its partial sum
            const double last = __shfl_sync(FULL, run_q, 31);
            cQrun = last;
            cA = __shfl_sync(FULL, A, 31);
            cB = __shfl_sync(FULL, B, 31);
        }
        if (end) {
            if (pos) {
                // run g (not the top one) starts at Q - 2 S(t_g), slot groups-1-g
                if (g < groups - 1) {
                    const int64_t D = Q - 2 * S;
                    a.lam[o + groups - 1 - g] = D > 0 ? fix_to_double(D, sigma) : 0.0;
                    a.val[o + groups - 1 - g] = Tr::value(keys[i]);
                }
            } else {
                // the run after g starts at 2 S(t_g) - Q; after the last, 0
                const int64_t D = 2 * S - Q;
                a.lam[o + g + 1] = D > 0 ? fix_to_double(D, sigma) : 0.0;
                a.val[o + g + 1] = g + 1 < groups ? Tr::value(keys[i + 1]) : T(0);
            }
        }
        carry = __shfl_sync(FULL, S, 31);
        gbase += __popc(em);
    }
    if (lane == 0) {
        a.lam[o] = 0.0;
        a.val[o] = v0;
        if (pos) {
            const int64_t D = Q - 2 * Sbelow;
            a.lam[o + groups] = D > 0 ? fix_to_double(D, sigma) : 0.0;
            a.val[o + groups] = T(0);
        }
        // v = 0: R = Btot - 2 B(0) + C0 with B(0) the signed sum over ratios <= 0
        if (a.res) a.res[o + groups] = rs.Btot - 2.0 * (pos ? rs.Bb : cB) + rs.C0;
        a.len[p] = groups + 1;
    }
}

// One pass over the rows of pair (j, k) by one warp.  COUNT: rows in range.
// Else: append in-range rows (exact key, row) to the list (at most cap; the
// total is returned either way) and sum the exact weight below the range.
// Without residual sums the rows are visited four per lane per step, the
// step's loads of the float copy issued together (measured 14% faster for the
// count and write passes); with them, one per lane per step (the double sums
// bound that pass, and the wider step measured 3% slower).
template <typename T, bool COUNT>
__device__ int scan_rows(const PathArgs<T> &a, int64_t j, int64_t k, const T *colb,
                         const float *inv, const int64_t *colq, bool wide, bool pos,
                         uint32_t ck_lo, uint32_t ck_hi, typename Traits<T>::K kv,
                         typename Traits<T>::K *keys, uint32_t *rows, int cap, int64_t &Sbelow,
                         RowSums &rs, int lane) {
    using Tr = Traits<T>;
    using K = typename Tr::K;
    const unsigned FULL = 0xFFFFFFFFu;
    const T *xk = a.Xt + k * a.ldn;
    const float *xf = a.Xf + k * a.ldn;
    const bool want_r = !COUNT && a.res != nullptr;
    const int n = (int)a.n;
    int c = 0;
    int64_t sb = 0;
    // one row: classify, weight below, exact key, list append
    auto visit = [&](int i, float xv, double *sums) {
        const bool inb = i < n;
        int cls = 1;
        K ke = Tr::NONE;
        const T b = inb ? colb[i] : T(0);
        const bool valid = b != T(0);
        if (valid) cls = classify<T>(xv, inv[i], xk + i, b, wide, pos, ck_lo, ck_hi, kv, ke);
        if (!COUNT) {
            if (cls < 0) sb += colq[i];
            if (cls == 0 && ke == Tr::NONE) ke = Tr::key(Tr::div_rn(xk[i], b));
        }
        if (sums && inb) {  // bt, wv, c0, ab, bb of RowSums
            // float input: the float copy is the input itself
            const double x = sizeof(T) == 4 ? (double)xv : (double)xk[i];
            const double bd = (double)b;
            if (valid) {
                const double sx = bd < 0.0 ? -x : x;
                sums[0] += sx;
                sums[1] += fabs(bd);
                if (cls < 0) {
                    sums[3] += fabs(bd);
                    sums[4] += sx;
                }
            } else {
                sums[2] += fabs(x);
            }
        }
        const unsigned im = __ballot_sync(FULL, cls == 0);
        if (!COUNT && cls == 0) {
            const int pos_i = c + __popc(im & ((1u << lane) - 1u));
            if (pos_i < cap) {
                keys[pos_i] = ke;
                rows[pos_i] = (uint32_t)i;
            }
        }
        c += __popc(im);
    };
    if (want_r) {
        double sums[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        for (int i0 = 0; i0 < n; i0 += 32) {
            const int i = i0 + lane;
            visit(i, i < n ? xf[i] : 0.0f, sums);
        }
        rs.Btot = warp_sum_f64(sums[0]);
        rs.Wv = warp_sum_f64(sums[1]);
        rs.C0 = warp_sum_f64(sums[2]);
        rs.Ab = warp_sum_f64(sums[3]);
        rs.Bb = warp_sum_f64(sums[4]);
    } else {
        constexpr int U = 4;
        for (int i0 = 0; i0 < n; i0 += 32 * U) {
            float xv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int i = i0 + u * 32 + lane;
                xv[u] = i < n ? xf[i] : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) visit(i0 + u * 32 + lane, xv[u], nullptr);
        }
    }
    if (!COUNT) Sbelow = warp_sum_i64(sb);
    __syncwarp();
    return c;
}

template <typename T>
__device__ __forceinline__ bool pair_is_wide(const PathArgs<T> &a, const ColInfo &cj, int64_t k) {
    return (cj.flags & COL_WIDE) != 0 || (sizeof(T) == 8 && (a.ci[k].flags & COL_WIDE));
}

template <typename T, bool COUNT>
__global__ void __launch_bounds__(PW * 32) k_path_pass(PathArgs<T> a, int kchunk) {
    using Tr = Traits<T>;
    using K = typename Tr::K;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int npad = ((int)a.n + 31) & ~31;
    T *colb = reinterpret_cast<T *>(smem);
    size_t o = al16((size_t)npad * sizeof(T));
    float *inv = reinterpret_cast<float *>(smem + o);
    o += al16((size_t)npad * 4);
    int64_t *colq = reinterpret_cast<int64_t *>(smem + o);
    o += al16((size_t)npad * 8);
    K *keys = reinterpret_cast<K *>(smem + o + (size_t)warp * PATH_CAP * (sizeof(K) + 4));
    uint32_t *rows = reinterpret_cast<uint32_t *>(keys + PATH_CAP);
    const int64_t j = blockIdx.x;
    stage_column<T>(a, j, colb, inv, colq, npad);
    __syncthreads();
    const ColInfo cj = a.ci[j];
    const int64_t k0 = (int64_t)blockIdx.y * kchunk, k1 = min(a.m, k0 + kchunk);
    for (int64_t k = k0 + warp; k < k1; k += PW) {
        const int64_t p = j * a.m + k;
        const T v0 = a.v0[p];
        if (k == j || v0 == T(0) || cj.n_valid == 0) {  // constant path
            double r = 0.0;  // v = 1 for k == jhat: zero residual; v = 0: sum |x_ik|
            if (!COUNT && a.res && k != j) {
                const T *xk = a.Xt + k * a.ldn;
                for (int i = lane; i < (int)a.n; i += 32) r += fabs((double)xk[i]);
                r = warp_sum_f64(r);
            }
            if (lane == 0) {
                if (COUNT) {
                    a.bound[p] = 1;
                } else {
                    const int64_t off = a.off[p];
                    a.lam[off] = 0.0;
                    a.val[off] = k == j ? T(1) : T(0);
                    if (a.res) a.res[off] = r;
                    a.len[p] = 1;
                }
            }
            continue;
        }
        bool pos;
        uint32_t ck_lo, ck_hi;
        K kv;
        range_of<T>(v0, pos, ck_lo, ck_hi, kv);
        const bool wide = pair_is_wide<T>(a, cj, k);
        int64_t Sbelow = 0;
        RowSums rs{};
        const int c = scan_rows<T, COUNT>(a, j, k, colb, inv, colq, wide, pos, ck_lo, ck_hi, kv,
                                          keys, rows, PATH_CAP, Sbelow, rs, lane);
        if (COUNT) {
            if (lane == 0) a.bound[p] = (int64_t)c + 1;
            continue;
        }
        if (c > PATH_CAP) {  // the big-pair kernel takes it
            if (lane == 0) a.big[atomicAdd(a.big_count, 1u)] = (int32_t)(p);
            continue;
        }
        int P = 32;
        while (P < c) P <<= 1;
        warp_list_sort<K>(keys, rows, c, P, lane);
        emit_path<T>(a, p, v0, pos, keys, rows, c, colq, cj.Q, Sbelow, cj.sigma, colb,
                     a.Xt + k * a.ldn, rs, lane);
        __syncwarp();
    }
}

// Pairs with more rows in range than a warp's shared list: one warp per pair,
// the list in a global scratch slice (a pair's rows never exceed n).
template <typename T>
__global__ void __launch_bounds__(128) k_path_big(PathArgs<T> a) {
    using Tr = Traits<T>;
    using K = typename Tr::K;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;  // worker warp
    const int npad = ((int)a.n + 31) & ~31;
    unsigned char *sl = a.scratch + (size_t)gw * (size_t)a.slice * (sizeof(K) + 4 + sizeof(T) + 12);
    K *keys = reinterpret_cast<K *>(sl);
    uint32_t *rows = reinterpret_cast<uint32_t *>(keys + a.slice);
    // the column arrays of jhat live in the slice too (each warp may hold a different jhat)
    T *cb = reinterpret_cast<T *>(rows + a.slice);
    float *ci_inv = reinterpret_cast<float *>(cb + a.slice);
    int64_t *cq = reinterpret_cast<int64_t *>(ci_inv + a.slice);
    const uint32_t total = *a.big_count;
    for (;;) {
        uint32_t w = 0;
        if (lane == 0) w = atomicAdd(a.big_next, 1u);
        w = __shfl_sync(0xFFFFFFFFu, w, 0);
        if (w >= total) break;
        const int64_t p = a.big[w];
        const int64_t j = p / a.m, k = p - j * a.m;
        const ColInfo cj = a.ci[j];
        const T *xj = a.Xt + j * a.ldn;
        for (int i = lane; i < npad; i += 32) {
            const T b = i < a.n ? xj[i] : T(0);
            cb[i] = b;
            ci_inv[i] = b != T(0) ? Approx<T>::inv_of(b) : 0.0f;
            int e = 0;
            cq[i] = b != T(0) ? fixq(b < T(0) ? -b : b, cj.sigma, e) : 0;
        }
        __syncwarp();
        const T v0 = a.v0[p];
        bool pos;
        uint32_t ck_lo, ck_hi;
        K kv;
        range_of<T>(v0, pos, ck_lo, ck_hi, kv);
        int64_t Sbelow = 0;
        RowSums rs{};
        const int c = scan_rows<T, false>(a, j, k, cb, ci_inv, cq, pair_is_wide<T>(a, cj, k), pos,
                                          ck_lo, ck_hi, kv, keys, rows, (int)a.slice, Sbelow,
                                          rs, lane);
        int P = 32;
        while (P < c) P <<= 1;
        warp_list_sort<K>(keys, rows, c, P, lane);
        emit_path<T>(a, p, v0, pos, keys, rows, c, cq, cj.Q, Sbelow, cj.sigma, cb,
                     a.Xt + k * a.ldn, rs, lane);
        __syncwarp();
    }
}

// Exclusive scan of bound[0..N) into off[0..N] (off[N] = total), three steps.
constexpr int SCAN_B = 1024;
__global__ void __launch_bounds__(SCAN_B) k_scan_blocks(const int64_t *in, int64_t *out,
                                                        int64_t *bsum, int64_t N) {
    __shared__ int64_t ws[32];
    const int64_t i = (int64_t)blockIdx.x * SCAN_B + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t x = i < N ? in[i] : 0;
    const int64_t incl = warp_scan_add(x, lane);
    if (lane == 31) ws[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int64_t v = ws[lane];
        ws[lane] = warp_scan_add(v, lane) - v;
    }
    __syncthreads();
    const int64_t e = ws[warp] + incl - x;
    if (i < N) out[i] = e;
    if (threadIdx.x == SCAN_B - 1) bsum[blockIdx.x] = e + x;
}

__global__ void __launch_bounds__(SCAN_B) k_scan_tops(int64_t *bsum, int64_t nb, int64_t *total) {
    __shared__ int64_t ws[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t carry = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += SCAN_B) {
        const int64_t b = b0 + threadIdx.x;
        const int64_t x = b < nb ? bsum[b] : 0;
        const int64_t incl = warp_scan_add(x, lane);
        if (lane == 31) ws[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const int64_t v = ws[lane];
            ws[lane] = warp_scan_add(v, lane) - v;
        }
        __syncthreads();
        const int64_t e = carry + ws[warp] + incl - x;
        if (b < nb) bsum[b] = e;
        __syncthreads();
        if (threadIdx.x == SCAN_B - 1) ws[0] = e + x;
        __syncthreads();
        carry = ws[0];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_add(int64_t *out, const int64_t *bsum, int64_t N) {
    const int64_t i = (int64_t)blockIdx.x * SCAN_B + threadIdx.x;
    if (i < N) out[i] += bsum[blockIdx.x];
}

}  // namespace

size_t path_scan_scratch(int64_t N) { return (size_t)((N + SCAN_B - 1) / SCAN_B) * 8; }

cudaError_t launch_scan_i64(int64_t *a, int64_t N, int64_t *tmp, cudaStream_t st, int &launches) {
    const int64_t nb = (N + SCAN_B - 1) / SCAN_B;
    k_scan_blocks<<<(unsigned)nb, SCAN_B, 0, st>>>(a, a, tmp, N);
    k_scan_tops<<<1, SCAN_B, 0, st>>>(tmp, nb, a + N);
    k_scan_add<<<(unsigned)nb, SCAN_B, 0, st>>>(a, tmp, N);
    launches += 3;
    return cudaGetLastError();
}
int path_big_workers() { return 64; }

template <typename T> size_t path_slice_bytes(int64_t n) {
    int64_t P = 32;
    while (P < n) P <<= 1;
    return (size_t)P * (sizeof(typename Traits<T>::K) + 4 + sizeof(T) + 12);
}

template <typename T> size_t path_smem_bytes(int64_t n) {
    const int npad = ((int)n + 31) & ~31;
    return al16((size_t)npad * sizeof(T)) + al16((size_t)npad * 4) + al16((size_t)npad * 8) +
           (size_t)PW * PATH_CAP * (sizeof(typename Traits<T>::K) + 4);
}

// Largest n whose staged column and lists fit one CTA of the path kernels
// (and that the fit, which solves lambda = 0, accepts).
template <typename T> int64_t path_max_rows() {
    int64_t n = 32;
    while (n + 32 <= max_rows_pairs<T>() && path_smem_bytes<T>(n + 32) <= 227 * 1024) n += 32;
    return n;
}

template <typename T>
cudaError_t launch_path(bool count, const T *Xt, const float *Xf, const ColInfo *ci, int64_t n,
                        int64_t m, int64_t ldn, const T *v0, int64_t *bound_or_off,
                        int64_t *scan_tmp, double *lam, T *val, double *res, int32_t *len,
                        int32_t *big, uint32_t *big_count, unsigned char *scratch,
                        uint32_t *status, int num_sms, cudaStream_t st, int &launches) {
    PathArgs<T> a{};
    a.Xt = Xt;
    a.Xf = Xf;
    a.ci = ci;
    a.n = n;
    a.m = m;
    a.ldn = ldn;
    a.v0 = v0;
    a.status = status;
    const size_t smem = path_smem_bytes<T>(n);
    const int64_t chunks = std::max<int64_t>(1, std::min<int64_t>((m + PW - 1) / PW,
                                                                  (num_sms * 8 + m - 1) / m));
    const int kchunk = (int)((m + chunks - 1) / chunks);
    dim3 grid((unsigned)m, (unsigned)((m + kchunk - 1) / kchunk));
    cudaError_t e;
    if (count) {
        a.bound = bound_or_off;
        auto kern = k_path_pass<T, true>;
        if ((e = ensure_smem(reinterpret_cast<const void *>(kern), smem)) != cudaSuccess) return e;
        kern<<<grid, PW * 32, smem, st>>>(a, kchunk);
        launches++;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        // exclusive scan of the m*m bounds, in place, total at [m*m]
        return launch_scan_i64(bound_or_off, m * m, scan_tmp, st, launches);
    }
    a.off = bound_or_off;
    a.lam = lam;
    a.val = val;
    a.res = res;
    a.len = len;
    a.big = big;
    a.big_count = big_count;
    a.big_next = big_count + 1;
    a.scratch = scratch;
    int64_t P = 32;
    while (P < n) P <<= 1;
    a.slice = P;
    if ((e = cudaMemsetAsync(big_count, 0, 2 * sizeof(uint32_t), st)) != cudaSuccess) return e;
    auto kern = k_path_pass<T, false>;
    if ((e = ensure_smem(reinterpret_cast<const void *>(kern), smem)) != cudaSuccess) return e;
    kern<<<grid, PW * 32, smem, st>>>(a, kchunk);
    launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_path_big<T><<<path_big_workers() / 4, 128, 0, st>>>(a);
    launches++;
    return cudaGetLastError();
}

template size_t path_slice_bytes<float>(int64_t);
template size_t path_slice_bytes<double>(int64_t);
template int64_t path_max_rows<float>();
template int64_t path_max_rows<double>();
template cudaError_t launch_path<float>(bool, const float *, const float *, const ColInfo *,
                                        int64_t, int64_t, int64_t, const float *, int64_t *,
                                        int64_t *, double *, float *, double *, int32_t *,
                                        int32_t *, uint32_t *, unsigned char *, uint32_t *, int,
                                        cudaStream_t, int &);
template cudaError_t launch_path<double>(bool, const double *, const float *, const ColInfo *,
                                         int64_t, int64_t, int64_t, const double *, int64_t *,
                                         int64_t *, double *, double *, double *, int32_t *,
                                         int32_t *, uint32_t *, unsigned char *, uint32_t *, int,
                                         cudaStream_t, int &);

L1L_CHECKS_READER(l1l_checks_path)

}  // namespace l1l
