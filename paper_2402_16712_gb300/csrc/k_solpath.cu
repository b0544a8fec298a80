// k_solpath.cu -- Algorithm 3: the solution path over all lambda >= 0.
//
// From the pair paths of Algorithm 2 (with each entry's residual R), the
// objective of preserved coordinate jhat is z_jhat(lambda) = sum_k (R + lambda
// |v|) of the entry of pair (jhat, k) holding at lambda: piecewise linear and
// concave in lambda.  Algorithm 3 finds, interval by interval, which jhat's
// line is lowest and where two lines cross (beta_L, beta_U).  Here the same
// result comes from two GPU steps:
//   1. per jhat (one CTA), merge the m sorted entry lists of its pairs by
//      lambda (a tree of merge-path merges, one warp per merge) and prefix-sum
//      the changes of intercept and slope: the pieces (lambda_start, I, s) of
//      z_jhat;
//   2. the lower envelope min_jhat z_jhat by a tree of pairwise minimum
//      merges (one thread sweeps two concave functions; each piece of either
//      contributes at most one interval to their minimum, so a merge never
//      outgrows its inputs).
// The root's pieces are the solution path: from lambda_start on, jhat* and
// z* = I + s lambda; v* is read from the pair paths of jhat*.
#include <cmath>

#include "common.cuh"
#include "launch.h"
#include "pairs.cuh"

namespace l1l {

namespace {

struct Piece {
    double lam;    // start of the piece (for deltas: where the change happens)
    double I, s;   // intercept and slope (for deltas: their changes)
    int32_t owner; // jhat
    int32_t pad;
};
static_assert(sizeof(Piece) == 32, "piece layout");

constexpr int ZB = 512;  // threads of the per-jhat build kernel

// Deltas of jhat: count = 1 (the base) + sum_k (len_k - 1).
__global__ void __launch_bounds__(256) k_zcount(const int32_t *len, int64_t m, int64_t *cnt) {
    const int64_t j = blockIdx.x;
    int64_t c = 0;
    for (int64_t k = threadIdx.x; k < m; k += blockDim.x) c += len[j * m + k] - 1;
    c = warp_sum_i64(c);
    __shared__ int64_t ws[8];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t t = 1;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
        cnt[j] = t;
    }
}

// Stable merge of sorted A[0..na) and B[0..nb) (by lam; A first on ties) into
// out, by one warp: lane l produces outputs [l*L/32, (l+1)*L/32).
__device__ void warp_merge(const Piece *A, int64_t na, const Piece *B, int64_t nb, Piece *out,
                           int lane) {
    const int64_t L = na + nb;
    const int64_t d0 = L * lane / 32, d1 = L * (lane + 1) / 32;
    // merge-path split for diagonal d: i elements from A, d - i from B
    auto split = [&](int64_t d) -> int64_t {
        int64_t lo = d > nb ? d - nb : 0, hi = d < na ? d : na;
        while (lo < hi) {
            const int64_t i = (lo + hi) >> 1;
            // take A[i] before B[d-1-i] when A[i].lam <= B[d-1-i].lam
            if (A[i].lam <= B[d - 1 - i].lam)
                lo = i + 1;
            else
                hi = i;
        }
        return lo;
    };
    int64_t i = split(d0), jx = d0 - i;
    for (int64_t d = d0; d < d1; ++d) {
        const bool takeA = jx >= nb || (i < na && A[i].lam <= B[jx].lam);
        out[d] = takeA ? A[i++] : B[jx++];
    }
}

// Block-wide exclusive scan of one int64 / double per thread (fixed order).
template <typename V> __device__ V block_excl_scan(V x, V *sm, V &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    V incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const V y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
    }
    __syncthreads();
    if (lane == 31) sm[warp] = incl;
    __syncthreads();
    V before = 0, tot = 0;
    for (int w = 0; w < nw; ++w) {
        if (w < warp) before += sm[w];
        tot += sm[w];
    }
    total = tot;
    return before + incl - x;
}

// Build z_jhat's pieces for jhat = blockIdx.x.  Buffers A and B hold this
// jhat's region [base, base + cnt); runs of the merge tree are tracked in
// rs0 / rs1 (m + 2 starts each, per jhat).  The pieces end in P at base, their
// count in pcount[jhat].
template <typename T>
__global__ void __launch_bounds__(ZB) k_zbuild(int64_t m, const int64_t *off, const int32_t *len,
                                                const double *lam, const T *val, const double *res,
                                                const int64_t *dbase, Piece *A, Piece *B,
                                                int64_t *rs0, int64_t *rs1, Piece *P,
                                                int64_t *pcount) {
    __shared__ double smd[ZB / 32];
    __shared__ int64_t smi[ZB / 32];
    __shared__ int64_t s_carry;
    const int64_t j = blockIdx.x;
    const int64_t base = dbase[j], cnt = dbase[j + 1] - base;
    int64_t *st0 = rs0 + j * (m + 2), *st1 = rs1 + j * (m + 2);
    Piece *a = A + base, *b = B + base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = ZB / 32;
    // run starts: run 0 = the base element, run k + 1 = pair k's changes
    if (threadIdx.x == 0) s_carry = 1;
    __syncthreads();
    for (int64_t k0 = 0; k0 < m; k0 += ZB) {
        const int64_t k = k0 + threadIdx.x;
        const int64_t c = k < m ? (int64_t)len[j * m + k] - 1 : 0;
        int64_t tot;
        const int64_t ex = block_excl_scan<int64_t>(c, smi, tot);
        if (k < m) st0[k + 1] = s_carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) s_carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        st0[0] = 0;
        st0[m + 1] = cnt;
    }
    __syncthreads();
    // fill: the base (sum of first entries) and each pair's changes
    double I0 = 0.0, s0 = 0.0;
    for (int64_t k = warp; k < m; k += nw) {
        const int64_t p = j * m + k, o = off[p], L = len[p];
        if (lane == 0) {
            I0 += res[o];
            s0 += fabs((double)val[o]);
        }
        const int64_t dst = st0[k + 1];
        for (int64_t g = 1 + lane; g < L; g += 32) {
            Piece d;
            d.lam = lam[o + g];
            d.I = res[o + g] - res[o + g - 1];
            d.s = fabs((double)val[o + g]) - fabs((double)val[o + g - 1]);
            d.owner = (int32_t)j;
            d.pad = 0;
            a[dst + g - 1] = d;
        }
    }
    double tI;
    {
        double x = I0;
        block_excl_scan<double>(x, smd, tI);
    }
    double ts;
    {
        double x = s0;
        block_excl_scan<double>(x, smd, ts);
    }
    if (threadIdx.x == 0) {
        Piece d;
        d.lam = 0.0;
        d.I = tI;
        d.s = ts;
        d.owner = (int32_t)j;
        d.pad = 0;
        a[0] = d;
    }
    __syncthreads();
    // merge tree over the m + 1 runs
    int64_t runs = m + 1;
    Piece *src = a, *dstb = b;
    int64_t *sa = st0, *sb = st1;
    while (runs > 1) {
        const int64_t pairs = runs / 2;
        for (int64_t r = warp; r < pairs; r += nw) {
            const int64_t x0 = sa[2 * r], x1 = sa[2 * r + 1], x2 = sa[2 * r + 2];
            warp_merge(src + x0, x1 - x0, src + x1, x2 - x1, dstb + x0, lane);
        }
        if (runs & 1) {  // the unpaired last run is copied
            const int64_t x0 = sa[runs - 1], x1 = sa[runs];
            for (int64_t e = x0 + threadIdx.x; e < x1; e += ZB) dstb[e] = src[e];
        }
        __syncthreads();
        const int64_t nr = (runs + 1) / 2;
        for (int64_t r = threadIdx.x; r < nr; r += ZB) sb[r] = sa[2 * r];
        if (threadIdx.x == 0) sb[nr] = sa[runs];
        __syncthreads();
        runs = nr;
        Piece *t = src;
        src = dstb;
        dstb = t;
        int64_t *u = sa;
        sa = sb;
        sb = u;
    }
    // prefix sums of the changes, one piece per distinct lambda (the last
    // change at that lambda closes it)
    const int64_t chunk = (cnt + ZB - 1) / ZB;
    const int64_t e0 = min(cnt, (int64_t)threadIdx.x * chunk), e1 = min(cnt, e0 + chunk);
    // Neumaier-compensated running sums (each thread's chunk, then the chunk
    // totals by a block scan)
    auto nadd = [](double &sum, double &comp, double x) {
        const double t = sum + x;
        comp += fabs(sum) >= fabs(x) ? (sum - t) + x : (x - t) + sum;
        sum = t;
    };
    double lI = 0.0, ls = 0.0, lIc = 0.0, lsc = 0.0;
    int64_t nends = 0;
    for (int64_t e = e0; e < e1; ++e) {
        nadd(lI, lIc, src[e].I);
        nadd(ls, lsc, src[e].s);
        nends += (e == cnt - 1 || src[e + 1].lam != src[e].lam) ? 1 : 0;
    }
    lI += lIc;
    ls += lsc;
    double totI, tots;
    int64_t totn;
    const double bI = block_excl_scan<double>(lI, smd, totI);
    const double bs = block_excl_scan<double>(ls, smd, tots);
    const int64_t bn = block_excl_scan<int64_t>(nends, smi, totn);
    double cI = bI, cs = bs, cIc = 0.0, csc = 0.0;
    int64_t w = bn;
    Piece *out = P + base;
    for (int64_t e = e0; e < e1; ++e) {
        nadd(cI, cIc, src[e].I);
        nadd(cs, csc, src[e].s);
        if (e == cnt - 1 || src[e + 1].lam != src[e].lam) {
            Piece q;
            q.lam = src[e].lam;
            q.I = cI + cIc;
            q.s = cs + csc;
            q.owner = (int32_t)j;
            q.pad = 0;
            out[w++] = q;
        }
    }
    if (threadIdx.x == 0) pcount[j] = totn;
}

// Minimum of two concave piecewise-linear functions F, G (pieces ordered by
// start, both starting at 0), written to out; returns the piece count.
// Intercepts and slopes are double sums of many terms, so values and slopes
// that agree to a relative 1e-12 are taken as equal: equal lines go to the
// smaller owner, and lines of equal slope never cross (far beyond the last
// breakpoint every slope is exactly 1 and rounding would otherwise invent a
// crossing).
constexpr double SOL_RTOL = 1e-12;
// The winner(s) on one elementary interval [cur, end) where F is the line f
// and G the line g: calls emit(line, start) once or twice (a crossing).
template <typename E>
__device__ __forceinline__ void interval_min(const Piece &f, const Piece &g, double cur,
                                             double end, E &&emit) {
    double dI = f.I - g.I, ds = f.s - g.s;  // (f - g)(lambda) = dI + ds lambda
    if (fabs(ds) <= SOL_RTOL * fmax(fabs(f.s), fabs(g.s))) ds = 0.0;
    double d0 = dI + ds * cur;
    if (fabs(d0) <= SOL_RTOL * (fabs(f.I) + fabs(g.I) + (fabs(f.s) + fabs(g.s)) * cur)) d0 = 0.0;
    const bool f_first =
        d0 < 0.0 || (d0 == 0.0 && (ds < 0.0 || (ds == 0.0 && f.owner <= g.owner)));
    emit(f_first ? f : g, cur);
    if (ds != 0.0) {
        const double x = -dI / ds;  // the lines cross at x
        if (x > cur && x < end) {
            // past the crossing, f is lower exactly when f - g decreases
            const bool f_after = ds < 0.0;
            if (f_after != f_first) emit(f_after ? f : g, x);
        }
    }
}

__device__ __forceinline__ bool same_line(const Piece &a, const Piece &b) {
    return a.owner == b.owner && a.I == b.I && a.s == b.s;
}

constexpr int EB = 256;  // threads per envelope merge

// Minimum of two concave piecewise-linear functions F (a pieces) and G (b
// pieces), both starting at 0, by one CTA.  The merged sequence of piece
// starts is split evenly (merge path); each thread handles the elementary
// intervals that end at its consumed starts: a counting pass, a block scan of
// the counts (dropping a thread's first piece when it repeats the previous
// thread's last one), then the writing pass.  Returns the piece count, or -1
// when it would exceed cap.
__device__ int64_t block_min_merge(const Piece *F, int64_t a, const Piece *G, int64_t b,
                                   Piece *out, int64_t cap) {
    __shared__ int64_t s_cnt[EB / 32];
    __shared__ int s_last[EB];
    __shared__ Piece s_lastp[EB], s_firstp[EB];
    const int t = threadIdx.x;
    const int64_t L = a + b;
    const int64_t p0 = L * t / EB, p1 = L * (t + 1) / EB;
    // merge-path split: i starts of F among the first p0 consumed
    int64_t lo = p0 > b ? p0 - b : 0, hi = p0 < a ? p0 : a;
    while (lo < hi) {
        const int64_t i = (lo + hi) >> 1;
        if (F[i].lam <= G[p0 - 1 - i].lam)
            lo = i + 1;
        else
            hi = i;
    }
    const int64_t i_start = lo, j_start = p0 - lo;
    // one walk, run twice: count (write == false) or write at base
    auto walk = [&](bool write, int64_t base, bool drop_first, Piece &first, Piece &last,
                    int64_t &count) {
        int64_t i = i_start, j = j_start, w = 0;
        bool have = false;
        Piece prev;
        auto emit = [&](const Piece &ln, double start) {
            if (have && same_line(prev, ln)) return;
            if (!have) first = ln;
            const bool skip = !have && drop_first;
            have = true;
            prev = ln;
            if (skip) return;
            if (write && base + w < cap) {
                Piece q = ln;
                q.lam = start;
                out[base + w] = q;
            }
            ++w;
        };
        for (int64_t p = p0; p < p1; ++p) {
            if (j >= b || (i < a && F[i].lam <= G[j].lam))
                ++i;
            else
                ++j;
            if (i < 1 || j < 1) continue;
            const double cur = fmax(F[i - 1].lam, G[j - 1].lam);
            const double end = fmin(i < a ? F[i].lam : INFINITY, j < b ? G[j].lam : INFINITY);
            if (!(cur < end)) continue;
            interval_min(F[i - 1], G[j - 1], cur, end, emit);
        }
        if (have) last = prev;
        count = w;
        return have;
    };
    Piece first{}, last{};
    int64_t c = 0;
    const bool have = walk(false, 0, false, first, last, c);
    s_last[t] = have ? t : -1;
    s_lastp[t] = last;
    s_firstp[t] = first;
    __syncthreads();
    // nearest earlier thread that produced a piece (its last line)
    int prev_t = -1;
    for (int u = t - 1; u >= 0; --u)
        if (s_last[u] >= 0) {
            prev_t = u;
            break;
        }
    const bool drop = have && prev_t >= 0 && same_line(s_lastp[prev_t], s_firstp[t]);
    const int64_t mine = c - (drop ? 1 : 0);
    // block exclusive scan of the counts
    int64_t incl = mine;
    const int lane = t & 31, warp = t >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_cnt[warp] = incl;
    __syncthreads();
    int64_t before = 0, total = 0;
    for (int w = 0; w < EB / 32; ++w) {
        if (w < warp) before += s_cnt[w];
        total += s_cnt[w];
    }
    const int64_t base = before + incl - mine;
    int64_t c2 = 0;
    walk(true, base, drop, first, last, c2);
    __syncthreads();
    return total > cap ? -1 : total;
}

// One level of the envelope tree, one CTA per merge: function i (a multiple
// of 2 * half) absorbs function i + half.  Regions at dbase[i]; counts in
// pcount[i]; a piece count beyond the region sets status bit ST_INTERNAL.
__global__ void __launch_bounds__(EB) k_envelope_level(int64_t m, int64_t half,
                                                        const int64_t *dbase, const Piece *in,
                                                        Piece *outb, int64_t *pcount,
                                                        uint32_t *status) {
    const int64_t i = (int64_t)blockIdx.x * 2 * half;
    if (i >= m) return;
    const int64_t bi = dbase[i];
    const int64_t a = pcount[i];
    if (i + half < m) {
        const int64_t bg = dbase[i + half];
        const int64_t cap = dbase[min(m, i + 2 * half)] - bi;
        const int64_t r = block_min_merge(in + bi, a, in + bg, pcount[i + half], outb + bi, cap);
        if (threadIdx.x == 0) {
            if (r < 0) atomicOr(status, ST_INTERNAL);
            pcount[i] = r < 0 ? cap : r;
        }
    } else {
        for (int64_t e = threadIdx.x; e < a; e += blockDim.x) outb[bi + e] = in[bi + e];
    }
}

// v* of each solution piece: for pair (jhat*, k), the value holding just
// after the piece's start (last entry whose lambda is <= the start).
template <typename T>
__global__ void k_solution_v(int64_t m, int64_t cap, const int64_t *pcount, const Piece *env,
                             const int64_t *off, const int32_t *len, const double *lam,
                             const T *val, T *out_v) {
    const int64_t count = min(pcount[0], cap);
    for (int64_t e = blockIdx.x; e < count; e += gridDim.x) {
    const Piece p = env[e];
    const int64_t j = p.owner;
    for (int64_t k = threadIdx.x; k < m; k += blockDim.x) {
        const int64_t q = j * m + k, o = off[q], L = len[q];
        int64_t lo = 0, hi = L;  // first entry with lam > start
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (lam[o + mid] <= p.lam)
                lo = mid + 1;
            else
                hi = mid;
        }
        out_v[e * m + k] = val[o + (lo > 0 ? lo - 1 : 0)];
    }
    }
}

__global__ void k_solution_out(const Piece *env, const int64_t *pcount, int64_t cap,
                               double *start, int32_t *jhat, double *I, double *s,
                               int64_t *count) {
    const int64_t c = pcount[0];
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < min(c, cap);
         e += (int64_t)gridDim.x * blockDim.x) {
        start[e] = env[e].lam;
        jhat[e] = env[e].owner;
        I[e] = env[e].I;
        s[e] = env[e].s;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *count = c;
}

}  // namespace

// Workspace: dbase [m+1], pcount [m], run starts 2 x m (m+2), scan scratch,
// then three piece buffers of (entries + m).
size_t solpath_bytes(int64_t m, int64_t entries) {
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    size_t o = 256;  // status word
    o += al((size_t)(m + 1) * 8);
    o += al((size_t)m * 8);
    o += 2 * al((size_t)m * (m + 2) * 8);
    o += al(path_scan_scratch(m));
    o += 3 * al((size_t)(entries + m) * sizeof(Piece));
    return o;
}

template <typename T>
cudaError_t launch_solpath(int64_t m, const int64_t *off, const int32_t *len, const double *lam,
                           const T *val, const double *res, unsigned char *ws, int64_t entries,
                           double *out_start, int32_t *out_jhat, double *out_I, double *out_s,
                           T *out_v, int64_t *out_count, int64_t cap, cudaStream_t st,
                           int &launches) {
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    size_t o = 0;
    uint32_t *status = reinterpret_cast<uint32_t *>(ws + o);  // read by l1line_status
    o += 256;
    int64_t *dbase = reinterpret_cast<int64_t *>(ws + o);
    o += al((size_t)(m + 1) * 8);
    int64_t *pcount = reinterpret_cast<int64_t *>(ws + o);
    o += al((size_t)m * 8);
    int64_t *rs0 = reinterpret_cast<int64_t *>(ws + o);
    o += al((size_t)m * (m + 2) * 8);
    int64_t *rs1 = reinterpret_cast<int64_t *>(ws + o);
    o += al((size_t)m * (m + 2) * 8);
    int64_t *stmp = reinterpret_cast<int64_t *>(ws + o);
    o += al(path_scan_scratch(m));
    const size_t pb = al((size_t)(entries + m) * sizeof(Piece));
    Piece *A = reinterpret_cast<Piece *>(ws + o);
    Piece *B = reinterpret_cast<Piece *>(ws + o + pb);
    Piece *P = reinterpret_cast<Piece *>(ws + o + 2 * pb);
    cudaError_t e;
    if ((e = cudaMemsetAsync(status, 0, sizeof(uint32_t), st)) != cudaSuccess) return e;
    k_zcount<<<(unsigned)m, 256, 0, st>>>(len, m, dbase);
    launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_scan_i64(dbase, m, stmp, st, launches)) != cudaSuccess) return e;
    k_zbuild<T><<<(unsigned)m, ZB, 0, st>>>(m, off, len, lam, val, res, dbase, A, B, rs0, rs1, P,
                                            pcount);
    launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // envelope: ping-pong between P and A
    Piece *in = P, *outb = A;
    for (int64_t half = 1; half < m; half *= 2) {
        const int64_t merges = (m + 2 * half - 1) / (2 * half);
        k_envelope_level<<<(unsigned)merges, EB, 0, st>>>(m, half, dbase, in, outb, pcount,
                                                          status);
        launches++;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        Piece *t = in;
        in = outb;
        outb = t;
    }
    k_solution_out<<<64, 256, 0, st>>>(in, pcount, cap, out_start, out_jhat, out_I, out_s,
                                       out_count);
    launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (out_v) {
        k_solution_v<T><<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(cap, 4096)), 128, 0,
                          st>>>(m, cap, pcount, in, off, len, lam, val, out_v);
        launches++;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template cudaError_t launch_solpath<float>(int64_t, const int64_t *, const int32_t *,
                                           const double *, const float *, const double *,
                                           unsigned char *, int64_t, double *, int32_t *,
                                           double *, double *, float *, int64_t *, int64_t,
                                           cudaStream_t, int &);
template cudaError_t launch_solpath<double>(int64_t, const int64_t *, const int32_t *,
                                            const double *, const double *, const double *,
                                            unsigned char *, int64_t, double *, int32_t *,
                                            double *, double *, double *, int64_t *, int64_t,
                                            cudaStream_t, int &);

L1L_CHECKS_READER(l1l_checks_solpath)

}  // namespace l1l
