// common.cuh -- shared device helpers of the sm_103a hot path.
//
// Notation follows the paper (Lemma 1, Algorithm 1): X is n x m with rows the
// points x_i; jhat is the preserved coordinate, k another coordinate;
// r_i = x_ik / x_ijhat, w_i = |x_ijhat|, lambda the penalty.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace l1l {

// ---------------------------------------------------------------------------
// Status bits written to the workspace status word (atomicOr).
// ---------------------------------------------------------------------------
enum : uint32_t {
    ST_NONFINITE = 1u << 0,
    ST_INTERNAL = 1u << 1,
    ST_TIMEOUT = 1u << 2,    // reserved: no kernel waits on another
    ST_BADINDEX = 1u << 3,  // a jhat list entry outside [0, m)
};

// ---------------------------------------------------------------------------
// Order-preserving integer image of a ratio ("key").  -0 maps like +0, so the
// zero ratio and the penalty point share one key.  Negative values map below
// KEY0 (the key of 0), positive above.  The all-ones key never arises from a
// finite or infinite ratio and marks "no element".
// ---------------------------------------------------------------------------
template <typename T> struct Traits;

template <> struct Traits<float> {
    using K = uint32_t;
    static constexpr K KEY0 = 0x80000000u;
    static constexpr K NONE = 0xFFFFFFFFu;
    static constexpr int KEY_BITS = 32;
    static __device__ __forceinline__ K key(float r) {
        uint32_t u = __float_as_uint(r);
        if (u == 0x80000000u) u = 0u;
        return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    }
    static __device__ __forceinline__ float value(K k) {
        uint32_t u = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
        return __uint_as_float(u);
    }
    static __device__ __forceinline__ float div_rn(float a, float b) { return __fdiv_rn(a, b); }
};

template <> struct Traits<double> {
    using K = uint64_t;
    static constexpr K KEY0 = 0x8000000000000000ull;
    static constexpr K NONE = 0xFFFFFFFFFFFFFFFFull;
    static constexpr int KEY_BITS = 64;
    static __device__ __forceinline__ K key(double r) {
        uint64_t u = (uint64_t)__double_as_longlong(r);
        if (u == 0x8000000000000000ull) u = 0ull;
        return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
    }
    static __device__ __forceinline__ double value(K k) {
        uint64_t u = (k & 0x8000000000000000ull) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
        return __longlong_as_double((long long)u);
    }
    static __device__ __forceinline__ double div_rn(double a, double b) { return __ddiv_rn(a, b); }
};

// ---------------------------------------------------------------------------
// Fixed-point weights.  Per column jhat a scale sigma is chosen so that every
// weight w_i = |x_ijhat| maps to q_i = floor(w_i * 2^sigma) < 2^(61 - L) with
// L = ceil(log2(n_valid + 1)); the column total Q = sum q_i then stays below
// 2^61 and 2*S - Q fits an int64 with room to spare.  A weight whose lowest
// set bit lies below 2^-sigma loses bits ("inexact"); the column records how
// many did, and the decision logic widens its certainty margin by that count.
// ---------------------------------------------------------------------------
struct ColInfo {
    int64_t Q;          // sum of q_i over valid rows
    int32_t sigma;      // scale exponent
    int32_t n_valid;    // rows with x_ijhat != 0
    int32_t n_inexact;  // rows whose q_i was truncated
    int32_t flags;      // COL_WIDE: magnitudes outside the approximate-key range
    // The same weights at 32 bits (float input's fast path): q32_i =
    // q_i >> shift32 = floor(w_i 2^(sigma - shift32)), with shift32 the
    // fewest bits that bring the total Q32 below 2^32, so every partial sum
    // of q32 fits a uint32 exactly.  n_inexact32 counts the rows whose q32
    // was truncated (the certainty band of the 32-bit decisions).
    uint32_t Q32;
    int32_t shift32;
    int32_t n_inexact32;
    // sum_i |x_i| bounded above, as a float: (Q + n_inexact) 2^-sigma rounded up
    // (the certificate of the float-float residual of double pairs reads it)
    float l1_up;
};

// A column is "wide" when some nonzero |x| lies outside the range in which the
// reciprocal-multiply approximation of a ratio is within the guard band of
// the correctly rounded ratio (float: 2^-126 <= |x_ijhat| < 2^126, so 1/x is a
// normal float; double: 2^-60 <= |x| < 2^60 for both columns of a pair, so
// every float intermediate stays normal).  Pairs touching such a column take
// the exact path.
enum : int32_t { COL_WIDE = 1 };
template <typename T> struct WideRange;
template <> struct WideRange<float> { static constexpr int lo = -126, hi = 125; };
template <> struct WideRange<double> { static constexpr int lo = -60, hi = 59; };

__device__ __forceinline__ int64_t fixq(float w, int sigma, int &inexact) {
    uint32_t u = __float_as_uint(w) & 0x7FFFFFFFu;
    uint32_t be = u >> 23;
    uint32_t mant = u & 0x7FFFFFu;
    if (be) mant |= 0x800000u;
    int s = (be ? (int)be : 1) - 150 + sigma;
    if (s >= 0) return (int64_t)((uint64_t)mant << s);
    int rs = -s;
    if (rs >= 32) {
        inexact |= (mant != 0);
        return 0;
    }
    inexact |= ((mant & ((1u << rs) - 1u)) != 0);
    return (int64_t)(mant >> rs);
}

__device__ __forceinline__ int64_t fixq(double w, int sigma, int &inexact) {
    uint64_t u = (uint64_t)__double_as_longlong(w) & 0x7FFFFFFFFFFFFFFFull;
    uint64_t be = u >> 52;
    uint64_t mant = u & 0xFFFFFFFFFFFFFull;
    if (be) mant |= 0x10000000000000ull;
    int s = (be ? (int)be : 1) - 1075 + sigma;
    if (s >= 0) return (int64_t)(mant << s);
    int rs = -s;
    if (rs >= 64) {
        inexact |= (mant != 0);
        return 0;
    }
    inexact |= ((mant & ((1ull << rs) - 1ull)) != 0);
    return (int64_t)(mant >> rs);
}

// floor(log2(w)) for finite w != 0, read off the bit pattern (subnormals
// included).
__device__ __forceinline__ int ilog2_pos(float w) {
    uint32_t u = __float_as_uint(w) & 0x7FFFFFFFu;
    int be = (int)(u >> 23);
    if (be) return be - 127;
    return (31 - __clz((int)u)) - 149;
}
__device__ __forceinline__ int ilog2_pos(double w) {
    uint64_t u = (uint64_t)__double_as_longlong(w) & 0x7FFFFFFFFFFFFFFFull;
    int be = (int)(u >> 52);
    if (be) return be - 1023;
    return (63 - __clzll((long long)u)) - 1074;
}

// ---------------------------------------------------------------------------
// Exact decision.  With S = (fixed-point) weight of valid rows whose key is
// <= t, the test of Lemma 1 "weight at or below t exceeds W/2", W including
// lambda and the penalty point counted when t >= 0, reads
//     t <  0:  2 S - Q  >  lambda'        t >= 0:  2 S - Q  >  -lambda'
// with lambda' = lambda * 2^sigma.  For integer D = 2S - Q this is
// D > floor(y).  When some weights were truncated (e = n_inexact > 0) the
// true D lies in (D - e, D + 2e) and the answer is certain only outside that
// band; otherwise the pair is handed to the exact wide-accumulator path.
// ---------------------------------------------------------------------------
struct Decide {
    int64_t Q;
    int64_t Lf;  // floor(lambda'), saturated at 2^62
    int64_t Lc;  // ceil(lambda'),  saturated at 2^62
    int64_t e;   // n_inexact

    __device__ __forceinline__ void init(const ColInfo &ci, double lambda) {
        init_at(ci.Q, ci.sigma, ci.n_inexact, lambda);
    }
    // The same test on the 32-bit weights q32 (scale sigma - shift32).
    __device__ __forceinline__ void init32(const ColInfo &ci, double lambda) {
        init_at((int64_t)ci.Q32, ci.sigma - ci.shift32, ci.n_inexact32, lambda);
    }
    __device__ __forceinline__ void init_at(int64_t Qs, int sigma, int64_t inexact,
                                            double lambda) {
        Q = Qs;
        e = inexact;
        const int64_t SAT = (int64_t)1 << 62;
        if (lambda == 0.0) {
            Lf = Lc = 0;
        } else {
            double lp = ldexp(lambda, sigma);
            if (!(lp < 4611686018427387904.0)) {
                Lf = Lc = SAT;
            } else if (lp < 1.0) {
                Lf = 0;
                Lc = 1;
            } else {
                Lf = (int64_t)floor(lp);
                Lc = (int64_t)ceil(lp);
            }
        }
    }
    // 1 = true, 0 = false, -1 = undecidable at this precision.
    __device__ __forceinline__ int cond(int64_t S, bool t_nonneg) const {
        int64_t D = 2 * S - Q;
        if (e == 0) return t_nonneg ? (D > -Lc) : (D > Lf);
        if (t_nonneg) {
            if (D - e >= -Lf) return 1;
            if (D + 2 * e <= -Lc) return 0;
        } else {
            if (D - e >= Lc) return 1;
            if (D + 2 * e <= Lf) return 0;
        }
        return -1;
    }
};

// ---------------------------------------------------------------------------
// Warp helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t warp_sum_i64(int64_t x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
    return x;
}
__device__ __forceinline__ int warp_sum_i32(int x) { return __reduce_add_sync(0xFFFFFFFFu, x); }
__device__ __forceinline__ float warp_sum_f32(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
    return x;
}
__device__ __forceinline__ double warp_sum_f64(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
    return x;
}

// Pair-list entry for the exact slow path.
struct SlowEntry {
    int32_t t;       // lambda index
    int32_t j;       // jhat
    int32_t k;
    int16_t inst;    // instance (batched calls), 0 otherwise
    int16_t reason;  // why the fast path gave up (SEL_* code), for diagnostics
};

// Shapes and device pointers of one scan, passed by value to every kernel.
template <typename T> struct ScanArgs {
    const T *Xt;       // [m][ldn] column-major copy of X
    const float *Xf;   // the same rounded to float (== Xt for float input); double
                       // input: [2][m][ldn], the remainders x - fl(x) second
    const ColInfo *ci;  // [m]
    int64_t n, m, ldn;
    int32_t n_lambda;
    T *v_all;          // [n_lambda][m][m]
    double *s_all;     // [n_lambda][m][m]
    uint32_t *status;  // workspace status word
    uint32_t *slow_count;
    SlowEntry *slow;   // capacity n_lambda * m * m
    int force_exact;
    int inst;          // instance index recorded in slow-list entries (batched calls)
    const int32_t *jlist;  // device list of the jhat to score (nullptr: all m)
    int64_t nj;            // entries of jlist (m when jlist is nullptr)
    int d0;                // first-bracket half-width of the selection, sample positions
};

// Default first-bracket half-width (of NSAMP = 64 weight-proportional samples).
// +-6 samples keep ~15-20% of the rows as candidates and rarely miss the
// median; narrower brackets (d0 = 4) are faster when the weights are not
// concentrated in few rows (5% outliers) but miss often when they are (20%
// outlier rows holding most of the weight), so the narrower choice is left to
// the autotuner, which measures it per shape.
constexpr int D0_DEFAULT = 6;

constexpr int MAX_LAMBDA_PER_LAUNCH = 256;

// Rows of the staged column-major copy (and of the pair kernel's shared
// column arrays) are padded with zeros to a multiple of ROW_PAD, so that the
// selection's unrolled passes (4 loads of 32 rows per lane group) never need
// a bound check: a padding row has a zero reciprocal and is not a valid row.
constexpr int ROW_PAD = 128;

// ---------------------------------------------------------------------------
// A batch of independent instances, described entirely by value so that the
// launches can be captured in a CUDA graph without host-memory copies.
// Instances are listed in processing order (largest work first); each owns a
// region of the workspace laid out by inst_layout().
// ---------------------------------------------------------------------------
constexpr int MAX_BATCH = 256;
constexpr int MAX_BATCH_LAMBDAS = 512;

template <typename T> struct BatchInst {
    const T *X;         // caller's row-major n x m matrix
    int64_t ws_off;     // this instance's workspace region
    int64_t out_v_off;  // first element of its v* rows in out_v
    int32_t n, m, ldn, nl;
    int32_t out_t_off;  // first slot of its objectives / jhat* in out_obj / out_jstar
    int16_t tl_min, tl_max;
};

template <typename T> struct BatchDesc {
    int32_t count;       // instances
    int32_t tiles;       // transpose tiles over all instances
    int64_t units;       // (instance, jhat) work units
    int32_t ztasks;      // (instance, lambda, jhat) objective sums
    int32_t lams;        // lambdas over all instances
    int32_t force_exact;
    int32_t d0;          // first-bracket half-width of the selection
    BatchInst<T> inst[MAX_BATCH];
    int64_t unit_begin[MAX_BATCH + 1];  // prefix of m over instances
    int32_t tile_begin[MAX_BATCH + 1];
    int32_t ztask_begin[MAX_BATCH + 1];  // prefix of nl * m
    int32_t lam_begin[MAX_BATCH + 1];    // prefix of nl (also the index into lam)
    double lam[MAX_BATCH_LAMBDAS];
};

// Layout of one instance's workspace region (host and device agree on it).
struct InstLayout {
    size_t ci, Xt, Xf, v_all, s_all, z_all, total;
};
__host__ __device__ inline size_t al256b(size_t x) { return (x + 255) & ~size_t(255); }
__host__ __device__ inline InstLayout inst_layout(int64_t m, int64_t ldn, int64_t nl, size_t es) {
    InstLayout L;
    size_t o = 0;
    L.ci = o;
    o = al256b(o + (size_t)m * sizeof(ColInfo));
    L.Xt = o;
    o = al256b(o + (size_t)m * (size_t)ldn * es);
    L.Xf = es == 8 ? o : L.Xt;  // double input: float copy, then its remainders
    if (es == 8) o = al256b(o + (size_t)m * (size_t)ldn * 8);
    L.v_all = o;
    o = al256b(o + (size_t)nl * (size_t)m * (size_t)m * es);
    L.s_all = o;
    o = al256b(o + (size_t)nl * (size_t)m * (size_t)m * 8);
    L.z_all = o;
    o = al256b(o + (size_t)nl * (size_t)m * 8);
    L.total = o;
    return L;
}
// Batch-wide workspace head: status word (@0), exact-path counter (@256), one
// unit counter per size class (@512 + 8 c).
constexpr size_t BATCH_HEAD = 768;
struct LambdaPack {
    double lam[MAX_LAMBDA_PER_LAUNCH];
    int tl_min, tl_max;  // positions of the smallest and largest lambda of the launch
};

}  // namespace l1l
