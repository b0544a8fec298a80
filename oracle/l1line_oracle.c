/*
 * l1line_oracle.c -- plain, slow CPU oracle for the l1-regularised l1 best-fit
 * line of Ling & Brooks (arXiv 2402.16712).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the tests, the smoke check and the bench's CPU-baseline
 * leg use it.  It shares no code, header, table or helper with the CUDA path.
 *
 * What it computes, for every penalty lambda, every preserved coordinate jhat
 * and every other coordinate k (Lemma 1 and Algorithm 1):
 *
 *   I   = { i : x[i][jhat] != 0 }
 *   r_i = fl(x[i][k] / x[i][jhat])     IEEE round-to-nearest, input precision
 *   w_i = |x[i][jhat]|
 *   B   = { (r_i, w_i) : i in I }  U  { (0, lambda) }      (penalty point)
 *   W   = sum_{i in I} w_i + lambda
 *   v_k = min { t in values(B) : sum_{(r,w) in B, r <= t} w  >  W / 2 }
 *
 * i.e. the weighted median of the ratios with the penalty point at zero; when
 * the minimiser of sum_i |x_ik - t x_ijhat| + lambda |t| is an interval this
 * is its right end point, which is what Algorithm 1's half-open test with
 * "last index wins" selects (Algorithm 1, inner loop).  v_jhat = 1.  If W = 0
 * (column jhat all zero and lambda = 0) no t qualifies and v_k keeps
 * Algorithm 1's initial value 0.
 *
 *   z_jhat = sum_i sum_k |x_ik - v_k x_ijhat| + lambda sum_k |v_k|   (Algorithm 1)
 *   jhat*  = smallest jhat attaining min z_jhat  (strict "z < z*" scanned in
 *            increasing jhat, Algorithm 1)
 *
 * Method: literally the paper's -- collect the list, sort it by ratio, scan
 * the cumulative weight.  The test "2 S(<=t) > W" is decided EXACTLY: the
 * running difference  D = sum_{r<=t} w - sum_{r>t} w  is kept in a
 * Kulisch-style long fixed-point accumulator whose unit is 2^-1074 (every
 * finite double is an integer multiple of it), so no rounding enters the
 * decision.  The objective is summed in double with Neumaier's compensated
 * summation; for float input every product v*x is exact in double.
 *
 * Build: plain C11, no fast-math, no FMA contraction (-ffp-contract=off),
 * optional OpenMP over jhat.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* Kulisch-style exact accumulator                                     */
/* ------------------------------------------------------------------ */
/* Two's complement integer of KL_LIMBS*64 bits; one unit = 2^-1074.
 * A finite double is mant * 2^(e) with mant < 2^53 and the unit position of
 * its lowest bit in [0, 2045], so it occupies bits [0, 2098).  36 limbs give
 * 2304 bits: sums of up to 2^200 doubles cannot overflow. */
#define KL_LIMBS 36

typedef struct {
    uint64_t limb[KL_LIMBS];
} kacc;

static void kacc_zero(kacc *a) { memset(a->limb, 0, sizeof(a->limb)); }

/* a += sgn * |x| * mult, mult in {1,2}; x finite. */
static void kacc_add(kacc *a, double x, int negate) {
    uint64_t bits;
    memcpy(&bits, &x, sizeof(bits));
    uint64_t bexp = (bits >> 52) & 0x7FF;
    uint64_t mant = bits & ((UINT64_C(1) << 52) - 1);
    if (bexp == 0 && mant == 0) return;
    unsigned shift;
    if (bexp) {
        mant |= UINT64_C(1) << 52;
        shift = (unsigned)(bexp - 1);
    } else {
        shift = 0; /* subnormal: value = mant * 2^-1074 */
    }
    int neg = ((bits >> 63) & 1) ^ (negate ? 1 : 0);
    unsigned idx = shift / 64, off = shift % 64;
    uint64_t lo = mant << off;
    uint64_t hi = off ? (mant >> (64 - off)) : 0;
    if (!neg) {
        uint64_t s = a->limb[idx] + lo;
        uint64_t c = s < lo;
        a->limb[idx] = s;
        unsigned j = idx + 1;
        uint64_t addend = hi;
        while (j < KL_LIMBS && (addend || c)) {
            uint64_t t = a->limb[j] + addend;
            uint64_t c1 = t < addend;
            uint64_t t2 = t + c;
            uint64_t c2 = t2 < c;
            a->limb[j] = t2;
            c = c1 | c2;
            addend = 0;
            j++;
        }
    } else {
        uint64_t s = a->limb[idx] - lo;
        uint64_t b = a->limb[idx] < lo;
        a->limb[idx] = s;
        unsigned j = idx + 1;
        uint64_t sub = hi;
        while (j < KL_LIMBS && (sub || b)) {
            uint64_t cur = a->limb[j];
            uint64_t t = cur - sub;
            uint64_t b1 = cur < sub;
            uint64_t t2 = t - b;
            uint64_t b2 = t < b;
            a->limb[j] = t2;
            b = b1 | b2;
            sub = 0;
            j++;
        }
    }
}

/* -1, 0 or +1 */
static int kacc_sign(const kacc *a) {
    if (a->limb[KL_LIMBS - 1] >> 63) return -1;
    for (int j = 0; j < KL_LIMBS; j++)
        if (a->limb[j]) return 1;
    return 0;
}

/* Exact sign of sum(vals[0..cnt)); exported so the tests can pin the
 * accumulator against an independent exact summation. */
int oracle_sign_of_sum(const double *vals, int64_t cnt) {
    kacc a;
    kacc_zero(&a);
    for (int64_t i = 0; i < cnt; i++) kacc_add(&a, vals[i], 0);
    return kacc_sign(&a);
}

/* ------------------------------------------------------------------ */
/* Weighted median of ratios for one (jhat, k) pair (Lemma 1)          */
/* ------------------------------------------------------------------ */
typedef struct {
    double r; /* ratio, already rounded to the input precision; -0 -> +0 */
    double w; /* weight |x_ijhat|, or lambda for the penalty point        */
} rw_t;

static int cmp_rw(const void *pa, const void *pb) {
    double a = ((const rw_t *)pa)->r, b = ((const rw_t *)pb)->r;
    return (a > b) - (a < b);
}

/* list[0..cnt) holds the ratios and weights, penalty point included.
 * Returns the chosen value, or 0 when no point satisfies the test (W = 0). */
static double weighted_median_exact(rw_t *list, int64_t cnt) {
    qsort(list, (size_t)cnt, sizeof(rw_t), cmp_rw);
    kacc D; /* D = sum_{r<=t} w - sum_{r>t} w = 2 S(<=t) - W */
    kacc_zero(&D);
    for (int64_t p = 0; p < cnt; p++) kacc_add(&D, list[p].w, 1);
    int64_t p = 0;
    while (p < cnt) {
        double t = list[p].r;
        while (p < cnt && list[p].r == t) {
            kacc_add(&D, list[p].w, 0);
            kacc_add(&D, list[p].w, 0);
            p++;
        }
        if (kacc_sign(&D) > 0) return t == 0.0 ? 0.0 : t;
    }
    return 0.0;
}

/* ------------------------------------------------------------------ */
/* Neumaier compensated sum                                            */
/* ------------------------------------------------------------------ */
typedef struct {
    double s, c;
} nsum;

static void nsum_add(nsum *a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x))
        a->c += (a->s - t) + x;
    else
        a->c += (x - t) + a->s;
    a->s = t;
}

static double nsum_get(const nsum *a) { return a->s + a->c; }

/* ------------------------------------------------------------------ */
/* Per-precision bodies                                                */
/* ------------------------------------------------------------------ */
#define ORACLE_OK 0
#define ORACLE_ERR_ARG -1
#define ORACLE_ERR_NONFINITE -2
#define ORACLE_ERR_ALLOC -3

#define DEFINE_ORACLE(SUFFIX, T, ABS)                                                     \
    /* One pair: a = column k (n values, stride sa), b = column jhat (stride sb). */      \
    static T pair_##SUFFIX(const T *a, int64_t sa, const T *b, int64_t sb, int64_t n,     \
                           double lambda, rw_t *scratch) {                                \
        int64_t cnt = 0;                                                                  \
        for (int64_t i = 0; i < n; i++) {                                                 \
            T bi = b[i * sb];                                                             \
            if (bi != (T)0) {                                                             \
                volatile T r = a[i * sa] / bi; /* rounded to T */                         \
                T rr = r;                                                                 \
                scratch[cnt].r = (rr == (T)0) ? 0.0 : (double)rr;                         \
                scratch[cnt].w = (double)ABS(bi);                                         \
                cnt++;                                                                    \
            }                                                                             \
        }                                                                                 \
        scratch[cnt].r = 0.0;                                                             \
        scratch[cnt].w = lambda;                                                          \
        cnt++;                                                                            \
        return (T)weighted_median_exact(scratch, cnt);                                    \
    }                                                                                     \
                                                                                          \
    int oracle_pair_##SUFFIX(const T *a, const T *b, int64_t n, double lambda, T *v_out) { \
        if (n < 0 || !v_out || (n > 0 && (!a || !b)) || !(lambda >= 0) || isinf(lambda))  \
            return ORACLE_ERR_ARG;                                                        \
        rw_t *scratch = (rw_t *)malloc(sizeof(rw_t) * (size_t)(n + 1));                   \
        if (!scratch) return ORACLE_ERR_ALLOC;                                            \
        *v_out = pair_##SUFFIX(a, 1, b, 1, n, lambda, scratch);                           \
        free(scratch);                                                                    \
        return ORACLE_OK;                                                                 \
    }                                                                                     \
                                                                                          \
    /* Full fit over the jhat listed in jlist (all jhat when jlist == NULL).             \
     * X row-major n x m.  Outputs (any may be NULL except where noted):                 \
     *   v_all [nl][m][m]  v^jhat for every lambda and jhat (rows for unlisted jhat      \
     *                     are left untouched)                                           \
     *   s_all [nl][m][m]  per-pair residual sum_i |x_ik - v_k x_ijhat| + lambda|v_k|    \
     *   z_all [nl][m]     z_jhat (NaN for unlisted jhat)                                \
     *   out_v [nl][m], out_obj [nl], out_jstar [nl]   the argmin over listed jhat.      \
     */                                                                                   \
    int oracle_fit_##SUFFIX(const T *X, int64_t n, int64_t m, const double *lambdas,      \
                            int64_t nl, const int32_t *jlist, int64_t nj, T *v_all,       \
                            double *s_all, double *z_all, T *out_v, double *out_obj,      \
                            int32_t *out_jstar, int nthreads) {                           \
        if (n < 1 || m < 1 || nl < 1 || !X || !lambdas) return ORACLE_ERR_ARG;            \
        for (int64_t t = 0; t < nl; t++)                                                  \
            if (!(lambdas[t] >= 0) || isinf(lambdas[t])) return ORACLE_ERR_ARG;           \
        for (int64_t e = 0; e < n * m; e++)                                               \
            if (!isfinite((double)X[e])) return ORACLE_ERR_NONFINITE;                     \
        if (!jlist) nj = m;                                                               \
        if (nj < 1) return ORACLE_ERR_ARG;                                                \
        for (int64_t q = 0; jlist && q < nj; q++)                                         \
            if (jlist[q] < 0 || jlist[q] >= m) return ORACLE_ERR_ARG;                     \
        T *vbuf = (T *)malloc(sizeof(T) * (size_t)(nl * nj * m));                         \
        double *zbuf = (double *)malloc(sizeof(double) * (size_t)(nl * nj));              \
        if (!vbuf || !zbuf) {                                                             \
            free(vbuf);                                                                   \
            free(zbuf);                                                                   \
            return ORACLE_ERR_ALLOC;                                                      \
        }                                                                                 \
        int failed = 0;                                                                   \
        int nth = nthreads > 0 ? nthreads : 1;                                            \
        (void)nth;                                                                        \
        _Pragma("omp parallel num_threads(nth)") {                                        \
            rw_t *scratch = (rw_t *)malloc(sizeof(rw_t) * (size_t)(n + 1));               \
            if (!scratch) {                                                               \
                _Pragma("omp atomic write") failed = 1;                                   \
            }                                                                             \
            _Pragma("omp for schedule(dynamic, 1)") for (int64_t q = 0; q < nj; q++) {    \
                if (!scratch) continue;                                                   \
                int64_t jh = jlist ? jlist[q] : q;                                        \
                const T *b = X + jh;                                                      \
                for (int64_t t = 0; t < nl; t++) {                                        \
                    double lam = lambdas[t];                                              \
                    T *v = vbuf + (t * nj + q) * m;                                       \
                    for (int64_t k = 0; k < m; k++)                                       \
                        v[k] = (k == jh) ? (T)1 : pair_##SUFFIX(X + k, m, b, m, n, lam,   \
                                                                scratch);                 \
                    nsum z = {0.0, 0.0};                                                  \
                    for (int64_t k = 0; k < m; k++) {                                     \
                        nsum s = {0.0, 0.0};                                              \
                        for (int64_t i = 0; i < n; i++) {                                 \
                            double prod = (double)v[k] * (double)b[i * m];                \
                            double term = fabs((double)X[i * m + k] - prod);              \
                            nsum_add(&s, term);                                           \
                            nsum_add(&z, term);                                           \
                        }                                                                 \
                        double pen = lam * fabs((double)v[k]);                            \
                        nsum_add(&s, pen);                                                \
                        nsum_add(&z, pen);                                                \
                        if (s_all) s_all[(t * m + jh) * m + k] = nsum_get(&s);            \
                    }                                                                     \
                    zbuf[t * nj + q] = nsum_get(&z);                                      \
                }                                                                         \
            }                                                                             \
            free(scratch);                                                                \
        }                                                                                 \
        if (failed) {                                                                     \
            free(vbuf);                                                                   \
            free(zbuf);                                                                   \
            return ORACLE_ERR_ALLOC;                                                      \
        }                                                                                 \
        for (int64_t t = 0; t < nl; t++) {                                                \
            if (z_all)                                                                    \
                for (int64_t j = 0; j < m; j++) z_all[t * m + j] = NAN;                   \
            int64_t best = -1;                                                            \
            double zbest = INFINITY;                                                      \
            /* scan in increasing jhat, strict "<" keeps the smallest index on ties */    \
            for (int64_t j = 0; j < m; j++) {                                             \
                int64_t q = -1;                                                           \
                if (!jlist)                                                               \
                    q = j;                                                                \
                else                                                                      \
                    for (int64_t u = 0; u < nj; u++)                                      \
                        if (jlist[u] == j) {                                              \
                            q = u;                                                        \
                            break;                                                        \
                        }                                                                 \
                if (q < 0) continue;                                                      \
                double zj = zbuf[t * nj + q];                                             \
                if (z_all) z_all[t * m + j] = zj;                                         \
                if (v_all) memcpy(v_all + (t * m + j) * m, vbuf + (t * nj + q) * m,       \
                                  sizeof(T) * (size_t)m);                                 \
                if (best < 0 || zj < zbest) {                                             \
                    zbest = zj;                                                           \
                    best = q;                                                             \
                }                                                                         \
            }                                                                             \
            int64_t jbest = jlist ? jlist[best] : best;                                   \
            if (out_obj) out_obj[t] = zbest;                                              \
            if (out_jstar) out_jstar[t] = (int32_t)jbest;                                 \
            if (out_v) memcpy(out_v + t * m, vbuf + (t * nj + best) * m,                  \
                              sizeof(T) * (size_t)m);                                     \
        }                                                                                 \
        free(vbuf);                                                                       \
        free(zbuf);                                                                       \
        return ORACLE_OK;                                                                 \
    }

DEFINE_ORACLE(f64, double, fabs)
DEFINE_ORACLE(f32, float, fabsf)

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Algorithm 2: the lambda path of one pair                            */
/* ------------------------------------------------------------------ */
/* Exact value of a rounded to the nearest double (ties to even). */
static double kacc_to_double(const kacc *a) {
    kacc m = *a;
    const int neg = kacc_sign(a) < 0;
    if (neg) { /* two's complement negation */
        uint64_t c = 1;
        for (int j = 0; j < KL_LIMBS; j++) {
            uint64_t t = ~m.limb[j] + c;
            c = (c && t == 0) ? 1 : 0;
            m.limb[j] = t;
        }
    }
    int top = -1;
    for (int j = KL_LIMBS - 1; j >= 0 && top < 0; j--)
        if (m.limb[j])
            for (int b = 63; b >= 0; b--)
                if ((m.limb[j] >> b) & 1) {
                    top = j * 64 + b;
                    break;
                }
    if (top < 0) return 0.0;
    double v;
    if (top <= 52) { /* fits 53 bits: exact (subnormal range included) */
        v = ldexp((double)m.limb[0], -1074);
    } else {
        const int shift = top - 52;
        /* the 53 bits [shift, top] */
        const int li = shift / 64, lo = shift % 64;
        uint64_t f = m.limb[li] >> lo;
        if (lo && li + 1 < KL_LIMBS) f |= m.limb[li + 1] << (64 - lo);
        uint64_t mant = f & ((UINT64_C(1) << 53) - 1);
        const int rb = shift - 1;
        const int round = (int)((m.limb[rb / 64] >> (rb % 64)) & 1);
        int sticky = 0;
        for (int b = 0; b < rb && !sticky; b++)
            if ((m.limb[b / 64] >> (b % 64)) & 1) sticky = 1;
        int e = shift;
        if (round && (sticky || (mant & 1))) {
            mant++;
            if (mant == (UINT64_C(1) << 53)) {
                mant >>= 1;
                e++;
            }
        }
        v = ldexp((double)mant, e - 1074);
    }
    return neg ? -v : v;
}

typedef struct {
    double lam;
    double v;
} bp_t;

static int cmp_bp(const void *pa, const void *pb) {
    const bp_t *a = (const bp_t *)pa, *b = (const bp_t *)pb;
    if (a->lam != b->lam) return (a->lam > b->lam) - (a->lam < b->lam);
    const double x = fabs(a->v), y = fabs(b->v); /* then moving toward 0 */
    return (x < y) - (x > y);
}

/* list[0..cnt): (ratio, weight) of the rows with x_ijhat != 0 (no penalty
 * point).  Writes the path into out (capacity cnt + 2; the merged result
 * has at most cnt + 1 entries) and returns its length.  Steps of Algorithm 2 for one (jhat, j): sort the ratios; for each
 * sorted position p, lambda_p = sgn(r_p) (S_after - S_before) - w_p (exact);
 * a row with lambda_p + 2 w_p > 0 starts the value r_p at max(0, lambda_p);
 * lambda_max = max(0, max_p lambda_p + 2 w_p) starts the value 0.  Readings
 * (the paper is silent): a zero ratio is the penalty point itself, so such a
 * row starts nothing (it still counts in the sums); the path starts with
 * Algorithm 1's value at lambda = 0, v0; breakpoints are ordered by lambda
 * and, at equal lambda, by decreasing |v|; consecutive equal values are
 * merged, keeping the first lambda.  Meaning: v(0) = the first value; on the
 * open interval between consecutive breakpoints, the later entry's value; at
 * a breakpoint lambda > 0, the earlier value when it is positive (the test
 * of Lemma 1 is strict there) and the later one when it is negative. */
static void kacc_neg(kacc *a) { /* a = -a (two's complement) */
    uint64_t c = 1;
    for (int j = 0; j < KL_LIMBS; j++) {
        const uint64_t t = ~a->limb[j] + c;
        c = (c && t == 0) ? 1 : 0;
        a->limb[j] = t;
    }
}

static void kacc_addk(kacc *a, const kacc *b) { /* a += b */
    uint64_t cy = 0;
    for (int j = 0; j < KL_LIMBS; j++) {
        const uint64_t s = a->limb[j] + b->limb[j];
        const uint64_t c1 = s < b->limb[j];
        const uint64_t s2 = s + cy;
        const uint64_t c2 = s2 < cy;
        a->limb[j] = s2;
        cy = c1 | c2;
    }
}

static int64_t path_pair(rw_t *list, int64_t cnt, double v0, bp_t *out) {
    qsort(list, (size_t)cnt, sizeof(rw_t), cmp_rw);
    kacc Q, before;
    kacc_zero(&Q);
    kacc_zero(&before);
    for (int64_t p = 0; p < cnt; p++) kacc_add(&Q, list[p].w, 0);
    int64_t e = 0;
    double lmax = 0.0;
    /* Algorithm 1's value at lambda = 0 (right end point of the minimiser
     * interval); when that interval is not a point, Algorithm 2's strict test
     * drops this value, which then holds at lambda = 0 only. */
    out[e].lam = 0.0;
    out[e].v = v0;
    e++;
    for (int64_t p = 0; p < cnt; p++) {
        const double r = list[p].r, w = list[p].w;
        if (r != 0.0) {
            /* x = S_after - S_before = Q - 2 S_before - w */
            kacc x = Q, nb = before;
            kacc_neg(&nb);
            kacc_addk(&x, &nb);
            kacc_addk(&x, &nb);
            kacc_add(&x, w, 1);
            /* lam_p = sgn(r) x - w;  lam_p + 2 w = sgn(r) x + w */
            if (r < 0.0) kacc_neg(&x);
            kacc lam = x, top = x;
            kacc_add(&lam, w, 1);
            kacc_add(&top, w, 0);
            if (kacc_sign(&top) > 0) {
                out[e].lam = kacc_sign(&lam) > 0 ? kacc_to_double(&lam) : 0.0;
                out[e].v = r;
                e++;
                const double tv = kacc_to_double(&top);
                if (tv > lmax) lmax = tv;
            }
        }
        kacc_add(&before, w, 0);
    }
    out[e].lam = lmax;
    out[e].v = 0.0;
    e++;
    qsort(out, (size_t)e, sizeof(bp_t), cmp_bp);
    int64_t k = 0;
    for (int64_t p = 0; p < e; p++)
        if (k == 0 || out[p].v != out[k - 1].v) out[k++] = out[p];
    return k;
}

/* The lambda path of v_k for preserved coordinate jhat (Algorithm 2), X
 * row-major n x m.  Writes up to cap entries: out_lam (double, increasing)
 * and out_v (the value from that lambda on).  k == jhat gives (0, 1).
 * Returns the path length, or -(length) when cap is too small, or an
 * ORACLE_ERR_* code (all <= -1 ... callers check cap >= n + 1 first). */
#define DEFINE_PATH(SUFFIX, T, ABS)                                                        \
    int64_t oracle_path_##SUFFIX(const T *X, int64_t n, int64_t m, int64_t jh, int64_t k,   \
                                 double *out_lam, T *out_v, int64_t cap) {                 \
        if (!X || n < 1 || m < 1 || jh < 0 || jh >= m || k < 0 || k >= m || cap < n + 1)   \
            return ORACLE_ERR_ARG;                                                         \
        if (k == jh) {                                                                     \
            out_lam[0] = 0.0;                                                              \
            out_v[0] = (T)1;                                                               \
            return 1;                                                                      \
        }                                                                                  \
        rw_t *list = (rw_t *)malloc(sizeof(rw_t) * (size_t)n);                             \
        /* before merging: v0, one entry per row, and the final 0 */                      \
        bp_t *bp = (bp_t *)malloc(sizeof(bp_t) * (size_t)(n + 2));                         \
        if (!list || !bp) {                                                                \
            free(list);                                                                    \
            free(bp);                                                                      \
            return ORACLE_ERR_ALLOC;                                                       \
        }                                                                                  \
        rw_t *med = (rw_t *)malloc(sizeof(rw_t) * (size_t)(n + 1));                        \
        if (!med) {                                                                        \
            free(list);                                                                    \
            free(bp);                                                                      \
            return ORACLE_ERR_ALLOC;                                                       \
        }                                                                                  \
        int64_t cnt = 0;                                                                   \
        for (int64_t i = 0; i < n; i++) {                                                  \
            T b = X[i * m + jh];                                                           \
            if (b != (T)0) {                                                               \
                volatile T r = X[i * m + k] / b;                                           \
                T rr = r;                                                                  \
                list[cnt].r = (rr == (T)0) ? 0.0 : (double)rr;                             \
                list[cnt].w = (double)ABS(b);                                              \
                med[cnt] = list[cnt];                                                      \
                cnt++;                                                                     \
            }                                                                              \
        }                                                                                  \
        med[cnt].r = 0.0; /* the penalty point, weight lambda = 0 */                       \
        med[cnt].w = 0.0;                                                                  \
        const double v0 = weighted_median_exact(med, cnt + 1);                             \
        free(med);                                                                         \
        const int64_t len = path_pair(list, cnt, v0, bp);                                  \
        for (int64_t p = 0; p < len; p++) {                                                \
            out_lam[p] = bp[p].lam;                                                        \
            out_v[p] = (T)bp[p].v;                                                         \
        }                                                                                  \
        free(list);                                                                        \
        free(bp);                                                                          \
        return len;                                                                        \
    }

DEFINE_PATH(f64, double, fabs)
DEFINE_PATH(f32, float, fabsf)
