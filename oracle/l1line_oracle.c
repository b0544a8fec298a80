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
