/*
 * l1line.h -- C ABI of the GB300 (sm_103a) hot path of the l1-norm
 * regularised l1-norm best-fit line (Ling & Brooks, arXiv 2402.16712).
 *
 * The method (Lemma 1 and Algorithm 1 of the paper): for data points x_i in
 * R^m (the n rows of X) and a penalty lambda >= 0, every coordinate jhat is
 * tried as the preserved coordinate with v_jhat = 1; for every other
 * coordinate k, v_k is the weighted median of the ratios x_ik / x_ijhat
 * (rows with x_ijhat != 0, weights |x_ijhat|) together with a penalty point at
 * 0 of weight lambda; the score of jhat is
 *     z_jhat = sum_i sum_k |x_ik - v_k x_ijhat| + lambda * sum_k |v_k|
 * and the fit returns the v of the smallest z (smallest jhat on ties).
 *
 * Conventions shared by every entry point
 *  - X is a DEVICE pointer to a row-major n x m matrix (row i = point x_i),
 *    n >= 1, m >= 1, all entries finite.  Pointers to device memory must be
 *    aligned to their element size.
 *  - lambdas is a HOST pointer to n_lambda >= 1 finite values >= 0; the
 *    values are copied into the launch parameters, so the host array may be
 *    reused as soon as the call returns.
 *  - Ratios are IEEE round-to-nearest divisions in the input precision; -0 is
 *    treated as +0.  The weighted-median decision "the weight at or below t
 *    exceeds half the total" is taken exactly (no rounding), so v is
 *    bit-identical to an exact evaluation of the definition.  When the
 *    minimiser is an interval, v_k is its right end point (Algorithm 1's
 *    half-open test, last index wins).  A column jhat that is all zero gets
 *    v = e_jhat (Algorithm 1's initial v_k = 0).
 *  - Objectives are double; per-pair residuals are accumulated in the input
 *    precision and combined in double.
 *  - workspace is a DEVICE buffer owned by the caller, at least
 *    l1line_workspace_bytes(...) bytes, 256-byte aligned; the library never
 *    allocates memory.  One workspace must not be used by two calls that run
 *    concurrently.
 *  - stream is a cudaStream_t (NULL = legacy default stream).  Every call is
 *    asynchronous on it.  Argument errors are reported by the return value
 *    before anything is launched.  Errors found on the device (non-finite
 *    input, an internal invariant) are recorded in the workspace and read with
 *    l1line_status(), which synchronises the stream.
 *  - Return values are l1l_status codes; none of the calls aborts.
 */
#ifndef L1LINE_H
#define L1LINE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Every entry point that enqueues work first clears a non-sticky CUDA error
 * left by an earlier, unrelated runtime call (cudaGetLastError), so that its
 * L1L_ERR_CUDA reports only its own failures; a sticky error (a lost
 * context) stays and is reported. */
typedef enum {
    L1L_OK = 0,
    L1L_ERR_ARG = -1,         /* bad argument (null, size, lambda < 0 / NaN / inf) */
    L1L_ERR_NONFINITE = -2,   /* X holds NaN or inf (reported by l1line_status)   */
    L1L_ERR_CUDA = -3,        /* a CUDA runtime call failed                        */
    L1L_ERR_WORKSPACE = -4,   /* workspace missing, too small or misaligned        */
    L1L_ERR_TIMEOUT = -5,     /* reserved: no kernel of this library waits on
                                 another, so no call returns it                    */
    L1L_ERR_UNSUPPORTED = -6, /* size beyond what the kernels support (see below)  */
    L1L_ERR_INTERNAL = -7     /* a device-side invariant failed                    */
} l1l_status;

enum { L1L_DTYPE_F32 = 0, L1L_DTYPE_F64 = 1 };

/* Flags for the *_ex entry points. */
enum {
    /* decide every pair with the exact wide-accumulator path instead of the
       fixed-point fast path (testing aid; same results, much slower) */
    L1L_FLAG_FORCE_EXACT = 1u << 0
};

/* Largest n (rows) the shared-memory pair kernel takes, per dtype (column
 * jhat is staged in one CTA's shared memory).  Scans and fits with larger n
 * run the global-memory path instead: per (lambda, jhat, k) a cluster of up
 * to 8 CTAs streams both columns from the staged copy, with a radix descent
 * over the ratio keys and the same exact decisions (Lemma 1 puts no limit on
 * n); the results obey the same bar.  n > 2^31 - 256, m > 2^31 - 1,
 * n_lambda > 65535, or m * m * min(n_lambda, 256) > 2^31 (the exact path's
 * pair list of one launch; m <= 46,340 for one lambda) return
 * L1L_ERR_UNSUPPORTED, as do the batched call, the proposer calls (features,
 * proposed fit) and the lambda-path calls for n beyond their own limits
 * (l1line_path_max_rows; the others: l1line_max_rows). */
int64_t l1line_max_rows(int dtype);

/* Bytes of device workspace needed by l1line_scan_* and l1line_fit_* for the
 * given shape; 0 on a bad argument.  Includes the per-(lambda, jhat, k) tables
 * the fit keeps internally. */
size_t l1line_workspace_bytes(int dtype, int64_t n, int64_t m, int64_t n_lambda);

/*
 * Steps A1-A5 for every (lambda, jhat, k): the weighted median v^jhat_k
 * (Lemma 1; Algorithm 1 inner loops) and z_jhat (Algorithm 1, objective line).
 *   v_all  DEVICE [n_lambda][m][m] in the input dtype: row (t, jhat) is v^jhat
 *          for lambdas[t], with v^jhat_jhat = 1.  May be NULL.
 *   s_all  DEVICE [n_lambda][m][m] double: per-pair residual
 *          sum_i |x_ik - v_k x_ijhat| + lambda |v_k|; the diagonal holds
 *          lambda (v_jhat = 1, zero residual), so z_jhat is the row sum.
 *          May be NULL.
 *   z_all  DEVICE [n_lambda][m] double: z_jhat.  May be NULL.
 */
int l1line_scan_f32(const float *X, int64_t n, int64_t m, const double *lambdas,
                    int64_t n_lambda, float *v_all, double *s_all, double *z_all,
                    void *workspace, size_t workspace_bytes, void *stream);
int l1line_scan_f64(const double *X, int64_t n, int64_t m, const double *lambdas,
                    int64_t n_lambda, double *v_all, double *s_all, double *z_all,
                    void *workspace, size_t workspace_bytes, void *stream);
/* Same with flags (L1L_FLAG_*). */
int l1line_scan_ex_f32(const float *X, int64_t n, int64_t m, const double *lambdas,
                       int64_t n_lambda, float *v_all, double *s_all, double *z_all,
                       void *workspace, size_t workspace_bytes, void *stream,
                       uint32_t flags);
int l1line_scan_ex_f64(const double *X, int64_t n, int64_t m, const double *lambdas,
                       int64_t n_lambda, double *v_all, double *s_all, double *z_all,
                       void *workspace, size_t workspace_bytes, void *stream,
                       uint32_t flags);

/*
 * Algorithm 1 for each lambda (steps A1-A6): the fitted line.
 *   out_v     DEVICE [n_lambda][m]  v* for lambdas[t] (v*[jhat*] = 1)
 *   out_obj   DEVICE [n_lambda]     z* = min_jhat z_jhat (double)
 *   out_jstar DEVICE [n_lambda]     jhat* (0-based; smallest index on ties,
 *                                   from Algorithm 1's strict "z < z*")
 */
int l1line_fit_f32(const float *X, int64_t n, int64_t m, const double *lambdas,
                   int64_t n_lambda, float *out_v, double *out_obj, int32_t *out_jstar,
                   void *workspace, size_t workspace_bytes, void *stream);
int l1line_fit_f64(const double *X, int64_t n, int64_t m, const double *lambdas,
                   int64_t n_lambda, double *out_v, double *out_obj, int32_t *out_jstar,
                   void *workspace, size_t workspace_bytes, void *stream);

/*
 * Batched fit (step A7 over independent instances of uneven size): `batch`
 * (1..256) independent problems, instance b with its own
 * X_b (DEVICE pointer, row-major ns[b] x ms[b]) and lambdas
 * lambdas[lambda_offsets[b] .. lambda_offsets[b+1]) (HOST arrays; at most 512
 * lambdas in total, lambda_offsets[0] = 0).  Each instance is fitted exactly
 * as l1line_fit_* would fit it.  Outputs are concatenated in instance order:
 *   out_v     DEVICE  instance b's [n_lambda_b][ms[b]] block starts at
 *                     sum_{b'<b} n_lambda_b' * ms[b']
 *   out_obj   DEVICE  instance b's n_lambda_b values start at lambda_offsets[b]
 *   out_jstar DEVICE  likewise (0-based jhat* per lambda)
 * The pair work runs in one persistent launch whose blocks take (instance,
 * jhat) units from an atomic counter, largest instances first.  All launch
 * parameters are passed by value; after one call with a given shape the
 * sequence issues only stream operations.  Workspace: see
 * l1line_batched_workspace_bytes (0 on a bad argument); l1line_status reads
 * its device status.
 */
size_t l1line_batched_workspace_bytes(int dtype, int64_t batch, const int64_t *ns,
                                      const int64_t *ms, const int64_t *lambda_offsets);
int l1line_fit_batched_f32(int64_t batch, const float *const *Xs, const int64_t *ns,
                           const int64_t *ms, const double *lambdas,
                           const int64_t *lambda_offsets, float *out_v, double *out_obj,
                           int32_t *out_jstar, void *workspace, size_t workspace_bytes,
                           void *stream);
int l1line_fit_batched_f64(int64_t batch, const double *const *Xs, const int64_t *ns,
                           const int64_t *ms, const double *lambdas,
                           const int64_t *lambda_offsets, double *out_v, double *out_obj,
                           int32_t *out_jstar, void *workspace, size_t workspace_bytes,
                           void *stream);

/*
 * Subset fit: Algorithm 1 restricted to the candidate jhat listed in
 * jhat_list (DEVICE int32[K], 1 <= K <= m, entries in [0, m); duplicates are
 * allowed and scored once each; K > m returns L1L_ERR_ARG).  Every k is still scanned for each listed jhat, so the
 * scores z_jhat of the listed jhat are exactly those of l1line_fit_*, and the
 * result is the listed jhat of smallest z (smallest index on ties).  Outputs
 * as for l1line_fit_*.  Workspace: l1line_workspace_bytes(dtype, n, m,
 * n_lambda).  An entry outside [0, m) is reported by l1line_status as
 * L1L_ERR_ARG (the list lives on the device, so it is checked there).
 */
int l1line_fit_subset_f32(const float *X, int64_t n, int64_t m, const double *lambdas,
                          int64_t n_lambda, const int32_t *jhat_list, int64_t K,
                          float *out_v, double *out_obj, int32_t *out_jstar,
                          void *workspace, size_t workspace_bytes, void *stream);
int l1line_fit_subset_f64(const double *X, int64_t n, int64_t m, const double *lambdas,
                          int64_t n_lambda, const int32_t *jhat_list, int64_t K,
                          double *out_v, double *out_obj, int32_t *out_jstar,
                          void *workspace, size_t workspace_bytes, void *stream);

/*
 * Algorithm 2: the lambda path of every (jhat, k) pair.  As lambda grows from
 * 0 the penalty point gains weight and v_k moves monotonically from its
 * lambda = 0 value to 0 through the distinct ratios in between.  Pair
 * p = jhat * m + k owns entries offsets[p] .. offsets[p] + out_len[p] - 1:
 * (out_lambda, out_v) with out_lambda increasing from 0 and out_v moving
 * toward 0 (the last entry is 0, except for k == jhat: one entry (0, 1)).
 * Meaning: v_k(0) = the first value; on the open interval between two
 * consecutive lambdas, the later entry's value; at an entry's lambda > 0, the
 * earlier value when that is positive and the later one when it is negative
 * (Lemma 1's test is strict).  Two entries share lambda = 0 when the lambda = 0
 * minimiser is an interval: the first (its right end point, Algorithm 1's
 * choice) holds at lambda = 0 only.  v is exact (bit-identical to
 * Algorithm 1 at every lambda); a lambda is the exact weight difference of
 * Algorithm 2, computed in fixed point (exactly, then rounded once to double,
 * when every |x_ijhat| of the column is a multiple of the column's
 * fixed-point unit; otherwise within 2^-40 of the column's l1 norm).
 *
 * Two calls with one workspace (l1line_path_workspace_bytes, 256-byte
 * aligned): l1line_path_count_* stages X, solves lambda = 0 exactly and writes
 * offsets (DEVICE int64 [m*m + 1]: an exclusive scan of per-pair upper
 * bounds; offsets[m*m] = entries to allocate); read offsets[m*m], then
 * l1line_path_write_* (same X, n, m and workspace, nothing else using the
 * workspace in between) fills out_lambda (DEVICE double), out_v (DEVICE, the
 * input dtype), both of at least offsets[m*m] entries, and out_len (DEVICE
 * int32 [m*m], the number of entries each pair used).  out_resid (DEVICE
 * double, same size, or NULL) receives each entry's residual
 * sum_i |x_ik - v x_ijhat| (double sums), so that on the entry's lambda
 * interval the pair's term of z_jhat is out_resid + lambda |out_v|.
 *
 * n is limited by the path kernels' shared memory (one staged column and
 * eight 256-entry lists per CTA): l1line_path_max_rows(dtype) returns the
 * largest n; larger n make l1line_path_workspace_bytes return 0 and the
 * calls return L1L_ERR_UNSUPPORTED.
 */
int64_t l1line_path_max_rows(int dtype);
size_t l1line_path_workspace_bytes(int dtype, int64_t n, int64_t m);
int l1line_path_count_f32(const float *X, int64_t n, int64_t m, int64_t *offsets,
                          void *workspace, size_t workspace_bytes, void *stream);
int l1line_path_count_f64(const double *X, int64_t n, int64_t m, int64_t *offsets,
                          void *workspace, size_t workspace_bytes, void *stream);
int l1line_path_write_f32(const float *X, int64_t n, int64_t m, const int64_t *offsets,
                          double *out_lambda, float *out_v, double *out_resid, int32_t *out_len,
                          void *workspace, size_t workspace_bytes, void *stream);
int l1line_path_write_f64(const double *X, int64_t n, int64_t m, const int64_t *offsets,
                          double *out_lambda, double *out_v, double *out_resid, int32_t *out_len,
                          void *workspace, size_t workspace_bytes, void *stream);

/*
 * Algorithm 3: the solution path over all lambda >= 0, from the pair paths
 * of the two calls above (with out_resid).  z_jhat(lambda) = sum_k (resid +
 * lambda |v|) over the entries holding at lambda is piecewise linear and
 * concave; the path is the lower envelope min_jhat z_jhat, as Algorithm 3's
 * per-interval line crossings (beta_L, beta_U) give it.  Outputs (DEVICE,
 * capacity cap entries): piece e holds from out_start[e] (increasing from 0)
 * to the next start: jhat* = out_jhat[e] and z* = out_intercept[e] +
 * out_slope[e] lambda; out_v (cap x m, may be NULL) receives v* on the open
 * interval after the start.  *out_count (DEVICE int64) = the number of
 * pieces (only the first cap are written).  entries = offsets[m*m].  Among
 * identical lines the smallest jhat is named.  z and crossing lambdas are
 * double sums of the residuals (relative error ~ entries x 2^-53); values and
 * slopes agreeing to a relative 1e-12 are taken as equal.  The workspace
 * (l1line_solution_path_workspace_bytes, 256-byte aligned) starts with a
 * status word that l1line_status reads.
 */
size_t l1line_solution_path_workspace_bytes(int64_t m, int64_t entries);
int l1line_solution_path_f32(int64_t m, const int64_t *offsets, const double *lambda,
                             const float *v, const double *resid, const int32_t *len,
                             int64_t entries, double *out_start, int32_t *out_jhat,
                             double *out_intercept, double *out_slope, float *out_v,
                             int64_t *out_count, int64_t cap, void *workspace,
                             size_t workspace_bytes, void *stream);
int l1line_solution_path_f64(int64_t m, const int64_t *offsets, const double *lambda,
                             const double *v, const double *resid, const int32_t *len,
                             int64_t entries, double *out_start, int32_t *out_jhat,
                             double *out_intercept, double *out_slope, double *out_v,
                             int64_t *out_count, int64_t cap, void *workspace,
                             size_t workspace_bytes, void *stream);

/*
 * Successive components (the paper's remark after Proposition 5: apply
 * Algorithm 1 again to the data projected onto the null space of the
 * components found so far).  Reading of the projection, which the paper does
 * not define: component (jhat, v) represents x_i by x_ijhat v, so the
 * projected point is the residual x_i - x_ijhat v, rounded per operation in
 * the input precision: x'_ik = fl(x_ik - fl(v_k x_ijhat)) (column jhat becomes
 * 0).  ncomp fits at one lambda, each on the data deflated by all earlier
 * components: out_v [ncomp][m], out_obj [ncomp], out_jstar [ncomp] (DEVICE).
 * Workspace: l1line_components_workspace_bytes (fit workspace + two copies
 * of X); l1line_status reads its status.
 */
size_t l1line_components_workspace_bytes(int dtype, int64_t n, int64_t m);
int l1line_components_f32(const float *X, int64_t n, int64_t m, double lambda, int64_t ncomp,
                          float *out_v, double *out_obj, int32_t *out_jstar, void *workspace,
                          size_t workspace_bytes, void *stream);
int l1line_components_f64(const double *X, int64_t n, int64_t m, double lambda, int64_t ncomp,
                          double *out_v, double *out_obj, int32_t *out_jstar, void *workspace,
                          size_t workspace_bytes, void *stream);

/*
 * Learned jhat proposer (not in the paper; an extension of Algorithm 1's
 * outer loop): a small network scores every candidate jhat from four
 * features, and only the K best-scored candidates are fitted exactly (the
 * exact objective still decides among them; the full scan stays the reference
 * for its regret).
 *
 * Features of column jhat: its l1 norm, l2 norm and the lower median of
 * |x_i,jhat| (0-based rank floor((n-1)/2) of the ascending order), and the
 * objective z_jhat of Algorithm 1 (penalty lambda) on the R =
 * l1line_proposer_rows(n) rows of X with the largest l1 norm (the double sum
 * of |x_ij| over j, left to right, rounded to float; ties to the smaller row),
 * computed by this library's own fit of those rows; each feature standardised
 * over the m columns of the instance (mean 0, population standard deviation
 * 1; a feature constant over the columns becomes 0).  Stored as float [m][4].
 *
 * Network: 4 -> 128 -> 128 -> 1, ReLU after both hidden layers; weight
 * matrices in binary16, biases in float, float arithmetic.  l1line_mlp is its
 * packed DEVICE image (35,088 bytes, 16-byte aligned); the flat float
 * parameter vector used for training holds L1L_MLP_PARAMS values in the order
 * W1 [128][4], b1 [128], W2 [128][128], b2 [128], w3 [128], b3.
 */
#define L1L_MLP_HIDDEN 128
#define L1L_MLP_FEATURES 4
#define L1L_MLP_PARAMS 17281
typedef struct l1line_mlp {
    uint16_t w1[L1L_MLP_HIDDEN * L1L_MLP_FEATURES]; /* binary16 bits, [o][c]  */
    float b1[L1L_MLP_HIDDEN];
    uint16_t w2[L1L_MLP_HIDDEN * L1L_MLP_HIDDEN]; /* binary16 bits, [o][i]  */
    float b2[L1L_MLP_HIDDEN];
    uint16_t w3[L1L_MLP_HIDDEN];                  /* binary16 bits          */
    float b3;
    float reserved[3];
} l1line_mlp;

/* Rows of the restricted fit behind the fourth feature: min(n, max(256,
 * ceil(n / 8))); 0 for n < 1. */
int64_t l1line_proposer_rows(int64_t n);

/* Bytes of device workspace l1line_features_* (n_lambda = 1) and
 * l1line_fit_proposed_* need: the fit's workspace, then the restricted fit's
 * (its rows, their copy and its own workspace); 0 on a bad argument. */
size_t l1line_proposed_workspace_bytes(int dtype, int64_t n, int64_t m, int64_t n_lambda);

/* Features of every column of X (raw and standardised, DEVICE float [m][4]
 * each; raw may be NULL); lambda (>= 0) is the penalty of the restricted
 * objective.  Workspace: l1line_proposed_workspace_bytes(dtype, n, m, 1). */
int l1line_features_f32(const float *X, int64_t n, int64_t m, double lambda, float *out_raw,
                        float *out_std, void *workspace, size_t workspace_bytes, void *stream);
int l1line_features_f64(const double *X, int64_t n, int64_t m, double lambda, float *out_raw,
                        float *out_std, void *workspace, size_t workspace_bytes, void *stream);

/* Network forward pass: scores[r] = net(feat[rows[r]]) for r < N (rows NULL:
 * row r).  feat DEVICE float [*][4], rows DEVICE int32 [N] or NULL, mlp
 * DEVICE, scores DEVICE float [N]. */
int l1line_mlp_forward(const float *feat, const int32_t *rows, int64_t N,
                       const l1line_mlp *mlp, float *scores, void *stream);

/* Bytes of DEVICE workspace l1line_mlp_backward needs for N samples. */
size_t l1line_mlp_workspace_bytes(int64_t N);

/* Gradient of sum_r dscores[r] * scores[r] with respect to the flat
 * parameters (through the binary16 weights as used), written (not added) to
 * grad (DEVICE float [L1L_MLP_PARAMS]).  Deterministic: per-CTA partial
 * gradients in the workspace are summed in a fixed order. */
int l1line_mlp_backward(const float *feat, const int32_t *rows, int64_t N,
                        const l1line_mlp *mlp, const float *dscores, float *grad,
                        void *workspace, size_t workspace_bytes, void *stream);

/* Listwise training loss.  Instance b owns positions offsets[b] ..
 * offsets[b+1]-1 (DEVICE int64 [n_inst + 1]) of scores; its loss is the cross
 * entropy between softmax(targets) and softmax(scores) over those positions
 * (targets[rows[r]], or targets[r] when rows is NULL).  Writes loss[b]
 * (DEVICE float [n_inst]) and dscores[r] = d(mean_b loss_b)/d scores[r]. */
int l1line_rank_loss(const float *scores, const float *targets, const int32_t *rows,
                     const int64_t *offsets, int64_t n_inst, float *dscores, float *loss,
                     void *stream);

/* One Adam step (step >= 1, with bias correction) on the flat float
 * parameters theta with moments m1, m2 (DEVICE float [L1L_MLP_PARAMS] each),
 * then writes the updated network into mlp (DEVICE; may be NULL). */
int l1line_adam_step(float *theta, const float *grad, float *m1, float *m2, int64_t step,
                     float lr, float beta1, float beta2, float eps, l1line_mlp *mlp,
                     void *stream);

/* Packs flat float parameters into the network image (weights rounded to
 * binary16, nearest even). */
int l1line_mlp_pack(const float *theta, l1line_mlp *mlp, void *stream);

/* Indices of the K (1 <= K <= m) highest scores, ties to the smaller index,
 * NaN lowest, written in ascending index order to out_idx (DEVICE int32 [K]). */
int l1line_topk(const float *scores, int64_t m, int64_t K, int32_t *out_idx, void *stream);

/* The whole learned path in one call: features (the restricted objective at
 * lambdas[0]), network, top-K, then the subset fit of those K candidates.
 * out_idx (DEVICE int32 [K]) receives the candidates (may be NULL).
 * Workspace: l1line_proposed_workspace_bytes(dtype, n, m, n_lambda). */
int l1line_fit_proposed_f32(const float *X, int64_t n, int64_t m, const double *lambdas,
                            int64_t n_lambda, const l1line_mlp *mlp, int64_t K,
                            int32_t *out_idx, float *out_v, double *out_obj,
                            int32_t *out_jstar, void *workspace, size_t workspace_bytes,
                            void *stream);
int l1line_fit_proposed_f64(const double *X, int64_t n, int64_t m, const double *lambdas,
                            int64_t n_lambda, const l1line_mlp *mlp, int64_t K,
                            int32_t *out_idx, double *out_v, double *out_obj,
                            int32_t *out_jstar, void *workspace, size_t workspace_bytes,
                            void *stream);

/*
 * No-allocation fit (the paper has no counterpart: this is an interface
 * convenience of the library).
 *
 * Some callers cannot call cudaMalloc at all: code embedded in an application
 * whose device memory is owned by its own allocator, a plugin given no access
 * to one, or a latency-critical loop that must not pay for the implicit
 * synchronisation of an allocation.  For them this entry point does what
 * l1line_fit_f32 does, with the same arguments and results, but takes no
 * workspace: it uses a fixed scratch array of
 * L1L_NOALLOC_SCRATCH_BYTES that the library declares in device memory, which
 * every GPU that loads the library holds until the process exits.
 *  - Sizes whose workspace (l1line_workspace_bytes(L1L_DTYPE_F32, n, m,
 *    n_lambda)) exceeds L1L_NOALLOC_SCRATCH_BYTES return L1L_ERR_UNSUPPORTED
 *    before anything is launched.
 *  - The first call on a device looks up the scratch's device address for
 *    that device (cudaGetSymbolAddress, with the device current); make that
 *    first call before any stream capture.  Later calls reuse the address.
 *  - Every call, from every thread and stream, shares the one scratch array:
 *    calls that overlap on the GPU race and corrupt each other's results.
 *    Serialise them (one stream, or events).  Each call resets the parts of
 *    the scratch that must start at zero and overwrites the rest.
 *  - Its return value carries only the host-side codes (L1L_ERR_ARG,
 *    L1L_ERR_UNSUPPORTED, L1L_ERR_CUDA, L1L_OK): the call does not wait for
 *    its kernels.  The device-side status of the fit (a NaN or infinity in X,
 *    an internal error) stays in the scratch until the next call on that
 *    device; l1line_noalloc_status reads it.
 * X, out_v, out_obj and out_jstar are device pointers as for l1line_fit_f32;
 * lambdas is a host pointer.  Nothing is allocated or freed.
 */
#define L1L_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)
int l1line_fit_noalloc_f32(const float *X, int64_t n, int64_t m, const double *lambdas,
                           int64_t n_lambda, float *out_v, double *out_obj,
                           int32_t *out_jstar, void *stream);

/* Synchronise `stream` and return the device-side status that the last
 * l1line_fit_noalloc_f32 call on the current device left in its scratch, with
 * the codes of l1line_status (L1L_OK before any call); L1L_ERR_CUDA if the
 * synchronisation or the read fails.  Allocates nothing. */
int l1line_noalloc_status(void *stream);

/* Synchronise `stream` and return the device-side status recorded in the
 * workspace by the last call that used it (L1L_OK, L1L_ERR_NONFINITE,
 * L1L_ERR_INTERNAL, or L1L_ERR_ARG for a jhat list entry out of range), or
 * L1L_ERR_CUDA. */
int l1line_status(void *workspace, void *stream);

/* Human-readable text of a status code (static storage). */
const char *l1line_status_string(int status);

/* Number of kernels the most recent scan or fit call launched (for launch
 * accounting); host-side counter, per calling thread. */
int l1line_last_launch_count(void);

/* Bounds-check counters (a diagnostic, not in the paper).  The library built
 * with L1L_CHECKS=1 checks the shared- and global-memory indices of its
 * kernels; an index out of range is counted, replaced by 0 (the kernel runs
 * on, no trap) and sets *line (when non-NULL) to a source line of the last
 * one.  Synchronises the device; returns the hits since the last reset and
 * clears them when `reset` is non-zero; -1 in the normal build, -2 on a CUDA
 * error. */
int64_t l1line_check_hits(int reset, int *line);

/*
 * Tuning of the pair kernel's launch (for an autotuner).  Every field 0 means
 * "the planner's choice".  Results do not depend on the tuning (every
 * decision stays exact); only the speed does.
 *   warps        warps per CTA, 1..16
 *   ctas_per_sm  CTAs per SM that the shared-memory plan is sized for, 1..3;
 *                at most 32 resident warps (warps x ctas_per_sm).  The
 *                kernel is compiled for three register budgets: 128 registers
 *                for up to 16 resident warps, 80 for 17-24 (CTAs of at most
 *                8 warps; 17-24 resident warps in larger CTAs is not a plan),
 *                64 for 25-32 (planner: the most resident warps whose
 *                candidate lists fit; on a tie the fewer CTAs)
 *   kchunk       k per CTA of single-instance calls (the batched call always
 *                gives a CTA a whole column jhat)
 *   d0           half-width, in positions of the 64 weight-proportional
 *                samples of column jhat, of the first bracket around the
 *                weighted median, 1..24 (planner: 6)
 *   batch_classes  size classes of a batched call, 1..3: the instances,
 *                ordered by n, are cut into that many runs (where the
 *                planner's occupancy model places the cuts), each run
 *                scored by its own pair launch with shared memory laid out
 *                for its largest n (planner: one more class while the
 *                model puts it at least 5% below the best with one fewer;
 *                l1line_plan reports 0)
 *   column       where the pair kernel keeps x_ijhat: 1 shared memory, 2 the
 *                column copy in global memory (L2), which leaves shared memory
 *                to more resident warps (planner: global for double input;
 *                for float input global only when that admits more resident
 *                warps; l1line_plan reports 1 or 2)
 * l1line_set_tuning applies to the later calls of the calling thread (NULL
 * restores the planner); a tuning whose candidate lists do not fit shared
 * memory makes those calls return L1L_ERR_UNSUPPORTED.  l1line_plan reports
 * the plan such a call would use for nj scored jhat (nj = m for a full scan)
 * on the current device.
 */
typedef struct l1line_tuning {
    int32_t warps;
    int32_t ctas_per_sm;
    int32_t kchunk;
    int32_t d0;
    int32_t batch_classes;
    int32_t column;
} l1line_tuning;
int l1line_set_tuning(const l1line_tuning *t);
int l1line_plan(int dtype, int64_t n, int64_t m, int64_t nj, l1line_tuning *out);
/* The same plan for a GPU of `sms` streaming multiprocessors, computed on the
 * host without touching a device (the planner is host code; l1line_plan
 * passes the current device's count).  For tests and for planning ahead of a
 * launch.  No passage of the paper: a launch heuristic.  Returns L1L_OK,
 * L1L_ERR_ARG (NULL out, n, m, nj or sms < 1, unknown dtype) or
 * L1L_ERR_UNSUPPORTED (n beyond the pair kernel's shared memory; such fits
 * take the global-memory path). */
int l1line_plan_for(int dtype, int64_t n, int64_t m, int64_t nj, int sms, l1line_tuning *out);

/* Measurement hook: when both are non-NULL (cudaEvent_t), later scan and fit
 * calls from this thread record `start` on their stream just before the pair
 * kernel (steps A2-A4) is launched and `stop` just after it, so the caller can
 * time that kernel alone with cudaEventElapsedTime.  With more than 256
 * lambdas the bracket spans every pair-kernel launch and the exact-path
 * launches between them.  Pass NULLs to switch it off.  Returns L1L_OK. */
int l1line_profile_events(void *start, void *stop);

/*
 * Bandwidth probes: the measured denominators of the pair kernel's L2 and
 * shared-memory ceilings (the fit path never calls them).  Asynchronous on
 * `stream`; the caller times the launch (CUDA events) and divides
 * *bytes_read by the time.
 *   L1L_PROBE_L2    reads `bytes` (>= 16) of the device buffer `buf`
 *                   (16-byte aligned) `reps` times with 16-byte loads that
 *                   bypass L1; size it well below the L2 so every pass after
 *                   the first hits L2.  *bytes_read = reps * floor(bytes/16)*16.
 *   L1L_PROBE_SMEM  4 CTAs of 512 threads per SM each read reps x 8
 *                   conflict-free 16-byte shared-memory words; `buf` and
 *                   `bytes` are ignored.
 * `sink` is a 4-byte device word the kernels may increment (it keeps the
 * loads live).  Errors: L1L_ERR_ARG (kind, reps < 1, NULL sink or bytes_read,
 * L2 probe buffer NULL, unaligned or under 16 bytes), L1L_ERR_CUDA.
 */
enum { L1L_PROBE_L2 = 0, L1L_PROBE_SMEM = 1 };
int l1line_probe(int kind, const void *buf, size_t bytes, int reps, void *sink, void *stream,
                 double *bytes_read);

#ifdef __cplusplus
}
#endif
#endif /* L1LINE_H */
