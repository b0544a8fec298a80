// launch.h -- host-side launchers of the kernels (internal to the library).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"
#include "l1line.h"

namespace l1l {

// Raise a kernel's dynamic shared-memory limit on the current device once;
// later calls asking for no more skip the runtime call, so that launches can
// be captured in a CUDA graph after one warm-up call.
cudaError_t ensure_smem(const void *fn, size_t bytes);
// Resident blocks per SM for (kernel, threads, dynamic shared memory), cached.
cudaError_t blocks_per_sm(const void *fn, int threads, size_t smem, int *out);

// Xf: the float copy of Xt for double input, followed by the remainders
// x - fl(x) at Xf + m ldn (unused for float input).
template <typename T>
cudaError_t launch_prep(const T *X, T *Xt, float *Xf, ColInfo *ci, int64_t n, int64_t m,
                        int64_t ldn, uint32_t *status, cudaStream_t st, int &launches);

// Launch shapes of the pair kernels: one compiled instantiation per register
// budget, which follows from the resident threads it is compiled for.
enum : int {
    SHAPE_R80 = 0,   // <= 8 warps per CTA, <= 24 warps per SM: 80 registers
    SHAPE_R64 = 1,   // <= 16 warps per CTA, <= 32 warps per SM: 64 registers
    SHAPE_R128 = 2,  // <= 16 warps per CTA, <= 16 warps per SM: 128 registers
};
// The shape of `warps` per CTA x `ctas` per SM: up to 16 resident warps
// SHAPE_R128, 17-24 SHAPE_R80 (CTAs of up to 8 warps only), 25-32 SHAPE_R64;
// -1 for any other plan.
int pair_shape(int warps, int ctas);

// Shared-memory plan of the pair kernel for a given n; warps == 0 if n is too
// large for the kernel.
struct PairPlan {
    int warps;
    size_t smem;
    int kchunk;
    int kchunks;
    int cap;    // per-warp candidate-list capacity
    int ctas;   // CTAs per SM the shared memory is sized for
    int d0;     // first-bracket half-width of the selection
    int cs;     // 1: x_ijhat staged in shared memory; 0: read from global memory
    int shape;  // SHAPE_*
};
// Caller overrides of the planner (0 = the planner's choice).
struct Tune {
    int warps = 0, ctas = 0, kchunk = 0, d0 = 0, batch_classes = 0;
    int column = 0;  // 1: x_ijhat in shared memory, 2: in global memory
};
// nj: number of jhat scored (m for a full scan).
template <typename T>
// single: a single-instance call (false for the batched call's size classes,
// whose persistent CTAs take whole columns).
PairPlan plan_pairs(int64_t n, int64_t m, int num_sms, int64_t nj, const Tune &tune = Tune(),
                    bool single = true);
template <typename T> int64_t max_rows_pairs();

// One launch of the pair kernel for lambdas[t0 .. t0+nlc) (nlc <= MAX_LAMBDA_PER_LAUNCH).
template <typename T>
cudaError_t launch_pairs(const ScanArgs<T> &a, const double *lambdas, int t0, int nlc,
                         const PairPlan &plan, cudaStream_t st, int &launches);
// The same for one shape S == plan.shape (k_pairs_shape.cu).
template <typename T, int S>
cudaError_t launch_pairs_sh(const ScanArgs<T> &a, const LambdaPack &lp, int t0, int nlc,
                            const PairPlan &plan, cudaStream_t st);

// Largest n of any scan or fit: the global-memory path's limit (row counts
// and the exact path's row loop are 32-bit).
constexpr int64_t large_max_rows() { return (int64_t)0x7FFFFF00; }
// CTAs per cluster of the global-memory path for a staged column of ldn rows.
int large_cluster_size(int64_t ldn);
// Steps A2-A4 for n beyond max_rows_pairs (k_large.cu): one launch for
// lambdas[t0 .. t0+nlc), every (lambda, listed jhat, k).
template <typename T>
cudaError_t launch_large(const ScanArgs<T> &a, const double *lambdas, int t0, int nlc,
                         cudaStream_t st, int &launches);

// Exact path for the pairs listed by the preceding pair launch (same chunk).
template <typename T>
cudaError_t launch_exact(const ScanArgs<T> &a, const double *lambdas, int t0, int nlc,
                         int num_sms, cudaStream_t st, int &launches);

// z of the listed jhat (jlist == nullptr: all m, nj == m).
cudaError_t launch_zreduce(const double *s_all, double *z_all, int64_t m, int64_t n_lambda,
                           const int32_t *jlist, int64_t nj, cudaStream_t st, int &launches);

// Argmin over the listed jhat (smallest jhat on ties) and gather of v*.
template <typename T>
cudaError_t launch_argmin(const double *z_all, const T *v_all, int64_t m, int64_t n_lambda,
                          const int32_t *jlist, int64_t nj, T *out_v, double *out_obj,
                          int32_t *out_jstar, cudaStream_t st, int &launches);

// Successive components: Y = X - x_jhat v^T, elementwise, rounded per operation.
template <typename T>
cudaError_t launch_deflate(const T *X, T *Y, int64_t n, int64_t m, const int32_t *jstar,
                           const T *v, int num_sms, cudaStream_t st, int &launches);

// ---- learned jhat proposer (k_propose.cu) ----
constexpr int MLP_TILE = 64;  // samples per CTA of the network kernels
size_t mlp_smem_bytes();
// Column features 0..2 of the staged copy into raw [m][L1L_MLP_FEATURES].
template <typename T>
cudaError_t launch_colfeat(const T *Xt, int64_t ldn, int64_t n, int64_t m, float *raw,
                           cudaStream_t st, int &launches);
// Standardises every feature column of raw over the m columns.
cudaError_t launch_featstd(const float *raw, int64_t m, float *stdz, cudaStream_t st,
                           int &launches);
// The R rows of largest l1 norm of the row-major X (rho: row norms [n],
// rows: their indices in ascending order [R]) copied into Y (R x m).
template <typename T>
cudaError_t launch_heavy_rows(const T *X, int64_t n, int64_t m, int64_t R, float *rho,
                              int32_t *rows, T *Y, cudaStream_t st, int &launches);
// *dst |= *src (device status words), one thread.
cudaError_t launch_status_or(uint32_t *dst, const uint32_t *src, cudaStream_t st, int &launches);
// raw[j][c] = z[j] for j < m.
cudaError_t launch_setfeat(const double *z, int64_t m, int c, float *raw, cudaStream_t st,
                           int &launches);
cudaError_t launch_mlp_forward(const float *feat, const int32_t *rows, int64_t N,
                               const l1line_mlp *p, float *score, cudaStream_t st, int &launches);
cudaError_t launch_mlp_backward(const float *feat, const int32_t *rows, int64_t N,
                                const l1line_mlp *p, const float *dscore, float *part,
                                float *grad, cudaStream_t st, int &launches);
cudaError_t launch_rank_loss(const float *score, const float *target, const int32_t *rows,
                             const int64_t *off, int64_t n_inst, float *ds, float *loss,
                             cudaStream_t st, int &launches);
cudaError_t launch_adam(float *theta, const float *grad, float *m1, float *m2, float lr,
                        float beta1, float beta2, float eps, float c1, float c2, l1line_mlp *out,
                        cudaStream_t st, int &launches);
cudaError_t launch_mlp_pack(const float *theta, l1line_mlp *out, cudaStream_t st, int &launches);
cudaError_t launch_topk(const float *score, int64_t m, int K, int32_t *out, cudaStream_t st,
                        int &launches);

// ---- Algorithm 3: the solution path (k_solpath.cu) ----
size_t solpath_bytes(int64_t m, int64_t entries);
template <typename T>
cudaError_t launch_solpath(int64_t m, const int64_t *off, const int32_t *len, const double *lam,
                           const T *val, const double *res, unsigned char *ws, int64_t entries,
                           double *out_start, int32_t *out_jhat, double *out_I, double *out_s,
                           T *out_v, int64_t *out_count, int64_t cap, cudaStream_t st,
                           int &launches);

// ---- Algorithm 2: lambda paths of every pair (k_path.cu) ----
size_t path_scan_scratch(int64_t N);
// In place: a[0..N) -> its exclusive prefix sums, a[N] = total (tmp: path_scan_scratch(N)).
cudaError_t launch_scan_i64(int64_t *a, int64_t N, int64_t *tmp, cudaStream_t st, int &launches);
int path_big_workers();
template <typename T> size_t path_slice_bytes(int64_t n);
template <typename T> int64_t path_max_rows();
// count: bound_or_off = [m*m + 1] offsets out (exclusive scan of the bounds);
// write: bound_or_off = those offsets in, lam / val / len out.
template <typename T>
cudaError_t launch_path(bool count, const T *Xt, const float *Xf, const ColInfo *ci, int64_t n,
                        int64_t m, int64_t ldn, const T *v0, int64_t *bound_or_off,
                        int64_t *scan_tmp, double *lam, T *val, double *res, int32_t *len,
                        int32_t *big, uint32_t *big_count, unsigned char *scratch,
                        uint32_t *status, int num_sms, cudaStream_t st, int &launches);

// A size class of a batch: units [u0, u1) run in one persistent launch whose
// shared memory is laid out for the class's largest n.
struct BatchClass {
    int64_t u0, u1;
    int lay_npad;
    PairPlan plan;
};
constexpr int MAX_BATCH_CLASSES = 3;

// The persistent pair kernel of one size class (shape S == bc.plan.shape;
// k_pairs_shape.cu): as many CTAs as stay resident, pulling units from the
// class's counter `slot`.
template <typename T, int S>
cudaError_t launch_persist_sh(const BatchDesc<T> &bd, unsigned char *ws, const BatchClass &bc,
                              int slot, bool multi, int num_sms, cudaStream_t st);

// The batched fit: staging, one persistent pair kernel per size class, exact
// path, sums, argmin.
template <typename T>
cudaError_t launch_batch(const BatchDesc<T> &bd, unsigned char *ws, T *out_v, double *out_obj,
                         int32_t *out_jstar, const BatchClass *classes, int nclasses, bool multi,
                         int num_sms, cudaStream_t st, int &launches);

// Bandwidth probes (k_probe.cu): L2 reads of a resident buffer, shared-memory reads.
enum { PROBE_L2 = 0, PROBE_SMEM = 1 };
cudaError_t launch_probe(int kind, const void *buf, size_t bytes, int reps, unsigned *sink,
                         int num_sms, cudaStream_t st, double *bytes_read, int &launches);

}  // namespace l1l
