// k_propose.cu -- the learned jhat proposer (not part of the paper): column
// features (and the row norms and row gather of the restricted-objective
// feature), the 4-128-128-1 ReLU network (forward, backward, Adam), the
// listwise training loss and the top-K selection of candidate columns.
//
// The network's weight matrices are stored in binary16 and widened to float
// in shared memory; every product and sum is float.  All reductions run in a
// fixed order, so every kernel here is deterministic.
#include <cfloat>
#include <cuda_fp16.h>

#include "checks.cuh"
#include "common.cuh"
#include "l1line.h"
#include "launch.h"

namespace l1l {

namespace {

constexpr int HID = L1L_MLP_HIDDEN;  // 128
constexpr int NF = L1L_MLP_FEATURES;  // 4
constexpr int NPAR = L1L_MLP_PARAMS;  // 17281
constexpr int OFF_B1 = HID * NF, OFF_W2 = OFF_B1 + HID, OFF_B2 = OFF_W2 + HID * HID,
              OFF_W3 = OFF_B2 + HID, OFF_B3 = OFF_W3 + HID;
static_assert(OFF_B3 + 1 == NPAR, "parameter layout");
static_assert(sizeof(l1line_mlp) == 35088, "packed network image");
constexpr int TS = MLP_TILE;  // samples per CTA
constexpr int LD = HID + 1;   // shared row stride in floats (conflict-free column walks)
constexpr int NT = 256;

__device__ __forceinline__ uint32_t warp_incl_scan_u32(uint32_t x, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Block-wide reduction of a double in a fixed order (warp butterflies, then
// the warp totals in index order).  `red` holds one slot per warp.
__device__ double block_sum_f64(double x, double *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    x = warp_sum_f64(x);
    __syncthreads();
    if (lane == 0) red[warp] = x;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += red[w];
    return t;
}

__device__ double block_max_f64(double x, double *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xFFFFFFFFu, x, o));
    __syncthreads();
    if (lane == 0) red[warp] = x;
    __syncthreads();
    double t = red[0];
    for (int w = 1; w < nw; ++w) t = fmax(t, red[w]);
    return t;
}

// One step of an MSB-first radix select over 8-bit digits: thread 0..31 scan
// the 256-bin histogram; the bin holding rank `rank` extends the prefix.
// Returns (through shared memory) the new prefix, the rank inside that bin and
// the number of keys in lower bins.
struct SelState {
    uint32_t prefix, rank, below;
};
__device__ void radix_pick(const uint32_t *hist, SelState &s, SelState *out) {
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 32) {
        uint32_t c[8], tot = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            c[q] = hist[8 * lane + q];
            tot += c[q];
        }
        const uint32_t incl = warp_incl_scan_u32(tot, lane);
        const uint32_t excl = incl - tot;
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, excl <= s.rank && s.rank < incl);
        const int src = bal ? __ffs(bal) - 1 : 31;
        if (lane == src) {
            uint32_t r = s.rank - min(s.rank, excl), below = excl;
            int b = 7;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                if (r < c[q]) {
                    b = q;
                    break;
                }
                r -= c[q];
                below += c[q];
            }
            out->prefix = (s.prefix << 8) | (uint32_t)(8 * lane + b);
            out->rank = r;
            out->below = s.below + below;
        }
    }
    __syncthreads();
    s = *out;
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Column features: l1 norm, l2 norm and the lower median of |x| (rank
// floor((n-1)/2) of the ascending order), one CTA per column of the
// column-major copy.  Sums in double; the median is selected exactly on the
// order-preserving bit patterns of |x| rounded to float.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(NT) k_colfeat(const T *__restrict__ Xt, int64_t ldn, int n,
                                                 float *__restrict__ raw) {
    extern __shared__ uint32_t keys[];
    __shared__ uint32_t hist[256];
    __shared__ double red[NT / 32];
    __shared__ SelState sel;
    const int64_t j = blockIdx.x;
    const T *x = Xt + j * ldn;
    double s1 = 0.0, s2 = 0.0;
    for (int i = threadIdx.x; i < n; i += NT) {
        const double a = fabs((double)x[i]);
        s1 += a;
        s2 += a * a;
        keys[i] = __float_as_uint(fminf((float)a, FLT_MAX));
    }
    s1 = block_sum_f64(s1, red);
    s2 = block_sum_f64(s2, red);
    SelState s{0u, (uint32_t)((n - 1) / 2), 0u};
    for (int pass = 0; pass < 4; ++pass) {
        const int shift = 24 - 8 * pass;
        for (int b = threadIdx.x; b < 256; b += NT) hist[b] = 0u;
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += NT) {
            const uint32_t k = keys[L1L_CHK(i, n)];
            if (pass == 0 || (uint32_t)((uint64_t)k >> (shift + 8)) == s.prefix)
                atomicAdd(&hist[(k >> shift) & 255u], 1u);
        }
        __syncthreads();
        radix_pick(hist, s, &sel);
    }
    if (threadIdx.x == 0) {
        raw[j * NF + 0] = (float)fmin(s1, (double)FLT_MAX);
        raw[j * NF + 1] = (float)fmin(sqrt(s2), (double)FLT_MAX);
        raw[j * NF + 2] = __uint_as_float(s.prefix);
    }
}

// Row weights of the restricted-objective feature: rho_i = sum_j |x_ij| in
// double, added left to right over j (one thread per row of the row-major X;
// the fixed order makes the sum reproducible), rounded to float.
template <typename T>
__global__ void __launch_bounds__(NT) k_rownorm(const T *__restrict__ X, int64_t n, int64_t m,
                                                 float *__restrict__ rho) {
    const int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (i >= n) return;
    const T *x = X + i * m;
    double s = 0.0;
    for (int64_t j = 0; j < m; ++j) s += fabs((double)x[j]);
    rho[i] = (float)fmin(s, (double)FLT_MAX);
}

// Rows[r] of X (row-major n x m) into Y (row-major R x m).
template <typename T>
__global__ void __launch_bounds__(NT) k_gather_rows(const T *__restrict__ X, int64_t n, int64_t m,
                                                     const int32_t *__restrict__ rows,
                                                     T *__restrict__ Y) {
    const int64_t r = blockIdx.x;
    const T *x = X + (int64_t)L1L_CHK(rows[r], (int32_t)n) * m;
    T *y = Y + r * m;
    for (int64_t j = threadIdx.x; j < m; j += NT) y[j] = x[j];
}

__global__ void k_status_or(uint32_t *dst, const uint32_t *src) { *dst |= *src; }

// raw[j][c] = z[j] (the restricted objective, rounded to float).
__global__ void __launch_bounds__(NT) k_setfeat(const double *__restrict__ z, int64_t m, int c,
                                                 float *__restrict__ raw) {
    const int64_t j = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (j < m) raw[j * NF + c] = (float)fmin(fmax(z[j], -(double)FLT_MAX), (double)FLT_MAX);
}

// Per feature: (f - mean) / population standard deviation over the m
// columns (0 where the deviation is 0).  One CTA.
__global__ void __launch_bounds__(NT) k_featstd(const float *__restrict__ raw, int64_t m,
                                                 float *__restrict__ out) {
    __shared__ double red[NT / 32];
    for (int c = 0; c < NF; ++c) {
        double s = 0.0;
        for (int64_t j = threadIdx.x; j < m; j += NT) s += raw[j * NF + c];
        const double mean = block_sum_f64(s, red) / (double)m;
        double v = 0.0;
        for (int64_t j = threadIdx.x; j < m; j += NT) {
            const double d = raw[j * NF + c] - mean;
            v += d * d;
        }
        const double sd = sqrt(block_sum_f64(v, red) / (double)m);
        for (int64_t j = threadIdx.x; j < m; j += NT)
            out[j * NF + c] = sd > 0.0 ? (float)((raw[j * NF + c] - mean) / sd) : 0.0f;
    }
}

// ---------------------------------------------------------------------------
// The network on a tile of TS samples.
// ---------------------------------------------------------------------------
struct MlpSmem {
    float w2[HID * LD];  // w2[o * LD + i]
    float w1[HID * NF];
    float b1[HID], b2[HID], w3[HID];
    float b3;
    float f[TS * NF];
    float h1[TS * LD];  // h1, then (backward) g1
    float h2[TS * LD];  // h2, then (backward) g2; forward-only: partial scores
    float ds[TS];
};

__device__ __forceinline__ float h2f(uint16_t b) { return __half2float(__ushort_as_half(b)); }

__device__ void mlp_load(const l1line_mlp *__restrict__ p, MlpSmem &S) {
    for (int e = threadIdx.x; e < HID * HID; e += NT) S.w2[(e >> 7) * LD + (e & 127)] = h2f(p->w2[e]);
    for (int e = threadIdx.x; e < HID * NF; e += NT) S.w1[e] = h2f(p->w1[e]);
    for (int e = threadIdx.x; e < HID; e += NT) {
        S.b1[e] = p->b1[e];
        S.b2[e] = p->b2[e];
        S.w3[e] = h2f(p->w3[e]);
    }
    if (threadIdx.x == 0) S.b3 = p->b3;
}

// Forward pass of the tile; leaves h1 and relu(a2) in shared memory when
// KEEP, else writes the scores.
template <bool KEEP>
__device__ void mlp_tile_forward(MlpSmem &S, int cnt, float *__restrict__ score_out) {
    for (int e = threadIdx.x; e < TS * HID; e += NT) {
        const int s = e >> 7, i = e & 127;
        float a = S.b1[i];
#pragma unroll
        for (int c = 0; c < NF; ++c) a = fmaf(S.w1[i * NF + c], S.f[s * NF + c], a);
        S.h1[s * LD + i] = fmaxf(a, 0.0f);
    }
    __syncthreads();
    // thread (og, sg): outputs og + 16p, samples sg + 16q
    const int og = threadIdx.x & 15, sg = threadIdx.x >> 4;
    float acc[4][8];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int p = 0; p < 8; ++p) acc[q][p] = 0.0f;
#pragma unroll 4
    for (int i = 0; i < HID; ++i) {
        float hv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) hv[q] = S.h1[(sg + 16 * q) * LD + i];
#pragma unroll
        for (int p = 0; p < 8; ++p) {
            const float w = S.w2[(og + 16 * p) * LD + i];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q][p] = fmaf(w, hv[q], acc[q][p]);
        }
    }
    if (KEEP) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int p = 0; p < 8; ++p)
                S.h2[(sg + 16 * q) * LD + og + 16 * p] = fmaxf(acc[q][p] + S.b2[og + 16 * p], 0.0f);
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float part = 0.0f;
#pragma unroll
            for (int p = 0; p < 8; ++p)
                part = fmaf(S.w3[og + 16 * p], fmaxf(acc[q][p] + S.b2[og + 16 * p], 0.0f), part);
            // the 16 lanes sharing sg are one half warp
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) part += __shfl_xor_sync(0xFFFFFFFFu, part, o);
            const int s = sg + 16 * q;
            if (og == 0 && s < cnt) score_out[s] = part + S.b3;
        }
    }
}

__device__ void load_tile_features(MlpSmem &S, const float *__restrict__ feat,
                                   const int32_t *__restrict__ rows, int64_t base, int cnt) {
    for (int e = threadIdx.x; e < TS * NF; e += NT) {
        const int s = e / NF, c = e - NF * (e / NF);
        float v = 0.0f;
        if (s < cnt) {
            const int64_t r = rows ? (int64_t)rows[base + s] : base + s;
            v = feat[r * NF + c];
        }
        S.f[e] = v;
    }
}

__global__ void __launch_bounds__(NT) k_mlp_fwd(const float *__restrict__ feat,
                                                 const int32_t *__restrict__ rows, int64_t N,
                                                 const l1line_mlp *__restrict__ p,
                                                 float *__restrict__ score) {
    extern __shared__ __align__(16) unsigned char smraw[];
    MlpSmem &S = *reinterpret_cast<MlpSmem *>(smraw);
    const int64_t base = (int64_t)blockIdx.x * TS;
    const int cnt = N - base < TS ? (int)(N - base) : TS;
    mlp_load(p, S);
    load_tile_features(S, feat, rows, base, cnt);
    __syncthreads();
    mlp_tile_forward<false>(S, cnt, score + base);
}

// Backward pass of sum_r ds[r] * score[r]: recomputes the tile's forward pass,
// then writes this CTA's parameter gradient (flat order W1, b1, W2, b2, w3, b3)
// to part[blockIdx.x]; k_grad_sum adds the CTAs' rows in index order.
__global__ void __launch_bounds__(NT) k_mlp_bwd(const float *__restrict__ feat,
                                                 const int32_t *__restrict__ rows, int64_t N,
                                                 const l1line_mlp *__restrict__ p,
                                                 const float *__restrict__ dscore,
                                                 float *__restrict__ part) {
    extern __shared__ __align__(16) unsigned char smraw[];
    MlpSmem &S = *reinterpret_cast<MlpSmem *>(smraw);
    const int64_t base = (int64_t)blockIdx.x * TS;
    const int cnt = N - base < TS ? (int)(N - base) : TS;
    float *g = part + (int64_t)blockIdx.x * NPAR;
    mlp_load(p, S);
    load_tile_features(S, feat, rows, base, cnt);
    for (int s = threadIdx.x; s < TS; s += NT) S.ds[s] = s < cnt ? dscore[base + s] : 0.0f;
    __syncthreads();
    mlp_tile_forward<true>(S, cnt, nullptr);
    __syncthreads();
    // output layer; g2 = ds * w3 * [a2 > 0] replaces h2 (same thread, same entries)
    if (threadIdx.x < HID) {
        const int o = threadIdx.x;
        float dw3 = 0.0f, db2 = 0.0f;
        for (int s = 0; s < TS; ++s) {
            const float h = S.h2[s * LD + o];
            dw3 = fmaf(S.ds[s], h, dw3);
            const float g2 = h > 0.0f ? S.ds[s] * S.w3[o] : 0.0f;
            S.h2[s * LD + o] = g2;
            db2 += g2;
        }
        g[OFF_W3 + o] = dw3;
        g[OFF_B2 + o] = db2;
    } else if (threadIdx.x == HID) {
        float db3 = 0.0f;
        for (int s = 0; s < TS; ++s) db3 += S.ds[s];
        g[OFF_B3] = db3;
    }
    __syncthreads();
    // dW2[o][i] = sum_s g2[s][o] h1[s][i]; thread (og, ig): o = og + 16p, i = ig + 16q
    {
        const int og = threadIdx.x & 15, ig = threadIdx.x >> 4;
        float acc[8][8];
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int b = 0; b < 8; ++b) acc[a][b] = 0.0f;
#pragma unroll 2
        for (int s = 0; s < TS; ++s) {
            float gv[8], hv[8];
#pragma unroll
            for (int a = 0; a < 8; ++a) gv[a] = S.h2[s * LD + og + 16 * a];
#pragma unroll
            for (int b = 0; b < 8; ++b) hv[b] = S.h1[s * LD + ig + 16 * b];
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(gv[a], hv[b], acc[a][b]);
        }
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int b = 0; b < 8; ++b) g[OFF_W2 + (og + 16 * a) * HID + ig + 16 * b] = acc[a][b];
    }
    __syncthreads();
    // g1[s][i] = [a1 > 0] sum_o w2[o][i] g2[s][o]; thread (ig, sg): i = ig + 16p, s = sg + 16q
    {
        const int ig = threadIdx.x & 15, sg = threadIdx.x >> 4;
        float acc[4][8];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int a = 0; a < 8; ++a) acc[q][a] = 0.0f;
#pragma unroll 4
        for (int o = 0; o < HID; ++o) {
            float gv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) gv[q] = S.h2[(sg + 16 * q) * LD + o];
#pragma unroll
            for (int a = 0; a < 8; ++a) {
                const float w = S.w2[o * LD + ig + 16 * a];
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[q][a] = fmaf(w, gv[q], acc[q][a]);
            }
        }
        // only this thread reads or writes these h1 entries in this phase
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int a = 0; a < 8; ++a) {
                float &h = S.h1[(sg + 16 * q) * LD + ig + 16 * a];
                h = h > 0.0f ? acc[q][a] : 0.0f;
            }
    }
    __syncthreads();
    if (threadIdx.x < HID) {
        const int i = threadIdx.x;
        float d[NF], db1 = 0.0f;
#pragma unroll
        for (int c = 0; c < NF; ++c) d[c] = 0.0f;
        for (int s = 0; s < TS; ++s) {
            const float g1 = S.h1[s * LD + i];
#pragma unroll
            for (int c = 0; c < NF; ++c) d[c] = fmaf(g1, S.f[s * NF + c], d[c]);
            db1 += g1;
        }
#pragma unroll
        for (int c = 0; c < NF; ++c) g[i * NF + c] = d[c];
        g[OFF_B1 + i] = db1;
    }
}

__global__ void k_grad_sum(const float *__restrict__ part, int nblk, float *__restrict__ grad) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= NPAR) return;
    float s = 0.0f;
    for (int b = 0; b < nblk; ++b) s += part[(int64_t)b * NPAR + e];
    grad[e] = s;
}

// ---------------------------------------------------------------------------
// Listwise loss: per instance, cross entropy between softmax(targets) and
// softmax(scores); ds = (p - q) / n_inst.  One CTA per instance.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) k_rank_loss(const float *__restrict__ score,
                                                   const float *__restrict__ target,
                                                   const int32_t *__restrict__ rows,
                                                   const int64_t *__restrict__ off, int64_t n_inst,
                                                   float *__restrict__ ds, float *__restrict__ loss) {
    __shared__ double red[NT / 32];
    const int64_t b = blockIdx.x;
    const int64_t r0 = off[b], r1 = off[b + 1];
    if (r1 <= r0) {
        if (threadIdx.x == 0) loss[b] = 0.0f;
        return;
    }
    auto tgt = [&](int64_t r) -> double { return target[rows ? (int64_t)rows[r] : r]; };
    double ms = -INFINITY, mu = -INFINITY;
    for (int64_t r = r0 + threadIdx.x; r < r1; r += NT) {
        ms = fmax(ms, (double)score[r]);
        mu = fmax(mu, tgt(r));
    }
    ms = block_max_f64(ms, red);
    mu = block_max_f64(mu, red);
    double es = 0.0, eu = 0.0, us = 0.0;
    for (int64_t r = r0 + threadIdx.x; r < r1; r += NT) {
        es += exp((double)score[r] - ms);
        const double e = exp(tgt(r) - mu);
        eu += e;
        us += e * (double)score[r];
    }
    es = block_sum_f64(es, red);
    eu = block_sum_f64(eu, red);
    us = block_sum_f64(us, red);
    const double inv_n = 1.0 / (double)n_inst;
    for (int64_t r = r0 + threadIdx.x; r < r1; r += NT) {
        const double pr = exp((double)score[r] - ms) / es, qr = exp(tgt(r) - mu) / eu;
        ds[r] = (float)((pr - qr) * inv_n);
    }
    if (threadIdx.x == 0) loss[b] = (float)(ms + log(es) - us / eu);
}

// ---------------------------------------------------------------------------
// Adam and packing of the float parameters into the binary16 network.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pack_one(int e, float v, l1line_mlp *out) {
    const uint16_t hb = __half_as_ushort(__float2half_rn(v));
    if (e < OFF_B1) out->w1[e] = hb;
    else if (e < OFF_W2) out->b1[e - OFF_B1] = v;
    else if (e < OFF_B2) out->w2[e - OFF_W2] = hb;
    else if (e < OFF_W3) out->b2[e - OFF_B2] = v;
    else if (e < OFF_B3) out->w3[e - OFF_W3] = hb;
    else out->b3 = v;
}

__global__ void k_mlp_pack(const float *__restrict__ theta, l1line_mlp *out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < NPAR) pack_one(e, theta[e], out);
}

__global__ void k_adam(float *__restrict__ theta, const float *__restrict__ grad,
                       float *__restrict__ m1, float *__restrict__ m2, float lr, float beta1,
                       float beta2, float eps, float c1, float c2, l1line_mlp *out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= NPAR) return;
    const float gv = grad[e];
    const float a = beta1 * m1[e] + (1.0f - beta1) * gv;
    const float b = beta2 * m2[e] + (1.0f - beta2) * gv * gv;
    m1[e] = a;
    m2[e] = b;
    const float t = theta[e] - lr * (a * c1) / (sqrtf(b * c2) + eps);
    theta[e] = t;
    if (out) pack_one(e, t, out);
}

// ---------------------------------------------------------------------------
// Top-K: the K highest scores (ties to the smaller index, NaN lowest), written
// in ascending index order.  One CTA of 1024 threads: radix select of the
// K-th key, then an ordered compaction.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t score_key(float s) {
    if (s != s) return 0xFFFFFFFFu;
    const uint32_t b = __float_as_uint(s == 0.0f ? 0.0f : s);
    const uint32_t ord = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
    return ~ord;  // ascending key = descending score
}

constexpr int TK_NT = 1024;

__device__ uint32_t block_excl_scan_u32(uint32_t x, uint32_t *wsum, uint32_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t incl = warp_incl_scan_u32(x, lane);
    __syncthreads();
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const uint32_t v = wsum[lane];
        const uint32_t vi = warp_incl_scan_u32(v, lane);
        wsum[lane] = vi - v;
        if (lane == 31) *total = vi;
    }
    __syncthreads();
    return wsum[warp] + incl - x;
}

__global__ void __launch_bounds__(TK_NT) k_topk(const float *__restrict__ score, int64_t m, int K,
                                                 int32_t *__restrict__ out) {
    __shared__ uint32_t hist[256];
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t total;
    __shared__ SelState sel;
    SelState s{0u, (uint32_t)(K - 1), 0u};
    for (int pass = 0; pass < 4; ++pass) {
        const int shift = 24 - 8 * pass;
        for (int b = threadIdx.x; b < 256; b += TK_NT) hist[b] = 0u;
        __syncthreads();
        for (int64_t i = threadIdx.x; i < m; i += TK_NT) {
            const uint32_t k = score_key(score[i]);
            if (pass == 0 || (uint32_t)((uint64_t)k >> (shift + 8)) == s.prefix)
                atomicAdd(&hist[(k >> shift) & 255u], 1u);
        }
        __syncthreads();
        radix_pick(hist, s, &sel);
    }
    const uint32_t T = s.prefix, need = (uint32_t)K - s.below;  // ties at T to take
    const int64_t chunk = (m + TK_NT - 1) / TK_NT;
    const int64_t i0 = min(m, (int64_t)threadIdx.x * chunk), i1 = min(m, i0 + chunk);
    uint32_t lt = 0, eq = 0;
    for (int64_t i = i0; i < i1; ++i) {
        const uint32_t k = score_key(score[i]);
        lt += k < T;
        eq += k == T;
    }
    const uint32_t eq_before = block_excl_scan_u32(eq, wsum, &total);
    const uint32_t take_eq = need > eq_before ? min(eq, need - eq_before) : 0u;
    uint32_t pos = block_excl_scan_u32(lt + take_eq, wsum, &total);
    uint32_t er = eq_before;
    for (int64_t i = i0; i < i1; ++i) {
        const uint32_t k = score_key(score[i]);
        bool in = k < T;
        if (k == T) in = er++ < need;
        if (in) out[L1L_CHK(pos++, (uint32_t)K)] = (int32_t)i;
    }
}

}  // namespace

size_t mlp_smem_bytes() { return sizeof(MlpSmem); }

L1L_CHECKS_READER(l1l_checks_propose)

template <typename T>
cudaError_t launch_colfeat(const T *Xt, int64_t ldn, int64_t n, int64_t m, float *raw,
                           cudaStream_t st, int &launches) {
    const size_t smem = (size_t)n * 4;
    cudaError_t e = ensure_smem(reinterpret_cast<const void *>(k_colfeat<T>), smem);
    if (e != cudaSuccess) return e;
    k_colfeat<T><<<(unsigned)m, NT, smem, st>>>(Xt, ldn, (int)n, raw);
    launches++;
    return cudaGetLastError();
}

cudaError_t launch_featstd(const float *raw, int64_t m, float *stdz, cudaStream_t st,
                           int &launches) {
    k_featstd<<<1, NT, 0, st>>>(raw, m, stdz);
    launches++;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_heavy_rows(const T *X, int64_t n, int64_t m, int64_t R, float *rho,
                              int32_t *rows, T *Y, cudaStream_t st, int &launches) {
    k_rownorm<T><<<(unsigned)((n + NT - 1) / NT), NT, 0, st>>>(X, n, m, rho);
    launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_topk<<<1, TK_NT, 0, st>>>(rho, n, (int)R, rows);
    launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_gather_rows<T><<<(unsigned)R, NT, 0, st>>>(X, n, m, rows, Y);
    launches++;
    return cudaGetLastError();
}

cudaError_t launch_status_or(uint32_t *dst, const uint32_t *src, cudaStream_t st,
                             int &launches) {
    k_status_or<<<1, 1, 0, st>>>(dst, src);
    launches++;
    return cudaGetLastError();
}

cudaError_t launch_setfeat(const double *z, int64_t m, int c, float *raw, cudaStream_t st,
                           int &launches) {
    k_setfeat<<<(unsigned)((m + NT - 1) / NT), NT, 0, st>>>(z, m, c, raw);
    launches++;
    return cudaGetLastError();
}

cudaError_t launch_mlp_forward(const float *feat, const int32_t *rows, int64_t N,
                               const l1line_mlp *p, float *score, cudaStream_t st, int &launches) {
    const size_t smem = sizeof(MlpSmem);
    cudaError_t e = ensure_smem(reinterpret_cast<const void *>(k_mlp_fwd), smem);
    if (e != cudaSuccess) return e;
    k_mlp_fwd<<<(unsigned)((N + TS - 1) / TS), NT, smem, st>>>(feat, rows, N, p, score);
    launches++;
    return cudaGetLastError();
}

cudaError_t launch_mlp_backward(const float *feat, const int32_t *rows, int64_t N,
                                const l1line_mlp *p, const float *dscore, float *part,
                                float *grad, cudaStream_t st, int &launches) {
    const size_t smem = sizeof(MlpSmem);
    cudaError_t e = ensure_smem(reinterpret_cast<const void *>(k_mlp_bwd), smem);
    if (e != cudaSuccess) return e;
    const int nblk = (int)((N + TS - 1) / TS);
    k_mlp_bwd<<<nblk, NT, smem, st>>>(feat, rows, N, p, dscore, part);
    launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_grad_sum<<<(NPAR + 255) / 256, 256, 0, st>>>(part, nblk, grad);
    launches++;
    return cudaGetLastError();
}

cudaError_t launch_rank_loss(const float *score, const float *target, const int32_t *rows,
                             const int64_t *off, int64_t n_inst, float *ds, float *loss,
                             cudaStream_t st, int &launches) {
    k_rank_loss<<<(unsigned)n_inst, NT, 0, st>>>(score, target, rows, off, n_inst, ds, loss);
    launches++;
    return cudaGetLastError();
}

cudaError_t launch_adam(float *theta, const float *grad, float *m1, float *m2, float lr,
                        float beta1, float beta2, float eps, float c1, float c2, l1line_mlp *out,
                        cudaStream_t st, int &launches) {
    k_adam<<<(NPAR + 255) / 256, 256, 0, st>>>(theta, grad, m1, m2, lr, beta1, beta2, eps, c1, c2,
                                               out);
    launches++;
    return cudaGetLastError();
}

cudaError_t launch_mlp_pack(const float *theta, l1line_mlp *out, cudaStream_t st, int &launches) {
    k_mlp_pack<<<(NPAR + 255) / 256, 256, 0, st>>>(theta, out);
    launches++;
    return cudaGetLastError();
}

cudaError_t launch_topk(const float *score, int64_t m, int K, int32_t *out, cudaStream_t st,
                        int &launches) {
    k_topk<<<1, TK_NT, 0, st>>>(score, m, K, out);
    launches++;
    return cudaGetLastError();
}

template cudaError_t launch_colfeat<float>(const float *, int64_t, int64_t, int64_t, float *,
                                           cudaStream_t, int &);
template cudaError_t launch_colfeat<double>(const double *, int64_t, int64_t, int64_t, float *,
                                            cudaStream_t, int &);
template cudaError_t launch_heavy_rows<float>(const float *, int64_t, int64_t, int64_t, float *,
                                              int32_t *, float *, cudaStream_t, int &);
template cudaError_t launch_heavy_rows<double>(const double *, int64_t, int64_t, int64_t,
                                               float *, int32_t *, double *, cudaStream_t, int &);

}  // namespace l1l
