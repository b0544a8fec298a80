// k_probe.cu -- bandwidth probes for the roofline denominators of the pair
// kernel: L2 read bandwidth (a buffer that fits in the L2, read over and over)
// and shared-memory read bandwidth.  Measurement only; nothing on the fit
// path calls them.
#include <algorithm>

#include "common.cuh"
#include "launch.h"

namespace l1l {

constexpr int PROBE_SMEM_WORDS = 2048;  // 32 KB of 16-byte words per CTA
constexpr int PROBE_SMEM_THREADS = 512;
constexpr int PROBE_SMEM_UNROLL = 8;

// Grid-stride 16-byte loads that bypass L1 (.cg), eight in flight per thread
// (the L2 latency under load times the SM's share of the bandwidth is more
// than four loads per thread cover), `reps` passes over the buffer.  The folded
// sum reaches memory only in the practically impossible case below, which
// keeps the loads live.
constexpr int PROBE_L2_UNROLL = 8;
__global__ void __launch_bounds__(256) k_probe_l2(const uint4 *__restrict__ buf, int64_t words,
                                                  int reps, unsigned *sink) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned acc[PROBE_L2_UNROLL] = {};
    for (int r = 0; r < reps; ++r) {
        int64_t w = t0;
        for (; w + (PROBE_L2_UNROLL - 1) * stride < words; w += PROBE_L2_UNROLL * stride) {
            uint4 v[PROBE_L2_UNROLL];
#pragma unroll
            for (int u = 0; u < PROBE_L2_UNROLL; ++u) v[u] = __ldcg(buf + w + u * stride);
#pragma unroll
            for (int u = 0; u < PROBE_L2_UNROLL; ++u)
                acc[u] += v[u].x ^ v[u].y ^ v[u].z ^ v[u].w;
        }
        for (; w < words; w += stride) {
            const uint4 v = __ldcg(buf + w);
            acc[0] += v.x ^ v.y ^ v.z ^ v.w;
        }
    }
    unsigned f = 0;
#pragma unroll
    for (int u = 0; u < PROBE_L2_UNROLL; ++u) f ^= acc[u];
    if (f == 0x9E3779B9u) atomicAdd(sink, 1u);
}

// Each thread reads PROBE_SMEM_UNROLL 16-byte shared words per rep; the 32
// lanes of a warp read 32 consecutive words (512 bytes, no bank conflicts).
__global__ void __launch_bounds__(PROBE_SMEM_THREADS) k_probe_smem(int reps, unsigned *sink) {
    __shared__ uint4 s[PROBE_SMEM_WORDS];
    for (int i = threadIdx.x; i < PROBE_SMEM_WORDS; i += blockDim.x)
        s[i] = make_uint4((unsigned)i, (unsigned)i * 3u, (unsigned)i * 5u, (unsigned)i * 7u);
    __syncthreads();
    unsigned a0 = 0, a1 = 0;
    const int base = threadIdx.x;
    for (int r = 0; r < reps; ++r) {
#pragma unroll
        for (int u = 0; u < PROBE_SMEM_UNROLL; u += 2) {
            const uint4 v0 = s[(base + u * 64 + r) & (PROBE_SMEM_WORDS - 1)];
            const uint4 v1 = s[(base + (u + 1) * 64 + r) & (PROBE_SMEM_WORDS - 1)];
            a0 += v0.x ^ v0.y ^ v0.z ^ v0.w;
            a1 += v1.x ^ v1.y ^ v1.z ^ v1.w;
        }
    }
    if ((a0 ^ a1) == 0x9E3779B9u) atomicAdd(sink, 1u);
}

cudaError_t launch_probe(int kind, const void *buf, size_t bytes, int reps, unsigned *sink,
                         int num_sms, cudaStream_t st, double *bytes_read, int &launches) {
    if (kind == PROBE_L2) {
        const int64_t words = (int64_t)(bytes / 16);
        k_probe_l2<<<num_sms * 4, 256, 0, st>>>(static_cast<const uint4 *>(buf), words, reps,
                                                sink);
        *bytes_read = (double)words * 16.0 * (double)reps;
    } else {
        const int grid = num_sms * 4;  // 4 x 512 threads and 4 x 32 KB fit one SM
        k_probe_smem<<<grid, PROBE_SMEM_THREADS, 0, st>>>(reps, sink);
        *bytes_read = (double)grid * PROBE_SMEM_THREADS * (double)reps * PROBE_SMEM_UNROLL * 16.0;
    }
    launches++;
    return cudaGetLastError();
}

}  // namespace l1l
