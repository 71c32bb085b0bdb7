// alu_probe.cu -- instruction-throughput probe for the integer roofline.
//
// The score pass is bound by integer ALU issue, not by memory or tensor
// cores, and the measured-peaks file only holds HBM and bf16 figures.  This
// kernel measures how many operations per second the GPU sustains for the
// instruction kinds the DP uses: every thread runs 8 independent dependency
// chains of one kind (enough independent work to hide latency at full
// occupancy), on every SM.
#include "sw_device.cuh"
#include "swgb_internal.h"

namespace swgb {

template <int KIND>
__global__ void __launch_bounds__(256) k_alu_probe(int64_t iters, uint32_t seed, uint32_t *out)
{
    uint32_t a[8];
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = (tid * 2654435761u) ^ (seed + 977u * q);
    const uint32_t b = seed * 3u + 0x00050005u, c = seed ^ 0x10001000u;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (KIND == 0) a[q] = (uint32_t)__viaddmax_s32((int)a[q], (int)b, (int)c);
            if (KIND == 1) a[q] = __viaddmax_s16x2(a[q], b, c);
            if (KIND == 2) a[q] = __vimax3_s16x2(a[q], a[(q + 1) & 7], b);
            if (KIND == 3) a[q] = a[q] + a[(q + 3) & 7];
            if (KIND == 4) a[q] = prmt(a[q], b, a[(q + 5) & 7]);
            if (KIND == 5) a[q] = a[q] * b + c;
            if (KIND == 6) {
                if (q & 1) a[q] = a[q] * b + c;
                else a[q] = __viaddmax_s16x2(a[q], b, c);
            }
        }
    }
    uint32_t x = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) x ^= a[q];
    out[tid] = x;
}

// Random 4-byte loads over a buffer much larger than L2: each thread keeps 8
// independent loads in flight, at addresses from a 64-bit LCG, and folds the
// values so that no load is dead.  The rate, in loads per second, is the
// ceiling for kernels whose traffic is scattered 32-byte sectors.
__global__ void __launch_bounds__(256) k_gather_probe(const uint32_t *__restrict__ buf, uint64_t mask,
                                                     int64_t rounds, uint32_t *out)
{
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    uint64_t x = tid * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
    uint32_t acc = 0;
    for (int64_t i = 0; i < rounds; ++i) {
        uint32_t v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            x = x * 6364136223846793005ull + 1442695040888963407ull;
            v[q] = __ldg(buf + ((x >> 17) & mask));
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) acc ^= v[q];
    }
    out[tid] = acc;
}

int launch_gather_probe(const uint32_t *buf, uint64_t mask, int64_t rounds, int blocks, int threads, uint32_t *out,
                        cudaStream_t st)
{
    k_gather_probe<<<blocks, threads, 0, st>>>(buf, mask, rounds, out);
    count_launch();
    return launch_status();
}

int launch_alu_probe(int kind, int64_t iters, int blocks, int threads, uint32_t *out, cudaStream_t st)
{
    const uint32_t seed = 12345u;
    switch (kind) {
    case 0: k_alu_probe<0><<<blocks, threads, 0, st>>>(iters, seed, out); break;
    case 1: k_alu_probe<1><<<blocks, threads, 0, st>>>(iters, seed, out); break;
    case 2: k_alu_probe<2><<<blocks, threads, 0, st>>>(iters, seed, out); break;
    case 3: k_alu_probe<3><<<blocks, threads, 0, st>>>(iters, seed, out); break;
    case 4: k_alu_probe<4><<<blocks, threads, 0, st>>>(iters, seed, out); break;
    case 5: k_alu_probe<5><<<blocks, threads, 0, st>>>(iters, seed, out); break;
    case 6: k_alu_probe<6><<<blocks, threads, 0, st>>>(iters, seed, out); break;
    default: return SW_ERR_INVALID_ARG;
    }
    count_launch();
    return launch_status();
}

}  // namespace swgb
