// bench_probes.cu -- measurement probes for bench.py's rooflines, built into
// their own shared library (libswgb_probes.so beside this file), outside the
// alignment library.
//
//   probe_alu     operations per second the GPU sustains for one of the
//                 instruction kinds the DP kernels use;
//   probe_gather  random 4-byte loads per second over a buffer much larger
//                 than L2, the ceiling of kernels whose traffic is scattered
//                 32-byte sectors.
//
// Both return 0 on success, -1 for invalid arguments and -3 when a CUDA call
// fails; they allocate and free their own buffers and time one launch with
// CUDA events on the given stream after one shorter warm-up launch.
#include <cstdint>
#include <cuda_runtime.h>

namespace {

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel)
{
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}

// Every thread runs 8 independent dependency chains of one instruction kind
// (enough independent work to hide latency at full occupancy), on every SM:
//   0 add-max (s32), 1 add-max (16x2), 2 three-way max (16x2), 3 add,
//   4 byte permute, 5 multiply-add, 6 add-max (16x2) and multiply-add mixed.
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

// Each thread keeps 8 independent loads in flight, at addresses from a 64-bit
// LCG, and folds the values so that no load is dead.
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

constexpr int kOk = 0, kBadArg = -1, kCuda = -3;

void launch_alu(int kind, int64_t iters, int blocks, int threads, uint32_t *out, cudaStream_t st)
{
    const uint32_t seed = 12345u;
    switch (kind) {
    case 0: k_alu_probe<0><<<blocks, threads, 0, st>>>(iters, seed, out); break;
    case 1: k_alu_probe<1><<<blocks, threads, 0, st>>>(iters, seed, out); break;
    case 2: k_alu_probe<2><<<blocks, threads, 0, st>>>(iters, seed, out); break;
    case 3: k_alu_probe<3><<<blocks, threads, 0, st>>>(iters, seed, out); break;
    case 4: k_alu_probe<4><<<blocks, threads, 0, st>>>(iters, seed, out); break;
    case 5: k_alu_probe<5><<<blocks, threads, 0, st>>>(iters, seed, out); break;
    default: k_alu_probe<6><<<blocks, threads, 0, st>>>(iters, seed, out); break;
    }
}

int sm_count(int *sms)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return kCuda;
    if (cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || *sms < 1) return kCuda;
    return kOk;
}

// Times launch(iterations) after launch(warm-up iterations); milliseconds.
template <typename F>
int time_launch(F launch, int64_t iters, cudaStream_t st, float *ms)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = kOk;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = kCuda;
    if (!rc) launch(iters / 8 + 1);
    if (!rc && cudaEventRecord(e0, st) != cudaSuccess) rc = kCuda;
    if (!rc) launch(iters);
    if (!rc && cudaEventRecord(e1, st) != cudaSuccess) rc = kCuda;
    if (!rc && (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(ms, e0, e1) != cudaSuccess))
        rc = kCuda;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return rc;
}

}  // namespace

extern "C" int probe_alu(int32_t kind, int64_t iters, double *ops_per_s, void *stream)
{
    if (!ops_per_s || iters < 1 || kind < 0 || kind > 6) return kBadArg;
    int sms = 0;
    if (sm_count(&sms)) return kCuda;
    cudaStream_t st = (cudaStream_t)stream;
    const int threads = 256, blocks = sms * 8;
    uint32_t *out = nullptr;
    if (cudaMalloc(&out, sizeof(uint32_t) * threads * blocks) != cudaSuccess) return kCuda;
    float ms = 0.f;
    const int rc = time_launch([&](int64_t it) { launch_alu(kind, it, blocks, threads, out, st); }, iters, st, &ms);
    cudaFree(out);
    if (rc) return rc;
    *ops_per_s = (double)blocks * threads * 8.0 * (double)iters / (ms * 1e-3);
    return kOk;
}

extern "C" int probe_gather(int32_t log2_words, int64_t rounds, double *loads_per_s, void *stream)
{
    if (!loads_per_s || log2_words < 20 || log2_words > 34 || rounds < 1) return kBadArg;
    int sms = 0;
    if (sm_count(&sms)) return kCuda;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t words = (size_t)1 << log2_words;
    const int threads = 256, blocks = sms * 8;
    uint32_t *buf = nullptr, *out = nullptr;
    if (cudaMalloc(&buf, words * sizeof(uint32_t)) != cudaSuccess) return kCuda;
    if (cudaMalloc(&out, sizeof(uint32_t) * threads * blocks) != cudaSuccess) {
        cudaFree(buf);
        return kCuda;
    }
    float ms = 0.f;
    int rc = cudaMemsetAsync(buf, 0x5A, words * sizeof(uint32_t), st) == cudaSuccess ? kOk : kCuda;
    if (!rc)
        rc = time_launch([&](int64_t r) { k_gather_probe<<<blocks, threads, 0, st>>>(buf, words - 1, r, out); }, rounds,
                         st, &ms);
    cudaFree(out);
    cudaFree(buf);
    if (rc) return rc;
    *loads_per_s = (double)blocks * threads * 8.0 * (double)rounds / (ms * 1e-3);
    return kOk;
}
