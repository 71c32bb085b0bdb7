// sw_filter.cu -- the learned candidate filter in front of Smith-Waterman.
//
// The paper's Stage E runs SW on every extended CAL of a read.  The filter
// ranks a read's candidates by a small network's prediction of the SW score
// so that only the top ones are aligned; reads whose ranking is not clear-cut
// fall back to aligning every candidate.  It never changes a reported score:
// the score of a read is the SW score of its best aligned candidate.
//
// Features: for pair (read of length m, window), the 4-mers q = 64 b0 + 16 b1
// + 4 b2 + b3 of both strings are counted; per 3-base prefix k = q >> 2 the
// shared counts min(c_read, c_window) are summed over the last base and
// divided by m - 3, giving 64 values stored as bf16.
//
// Network 64 -> 256 -> 64 -> 1 with ReLU: y = w3 . relu(W2^T relu(W1^T f +
// b1) + b2) + b3.  Serving runs on the tensor cores (tcgen05 with TMEM
// accumulators, sw_mlp_tc.cu; an mma.sync kernel here is the selectable
// alternative), bf16 operands and fp32 accumulation.  Training minimises the
// mean squared error against SW score / (match m): the gradient on the
// tensor cores as well (sw_mlp_tc.cu; an fp32 CUDA-core kernel here is the
// selectable alternative), then Adam.
#include <algorithm>

#include <cuda_bf16.h>

#include <atomic>

#include "sw_device.cuh"
#include "swgb_internal.h"

namespace swgb {

constexpr unsigned FM = 0xffffffffu;

// ---------------------------------------------------------------- features

// 4-mers are indexed in stream order, w = b0 + 4 b1 + 16 b2 + 64 b3 (b0 the
// first base, as the 2-bit packing stores it), so a 4-mer's counter address
// is one shift and one mask of the packed word.  Feature slot k = 16 b0 +
// 4 b1 + b2 is prefix p = w & 63 = slot_prefix(k) read the other way round,
// summed over the last base b3 = w >> 6.
__device__ __forceinline__ int slot_prefix(int k) { return (k >> 4) + 4 * ((k >> 2) & 3) + 16 * (k & 3); }

// The up-to-8 4-mers at positions base .. base + cnt - 1 of v (bases base ..
// base + 10 in bits 0 .. 21) as counter increments: 32-bit counters at word w.
__device__ __forceinline__ void bump8_words(uint32_t v, int cnt, uint32_t *hist)
{
#pragma unroll
    for (int t = 0; t < 8; ++t)
        if (t < cnt) atomicAdd(&hist[(v >> (2 * t)) & 0xFFu], 1u);
}

// Byte counters, four per word: word p = w & 63, byte b3 = w >> 6.
__device__ __forceinline__ void bump8_bytes(uint32_t v, int cnt, uint32_t *hist)
{
#pragma unroll
    for (int t = 0; t < 8; ++t)
        if (t < cnt) {
            const uint32_t w = v >> (2 * t);
            atomicAdd(&hist[w & 63u], 1u << ((w >> 3) & 0x18u));
        }
}

// Count the 4-mers of bases [s, s+len) into hist; lane l takes positions
// 8l .. 8l+7 of every 256.  BYTES: four byte counters per word (exact while
// no 4-mer occurs more than 255 times, i.e. for at most 258 bases), else
// 256 32-bit counters.
template <bool BYTES>
__device__ __forceinline__ void count_kmers(const uint32_t *__restrict__ buf, int64_t s, int32_t len,
                                            uint32_t *hist, int lane)
{
    const int nk = len - 3;  // number of 4-mers
    for (int base = lane * 8; base < nk; base += 32 * 8) {
        // 8 k-mers starting at base .. base+7 need bases base .. base+10
        const uint32_t v = load_bases(buf, s + base, min(11, len - base));
        if (BYTES) bump8_bytes(v, nk - base, hist);
        else bump8_words(v, nk - base, hist);
    }
}

constexpr int kByteCountMax = 258;

// Byte counters of the 4-mers at positions first .. first + cnt - 1 of a
// sequence (first + cnt <= len - 3), eight at a time.
__device__ __forceinline__ void count_run8(const uint32_t *__restrict__ buf, int64_t s, int32_t len, int first,
                                           int cnt, uint32_t *hist)
{
    for (int h = 0; h < cnt; h += 8) {
        const int q = first + h;
        const uint32_t v = load_bases(buf, s + q, min(11, len - q));
        bump8_bytes(v, cnt - h, hist);
    }
}

__global__ void __launch_bounds__(256) k_features(FeatureParams P)
{
    __shared__ uint32_t hist[8][2][256];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t *hr = hist[warp][0], *hw = hist[warp][1];
    // byte-counter path: four candidates at a time, 8 lanes and 64 words each
    const int sg = lane >> 3, sl = lane & 7;
    uint32_t *hs = hist[warp][1] + 64 * sg;
    // this lane's output slots: 8 sl .. 8 sl + 7 on the byte path, 2 lane
    // and 2 lane + 1 on the word path (prefixes p and p + 16)
    const int pw = slot_prefix(2 * lane);
    for (int64_t r = (int64_t)blockIdx.x * 8 + warp; r < P.n_reads; r += (int64_t)gridDim.x * 8) {
        const int64_t c0 = P.cand_off[r], c1 = P.cand_off[r + 1];
        if (c0 >= c1) continue;
        const int64_t rs = P.read_off[r];
        const int32_t m = (int32_t)(P.read_off[r + 1] - rs);
        const bool rbytes = m <= kByteCountMax;
        for (int q = lane; q < 256; q += 32) hr[q] = 0;
        __syncwarp();
        if (m >= 4) {
            if (rbytes) count_kmers<true>(P.reads, rs, m, hr, lane);
            else count_kmers<false>(P.reads, rs, m, hr, lane);
        }
        __syncwarp();
        const float inv = m >= 4 ? 1.f / (float)(m - 3) : 0.f;
        // the longest window of the read decides the path
        int32_t nmax = 0;
        for (int64_t p = c0 + lane; p < c1; p += 32) nmax = max(nmax, (int32_t)(P.win_off[p + 1] - P.win_off[p]));
        nmax = (int32_t)__reduce_max_sync(0xffffffffu, (unsigned)nmax);
        if (rbytes && nmax <= kByteCountMax) {
            for (int64_t pb = c0; pb < c1; pb += 4) {
                const int64_t p = pb + sg;
                const bool live = p < c1;
#pragma unroll
                for (int q = 0; q < 8; ++q) hs[8 * sl + q] = 0;
                __syncwarp();
                int32_t n = 0;
                if (live) {
                    const int64_t ws = P.win_off[p];
                    n = (int32_t)(P.win_off[p + 1] - ws);
                    const int nk = n - 3;
                    // lane sl counts k-mers sl*32 .. sl*32+31
                    if (m >= 4 && sl * 32 < nk) count_run8(P.wins, ws, n, sl * 32, min(32, nk - sl * 32), hs);
                }
                __syncwarp();
                if (live) {
                    uint32_t f2[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        // slots 8 sl + 2q and + 1: prefixes p and p + 16
                        const int p0 = slot_prefix(8 * sl + 2 * q);
                        const uint32_t a = (uint32_t)__dp4a(__vminu4(hr[p0], hs[p0]), 0x01010101u, 0u);
                        const uint32_t b = (uint32_t)__dp4a(__vminu4(hr[p0 + 16], hs[p0 + 16]), 0x01010101u, 0u);
                        const __nv_bfloat162 f = __floats2bfloat162_rn((float)a * inv, (float)b * inv);
                        f2[q] = *reinterpret_cast<const uint32_t *>(&f);
                    }
                    if (n < 4 || m < 4) f2[0] = f2[1] = f2[2] = f2[3] = 0u;
                    reinterpret_cast<uint4 *>(P.out)[p * 8 + sl] = make_uint4(f2[0], f2[1], f2[2], f2[3]);
                }
                __syncwarp();
            }
            continue;
        }
        for (int64_t p = c0; p < c1; ++p) {
            const int64_t ws = P.win_off[p];
            const int32_t n = (int32_t)(P.win_off[p + 1] - ws);
            uint32_t s0 = 0, s1 = 0;
            if (rbytes && n <= kByteCountMax) {
                // byte counters: feature p = byte sum of min(read word p, window word p)
                hw[lane] = 0;
                hw[lane + 32] = 0;
                __syncwarp();
                if (n >= 4 && m >= 4) count_kmers<true>(P.wins, ws, n, hw, lane);
                __syncwarp();
                s0 = (uint32_t)__dp4a(__vminu4(hr[pw], hw[pw]), 0x01010101u, 0u);
                s1 = (uint32_t)__dp4a(__vminu4(hr[pw + 16], hw[pw + 16]), 0x01010101u, 0u);
            } else {
                for (int q = lane; q < 256; q += 32) hw[q] = 0;
                __syncwarp();
                if (n >= 4 && m >= 4) count_kmers<false>(P.wins, ws, n, hw, lane);
                __syncwarp();
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const uint32_t r0 = rbytes ? (hr[pw] >> (8 * b)) & 0xFFu : hr[pw + 64 * b];
                    const uint32_t r1 = rbytes ? (hr[pw + 16] >> (8 * b)) & 0xFFu : hr[pw + 16 + 64 * b];
                    s0 += min(r0, hw[pw + 64 * b]);
                    s1 += min(r1, hw[pw + 16 + 64 * b]);
                }
            }
            const __nv_bfloat162 f = __floats2bfloat162_rn((float)s0 * inv, (float)s1 * inv);
            reinterpret_cast<__nv_bfloat162 *>(P.out)[p * 32 + lane] = f;
            __syncwarp();
        }
    }
}

// --------------------------------------------------------- model layout

// fp32 offsets into the model buffer (see include/swgb.h)

// bf16 copies of the weights, transposed for the tensor-core B operands
__global__ void k_mlp_refresh(float *model)
{
    const float *W1 = model + MD_W1, *W2 = model + MD_W2;
    __nv_bfloat16 *w1t = reinterpret_cast<__nv_bfloat16 *>(model + MD_W1T);
    __nv_bfloat16 *w2t = reinterpret_cast<__nv_bfloat16 *>(model + MD_W2T);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 16384; i += gridDim.x * blockDim.x) {
        const int a = i / 256, b = i % 256;      // W1[a][b] -> w1t[b][a]
        w1t[b * 64 + a] = __float2bfloat16_rn(W1[i]);
        const int j = i / 64, k = i % 64;        // W2[j][k] -> w2t[k][j]
        w2t[k * 256 + j] = __float2bfloat16_rn(W2[i]);
    }
}

__device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// He-scaled uniform weights from a counter-based generator; zero biases,
// Adam state and step; the output bias starts at 0.5 (mid-range target)
__global__ void k_mlp_init(float *model, uint64_t seed)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < MD_STEP + 1;
         i += (int64_t)gridDim.x * blockDim.x) {
        float v = 0.f;
        if (i < MD_NP) {
            const double u = (double)(mix64(seed * 0xD1B54A32D192ED03ULL ^ mix64((uint64_t)i)) >> 11) *
                                 (1.0 / 9007199254740992.0) * 2.0 - 1.0;
            if (i < MD_B1) v = (float)(u * sqrt(6.0 / 64.0));
            else if (i >= MD_W2 && i < MD_B2) v = (float)(u * sqrt(6.0 / 256.0));
            else if (i >= MD_W3 && i < MD_B3) v = (float)(u * sqrt(6.0 / 64.0) * 0.1);
            else if (i == MD_B3) v = 0.5f;
        }
        model[i] = v;
    }
}

// ------------------------------------------------------- forward (bf16 mma)

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                 "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Four 8x8 bf16 matrices from shared memory; lane l supplies the address of
// row l % 8 of matrix l / 8 and receives, for every matrix, the pair of
// elements (row l / 4, columns 2 (l % 4) and 2 (l % 4) + 1) -- the B
// fragment layout of mma.m16n8k16 when the rows are n and the columns k.
__device__ __forceinline__ void ldsm_x4(const void *smem_row, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(smem_row);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(a));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

constexpr int W1S = 72;   // padded row of w1t in shared memory (bf16)
constexpr int W2S = 264;  // padded row of w2t

// Each warp takes 16 pairs at a time.  Layer 1 is computed in four blocks of
// 64 hidden units; each block's ReLU output is repacked in registers as the
// A operand of layer 2 (the accumulator layout of two n8 tiles is the A
// layout of one k16 step), so hidden activations never leave registers.
__global__ void __launch_bounds__(128) k_mlp_forward(const float *__restrict__ model,
                                                     const __nv_bfloat16 *__restrict__ feat, int64_t n,
                                                     float *__restrict__ out)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __nv_bfloat16 *w1 = reinterpret_cast<__nv_bfloat16 *>(smem);            // [256][W1S]
    __nv_bfloat16 *w2 = w1 + 256 * W1S;                                      // [64][W2S]
    float *b1 = reinterpret_cast<float *>(w2 + 64 * W2S);                    // [256]
    float *b2 = b1 + 256;                                                    // [64]
    float *w3 = b2 + 64;                                                     // [64]
    {
        const __nv_bfloat16 *g1 = reinterpret_cast<const __nv_bfloat16 *>(model + MD_W1T);
        const __nv_bfloat16 *g2 = reinterpret_cast<const __nv_bfloat16 *>(model + MD_W2T);
        for (int i = threadIdx.x; i < 256 * 64; i += blockDim.x) {
            w1[(i / 64) * W1S + i % 64] = g1[i];
            w2[(i / 256) * W2S + i % 256] = g2[i];
        }
        for (int i = threadIdx.x; i < 256; i += blockDim.x) b1[i] = model[MD_B1 + i];
        for (int i = threadIdx.x; i < 64; i += blockDim.x) {
            b2[i] = model[MD_B2 + i];
            w3[i] = model[MD_W3 + i];
        }
        __syncthreads();
    }
    const float b3 = model[MD_B3];
    const int lane = threadIdx.x & 31, g = lane >> 2, tig = lane & 3;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const uint32_t *X = reinterpret_cast<const uint32_t *>(feat);  // bf16 pairs: row stride 32 words
    for (int64_t tile = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); tile * 16 < n;
         tile += warps) {
        const int64_t r0 = tile * 16 + g, r1 = r0 + 8;
        uint32_t xa[4][4];
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            const int c = kk * 8 + tig;  // word column (2 bf16)
            xa[kk][0] = r0 < n ? X[r0 * 32 + c] : 0u;
            xa[kk][1] = r1 < n ? X[r1 * 32 + c] : 0u;
            xa[kk][2] = r0 < n ? X[r0 * 32 + c + 4] : 0u;
            xa[kk][3] = r1 < n ? X[r1 * 32 + c + 4] : 0u;
        }
        float acc2[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const float c0 = b2[nt * 8 + tig * 2], c1 = b2[nt * 8 + tig * 2 + 1];
            acc2[nt][0] = c0; acc2[nt][1] = c1; acc2[nt][2] = c0; acc2[nt][3] = c1;
        }
#pragma unroll 1
        for (int nb = 0; nb < 4; ++nb) {
            float acc1[8][4];
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                const int col = nb * 64 + nt * 8 + tig * 2;
                acc1[nt][0] = b1[col]; acc1[nt][1] = b1[col + 1]; acc1[nt][2] = b1[col]; acc1[nt][3] = b1[col + 1];
            }
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
                for (int np = 0; np < 4; ++np) {
                    // n-tiles 2np, 2np+1: rows n0 .. n0+15, columns k0 .. k0+15
                    uint32_t b00, b01, b10, b11;
                    ldsm_x4(w1 + (nb * 64 + np * 16 + (lane >> 4) * 8 + (lane & 7)) * W1S + kk * 16 +
                                ((lane >> 3) & 1) * 8,
                            b00, b01, b10, b11);
                    mma_bf16(acc1[2 * np], xa[kk][0], xa[kk][1], xa[kk][2], xa[kk][3], b00, b01);
                    mma_bf16(acc1[2 * np + 1], xa[kk][0], xa[kk][1], xa[kk][2], xa[kk][3], b10, b11);
                }
            }
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
                const float *t0 = acc1[2 * ks], *t1 = acc1[2 * ks + 1];
                const uint32_t a0 = pack_bf16(fmaxf(t0[0], 0.f), fmaxf(t0[1], 0.f));
                const uint32_t a1 = pack_bf16(fmaxf(t0[2], 0.f), fmaxf(t0[3], 0.f));
                const uint32_t a2 = pack_bf16(fmaxf(t1[0], 0.f), fmaxf(t1[1], 0.f));
                const uint32_t a3 = pack_bf16(fmaxf(t1[2], 0.f), fmaxf(t1[3], 0.f));
#pragma unroll
                for (int np = 0; np < 4; ++np) {
                    uint32_t b00, b01, b10, b11;
                    ldsm_x4(w2 + (np * 16 + (lane >> 4) * 8 + (lane & 7)) * W2S + nb * 64 + ks * 16 +
                                ((lane >> 3) & 1) * 8,
                            b00, b01, b10, b11);
                    mma_bf16(acc2[2 * np], a0, a1, a2, a3, b00, b01);
                    mma_bf16(acc2[2 * np + 1], a0, a1, a2, a3, b10, b11);
                }
            }
        }
        float y0 = 0.f, y1 = 0.f;
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const float wa = w3[nt * 8 + tig * 2], wb = w3[nt * 8 + tig * 2 + 1];
            y0 += fmaxf(acc2[nt][0], 0.f) * wa + fmaxf(acc2[nt][1], 0.f) * wb;
            y1 += fmaxf(acc2[nt][2], 0.f) * wa + fmaxf(acc2[nt][3], 0.f) * wb;
        }
        y0 += __shfl_xor_sync(FM, y0, 1);
        y0 += __shfl_xor_sync(FM, y0, 2);
        y1 += __shfl_xor_sync(FM, y1, 1);
        y1 += __shfl_xor_sync(FM, y1, 2);
        if (tig == 0) {
            if (r0 < n) out[r0] = y0 + b3;
            if (r1 < n) out[r1] = y1 + b3;
        }
    }
}

// ------------------------------------------------- training (fp32, CUDA cores)

constexpr int GR_THREADS = 256;
constexpr int W2TS = 257;  // padded row of the transposed fp32 W2 in shared memory

// Mean-squared-error gradient over samples [s0, s1) of the batch, added
// into G.  Thread j owns hidden unit j of layer 1: its column of dW1 and its
// row of dW2 stay in registers for the whole chunk.
__global__ void __launch_bounds__(GR_THREADS, 1)
    k_mlp_grad(float *model, const __nv_bfloat16 *__restrict__ feat, const float *__restrict__ target,
               const int32_t *__restrict__ idx, int64_t n, int64_t per_block)
{
    extern __shared__ __align__(16) unsigned char smem[];
    float *W1 = reinterpret_cast<float *>(smem);        // [64][256]
    float *W2T = W1 + 64 * 256;                         // [64][W2TS]  (W2T[k][j] = W2[j][k])
    float *x = W2T + 64 * W2TS;                         // [64]
    float *a1 = x + 64;                                 // [256]
    float *part = a1 + 256;                             // [4][64]
    float *dz2 = part + 256;                            // [64]
    float *red = dz2 + 64;                              // [8]
    const int j = threadIdx.x;
    for (int i = j; i < 64 * 256; i += GR_THREADS) {
        W1[i] = model[MD_W1 + i];
        const int jj = i / 64, k = i % 64;
        W2T[k * W2TS + jj] = model[MD_W2 + i];
    }
    __syncthreads();
    const float b1j = model[MD_B1 + j];
    const float b2k = j < 64 ? model[MD_B2 + j] : 0.f;
    const float w3k = j < 64 ? model[MD_W3 + j] : 0.f;
    const float b3 = model[MD_B3];
    float gW1[64], gW2[64];
#pragma unroll
    for (int q = 0; q < 64; ++q) {
        gW1[q] = 0.f;
        gW2[q] = 0.f;
    }
    float gb1 = 0.f, gb2 = 0.f, gw3 = 0.f, gb3 = 0.f;
    const int64_t s0 = blockIdx.x * per_block, s1 = min(n, s0 + per_block);
    const float scale = 2.f / (float)n;
    for (int64_t s = s0; s < s1; ++s) {
        const int64_t row = idx ? idx[s] : s;
        if (j < 64) x[j] = __bfloat162float(feat[row * 64 + j]);
        __syncthreads();
        float z1 = b1j;
#pragma unroll 8
        for (int i = 0; i < 64; ++i) z1 += x[i] * W1[i * 256 + j];
        const float a = fmaxf(z1, 0.f);
        a1[j] = a;
        __syncthreads();
        {   // z2[k], four partial sums per output
            const int k = j & 63, pr = j >> 6;
            float z = 0.f;
#pragma unroll 8
            for (int jj = pr * 64; jj < pr * 64 + 64; ++jj) z += a1[jj] * W2T[k * W2TS + jj];
            part[pr * 64 + k] = z;
        }
        __syncthreads();
        float z2 = 0.f, a2 = 0.f;
        if (j < 64) {
            z2 = b2k + part[j] + part[64 + j] + part[128 + j] + part[192 + j];
            a2 = fmaxf(z2, 0.f);
            float yp = a2 * w3k;
            for (int o = 16; o > 0; o >>= 1) yp += __shfl_xor_sync(FM, yp, o);
            if ((j & 31) == 0) red[j >> 5] = yp;
        }
        __syncthreads();
        const float y = red[0] + red[1] + b3;
        const float dy = scale * (y - target[row]);
        if (j < 64) {
            const float d = z2 > 0.f ? dy * w3k : 0.f;
            dz2[j] = d;
            gw3 += a2 * dy;
            gb2 += d;
        }
        if (j == 0) gb3 += dy;
        __syncthreads();
        float da1 = 0.f;
#pragma unroll 8
        for (int k = 0; k < 64; ++k) {
            const float d = dz2[k];
            da1 += d * W2T[k * W2TS + j];
            gW2[k] += a * d;
        }
        const float dz1 = z1 > 0.f ? da1 : 0.f;
        gb1 += dz1;
#pragma unroll
        for (int i = 0; i < 64; ++i) gW1[i] += x[i] * dz1;
        __syncthreads();
    }
    float *G = model + MD_G;
#pragma unroll
    for (int i = 0; i < 64; ++i) atomicAdd(&G[MD_W1 + i * 256 + j], gW1[i]);
#pragma unroll
    for (int k = 0; k < 64; ++k) atomicAdd(&G[MD_W2 + j * 64 + k], gW2[k]);
    atomicAdd(&G[MD_B1 + j], gb1);
    if (j < 64) {
        atomicAdd(&G[MD_B2 + j], gb2);
        atomicAdd(&G[MD_W3 + j], gw3);
    }
    if (j == 0) atomicAdd(&G[MD_B3], gb3);
}

// One Adam step (Kingma & Ba) on the fp32 parameters from the gradient in G.
__global__ void k_mlp_adam(float *model, float lr, int32_t step)
{
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < MD_NP; i += (int64_t)gridDim.x * blockDim.x) {
        const float g = model[MD_G + i];
        const float m = b1 * model[MD_M + i] + (1.f - b1) * g;
        const float v = b2 * model[MD_V + i] + (1.f - b2) * g * g;
        model[MD_M + i] = m;
        model[MD_V + i] = v;
        model[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
    }
}

// ---------------------------------------------------- selection and best hit

// Per read, with the (k, tau, delta) of the rule for its length (the first
// rule whose bound is at least the read's length, else the last; without
// read offsets the first rule): the k best predictions (ties: lower
// candidate index first) and every other candidate whose prediction lies
// less than delta below the read's best; if the k-th and the (k+1)-th are
// closer than tau, every candidate.  The differences are taken in fp32.
__global__ void k_select(const float *__restrict__ pred, const int64_t *__restrict__ cand_off,
                         const int64_t *__restrict__ read_off, int64_t n_reads, const SelectRules rules,
                         uint8_t *__restrict__ mask)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n_reads;
         r += (int64_t)gridDim.x * blockDim.x) {
        int q = 0;
        if (read_off) {
            const int64_t m = read_off[r + 1] - read_off[r];
            while (q + 1 < rules.n && m > rules.max_len[q]) ++q;
        }
        const int k = rules.k[q];
        const float tau = rules.tau[q], delta = rules.delta[q];
        const int64_t a = cand_off[r], b = cand_off[r + 1];
        const int64_t c = b - a;
        if (c <= k) {
            for (int64_t p = a; p < b; ++p) mask[p] = 1;
            continue;
        }
        // the (k+1) best (value, index) kept sorted, best first
        float bv[SW_FILTER_MAX_K + 1];
        int64_t bi[SW_FILTER_MAX_K + 1];
        int cnt = 0;
        for (int64_t p = a; p < b; ++p) {
            const float v = pred[p];
            int pos = cnt;
            while (pos > 0 && bv[pos - 1] < v) --pos;  // strictly better moves up: ties keep index order
            if (pos > k) continue;
            const int last = cnt < k + 1 ? cnt : k;
            for (int q2 = last; q2 > pos; --q2) {
                bv[q2] = bv[q2 - 1];
                bi[q2] = bi[q2 - 1];
            }
            bv[pos] = v;
            bi[pos] = p;
            if (cnt < k + 1) ++cnt;
        }
        const bool all = bv[k - 1] - bv[k] < tau;
        const float top = bv[0];
        for (int64_t p = a; p < b; ++p) mask[p] = (all || top - pred[p] < delta) ? 1 : 0;
        if (!all)
            for (int q2 = 0; q2 < k; ++q2) mask[bi[q2]] = 1;
    }
}

__global__ void k_best_per_read(const int32_t *__restrict__ score, const int64_t *__restrict__ cand_off,
                                int64_t n_reads, const uint8_t *__restrict__ mask, int32_t *__restrict__ best,
                                int32_t *__restrict__ best_cand)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n_reads;
         r += (int64_t)gridDim.x * blockDim.x) {
        int32_t bs = -1, bc = -1;
        for (int64_t p = cand_off[r]; p < cand_off[r + 1]; ++p) {
            if (mask && !mask[p]) continue;
            if (score[p] > bs) {
                bs = score[p];
                bc = (int32_t)(p - cand_off[r]);
            }
        }
        best[r] = bs;
        if (best_cand) best_cand[r] = bc;
    }
}

// One thread: fold a status word into another (errors of one step of a
// composite call stay visible through the status word of its last step).
__global__ void k_or_status(int32_t *dst, const int32_t *src)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const int32_t v = *src;
        if (v) atomicOr(dst, v);
    }
}

// ------------------------------------------------------------ launchers

static int grid_for(int64_t items, int threads, int cap)
{
    int64_t b = (items + threads - 1) / threads;
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

int launch_features(const FeatureParams &P, int sm_count, cudaStream_t st)
{
    k_features<<<grid_for(P.n_reads, 8, (int64_t)sm_count * 16), 256, 0, st>>>(P);
    count_launch();
    return launch_status();
}

int launch_or_status(int32_t *dst, const int32_t *src, cudaStream_t st)
{
    k_or_status<<<1, 32, 0, st>>>(dst, src);
    count_launch();
    return launch_status();
}

int64_t mlp_floats() { return MD_TOTAL; }

int launch_mlp_init(float *model, uint64_t seed, cudaStream_t st)
{
    k_mlp_init<<<grid_for(MD_STEP + 1, 256, 152 * 4), 256, 0, st>>>(model, seed);
    k_mlp_refresh<<<64, 256, 0, st>>>(model);
    count_launch(2);
    return launch_status();
}

int launch_mlp_refresh(float *model, cudaStream_t st)
{
    k_mlp_refresh<<<64, 256, 0, st>>>(model);
    count_launch();
    return launch_status();
}

static size_t forward_smem() { return (size_t)(256 * W1S + 64 * W2S) * 2 + (256 + 64 + 64) * 4; }
static size_t grad_smem() { return (size_t)(64 * 256 + 64 * W2TS + 64 + 256 + 256 + 64 + 8) * 4; }

int launch_mlp_forward(const float *model, const uint16_t *feat, int64_t n, float *out, int sm_count,
                       cudaStream_t st)
{
    // per call: the attribute belongs to the current device, and calls may
    // come from several host threads at once
    if (cuda_failed(cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)forward_smem())))
        return SW_ERR_CUDA;
    int bps = 0;
    if (cuda_failed(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_mlp_forward, 128, forward_smem())))
        return SW_ERR_CUDA;
    const int64_t tiles = (n + 15) / 16;
    int64_t blocks = (tiles + 3) / 4;
    blocks = std::min<int64_t>(blocks, (int64_t)std::max(bps, 1) * sm_count);
    k_mlp_forward<<<(unsigned)std::max<int64_t>(blocks, 1), 128, forward_smem(), st>>>(
        model, reinterpret_cast<const __nv_bfloat16 *>(feat), n, out);
    count_launch();
    return launch_status();
}

int launch_mlp_grad(float *model, const uint16_t *feat, const float *target, const int32_t *idx, int64_t n,
                    int sm_count, cudaStream_t st)
{
    // per call: the attribute belongs to the current device, and calls may
    // come from several host threads at once
    if (cuda_failed(cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)grad_smem())))
        return SW_ERR_CUDA;
    if (cuda_failed(cudaMemsetAsync(model + MD_G, 0, sizeof(float) * MD_NP, st))) return SW_ERR_CUDA;
    // enough samples per block that the per-block gradient flush stays small
    const int64_t per_block = std::max<int64_t>(64, (n + sm_count - 1) / sm_count);
    const int64_t blocks = (n + per_block - 1) / per_block;
    k_mlp_grad<<<(unsigned)std::max<int64_t>(blocks, 1), GR_THREADS, grad_smem(), st>>>(
        model, reinterpret_cast<const __nv_bfloat16 *>(feat), target, idx, n, per_block);
    count_launch();
    return launch_status();
}

int launch_mlp_adam(float *model, float lr, int32_t step, cudaStream_t st)
{
    k_mlp_adam<<<grid_for(MD_NP, 256, 152 * 2), 256, 0, st>>>(model, lr, step);
    k_mlp_refresh<<<64, 256, 0, st>>>(model);
    count_launch(2);
    return launch_status();
}

int launch_select(const float *pred, const int64_t *cand_off, const int64_t *read_off, int64_t n_reads,
                  const SelectRules &rules, uint8_t *mask, cudaStream_t st)
{
    k_select<<<grid_for(n_reads, 128, 152 * 32), 128, 0, st>>>(pred, cand_off, read_off, n_reads, rules, mask);
    count_launch();
    return launch_status();
}

int launch_best_per_read(const int32_t *score, const int64_t *cand_off, int64_t n_reads, const uint8_t *mask,
                         int32_t *best, int32_t *best_cand, cudaStream_t st)
{
    k_best_per_read<<<grid_for(n_reads, 128, 152 * 32), 128, 0, st>>>(score, cand_off, n_reads, mask, best,
                                                                       best_cand);
    count_launch();
    return launch_status();
}

}  // namespace swgb

// ------------------------------------------------------------------ C ABI

using namespace swgb;

static std::atomic<int32_t> g_mlp_kind{SW_MLP_AUTO};  // set by sw_set_mlp_kernel
static std::atomic<int32_t> g_grad_kind{SW_GRAD_AUTO};  // set by sw_set_mlp_grad_kernel

static int sm_count_now(int *sms)
{
    int dev = 0;
    if (cuda_failed(cudaGetDevice(&dev))) return SW_ERR_NO_DEVICE;
    if (cuda_failed(cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev))) return SW_ERR_CUDA;
    return SW_OK;
}

extern "C" {

int sw_filter_features(const uint8_t *reads, const int64_t *read_offsets, int64_t n_reads, const uint8_t *windows,
                       const int64_t *window_offsets, const int64_t *cand_offsets, uint16_t *out_features,
                       sw_stream_t stream)
{
    if (n_reads < 0) return SW_ERR_INVALID_ARG;
    if (n_reads == 0) return SW_OK;
    if (!reads || !read_offsets || !windows || !window_offsets || !cand_offsets || !out_features)
        return SW_ERR_INVALID_ARG;
    if (((uintptr_t)reads & 15u) || ((uintptr_t)windows & 15u) || ((uintptr_t)out_features & 15u))
        return SW_ERR_INVALID_ARG;
    FeatureParams P{(const uint32_t *)reads, read_offsets, n_reads, (const uint32_t *)windows, window_offsets,
                    cand_offsets, out_features};
    int sms = 0;
    const int rc = sm_count_now(&sms);
    if (rc) return rc;
    return launch_features(P, sms, (cudaStream_t)stream);
}

int64_t sw_mlp_bytes(void) { return mlp_floats() * (int64_t)sizeof(float); }

int sw_mlp_init(float *model, uint64_t seed, sw_stream_t stream)
{
    if (!model || ((uintptr_t)model & 15u)) return SW_ERR_INVALID_ARG;
    return launch_mlp_init(model, seed, (cudaStream_t)stream);
}

int sw_mlp_refresh(float *model, sw_stream_t stream)
{
    if (!model || ((uintptr_t)model & 15u)) return SW_ERR_INVALID_ARG;
    return launch_mlp_refresh(model, (cudaStream_t)stream);
}

int sw_set_mlp_kernel(int32_t kind)
{
    if (kind != SW_MLP_AUTO && kind != SW_MLP_MMA_SYNC) return SW_ERR_INVALID_ARG;
    g_mlp_kind.store(kind);
    return SW_OK;
}

int sw_mlp_forward(const float *model, const uint16_t *features, int64_t n, float *out, sw_stream_t stream)
{
    if (n < 0 || !model || ((uintptr_t)model & 15u)) return SW_ERR_INVALID_ARG;
    if (n == 0) return SW_OK;
    if (!features || !out || ((uintptr_t)features & 3u)) return SW_ERR_INVALID_ARG;
    int sms = 0;
    int rc = sm_count_now(&sms);
    if (rc) return rc;
    // the tensor-memory kernel reads 16-byte feature rows
    if (g_mlp_kind.load() == SW_MLP_AUTO && !((uintptr_t)features & 15u)) {
        int32_t *status = nullptr;
        if ((rc = aux_status_word((cudaStream_t)stream, &status))) return rc;
        return launch_mlp_forward_tc(model, features, n, out, sms, status, (cudaStream_t)stream);
    }
    return launch_mlp_forward(model, features, n, out, sms, (cudaStream_t)stream);
}

int sw_set_mlp_grad_kernel(int32_t kind)
{
    if (kind != SW_GRAD_AUTO && kind != SW_GRAD_FP32) return SW_ERR_INVALID_ARG;
    g_grad_kind.store(kind);
    return SW_OK;
}

int sw_mlp_grad(float *model, const uint16_t *features, const float *target, const int32_t *idx, int64_t n,
                sw_stream_t stream)
{
    if (n < 1 || !model || !features || !target || ((uintptr_t)model & 15u)) return SW_ERR_INVALID_ARG;
    int sms = 0;
    int rc = sm_count_now(&sms);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    // the tensor-core kernel reads 16-byte feature rows
    if (g_grad_kind.load() == SW_GRAD_AUTO && !((uintptr_t)features & 15u)) {
        int32_t *status = nullptr;
        if ((rc = aux_status_word(st, &status))) return rc;
        float *partial = nullptr;
        if ((rc = grad_scratch(st, sizeof(float) * (size_t)MD_NP * mlp_grad_tc_parts(n, sms), &partial))) return rc;
        return launch_mlp_grad_tc(model, features, target, idx, n, sms, partial, status, st);
    }
    return launch_mlp_grad(model, features, target, idx, n, sms, st);
}

int sw_mlp_adam(float *model, float lr, int32_t step, sw_stream_t stream)
{
    if (!model || step < 1 || !(lr > 0.f)) return SW_ERR_INVALID_ARG;
    return launch_mlp_adam(model, lr, step, (cudaStream_t)stream);
}

// Host-side check of a rule table: 1..SW_FILTER_MAX_RULES rules with
// ascending bounds, 1 <= k <= SW_FILTER_MAX_K and delta >= 0 each.
static int make_rules(const sw_select_rule_t *rules, int32_t n_rules, SelectRules *out)
{
    if (!rules || n_rules < 1 || n_rules > SW_FILTER_MAX_RULES) return SW_ERR_INVALID_ARG;
    out->n = n_rules;
    for (int q = 0; q < n_rules; ++q) {
        const sw_select_rule_t &u = rules[q];
        if (u.k < 1 || u.k > SW_FILTER_MAX_K || !(u.delta >= 0.f)) return SW_ERR_INVALID_ARG;
        if (q > 0 && u.max_read_len < rules[q - 1].max_read_len) return SW_ERR_INVALID_ARG;
        out->max_len[q] = u.max_read_len;
        out->k[q] = u.k;
        out->tau[q] = u.tau;
        out->delta[q] = u.delta;
    }
    return SW_OK;
}

int sw_filter_select(const float *pred, const int64_t *cand_offsets, int64_t n_reads, int32_t k, float tau,
                     float delta, uint8_t *pair_mask, sw_stream_t stream)
{
    const sw_select_rule_t one{INT32_MAX, k, tau, delta};
    SelectRules rules;
    if (n_reads < 0 || make_rules(&one, 1, &rules)) return SW_ERR_INVALID_ARG;
    if (n_reads == 0) return SW_OK;
    if (!pred || !cand_offsets || !pair_mask) return SW_ERR_INVALID_ARG;
    return launch_select(pred, cand_offsets, nullptr, n_reads, rules, pair_mask, (cudaStream_t)stream);
}

int sw_filter_select_by_length(const float *pred, const int64_t *cand_offsets, const int64_t *read_offsets,
                               int64_t n_reads, const sw_select_rule_t *rules, int32_t n_rules, uint8_t *pair_mask,
                               sw_stream_t stream)
{
    SelectRules sr;
    if (n_reads < 0 || make_rules(rules, n_rules, &sr)) return SW_ERR_INVALID_ARG;
    if (n_reads == 0) return SW_OK;
    if (!pred || !cand_offsets || !pair_mask || (n_rules > 1 && !read_offsets)) return SW_ERR_INVALID_ARG;
    return launch_select(pred, cand_offsets, n_rules > 1 ? read_offsets : nullptr, n_reads, sr, pair_mask,
                         (cudaStream_t)stream);
}

int sw_best_per_read(const int32_t *score, const int64_t *cand_offsets, int64_t n_reads, const uint8_t *pair_mask,
                     int32_t *best_score, int32_t *best_cand, sw_stream_t stream)
{
    if (n_reads < 0) return SW_ERR_INVALID_ARG;
    if (n_reads == 0) return SW_OK;
    if (!score || !cand_offsets || !best_score) return SW_ERR_INVALID_ARG;
    return launch_best_per_read(score, cand_offsets, n_reads, pair_mask, best_score, best_cand,
                                (cudaStream_t)stream);
}

int sw_filter_align(const uint8_t *reads, const int64_t *read_offsets, int64_t n_reads, const uint8_t *windows,
                    const int64_t *window_offsets, const int64_t *pair_read, const int64_t *cand_offsets,
                    int64_t n_pairs, const float *model, const sw_select_rule_t *rules, int32_t n_rules,
                    const sw_scoring_t *scoring, int32_t *out_score, int32_t *out_end, uint8_t *pair_mask,
                    int32_t *best_score, int32_t *best_cand, sw_stream_t stream)
{
    SelectRules sr;
    if (n_reads < 0 || n_pairs < 0 || make_rules(rules, n_rules, &sr)) return SW_ERR_INVALID_ARG;
    if (n_reads == 0) return n_pairs == 0 ? SW_OK : SW_ERR_INVALID_ARG;
    if (!cand_offsets || !best_score) return SW_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (n_pairs == 0) {  // no candidates: every read gets -1, -1 (all bytes 0xFF)
        if (cuda_failed(cudaMemsetAsync(best_score, 0xFF, sizeof(int32_t) * (size_t)n_reads, st))) return SW_ERR_CUDA;
        if (best_cand && cuda_failed(cudaMemsetAsync(best_cand, 0xFF, sizeof(int32_t) * (size_t)n_reads, st)))
            return SW_ERR_CUDA;
        return SW_OK;
    }
    if (!reads || !read_offsets || !windows || !window_offsets || !pair_read || !model || !scoring || !out_score ||
        !out_end)
        return SW_ERR_INVALID_ARG;
    // library scratch of this stream: bf16 features (16-byte rows for the
    // tensor-core network), predictions, and the selection when the caller
    // passes no mask
    constexpr size_t kFeatures = 64;  // bf16 features per pair
    const size_t fb = ((size_t)n_pairs * kFeatures * 2 + 255) / 256 * 256;
    const size_t pb = ((size_t)n_pairs * 4 + 255) / 256 * 256;
    uint8_t *scr = nullptr;
    int rc = filter_scratch(st, fb + pb + (pair_mask ? 0 : (size_t)n_pairs), &scr);
    if (rc) return rc;
    uint16_t *feat = reinterpret_cast<uint16_t *>(scr);
    float *pred = reinterpret_cast<float *>(scr + fb);
    uint8_t *mask = pair_mask ? pair_mask : scr + fb + pb;
    // the network's status word, cleared here whichever kernel runs it
    int32_t *net_status = nullptr;
    if ((rc = aux_status_word(st, &net_status))) return rc;
    if ((rc = sw_filter_features(reads, read_offsets, n_reads, windows, window_offsets, cand_offsets, feat, stream)))
        return rc;
    if ((rc = sw_mlp_forward(model, feat, n_pairs, pred, stream))) return rc;
    if ((rc = launch_select(pred, cand_offsets, n_rules > 1 ? read_offsets : nullptr, n_reads, sr, mask, st)))
        return rc;
    if ((rc = sw_batch_align_masked(reads, read_offsets, n_reads, windows, window_offsets, pair_read, mask, n_pairs,
                                    scoring, out_score, out_end, nullptr, stream)))
        return rc;
    int32_t *align_status = nullptr;
    if ((rc = stream_status_word(st, &align_status))) return rc;
    if (align_status && align_status != net_status && (rc = launch_or_status(align_status, net_status, st)))
        return rc;
    return launch_best_per_read(out_score, cand_offsets, n_reads, mask, best_score, best_cand, st);
}

int sw_filter_train_step(float *model, const uint16_t *features, const float *target, const int32_t *idx, int64_t n,
                         float lr, int32_t step, sw_stream_t stream)
{
    if (n < 1 || !model || !features || !target || step < 1 || !(lr > 0.f)) return SW_ERR_INVALID_ARG;
    const int rc = sw_mlp_grad(model, features, target, idx, n, stream);
    return rc ? rc : sw_mlp_adam(model, lr, step, stream);
}

}  // extern "C"
