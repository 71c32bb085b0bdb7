// sw_mlp_tc.cu -- the candidate filter's network on the 5th-generation
// tensor cores (tcgen05): 64 -> 256 -> 64 -> 1, bf16 operands, fp32
// accumulation in tensor memory.
//
// Forward: one persistent CTA per SM holds both weight matrices in shared
// memory; two warp groups of 4 warps take alternate tiles of 128 pairs,
// each with its own 256 TMEM columns, so one group's epilogues run while
// the other's MMAs keep the tensor core busy.  Per tile:
//   1. the tile's features (128 x 64 bf16) are copied into the group's
//      shared-memory buffer;
//   2. one thread issues five tcgen05.mma (M 128, N 256, K 16; the fifth
//      carries the bias, see below) into the group's TMEM columns;
//   3. each warp reads its 32 rows back with tcgen05.ld, applies ReLU,
//      rounds to bf16 and writes the hidden units back into tensor memory
//      (tcgen05.st, two to a column);
//   4. seventeen tcgen05.mma (M 128, N 64, K 16) take that as their A
//      operand from tensor memory and compute layer 2;
//   5. each thread reads its row, applies ReLU and takes the dot product
//      with w3 (+ b3) in fp32.
// Shared-memory operands use the K-major layout without swizzle: 8-row x
// 16-byte core matrices, core matrices along K 128 bytes apart (leading
// byte offset) and 8-row groups K/8 x 128 bytes apart (stride byte offset).
// Completion of the MMAs is signalled through mbarriers that
// tcgen05.commit arrives on; every wait on one is bounded and a timeout is
// reported, never waited out.
#include <cuda_bf16.h>

#include <algorithm>

#include "sw_device.cuh"
#include "swgb_internal.h"

namespace swgb {

namespace {

constexpr int TC_ROWS = 128;        // pairs per tile (MMA M)
constexpr uint32_t TC_TMEM_COLS = 512;  // the whole tensor memory (one CTA per SM)
constexpr int64_t TC_WAIT_LIMIT = 1 << 20;  // polls of an mbarrier before giving up

// The forward's biases ride in the MMAs: each layer's K gets one more block
// of 16, whose first two columns are 1 in the A operand (features, hidden
// units) and the bias split into two bf16 parts, hi = bf16(b) and
// lo = bf16(b - hi), in the B operand (weights); the other 14 are 0.  The
// fp32 accumulator then holds x . W + hi + lo, and hi + lo equals the fp32
// bias to about 16 bits, so the epilogues only apply ReLU.
constexpr int FK1 = 64 + 16;                   // layer-1 K
constexpr int FK2 = 256 + 16;                  // layer-2 K

constexpr int SM_XSZ = 128 * FK1 * 2;          // one tile of features (A of layer 1)
constexpr int SM_TOTAL = 227 * 1024;           // all of it: headroom past the used bytes

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (r, k) of a K-major bf16 operand with K columns
__device__ __forceinline__ uint32_t kmajor_off(int r, int k, int K)
{
    return (uint32_t)((r >> 3) * (K / 8) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// shared-memory matrix descriptor: start, leading and stride byte offsets
// (16-byte units), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor of kind::f16: fp32 D, bf16 A and B, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy writes to shared memory, visible to the tensor core's reads
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// bounded wait for the given phase of an mbarrier; false on timeout
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase)
{
    for (int64_t it = 0; it < TC_WAIT_LIMIT; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred P1;\n\tmbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
            "selp.b32 %0, 1, 0, P1;\n\t}\n"
            : "=r"(ok)
            : "r"(mbar), "r"(phase)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// 16 consecutive 32-bit columns of this warp's 32 TMEM lanes from registers
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
            taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&v)[8])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(v[0]),
                 "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                 : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// an MMA whose A operand (M 128 rows, one per TMEM lane, K along columns,
// two bf16 per column) is in tensor memory
__device__ __forceinline__ void mma_bf16_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

// barrier `id` over the 128 threads of one warp group
__device__ __forceinline__ void group_sync(int id) { asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory"); }
// and-reduction of a predicate over the 128 threads of a warp group
__device__ __forceinline__ bool group_and(bool v, int id)
{
    int r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.b32 p, %1, 0;\n\tbar.red.and.pred q, %2, 128, p;\n\t"
        "selp.b32 %0, 1, 0, q;\n\t}\n"
        : "=r"(r)
        : "r"((int)v), "r"(id)
        : "memory");
    return r != 0;
}

// Two warp groups of 4 warps, each with its own tiles (alternate tiles of
// the CTA), its own 256 TMEM columns and its own feature buffer, so that one
// group's epilogues run while the other group's MMAs occupy the tensor core.
// The hidden layer stays in tensor memory: the group's epilogue reads the
// layer-1 accumulator (fp32, columns 0..255 of its region), applies ReLU,
// rounds to bf16 and writes the 256 hidden units two to a column into
// columns 0..127 of the same region (each column is read before it is
// overwritten), plus the bias block (ones) in columns 128..135; layer 2
// then takes its A operand from there and accumulates into columns
// 192..255.  Shared memory holds only the weights and the feature buffers.
constexpr int FW_W1 = 0;
constexpr int FW_W2 = FW_W1 + 256 * FK1 * 2;
constexpr int FW_X = FW_W2 + 64 * FK2 * 2;       // 2 groups x (128 x FK1 bf16)
constexpr int FW_W3 = FW_X + 2 * SM_XSZ;
constexpr int FW_BAR = FW_W3 + 64 * 4;          // 4 mbarriers (bar1, bar2 per group), TMEM base
constexpr int FW_USED = FW_BAR + 64;

__global__ void __launch_bounds__(256, 1) k_mlp_forward_tc(const float *__restrict__ model,
                                                            const __nv_bfloat16 *__restrict__ feat, int64_t n,
                                                            float *__restrict__ out, int32_t *status)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int grp = warp >> 2, quarter = warp & 3, gtid = tid & 127;
    const int bar_id = 1 + grp;  // named barrier of the group
    float *w3 = reinterpret_cast<float *>(smem + FW_W3);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + FW_BAR);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + FW_BAR + 32);
    const uint32_t s_base = smem_u32(smem);
    const uint32_t bar1 = smem_u32(bar + 2 * grp), bar2 = smem_u32(bar + 2 * grp + 1);
    const uint32_t xoff = FW_X + grp * SM_XSZ;

    {
        const uint4 *g1 = reinterpret_cast<const uint4 *>(model + MD_W1T);  // [256][64] bf16
        const uint4 *g2 = reinterpret_cast<const uint4 *>(model + MD_W2T);  // [64][256] bf16
        for (int c = tid; c < 256 * 8; c += blockDim.x) {
            const int r = c >> 3, k = (c & 7) * 8;
            *reinterpret_cast<uint4 *>(smem + FW_W1 + kmajor_off(r, k, FK1)) = g1[c];
        }
        for (int c = tid; c < 64 * 32; c += blockDim.x) {
            const int r = c >> 5, k = (c & 31) * 8;
            *reinterpret_cast<uint4 *>(smem + FW_W2 + kmajor_off(r, k, FK2)) = g2[c];
        }
        auto bias8 = [](float b) {
            const __nv_bfloat16 hi = __float2bfloat16_rn(b);
            const __nv_bfloat16 lo = __float2bfloat16_rn(b - __bfloat162float(hi));
            return make_uint4((uint32_t)__bfloat16_as_ushort(hi) | ((uint32_t)__bfloat16_as_ushort(lo) << 16), 0u,
                              0u, 0u);
        };
        const uint4 ones = make_uint4(0x3F803F80u, 0u, 0u, 0u), zero = make_uint4(0u, 0u, 0u, 0u);
        for (int r = tid; r < 256; r += blockDim.x) {
            *reinterpret_cast<uint4 *>(smem + FW_W1 + kmajor_off(r, 64, FK1)) = bias8(model[MD_B1 + r]);
            *reinterpret_cast<uint4 *>(smem + FW_W1 + kmajor_off(r, 72, FK1)) = zero;
        }
        for (int r = tid; r < 64; r += blockDim.x) {
            *reinterpret_cast<uint4 *>(smem + FW_W2 + kmajor_off(r, 256, FK2)) = bias8(model[MD_B2 + r]);
            *reinterpret_cast<uint4 *>(smem + FW_W2 + kmajor_off(r, 264, FK2)) = zero;
            w3[r] = model[MD_W3 + r];
        }
        for (int r = tid; r < TC_ROWS; r += blockDim.x) {
            for (int xb = 0; xb < 2; ++xb) {
                *reinterpret_cast<uint4 *>(smem + FW_X + xb * SM_XSZ + kmajor_off(r, 64, FK1)) = ones;
                *reinterpret_cast<uint4 *>(smem + FW_X + xb * SM_XSZ + kmajor_off(r, 72, FK1)) = zero;
            }
        }
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid < 4) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar + tid)));
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    const uint32_t region = tmem + 256u * (uint32_t)grp;            // this group's 256 columns
    const uint32_t lane_q = (uint32_t)(32 * quarter) << 16;         // this warp's TMEM lanes
    const float b3 = model[MD_B3];
    const int64_t tiles = (n + TC_ROWS - 1) / TC_ROWS;
    const int64_t stride = 2 * (int64_t)gridDim.x;
    // the features of one tile into the group's buffer (rows past n read as zero)
    auto load_x = [&](int64_t tile) {
        const int64_t row0 = tile * TC_ROWS;
        const uint4 *g = reinterpret_cast<const uint4 *>(feat);
        for (int c = gtid; c < TC_ROWS * 8; c += 128) {
            const int r = c >> 3, k = (c & 7) * 8;
            const bool in = row0 + r < n;
            cp_async16(s_base + xoff + kmajor_off(r, k, FK1), g + (in ? (row0 + r) * 8 + (c & 7) : 0), in ? 16u : 0u);
        }
        cp_async_commit();
    };
    auto layer1 = [&]() {
#pragma unroll
        for (int ks = 0; ks < FK1 / 16; ++ks)
            mma_bf16(region, smem_desc(s_base + xoff + 256 * ks, 128, FK1 / 8 * 128),
                     smem_desc(s_base + FW_W1 + 256 * ks, 128, FK1 / 8 * 128), idesc_bf16(128, 256), ks > 0);
        mma_commit(bar1);
    };
    uint32_t ph1 = 0, ph2 = 0;
    bool ok = true, pend1 = false, pend2 = false;
    uint32_t pph1 = 0, pph2 = 0;
    auto wait_group = [&](uint32_t b, uint32_t &ph, bool &pend, uint32_t &pph) -> bool {
        pph = ph;
        const bool got = mbar_wait(b, ph);
        ph ^= 1u;
        const bool all = group_and(got, bar_id);
        pend = !all;
        return all;
    };

    int64_t tile = blockIdx.x + (int64_t)grp * gridDim.x;
    if (tile < tiles) {
        load_x(tile);
        cp_async_wait_all();
        fence_async_smem();
        group_sync(bar_id);
        if (gtid == 0) layer1();
        pend1 = true;
        pph1 = ph1;
    }
    for (; tile < tiles && ok; tile += stride) {
        const int64_t next = tile + stride;
        ok = wait_group(bar1, ph1, pend1, pph1);  // layer 1 of this tile: the feature buffer is free again
        fence_after_sync();
        if (!ok) break;
        if (next < tiles) load_x(next);
        // hidden units: relu(D) as bf16, two to a column, into columns 0..127
#pragma unroll 1
        for (int c0 = 0; c0 < 256; c0 += 64) {
            uint32_t v[4][16];
#pragma unroll
            for (int q = 0; q < 4; ++q) tmem_ld16(region + lane_q + (uint32_t)(c0 + 16 * q), v[q]);
            tmem_wait_ld();
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2) {
                uint32_t pk[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int q = 2 * h2 + (j >> 3), e = 2 * (j & 7);
                    const __nv_bfloat162 hh = __floats2bfloat162_rn(fmaxf(__uint_as_float(v[q][e]), 0.f),
                                                                    fmaxf(__uint_as_float(v[q][e + 1]), 0.f));
                    pk[j] = *reinterpret_cast<const uint32_t *>(&hh);
                }
                tmem_st16(region + lane_q + (uint32_t)(c0 / 2 + 16 * h2), pk);
            }
        }
        {
            const uint32_t bias_blk[8] = {0x3F803F80u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
            tmem_st8(region + lane_q + 128u, bias_blk);
        }
        tmem_wait_st();
        fence_before_sync();
        group_sync(bar_id);
        fence_after_sync();
        if (gtid == 0) {
#pragma unroll
            for (int ks = 0; ks < FK2 / 16; ++ks)
                mma_bf16_ta(region + 192u, region + (uint32_t)(8 * ks),
                            smem_desc(s_base + FW_W2 + 256 * ks, 128, FK2 / 8 * 128), idesc_bf16(128, 64), ks > 0);
            mma_commit(bar2);
        }
        pend2 = true;
        pph2 = ph2;
        ok = wait_group(bar2, ph2, pend2, pph2);
        fence_after_sync();
        if (!ok) break;
        // y = w3 . relu(D) + b3: each thread its row, all 64 columns
        {
            float acc = 0.f;
            uint32_t v[4][16];
#pragma unroll
            for (int q = 0; q < 4; ++q) tmem_ld16(region + lane_q + 192u + (uint32_t)(16 * q), v[q]);
            tmem_wait_ld();
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int j = 0; j < 16; ++j) acc += fmaxf(__uint_as_float(v[q][j]), 0.f) * w3[16 * q + j];
            const int64_t row = tile * TC_ROWS + 32 * quarter + lane;
            if (row < n) out[row] = acc + b3;
        }
        // the next tile's features have landed; its layer 1 may now overwrite the region
        cp_async_wait_all();
        fence_async_smem();
        fence_before_sync();
        group_sync(bar_id);
        fence_after_sync();
        if (next < tiles) {
            if (gtid == 0) layer1();
            pend1 = true;
            pph1 = ph1;
        }
    }
    if (!ok && gtid == 0) atomicOr(status, ST_TIMEOUT);
    // a wait that ran out can leave tensor-core work in flight: wait for it
    // once more (bounded) before the memory is freed
    if (pend1) group_and(mbar_wait(bar1, pph1), bar_id);
    if (pend2) group_and(mbar_wait(bar2, pph2), bar_id);
    cp_async_wait_all();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
}

// ------------------------------------------------------------------ training
//
// The gradient of mean((y - target)^2) over a minibatch on the tensor cores.
// A CTA takes tiles of 128 samples; per tile five MMAs (M 128, bf16 operands
// in shared memory, fp32 accumulators in tensor memory):
//   Z1   = X . W1              (K 64,  N 256)   TMEM columns 0..255
//   Z2   = A1 . W2             (K 256, N 64)    columns 0..63
//   dA1  = dZ2 . W2^T          (K 64,  N 256)   columns 0..255
//   gW2  += A1^T . dZ2         (K 128, N 64)    columns 256..383, two M halves
//   gW1^T += dZ1^T . X         (K 128, N 64)    columns 384..511, two M halves
// with the CUDA cores in between: A1 = bf16(relu(Z1 + b1)), the output y,
// dy = 2 (y - t), dZ2 = dy w3 [Z2 + b2 > 0], dZ1 = dA1 [A1 > 0], and the
// bias gradients (column sums in fp32); the 1/n of the mean multiplies the
// final sums.  The weight-gradient sums stay in
// tensor memory across the CTA's tiles; at the end each CTA writes its
// partial gradient, and k_mlp_grad_reduce adds the partials in CTA order (so
// the result does not depend on scheduling).  Every operand is K-major: the
// transposed copies (X^T, A1^T, dZ2^T, dZ1^T) are written by the epilogues.
// Shared memory regions are reused as their contents die:
//   R1  A1 [128][256]           -> dZ1^T [256][128]
//   R2  A1^T [256][128]
//   R3  W1^T [256][64] -> W2^T [64][256] -> W2 [256][64]
//   R5  X [128][64]             -> dZ2 [128][64]
//   R6  X^T [64][128]
//   R7  dZ2^T [64][128]

constexpr int GB_R1 = 0;
constexpr int GB_R2 = GB_R1 + 65536;
constexpr int GB_R3 = GB_R2 + 65536;
constexpr int GB_R5 = GB_R3 + 32768;
constexpr int GB_R6 = GB_R5 + 16384;
constexpr int GB_R7 = GB_R6 + 16384;
constexpr int GB_B1 = GB_R7 + 16384;      // b1 [256]
constexpr int GB_B2 = GB_B1 + 1024;       // b2 [64]
constexpr int GB_W3 = GB_B2 + 256;        // w3 [64]
constexpr int GB_T = GB_W3 + 256;         // targets of the tile [128]
constexpr int GB_YP = GB_T + 512;         // partial outputs [2][128]
// bias gradients, one row per TMEM lane quarter (each warp adds only to its
// own quarter's row and column half, and the rows are added in order at the
// end, so the sums do not depend on warp scheduling)
constexpr int GB_GB1 = GB_YP + 1024;      // gb1 [4][256]
constexpr int GB_GB2 = GB_GB1 + 4096;     // gb2 [4][64]
constexpr int GB_GW3 = GB_GB2 + 1024;     // gw3 [4][64]
constexpr int GB_GB3 = GB_GW3 + 1024;     // gb3 [4]
constexpr int GB_BAR = GB_GB3 + 16;       // mbarrier (8 B), TMEM base (4 B)
constexpr int GB_USED = GB_BAR + 64;

// 2-byte bf16 store of v at byte offset off of shared memory
__device__ __forceinline__ void st_bf16(unsigned char *smem, uint32_t off, float v)
{
    *reinterpret_cast<__nv_bfloat16 *>(smem + off) = __float2bfloat16_rn(v);
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int d = 16; d; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    return v;
}

__global__ void __launch_bounds__(256, 1) k_mlp_grad_tc(const float *__restrict__ model,
                                                        const __nv_bfloat16 *__restrict__ feat,
                                                        const float *__restrict__ target,
                                                        const int32_t *__restrict__ idx, int64_t n,
                                                        float *__restrict__ partial, int32_t *status)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, half = warp >> 2;
    float *b1 = reinterpret_cast<float *>(smem + GB_B1);
    float *b2 = reinterpret_cast<float *>(smem + GB_B2);
    float *w3 = reinterpret_cast<float *>(smem + GB_W3);
    float *ts = reinterpret_cast<float *>(smem + GB_T);
    float *yp = reinterpret_cast<float *>(smem + GB_YP);
    float *gb1 = reinterpret_cast<float *>(smem + GB_GB1);
    float *gb2 = reinterpret_cast<float *>(smem + GB_GB2);
    float *gw3 = reinterpret_cast<float *>(smem + GB_GW3);
    float *gb3 = reinterpret_cast<float *>(smem + GB_GB3);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + GB_BAR);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + GB_BAR + 8);
    const uint32_t s_base = smem_u32(smem);
    const uint32_t mbar = smem_u32(bar);

    for (int i = tid; i < 256; i += blockDim.x) b1[i] = model[MD_B1 + i];
    for (int i = tid; i < 64; i += blockDim.x) {
        b2[i] = model[MD_B2 + i];
        w3[i] = model[MD_W3 + i];
    }
    for (int i = tid; i < 4 * 256; i += blockDim.x) gb1[i] = 0.f;
    for (int i = tid; i < 4 * 64; i += blockDim.x) {
        gb2[i] = 0.f;
        gw3[i] = 0.f;
    }
    if (tid < 4) gb3[tid] = 0.f;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar));
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    const uint32_t accA = tmem, accB = tmem + 256u, accC = tmem + 384u;
    const uint32_t lane_off = (uint32_t)(32 * quarter) << 16;
    const float b3 = model[MD_B3];
    const int64_t tiles = (n + TC_ROWS - 1) / TC_ROWS;
    uint32_t ph = 0, pending_ph = 0;
    bool ok = true, pending = false;
    // one commit, then every thread waits for it (bounded, uniform verdict);
    // a wait that runs out leaves the commit pending
    auto commit_wait = [&]() -> bool {
        if (tid == 0) mma_commit(mbar);
        pending = true;
        pending_ph = ph;
        const bool got = mbar_wait(mbar, ph);
        ph ^= 1u;
        const bool all = __syncthreads_and(got) != 0;
        if (all) pending = false;
        fence_after_sync();
        return all;
    };
    // generic-proxy shared-memory writes, visible to the next MMAs
    auto publish = [&]() {
        fence_async_smem();
        fence_before_sync();
        __syncthreads();
        fence_after_sync();
    };
    // copies a [rows][cols] bf16 matrix from global memory into K-major layout
    auto load_kmajor = [&](int region, const uint4 *g, int rows, int cols) {
        const int per_row = cols / 8;
        for (int c = tid; c < rows * per_row; c += blockDim.x) {
            const int r = c / per_row, k = (c % per_row) * 8;
            *reinterpret_cast<uint4 *>(smem + region + kmajor_off(r, k, cols)) = g[c];
        }
    };
    bool first = true;
    for (int64_t tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
        const int64_t row0 = tile * TC_ROWS;
        // 1. X (K-major along features), X^T (along samples), targets, W1^T
        for (int c = tid; c < TC_ROWS * 8; c += blockDim.x) {
            const int r = c >> 3, k = (c & 7) * 8;
            const int64_t s = row0 + r;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (s < n) {
                const int64_t row = idx ? idx[s] : s;
                v = reinterpret_cast<const uint4 *>(feat)[row * 8 + (c & 7)];
            }
            *reinterpret_cast<uint4 *>(smem + GB_R5 + kmajor_off(r, k, 64)) = v;
            const __nv_bfloat16 *e = reinterpret_cast<const __nv_bfloat16 *>(&v);
#pragma unroll
            for (int q = 0; q < 8; ++q)
                *reinterpret_cast<__nv_bfloat16 *>(smem + GB_R6 + kmajor_off(k + q, r, 128)) = e[q];
        }
        for (int r = tid; r < TC_ROWS; r += blockDim.x) {
            const int64_t s = row0 + r;
            ts[r] = s < n ? target[idx ? idx[s] : s] : 0.f;
        }
        load_kmajor(GB_R3, reinterpret_cast<const uint4 *>(model + MD_W1T), 256, 64);
        publish();
        // 2. Z1 = X . W1
        if (tid == 0)
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)
                mma_bf16(accA, smem_desc(s_base + GB_R5 + 256 * ks, 128, 1024),
                         smem_desc(s_base + GB_R3 + 256 * ks, 128, 1024), idesc_bf16(128, 256), ks > 0);
        if (!(ok = commit_wait())) break;
        // 3. W2^T for layer 2; A1 = bf16(relu(Z1 + b1)) as A1 and A1^T
        load_kmajor(GB_R3, reinterpret_cast<const uint4 *>(model + MD_W2T), 64, 256);
        {
            const int r = 32 * quarter + lane;
            for (int c0 = 128 * half; c0 < 128 * half + 128; c0 += 16) {
                uint32_t v[16];
                tmem_ld16(accA + lane_off + (uint32_t)c0, v);
                tmem_wait_ld();
                uint32_t pk[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float x0 = fmaxf(__uint_as_float(v[2 * j]) + b1[c0 + 2 * j], 0.f);
                    const float x1 = fmaxf(__uint_as_float(v[2 * j + 1]) + b1[c0 + 2 * j + 1], 0.f);
                    const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
                    pk[j] = *reinterpret_cast<const uint32_t *>(&h);
                    *reinterpret_cast<__nv_bfloat16 *>(smem + GB_R2 + kmajor_off(c0 + 2 * j, r, 128)) = h.x;
                    *reinterpret_cast<__nv_bfloat16 *>(smem + GB_R2 + kmajor_off(c0 + 2 * j + 1, r, 128)) = h.y;
                }
                *reinterpret_cast<uint4 *>(smem + GB_R1 + kmajor_off(r, c0, 256)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                *reinterpret_cast<uint4 *>(smem + GB_R1 + kmajor_off(r, c0 + 8, 256)) =
                    make_uint4(pk[4], pk[5], pk[6], pk[7]);
            }
        }
        publish();
        // 4. Z2 = A1 . W2
        if (tid == 0)
#pragma unroll
            for (int ks = 0; ks < 16; ++ks)
                mma_bf16(accA, smem_desc(s_base + GB_R1 + 256 * ks, 128, 4096),
                         smem_desc(s_base + GB_R3 + 256 * ks, 128, 4096), idesc_bf16(128, 64), ks > 0);
        if (!(ok = commit_wait())) break;
        // 5. W2 for dA1 (bf16 of the fp32 parameters, as the serving copies
        // round them); y, dy, dZ2 (as dZ2 and dZ2^T) and the small gradients
        for (int c = tid; c < 256 * 8; c += blockDim.x) {
            const int r = c >> 3, k = (c & 7) * 8;
            const float4 *src = reinterpret_cast<const float4 *>(model + MD_W2 + r * 64 + k);
            const float4 lo = src[0], hi = src[1];
            const __nv_bfloat162 p0 = __floats2bfloat162_rn(lo.x, lo.y), p1 = __floats2bfloat162_rn(lo.z, lo.w);
            const __nv_bfloat162 p2 = __floats2bfloat162_rn(hi.x, hi.y), p3 = __floats2bfloat162_rn(hi.z, hi.w);
            *reinterpret_cast<uint4 *>(smem + GB_R3 + kmajor_off(r, k, 64)) =
                make_uint4(*reinterpret_cast<const uint32_t *>(&p0), *reinterpret_cast<const uint32_t *>(&p1),
                           *reinterpret_cast<const uint32_t *>(&p2), *reinterpret_cast<const uint32_t *>(&p3));
        }
        {
            const int r = 32 * quarter + lane;
            const bool valid = row0 + r < n;
            float z[32];
            for (int c0 = 0; c0 < 32; c0 += 16) {
                uint32_t v[16];
                tmem_ld16(accA + lane_off + (uint32_t)(32 * half + c0), v);
                tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 16; ++j) z[c0 + j] = __uint_as_float(v[j]) + b2[32 * half + c0 + j];
            }
            float y = 0.f;
#pragma unroll
            for (int j = 0; j < 32; ++j) y += fmaxf(z[j], 0.f) * w3[32 * half + j];
            yp[half * 128 + r] = y;
            __syncthreads();
            // per-sample 2 (y - t); the 1/n of the mean is applied once, to
            // the sums, so the bf16 signals do not depend on the batch size
            const float dy = valid ? 2.f * (yp[r] + yp[128 + r] + b3 - ts[r]) : 0.f;
            float dz[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int c = 32 * half + j;
                dz[j] = z[j] > 0.f ? dy * w3[c] : 0.f;
                st_bf16(smem, GB_R7 + kmajor_off(c, r, 128), dz[j]);
                const float s2 = warp_sum(dz[j]);
                const float s3 = warp_sum(fmaxf(z[j], 0.f) * dy);
                if (lane == 0) {
                    gb2[quarter * 64 + c] += s2;
                    gw3[quarter * 64 + c] += s3;
                }
            }
#pragma unroll
            for (int j = 0; j < 32; j += 8) {
                uint32_t pk[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const __nv_bfloat162 h = __floats2bfloat162_rn(dz[j + 2 * q], dz[j + 2 * q + 1]);
                    pk[q] = *reinterpret_cast<const uint32_t *>(&h);
                }
                *reinterpret_cast<uint4 *>(smem + GB_R5 + kmajor_off(r, 32 * half + j, 64)) =
                    make_uint4(pk[0], pk[1], pk[2], pk[3]);
            }
            if (half == 0) {
                const float s = warp_sum(dy);
                if (lane == 0) gb3[quarter] += s;
            }
        }
        publish();
        // 6. dA1 = dZ2 . W2^T, and gW2 += A1^T . dZ2 (two 128-row halves)
        if (tid == 0) {
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)
                mma_bf16(accA, smem_desc(s_base + GB_R5 + 256 * ks, 128, 1024),
                         smem_desc(s_base + GB_R3 + 256 * ks, 128, 1024), idesc_bf16(128, 256), ks > 0);
#pragma unroll
            for (int hh = 0; hh < 2; ++hh)
#pragma unroll
                for (int ks = 0; ks < 8; ++ks)
                    mma_bf16(accB + 64u * hh, smem_desc(s_base + GB_R2 + 32768 * hh + 256 * ks, 128, 2048),
                             smem_desc(s_base + GB_R7 + 256 * ks, 128, 2048), idesc_bf16(128, 64),
                             (!first || ks > 0) ? 1u : 0u);
        }
        if (!(ok = commit_wait())) break;
        // 7. dZ1 = dA1 [A1 > 0], as dZ1^T; gb1
        {
            const int r = 32 * quarter + lane;
            for (int c0 = 128 * half; c0 < 128 * half + 128; c0 += 16) {
                uint32_t v[16];
                tmem_ld16(accA + lane_off + (uint32_t)c0, v);
                tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int c = c0 + j;
                    const float a = __bfloat162float(
                        *reinterpret_cast<const __nv_bfloat16 *>(smem + GB_R2 + kmajor_off(c, r, 128)));
                    const float d = a > 0.f ? __uint_as_float(v[j]) : 0.f;
                    st_bf16(smem, GB_R1 + kmajor_off(c, r, 128), d);
                    const float s1 = warp_sum(d);
                    if (lane == 0) gb1[quarter * 256 + c] += s1;
                }
            }
        }
        publish();
        // 8. gW1^T += dZ1^T . X (two 128-row halves)
        if (tid == 0)
#pragma unroll
            for (int hh = 0; hh < 2; ++hh)
#pragma unroll
                for (int ks = 0; ks < 8; ++ks)
                    mma_bf16(accC + 64u * hh, smem_desc(s_base + GB_R1 + 32768 * hh + 256 * ks, 128, 2048),
                             smem_desc(s_base + GB_R6 + 256 * ks, 128, 2048), idesc_bf16(128, 64),
                             (!first || ks > 0) ? 1u : 0u);
        if (!(ok = commit_wait())) break;
        first = false;
    }
    // the CTA's partial gradient: gW1, gW2 from tensor memory, biases
    if (ok && !first) {
        float *out = partial + (int64_t)blockIdx.x * MD_NP;
        const int j = 128 * half + 32 * quarter + lane;  // hidden unit of this lane
        for (int c0 = 0; c0 < 64; c0 += 16) {
            uint32_t v[16];
            tmem_ld16(accB + 64u * (uint32_t)half + lane_off + (uint32_t)c0, v);
            tmem_wait_ld();
#pragma unroll
            for (int q = 0; q < 16; ++q) out[MD_W2 + j * 64 + c0 + q] = __uint_as_float(v[q]);
            tmem_ld16(accC + 64u * (uint32_t)half + lane_off + (uint32_t)c0, v);
            tmem_wait_ld();
#pragma unroll
            for (int q = 0; q < 16; ++q) out[MD_W1 + (c0 + q) * 256 + j] = __uint_as_float(v[q]);
        }
        __syncthreads();
        for (int i = tid; i < 256; i += blockDim.x)
            out[MD_B1 + i] = ((gb1[i] + gb1[256 + i]) + gb1[512 + i]) + gb1[768 + i];
        for (int i = tid; i < 64; i += blockDim.x) {
            out[MD_B2 + i] = ((gb2[i] + gb2[64 + i]) + gb2[128 + i]) + gb2[192 + i];
            out[MD_W3 + i] = ((gw3[i] + gw3[64 + i]) + gw3[128 + i]) + gw3[192 + i];
        }
        if (tid == 0) out[MD_B3] = ((gb3[0] + gb3[1]) + gb3[2]) + gb3[3];
    } else if (!ok && tid == 0) {
        atomicOr(status, ST_TIMEOUT);
    }
    // a commit whose wait ran out may still have tensor-core work in flight:
    // wait for it once more (bounded) before the tensor memory is released
    if (pending) {
        const bool got = mbar_wait(mbar, pending_ph);
        __syncthreads_and(got);
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
}

// G = the sum of the CTAs' partial gradients, in CTA order, over n samples.
__global__ void k_mlp_grad_reduce(const float *__restrict__ partial, int n_part, float inv_n, float *__restrict__ G)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < MD_NP; i += (int64_t)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int p = 0; p < n_part; ++p) s += partial[(int64_t)p * MD_NP + i];
        G[i] = s * inv_n;
    }
}

}  // namespace

int launch_mlp_forward_tc(const float *model, const uint16_t *feat, int64_t n, float *out, int sm_count,
                          int32_t *status, cudaStream_t st)
{
    // per call: the attribute belongs to the current device, and calls may
    // come from several host threads at once
    if (cuda_failed(cudaFuncSetAttribute(k_mlp_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         FW_USED)))
        return SW_ERR_CUDA;
    static_assert(FW_USED <= SM_TOTAL, "shared memory layout");
    const int64_t tiles = (n + TC_ROWS - 1) / TC_ROWS;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((tiles + 1) / 2, sm_count));
    k_mlp_forward_tc<<<grid, 256, FW_USED, st>>>(model, reinterpret_cast<const __nv_bfloat16 *>(feat), n, out,
                                                   status);
    count_launch();
    return launch_status();
}

int mlp_grad_tc_parts(int64_t n, int sm_count)
{
    const int64_t tiles = (n + TC_ROWS - 1) / TC_ROWS;
    return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, sm_count));
}

int launch_mlp_grad_tc(float *model, const uint16_t *feat, const float *target, const int32_t *idx, int64_t n,
                       int sm_count, float *partial, int32_t *status, cudaStream_t st)
{
    if (cuda_failed(cudaFuncSetAttribute(k_mlp_grad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, GB_USED)))
        return SW_ERR_CUDA;
    static_assert(GB_USED <= SM_TOTAL, "shared memory layout");
    const int grid = mlp_grad_tc_parts(n, sm_count);
    k_mlp_grad_tc<<<grid, 256, GB_USED, st>>>(model, reinterpret_cast<const __nv_bfloat16 *>(feat), target, idx, n,
                                               partial, status);
    k_mlp_grad_reduce<<<(int)((MD_NP + 255) / 256), 256, 0, st>>>(partial, grid, (float)(1.0 / (double)n),
                                                                    model + MD_G);
    count_launch(2);
    return launch_status();
}

}  // namespace swgb
