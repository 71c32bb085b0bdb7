// sw_hostio.cu -- the host entry point's output path.
//
// A CIGAR slot holds capacity (2m + 3 runs) but a pair uses a few runs, so
// copying the slots back moves about 50x more bytes than the CIGARs hold.
// When the caller's op buffer is pinned host memory mapped into the
// device's address space, this kernel writes each pair's used runs straight
// into its host slot (the device reaches host memory over the chip-to-chip
// link); the rest of each slot is left as it was.
#include "sw_device.cuh"
#include "swgb_internal.h"

namespace swgb {

__global__ void k_cigar_to_host(const uint32_t *__restrict__ ops, const int64_t *__restrict__ off,
                                const int32_t *__restrict__ n_ops, int64_t n_pairs, uint32_t *host_ops)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n_pairs;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t n = n_ops[p];
        const int64_t o = off[p];
        for (int32_t k = 0; k < n; ++k) host_ops[o + k] = ops[o + k];
    }
}

int launch_cigar_to_host(const uint32_t *ops, const int64_t *off, const int32_t *n_ops, int64_t n_pairs,
                         uint32_t *host_ops, cudaStream_t st)
{
    int64_t blocks = (n_pairs + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    k_cigar_to_host<<<(unsigned)blocks, 256, 0, st>>>(ops, off, n_ops, n_pairs, host_ops);
    count_launch();
    return launch_status();
}

}  // namespace swgb

namespace swgb {

namespace {

// Exclusive scan of per-pair values v(p) in three passes (block sums, a
// one-block scan of the sums, block-local scans), writing out[0..n] with
// out[n] = the total.
template <class F>
__global__ void k_block_sums(F v, int64_t n, int64_t *blk)
{
    __shared__ int64_t ws[8];
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t x = p < n ? v(p) : 0;
    for (int d = 16; d > 0; d >>= 1) x += __shfl_down_sync(0xffffffffu, x, d);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
        blk[blockIdx.x] = t;
    }
}

__global__ void k_scan_blocks(int64_t *blk, int64_t n_blk, int64_t *total)
{
    __shared__ int64_t ws[32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < n_blk; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const int64_t v = i < n_blk ? blk[i] : 0;
        int64_t x = v;
        for (int d = 1; d < 32; d <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, x, d);
            if ((threadIdx.x & 31) >= d) x += y;
        }
        if ((threadIdx.x & 31) == 31) ws[threadIdx.x >> 5] = x;
        __syncthreads();
        int64_t wpre = 0;
        for (int w = 0; w < (int)(threadIdx.x >> 5); ++w) wpre += ws[w];
        if (i < n_blk) blk[i] = carry + wpre + x - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += wpre + x;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

template <class F>
__global__ void k_scan_write(F v, int64_t n, const int64_t *blk, int64_t *out)
{
    __shared__ int64_t ws[8];
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t val = p < n ? v(p) : 0;
    int64_t x = val;
    for (int d = 1; d < 32; d <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, d);
        if ((threadIdx.x & 31) >= d) x += y;
    }
    if ((threadIdx.x & 31) == 31) ws[threadIdx.x >> 5] = x;
    __syncthreads();
    int64_t wpre = 0;
    for (int w = 0; w < (int)(threadIdx.x >> 5); ++w) wpre += ws[w];
    if (p < n) out[p] = blk[blockIdx.x] + wpre + x - val;
}

template <class F>
int exclusive_scan(F v, int64_t n, int64_t *out, int64_t *blk, cudaStream_t st)
{
    const int64_t n_blk = (n + 255) / 256;
    k_block_sums<<<(unsigned)n_blk, 256, 0, st>>>(v, n, blk);
    k_scan_blocks<<<1, 1024, 0, st>>>(blk, n_blk, out + n);
    k_scan_write<<<(unsigned)n_blk, 256, 0, st>>>(v, n, blk, out);
    count_launch(3);
    return launch_status();
}

struct CapOf {  // CIGAR capacity of pair p: 2 m + 3 runs
    const int64_t *roff;
    __device__ int64_t operator()(int64_t p) const { return 2 * (roff[p + 1] - roff[p]) + 3; }
};

struct I32Of {  // a plain int32 array
    const int32_t *v;
    __device__ int64_t operator()(int64_t p) const { return v[p]; }
};

struct CapOfIndexed {  // capacity of pair p whose read is pair_read[p]
    const int64_t *roff;
    const int64_t *pair_read;
    __device__ int64_t operator()(int64_t p) const
    {
        const int64_t r = pair_read[p];
        return 2 * (roff[r + 1] - roff[r]) + 3;
    }
};

struct RunsOf {  // runs pair p's CIGAR holds (an overflowed slot holds none)
    const int32_t *n_ops;
    __device__ int64_t operator()(int64_t p) const { return n_ops[p] > 0 ? n_ops[p] : 0; }
};

__global__ void k_dense_copy(const uint32_t *__restrict__ ops, const int64_t *__restrict__ off,
                             const int32_t *__restrict__ n_ops, const int64_t *__restrict__ doff, int64_t n_pairs,
                             uint32_t *__restrict__ dense, int64_t dense_cap)
{
    // a warp per 32 pairs; each pair's runs are copied by consecutive lanes
    const int lane = threadIdx.x & 31;
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p0 = w * 32; p0 < n_pairs; p0 += nw * 32) {
        for (int q = 0; q < 32 && p0 + q < n_pairs; ++q) {
            const int64_t p = p0 + q;
            const int32_t n = n_ops[p];
            for (int32_t k = lane; k < n; k += 32)
                if (doff[p] + k < dense_cap) dense[doff[p] + k] = ops[off[p] + k];
        }
    }
}

}  // namespace

int launch_cap_offsets(const int64_t *read_off, int64_t n_pairs, int64_t *cig_off, int64_t *blk, cudaStream_t st)
{
    return exclusive_scan(CapOf{read_off}, n_pairs, cig_off, blk, st);
}

int launch_cap_offsets_indexed(const int64_t *read_off, const int64_t *pair_read, int64_t n_pairs, int64_t *cig_off,
                               int64_t *blk, cudaStream_t st)
{
    if (n_pairs == 0)
        return cuda_failed(cudaMemsetAsync(cig_off, 0, sizeof(int64_t), st)) ? SW_ERR_CUDA : SW_OK;
    if (!pair_read) return exclusive_scan(CapOf{read_off}, n_pairs, cig_off, blk, st);
    return exclusive_scan(CapOfIndexed{read_off, pair_read}, n_pairs, cig_off, blk, st);
}

int launch_scan_i32(const int32_t *v, int64_t n, int64_t *out, int64_t *blk, cudaStream_t st)
{
    if (n == 0) return !cuda_failed(cudaMemsetAsync(out, 0, sizeof(int64_t), st)) ? SW_OK : SW_ERR_CUDA;
    return exclusive_scan(I32Of{v}, n, out, blk, st);
}

int launch_dense_cigar(const uint32_t *ops, const int64_t *off, const int32_t *n_ops, int64_t n_pairs,
                       int64_t *doff, uint32_t *dense, int64_t dense_cap, int64_t *blk, cudaStream_t st)
{
    int rc = exclusive_scan(RunsOf{n_ops}, n_pairs, doff, blk, st);
    if (rc) return rc;
    int64_t blocks = (n_pairs + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    k_dense_copy<<<(unsigned)blocks, 256, 0, st>>>(ops, off, n_ops, doff, n_pairs, dense, dense_cap);
    count_launch();
    return launch_status();
}

}  // namespace swgb
