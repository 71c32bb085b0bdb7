// sw_noalloc.cu -- score-and-end alignment that allocates no memory.
//
// For callers that must not have the library allocate device memory: for
// example applications that hand every byte of device memory to their own
// pool allocator, or latency-sensitive services for which cudaMalloc and
// cudaFree (which synchronise the device) are not acceptable.  The entry
// point runs the same score kernel as sw_batch_align (score and end cell, no
// CIGAR), but its scratch -- the work counter, the status word and the pair
// order -- lives in one file-scope device array of fixed size instead of in
// library-allocated buffers.
#include <algorithm>

#include "sw_device.cuh"
#include "swgb_internal.h"

namespace swgb {

// Scratch layout (int32 words): [0] work counter, [1] status, [2] longest
// read, [3..63] unused, [64 ..] pair order.
constexpr int kNaHeader = 64;
static __device__ __align__(256) int32_t g_sw_noalloc_scratch[kNaHeader + SW_NOALLOC_MAX_PAIRS];

namespace {

// Validation and identity order.  Pairs with an empty window simply run as
// all-padding columns in the score kernel and come out with score 0.
__global__ void k_noalloc_prepare(PairSet ps, int64_t n_pairs, int32_t *scratch)
{
    int32_t *status = scratch + 1, *max_m = scratch + 2, *order = scratch + kNaHeader;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n_pairs;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r0 = ps.read_off[p], r1 = ps.read_off[p + 1];
        const int64_t w0 = ps.win_off[p], w1 = ps.win_off[p + 1];
        const int64_t m = r1 - r0, n = w1 - w0;
        if (r0 < 0 || w0 < 0 || m < 1 || n < 0 || n > SW_MAX_WINDOW_LEN) atomicOr(status, ST_BAD_INPUT);
        else if (m > SW_NOALLOC_MAX_READ_LEN) atomicOr(status, ST_UNSUPPORTED);
        else atomicMax(max_m, (int32_t)m);
        order[p] = (int32_t)p;
    }
}

}  // namespace
}  // namespace swgb

using namespace swgb;

extern "C" int sw_batch_align_noalloc(const uint8_t *reads, const int64_t *read_offsets, const uint8_t *windows,
                                      const int64_t *window_offsets, int64_t n_pairs,
                                      const sw_scoring_t *scoring, int32_t *out_score, int32_t *out_end,
                                      sw_stream_t stream)
{
    if (n_pairs < 0 || !scoring) return SW_ERR_INVALID_ARG;
    const sw_scoring_t *s = scoring;
    if (!(s->match >= 1 && s->match <= 127 && s->mismatch >= -127 && s->mismatch <= 0 &&
          s->gap_open <= s->gap_extend && s->gap_extend <= 0 && s->gap_open < 0 && s->match - s->gap_open <= 127))
        return SW_ERR_INVALID_ARG;
    if (n_pairs > SW_NOALLOC_MAX_PAIRS) return SW_ERR_UNSUPPORTED;
    if (n_pairs == 0) return SW_OK;
    if (!reads || !read_offsets || !windows || !window_offsets || !out_score || !out_end) return SW_ERR_INVALID_ARG;
    if (((uintptr_t)reads & 15u) || ((uintptr_t)windows & 15u)) return SW_ERR_INVALID_ARG;

    int dev = 0, sms = 0;
    if (cuda_failed(cudaGetDevice(&dev))) return SW_ERR_NO_DEVICE;
    if (cuda_failed(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) || sms < 1)
        return SW_ERR_CUDA;
    // The array's device address on the current device.  In host code the
    // array's name is only a host-side stand-in, so the address is looked up
    // with the device current.  The first call on a device also loads the
    // library's device code there (set-up: make it before any stream
    // capture).  The lookup allocates nothing and is cheap once the code is
    // loaded, so it is repeated on every call: after a device reset the code
    // is loaded again at another address, and a cached pointer would be stale.
    int32_t *scratch = nullptr;
    {
        void *ptr = nullptr;
        if (cuda_failed(cudaGetSymbolAddress(&ptr, g_sw_noalloc_scratch)) || !ptr) {
            cudaGetLastError();
            return SW_ERR_CUDA;
        }
        scratch = (int32_t *)ptr;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const PairSet ps{(const uint32_t *)reads, read_offsets, nullptr, (const uint32_t *)windows, window_offsets};

    // the array keeps the previous call's contents: clear counter, status, max
    if (cuda_failed(cudaMemsetAsync(scratch, 0, kNaHeader * sizeof(int32_t), st))) return SW_ERR_CUDA;
    const int64_t pblocks = std::min<int64_t>((n_pairs + 255) / 256, (int64_t)sms * 8);
    k_noalloc_prepare<<<(unsigned)pblocks, 256, 0, st>>>(ps, n_pairs, scratch);
    count_launch();
    if (cuda_failed(cudaGetLastError())) return SW_ERR_CUDA;
    int32_t hdr[3] = {0, 0, 0};
    if (cuda_failed(cudaMemcpyAsync(hdr, scratch, sizeof(hdr), cudaMemcpyDeviceToHost, st))) return SW_ERR_CUDA;
    if (cuda_failed(cudaStreamSynchronize(st))) return SW_ERR_CUDA;
    if (hdr[1] & ST_BAD_INPUT) return SW_ERR_DEVICE_INPUT;
    if (hdr[1] & ST_UNSUPPORTED) return SW_ERR_UNSUPPORTED;

    // int32 lanes cover every score; 32 rows per lane, lanes for the longest
    // read, so every read fits one row chunk and no boundary row is needed
    const int rows = 32;
    const int lanes = std::max(1, std::min(32, (hdr[2] + rows - 1) / rows));
    ScoreLaunch L{};
    L.ps = ps;
    L.sc = Scoring{s->match, s->mismatch, s->gap_open, s->gap_extend};
    L.order = scratch + kNaHeader;
    L.n_items = n_pairs;
    L.lanes = lanes;
    L.out_score = out_score;
    L.out_end = out_end;
    L.boundary = nullptr;
    L.boundary_group_bytes = 0;
    L.work_counter = scratch;
    L.status = scratch + 1;
    int regs = 0, bps = 0;
    if (score_kernel_regs(rows, MODE_I32, &regs, &bps, 128) != SW_OK || bps < 1) return SW_ERR_INTERNAL;
    const int64_t groups = 32 / lanes;
    const int64_t warps = (n_pairs + groups - 1) / groups;
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((warps + 3) / 4, (int64_t)bps * sms));
    return launch_score(rows, MODE_I32, L, (int)blocks, 128, st);
}
