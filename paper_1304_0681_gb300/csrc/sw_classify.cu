// sw_classify.cu -- validation and length-class ordering of a batch of pairs.
//
// Every pair gets a sort key (arithmetic mode, read-length class, window
// length bucket in descending order).  A counting sort over the keys then
// lays the pairs out class by class, longest windows first, so that each
// class can run under its own lane plan and lanes that share a warp see
// windows of similar length.
#include "sw_device.cuh"
#include "swgb_internal.h"

namespace swgb {

__global__ void k_classify(PairSet ps, int64_t n_reads, int64_t n_pairs, Scoring sc, int score_setting,
                           int32_t *__restrict__ keys, int32_t *__restrict__ hist, ClassInfo *__restrict__ info,
                           int32_t *__restrict__ out_score, int32_t *__restrict__ out_end,
                           int32_t *__restrict__ cig_n)
{
    // the block's per-class count and maxima, added to the global table once
    // at the end: a batch has few classes, and a global atomic per key group
    // would send every warp to the same few addresses
    __shared__ int32_t s_count[N_CLASS], s_max_n[N_CLASS], s_max_m[N_CLASS];
    for (int c = threadIdx.x; c < N_CLASS; c += blockDim.x) {
        s_count[c] = 0;
        s_max_n[c] = 0;
        s_max_m[c] = 0;
    }
    __syncthreads();
    // warp-strided so that every lane of a warp takes part in the key groups
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) * 32; base < n_pairs;
         base += nwarps * 32) {
        const int64_t p = base + lane;
        int32_t key = -1, cls = 0;
        int64_t m = 0, n = 0;
        if (p < n_pairs) {
            const int64_t rd = ps.pair_read ? ps.pair_read[p] : p;
            bool bad = rd < 0 || rd >= n_reads;
            if (!bad) {
                const int64_t r0 = ps.read_off[rd], r1 = ps.read_off[rd + 1];
                const int64_t w0 = ps.win_off[p], w1 = ps.win_off[p + 1];
                m = r1 - r0;
                n = w1 - w0;
                bad = r0 < 0 || w0 < 0 || m < 1 || m > SW_MAX_READ_LEN || n < 0 || n > SW_MAX_WINDOW_LEN;
            }
            if (bad) {
                atomicOr(&info->status, ST_BAD_INPUT);
            } else if (ps.mask && !ps.mask[p]) {
                // not selected: no alignment
                out_score[p] = -1;
                out_end[2 * p] = -1;
                out_end[2 * p + 1] = -1;
                if (cig_n) cig_n[p] = 0;
            } else if (n == 0) {
                // an empty window aligns nothing: score 0, no end cell, no CIGAR
                out_score[p] = 0;
                out_end[2 * p] = -1;
                out_end[2 * p + 1] = -1;
                if (cig_n) cig_n[p] = 0;
            } else {
                const int64_t hmax = (int64_t)sc.ma * (m < n ? m : n);
                const int mode = score_mode_for(hmax, score_setting);
                cls = mode * N_MCLASS + mclass_of((int32_t)m);
                int nb = (int)((n - 1) >> 5);
                nb = nb > N_NBUCKET - 1 ? N_NBUCKET - 1 : nb;
                key = cls * N_NBUCKET + (N_NBUCKET - 1 - nb);
            }
            keys[p] = key;
        }
        // one set of atomics per distinct key in the warp (the key fixes the class)
        const KeyGroup g = key_group(key);
        if (key >= 0) {
            const unsigned mx_n = __reduce_max_sync(g.mask, (unsigned)n);
            const unsigned mx_m = __reduce_max_sync(g.mask, (unsigned)m);
            if (g.rank == 0) {
                atomicAdd(&hist[key], g.size);
                atomicAdd(&s_count[cls], g.size);
                atomicMax(&s_max_n[cls], (int32_t)mx_n);
                atomicMax(&s_max_m[cls], (int32_t)mx_m);
            }
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < N_CLASS; c += blockDim.x)
        if (s_count[c]) {
            atomicAdd(&info->count[c], s_count[c]);
            atomicMax(&info->max_n[c], s_max_n[c]);
            atomicMax(&info->max_m[c], s_max_m[c]);
        }
}

// Exclusive scan of the key histogram.  Keys are class-major (N_NBUCKET
// buckets per class) and the per-class counts are known, so block c scans
// class c's buckets after the counts of the classes before it; empty classes
// return at once.
__global__ void __launch_bounds__(N_NBUCKET) k_scan(const int32_t *__restrict__ hist,
                                                    const int32_t *__restrict__ class_count,
                                                    int32_t *__restrict__ start, int32_t *__restrict__ cursor)
{
    const int cls = blockIdx.x, t = threadIdx.x;
    if (class_count[cls] == 0) return;
    __shared__ int32_t part[N_NBUCKET / 32];
    __shared__ int32_t base_s;
    // classes before this one
    int32_t pre = 0;
    for (int c = t; c < cls; c += N_NBUCKET) pre += class_count[c];
    pre = __reduce_add_sync(0xffffffffu, pre);
    if ((t & 31) == 0) part[t >> 5] = pre;
    __syncthreads();
    if (t == 0) {
        int32_t b = 0;
        for (int w = 0; w < N_NBUCKET / 32; ++w) b += part[w];
        base_s = b;
    }
    __syncthreads();
    // block scan of this class's buckets
    const int32_t v = hist[cls * N_NBUCKET + t];
    int32_t x = v;
    for (int d = 1; d < 32; d <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, x, d);
        if ((t & 31) >= d) x += y;
    }
    if ((t & 31) == 31) part[t >> 5] = x;
    __syncthreads();
    int32_t wpre = base_s;
    for (int w = 0; w < (t >> 5); ++w) wpre += part[w];
    const int32_t s = wpre + x - v;
    start[cls * N_NBUCKET + t] = s;
    cursor[cls * N_NBUCKET + t] = s;
}

__global__ void k_scatter(const int32_t *__restrict__ keys, int64_t n_pairs, int32_t *__restrict__ cursor,
                          int32_t *__restrict__ order)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) * 32; base < n_pairs;
         base += nwarps * 32) {
        const int64_t p = base + lane;
        const int32_t k = p < n_pairs ? keys[p] : -1;
        const KeyGroup g = key_group(k);
        if (k >= 0) {
            int32_t at = 0;
            if (g.rank == 0) at = atomicAdd(&cursor[k], g.size);
            at = __shfl_sync(g.mask, at, g.leader);
            order[at + g.rank] = (int32_t)p;
        }
    }
}

// A planned batch must classify into the class counts its plan was made for,
// with no read or window longer than the plan's for its class (the plan's
// scratch is sized from those maxima).  expect: counts, then longest read,
// then longest window, N_CLASS each.
__global__ void k_check_counts(const ClassInfo *__restrict__ info, const int32_t *__restrict__ expect,
                               int32_t *__restrict__ status)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N_CLASS; c += gridDim.x * blockDim.x)
        if (info->count[c] != expect[c] || info->max_m[c] > expect[N_CLASS + c] ||
            info->max_n[c] > expect[2 * N_CLASS + c])
            atomicOr(status, ST_BAD_INPUT);
}

int launch_check_counts(const ClassInfo *info, const int32_t *expect, int32_t *status, cudaStream_t st)
{
    k_check_counts<<<(N_CLASS + 255) / 256, 256, 0, st>>>(info, expect, status);
    count_launch();
    return launch_status();
}

int launch_classify(const PairSet &ps, int64_t n_reads, int64_t n_pairs, Scoring sc, int score_setting,
                    int32_t *keys, int32_t *hist, int32_t *bucket_start, int32_t *cursor,
                    ClassInfo *info, int32_t *order, int32_t *out_score, int32_t *out_end,
                    int32_t *cig_n, cudaStream_t st)
{
    const int threads = 256;
    int64_t blocks = (n_pairs + threads - 1) / threads;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    k_classify<<<(unsigned)blocks, threads, 0, st>>>(ps, n_reads, n_pairs, sc, score_setting, keys, hist, info, out_score,
                                                     out_end, cig_n);
    k_scan<<<N_CLASS, N_NBUCKET, 0, st>>>(hist, info->count, bucket_start, cursor);
    k_scatter<<<(unsigned)blocks, threads, 0, st>>>(keys, n_pairs, cursor, order);
    count_launch(3);
    return launch_status();
}

int launch_scan_scatter(const int32_t *keys, int64_t n_pairs, const int32_t *class_count, int32_t *hist,
                        int32_t *bucket_start, int32_t *cursor, int32_t *order, cudaStream_t st)
{
    const int threads = 256;
    int64_t blocks = (n_pairs + threads - 1) / threads;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    k_scan<<<N_CLASS, N_NBUCKET, 0, st>>>(hist, class_count, bucket_start, cursor);
    k_scatter<<<(unsigned)blocks, threads, 0, st>>>(keys, n_pairs, cursor, order);
    count_launch(2);
    return launch_status();
}

}  // namespace swgb
