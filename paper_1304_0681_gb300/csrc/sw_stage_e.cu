// sw_stage_e.cu -- Stage E, task iv: alignment records and splice junctions.
//
// The paper turns every alignment whose score passes a threshold into a
// record (reference position, strand, ...) and looks in its CIGAR for long
// deletion runs whose ends carry the intron marks GT ... AG or CT ... AC;
// such a run is a splice junction, counted over all batches (§2, Stage E).
// The SW task also reports statistics of each alignment, a quality score
// among them, which the paper does not define; here a read's top hit and a
// mapping quality from the gap between its best and second-best scores.
//
// Records: one thread per pair computes the aligned span from its CIGAR;
// a block count, a scan of the block counts and a second pass write the
// records in pair order.  Junctions: one thread per record walks its CIGAR,
// reads the four mark bases of each long D run from the packed window and
// counts the junction in an open-addressing hash table of packed 64-bit
// keys (insertion by atomicCAS, at most `capacity` probes).
#include <algorithm>

#include "sw_device.cuh"
#include "swgb_internal.h"

namespace swgb {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr uint64_t KEY_EMPTY = ~0ull;

struct Span {
    bool rec;
    int32_t read_start, j_start, n;
};

// The aligned span of pair p, or rec = false when it is no record.
__device__ __forceinline__ Span pair_span(const int32_t *score, const int32_t *end, const uint32_t *ops,
                                          const int64_t *cig_off, const int32_t *cig_n, int64_t p, int32_t min_score)
{
    Span s{false, 0, 0, 0};
    const int32_t sc = score[p];
    const int32_t n = cig_n[p];
    if (sc <= 0 || sc < min_score || n <= 0) return s;
    const uint32_t *o = ops + cig_off[p];
    int32_t ref = 0;
    for (int32_t k = 0; k < n; ++k) {
        const uint32_t v = o[k], op = v & 0xFu, len = v >> 4;
        if (op == 0u || op == 2u) ref += (int32_t)len;
        if (k == 0 && op == 4u) s.read_start = (int32_t)len;
    }
    s.rec = true;
    s.j_start = end[2 * p + 1] + 1 - ref;
    s.n = n;
    return s;
}

__global__ void k_record_counts(const int32_t *score, const int32_t *end, const uint32_t *ops, const int64_t *cig_off,
                                const int32_t *cig_n, int64_t n_pairs, int32_t min_score, int32_t *blk_count)
{
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool rec = p < n_pairs && pair_span(score, end, ops, cig_off, cig_n, p, min_score).rec;
    const int c = __syncthreads_count(rec);
    if (threadIdx.x == 0) blk_count[blockIdx.x] = c;
}

// Exclusive scan of the block counts in one block; the total goes to *total.
__global__ void k_scan_counts(const int32_t *blk_count, int64_t n_blk, int64_t *blk_off, int64_t *total)
{
    __shared__ int64_t warp_sum[32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < n_blk; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const int64_t v = i < n_blk ? blk_count[i] : 0;
        int64_t x = v;
        for (int d = 1; d < 32; d <<= 1) {
            const int64_t y = __shfl_up_sync(FULL, x, d);
            if ((threadIdx.x & 31) >= d) x += y;
        }
        if ((threadIdx.x & 31) == 31) warp_sum[threadIdx.x >> 5] = x;
        __syncthreads();
        int64_t wpre = 0;
        for (int w = 0; w < (int)(threadIdx.x >> 5); ++w) wpre += warp_sum[w];
        if (i < n_blk) blk_off[i] = carry + wpre + x - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += wpre + x;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void k_record_write(const int32_t *score, const int32_t *end, const uint32_t *ops, const int64_t *cig_off,
                               const int32_t *cig_n, int64_t n_pairs, const int32_t *chrom, const int64_t *pos,
                               const int8_t *strand, int32_t min_score, const int64_t *blk_off, sw_record_t *out)
{
    __shared__ int32_t warp_cnt[32];
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    Span s{false, 0, 0, 0};
    if (p < n_pairs) s = pair_span(score, end, ops, cig_off, cig_n, p, min_score);
    const unsigned bal = __ballot_sync(FULL, s.rec);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) warp_cnt[wid] = __popc(bal);
    __syncthreads();
    int pre = 0;
    for (int w = 0; w < wid; ++w) pre += warp_cnt[w];
    if (s.rec) {
        const int64_t at = blk_off[blockIdx.x] + pre + __popc(bal & ((1u << lane) - 1u));
        sw_record_t r;
        r.pair = p;
        r.ref_start = pos[p] + s.j_start;
        r.ref_end = pos[p] + end[2 * p + 1];
        r.chrom = chrom[p];
        r.score = score[p];
        r.read_start = s.read_start;
        r.read_end = end[2 * p];
        r.strand = strand[p];
        r.n_ops = s.n;
        out[at] = r;
    }
}

__device__ __forceinline__ uint32_t base_at(const uint32_t *wins, int64_t q) { return load_bases(wins, q, 1) & 3u; }

__device__ __forceinline__ uint64_t slot_of(uint64_t key, int log2cap)
{
    return (key * 0x9E3779B97F4A7C15ull) >> (64 - log2cap);
}

__global__ void k_junctions(const uint32_t *wins, const int64_t *win_off, const int32_t *score, const int32_t *end,
                            const uint32_t *ops, const int64_t *cig_off, const int32_t *cig_n, int64_t n_pairs,
                            const int32_t *chrom, const int64_t *pos, int32_t min_score, int32_t min_intron,
                            uint64_t *keys, unsigned long long *counts, int64_t capacity, int log2cap,
                            int32_t *status)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n_pairs;
         p += (int64_t)gridDim.x * blockDim.x) {
        const Span s = pair_span(score, end, ops, cig_off, cig_n, p, min_score);
        if (!s.rec) continue;
        const uint32_t *o = ops + cig_off[p];
        const int64_t w0 = win_off[p], wn = win_off[p + 1] - w0;
        int64_t j = s.j_start;
        for (int32_t k = 0; k < s.n; ++k) {
            const uint32_t v = o[k], op = v & 0xFu;
            const int64_t len = v >> 4;
            if (op == 0u) {
                j += len;
            } else if (op == 2u) {
                if (len >= min_intron && j >= 0 && j + len <= wn) {
                    const uint32_t b0 = base_at(wins, w0 + j), b1 = base_at(wins, w0 + j + 1);
                    const uint32_t e0 = base_at(wins, w0 + j + len - 2), e1 = base_at(wins, w0 + j + len - 1);
                    int st = -1;
                    if (b0 == 2u && b1 == 3u && e0 == 0u && e1 == 2u) st = 0;       // GT ... AG
                    else if (b0 == 1u && b1 == 3u && e0 == 0u && e1 == 1u) st = 1;  // CT ... AC
                    if (st >= 0) {
                        const int64_t c = chrom[p], start = pos[p] + j;
                        if (c < 0 || c >= 4096 || start < 0 || start >= 0xFFFFFFFFll || len > (1 << 19)) {
                            atomicOr(status, ST_UNSUPPORTED);
                        } else {
                            const uint64_t key = ((uint64_t)c << 52) | ((uint64_t)st << 51) |
                                                 ((uint64_t)start << 19) | (uint64_t)(len - 1);
                            uint64_t h = slot_of(key, log2cap);
                            bool done = false;
                            for (int64_t probe = 0; probe < capacity; ++probe) {
                                const unsigned long long prev = atomicCAS(
                                    (unsigned long long *)&keys[h], (unsigned long long)KEY_EMPTY,
                                    (unsigned long long)key);
                                if (prev == KEY_EMPTY || prev == key) {
                                    atomicAdd(&counts[h], 1ull);
                                    done = true;
                                    break;
                                }
                                h = (h + 1) & (uint64_t)(capacity - 1);
                            }
                            if (!done) atomicOr(status, ST_CAPACITY);
                        }
                    }
                }
                j += len;
            }
        }
    }
}

__global__ void k_table_clear(uint64_t *keys, unsigned long long *counts, int64_t capacity)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < capacity; i += (int64_t)gridDim.x * blockDim.x) {
        keys[i] = KEY_EMPTY;
        counts[i] = 0ull;
    }
}

__global__ void k_table_export(const uint64_t *keys, const unsigned long long *counts, int64_t capacity,
                               sw_junction_t *out, int64_t max_out, unsigned long long *n_out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < capacity; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = keys[i];
        if (key == KEY_EMPTY) continue;
        const unsigned long long at = atomicAdd(n_out, 1ull);
        if ((int64_t)at < max_out) {
            sw_junction_t jn;
            jn.chrom = (int32_t)(key >> 52);
            jn.strand = (int32_t)((key >> 51) & 1u);
            jn.start = (int64_t)((key >> 19) & 0xFFFFFFFFull);
            jn.end = jn.start + (int64_t)(key & ((1u << 19) - 1u));
            jn.count = (int64_t)counts[i];
            out[at] = jn;
        }
    }
}

int grid_for(int64_t n, int threads) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, 152 * 32)); }

// Top hit per read: best score S1 and its candidate (first on ties), the best
// score S2 of the other candidates (0 when there are none), and the mapping
// quality min(60, floor(60 (S1 - S2) / S1)), 0 when S1 <= 0.  Masked-out
// candidates are skipped; a read without candidates gets -1, -1, -1, 0.
__global__ void k_top_hits(const int32_t *__restrict__ score, const int64_t *__restrict__ cand_off, int64_t n_reads,
                           const uint8_t *__restrict__ mask, int32_t *__restrict__ best, int32_t *__restrict__ best_cand,
                           int32_t *__restrict__ second, int32_t *__restrict__ mapq)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n_reads;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p0 = cand_off[r], p1 = cand_off[r + 1];
        int32_t s1 = 0, s2 = 0, c1 = -1;
        bool any = false, two = false;
        for (int64_t p = p0; p < p1; ++p) {
            if (mask && !mask[p]) continue;
            const int32_t s = score[p];
            if (!any) {
                s1 = s;
                c1 = (int32_t)(p - p0);
                any = true;
            } else if (s > s1) {
                s2 = s1;  // the old best is now the best of the others
                s1 = s;
                c1 = (int32_t)(p - p0);
                two = true;
            } else {
                s2 = two ? max(s2, s) : s;
                two = true;
            }
        }
        int32_t q = 0;
        if (!any) {
            s1 = -1;
            s2 = -1;
        } else {
            if (!two) s2 = 0;
            if (s1 > 0) {
                const int64_t g = 60 * ((int64_t)s1 - s2) / s1;
                q = (int32_t)(g < 60 ? g : 60);
            }
        }
        best[r] = s1;
        if (best_cand) best_cand[r] = c1;
        if (second) second[r] = s2;
        if (mapq) mapq[r] = q;
    }
}

}  // namespace

int launch_top_hits(const int32_t *score, const int64_t *cand_off, int64_t n_reads, const uint8_t *mask, int32_t *best,
                    int32_t *best_cand, int32_t *second, int32_t *mapq, cudaStream_t st)
{
    int64_t blocks = (n_reads + 127) / 128;
    blocks = std::max<int64_t>(1, std::min<int64_t>(blocks, 152 * 32));
    k_top_hits<<<(unsigned)blocks, 128, 0, st>>>(score, cand_off, n_reads, mask, best, best_cand, second, mapq);
    count_launch();
    return launch_status();
}

int launch_records(const int32_t *score, const int32_t *end, const sw_cigar_t &cig, int64_t n_pairs,
                   const int32_t *chrom, const int64_t *pos, const int8_t *strand, int32_t min_score,
                   sw_record_t *out, int64_t *out_count, int32_t *blk_count, int64_t *blk_off, cudaStream_t st)
{
    const int threads = 256;
    const int64_t n_blk = (n_pairs + threads - 1) / threads;
    k_record_counts<<<(unsigned)n_blk, threads, 0, st>>>(score, end, cig.ops, cig.offsets, cig.n_ops, n_pairs,
                                                          min_score, blk_count);
    k_scan_counts<<<1, 1024, 0, st>>>(blk_count, n_blk, blk_off, out_count);
    k_record_write<<<(unsigned)n_blk, threads, 0, st>>>(score, end, cig.ops, cig.offsets, cig.n_ops, n_pairs, chrom,
                                                         pos, strand, min_score, blk_off, out);
    count_launch(3);
    return launch_status();
}

int launch_junctions(const uint32_t *wins, const int64_t *win_off, const int32_t *score, const int32_t *end,
                     const sw_cigar_t &cig, int64_t n_pairs, const int32_t *chrom, const int64_t *pos,
                     int32_t min_score, int32_t min_intron, uint64_t *table, int64_t capacity, int32_t *status,
                     cudaStream_t st)
{
    int log2cap = 0;
    while ((1ll << log2cap) < capacity) ++log2cap;
    k_junctions<<<grid_for(n_pairs, 256), 256, 0, st>>>(wins, win_off, score, end, cig.ops, cig.offsets, cig.n_ops,
                                                         n_pairs, chrom, pos, min_score, min_intron, table,
                                                         (unsigned long long *)(table + capacity), capacity, log2cap,
                                                         status);
    count_launch();
    return launch_status();
}

int launch_table_clear(uint64_t *table, int64_t capacity, cudaStream_t st)
{
    k_table_clear<<<grid_for(capacity, 256), 256, 0, st>>>(table, (unsigned long long *)(table + capacity), capacity);
    count_launch();
    return launch_status();
}

int launch_table_export(const uint64_t *table, int64_t capacity, sw_junction_t *out, int64_t max_out,
                        int64_t *out_count, cudaStream_t st)
{
    if (cuda_failed(cudaMemsetAsync(out_count, 0, sizeof(int64_t), st))) return SW_ERR_CUDA;
    k_table_export<<<grid_for(capacity, 256), 256, 0, st>>>(table, (const unsigned long long *)(table + capacity),
                                                             capacity, out, max_out, (unsigned long long *)out_count);
    count_launch();
    return launch_status();
}

}  // namespace swgb
