// sw_seed.cu -- seeding: reads to the reference windows SW aligns them against.
//
// The paper's Stage C splits each read into overlapping 15-base seeds at two
// phases and maps them exactly onto the reference (every hit is a region);
// Stage D merges the regions of a read that lie close together and keeps the
// long merged regions as candidate alignment locations (CALs); Stage E
// extends each CAL by 30 bases on both sides (task i) and joins extended
// CALs closer than the longest known intron into one window (task ii).
//
// The paper maps seeds with a BWT; here the reference index is a direct
// address table over all 4^k k-mers: table[x] is the end of k-mer x's bucket
// in a positions array, so a lookup is two adjacent loads and the bucket.
// With 280 GB of HBM the table (4^15 words = 4.3 GB) and the positions of a
// human-sized reference (12.4 GB) stay resident.
//
// Seeding runs one warp per (read, strand): seed lookups fill a hit list in
// shared memory, a bitonic sort orders it, ballots find the region breaks,
// and lane 0 joins the few CALs.  Read-strands with more hits than a warp's
// list holds go to a second kernel with one block per item and a larger
// list.  Windows land in a scratch area in any order; a count scan puts them
// in (read, strand, reference) order.
#include <algorithm>

#include "sw_device.cuh"
#include "swgb_internal.h"

namespace swgb {

namespace {

constexpr int kWarpHits = 512;            // hit list of one warp (2 KB of shared memory)
constexpr int kSeedWarps = 8;             // warps per block of the main kernel
constexpr int kBinWords = 512;            // 1024 16-bit bin counters per warp (2 KB)
constexpr int kTabTile = 4096;            // table entries per block of the table scan

__device__ __forceinline__ uint32_t kmask(int k) { return k >= 16 ? 0xFFFFFFFFu : ((1u << (2 * k)) - 1u); }

// Reverse complement of the `cnt` bases held in the low bits of x (first
// base lowest): the order of the 2-bit groups is reversed and each base
// becomes 3 - base.
__device__ __forceinline__ uint32_t revcomp_bits(uint32_t x, int cnt)
{
    uint32_t v = __brev(~x);
    v = ((v >> 1) & 0x55555555u) | ((v & 0x55555555u) << 1);
    return cnt >= 16 ? v : (v >> (32 - 2 * cnt));
}

// Chromosome holding position q: the largest c with off[c] <= q.
__device__ __forceinline__ int chrom_of(const int64_t *__restrict__ off, int n_chrom, int64_t q)
{
    int lo = 0, hi = n_chrom - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= q) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ---- index ---------------------------------------------------------------

// Each thread walks 16 consecutive positions (one packed word); the k-mer at
// q counts when q .. q+k-1 lie in one chromosome.  COUNT adds one to its
// table entry; otherwise the entry (the bucket's fill cursor) hands out its
// slot in `positions`.
template <bool COUNT>
__global__ void k_index_pass(const uint32_t *__restrict__ g, int64_t n_bases, const int64_t *__restrict__ off,
                             int n_chrom, int k, uint32_t *table, uint32_t *__restrict__ positions,
                             const int32_t *status)
{
    if (*(volatile const int32_t *)status & ST_BAD_INPUT) return;
    const uint32_t mask = kmask(k);
    const int64_t n_words = (n_bases + 15) >> 4;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n_words;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q0 = t << 4;
        if (q0 + k > n_bases) continue;
        const uint64_t bits = (uint64_t)__ldg(g + t) | ((t + 1 < n_words ? (uint64_t)__ldg(g + t + 1) : 0ull) << 32);
        int c = chrom_of(off, n_chrom, q0);
        int64_t cend = __ldg(off + c + 1);
        for (int u = 0; u < 16; ++u) {
            const int64_t q = q0 + u;
            if (q + k > n_bases) break;
            while (q >= cend && c + 1 < n_chrom) cend = __ldg(off + (++c) + 1);
            if (q + k > cend) continue;
            const uint32_t code = (uint32_t)(bits >> (2 * u)) & mask;
            if (COUNT) {
                atomicAdd(table + code, 1u);
            } else {
                const uint32_t slot = atomicAdd(table + code, 1u);
                positions[slot] = (uint32_t)q;
            }
        }
    }
}

// Exclusive scan of the table in place (uint32; the total fits: positions
// are 32-bit).  Pass 1: per-tile sums.
__global__ void k_tab_sums(const uint4 *__restrict__ tab, uint32_t *__restrict__ blk)
{
    __shared__ uint32_t ws[8];
    const uint4 *t = tab + blockIdx.x * (int64_t)(kTabTile / 4) + threadIdx.x * 4;
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint4 v = t[i];
        s += v.x + v.y + v.z + v.w;
    }
    for (int d = 16; d > 0; d >>= 1) s += __shfl_down_sync(0xffffffffu, s, d);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t x = 0;
        for (int w = 0; w < 8; ++w) x += ws[w];
        blk[blockIdx.x] = x;
    }
}

// Pass 2: one block scans the tile sums (exclusive, in place) and writes the
// total.
__global__ void k_tab_scan_blocks(uint32_t *blk, int64_t n_blk, int64_t *total)
{
    __shared__ uint32_t ws[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < n_blk; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const uint32_t v = i < n_blk ? blk[i] : 0u;
        uint32_t x = v;
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
            if ((threadIdx.x & 31) >= d) x += y;
        }
        if ((threadIdx.x & 31) == 31) ws[threadIdx.x >> 5] = x;
        __syncthreads();
        uint32_t wpre = 0;
        for (int w = 0; w < (int)(threadIdx.x >> 5); ++w) wpre += ws[w];
        if (i < n_blk) blk[i] = carry + wpre + x - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += wpre + x;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = (int64_t)carry;
}

// Pass 3: each thread scans its 16 entries, the block its threads' sums.
__global__ void k_tab_write(uint4 *tab, const uint32_t *__restrict__ blk)
{
    __shared__ uint32_t ws[8];
    uint4 *t = tab + blockIdx.x * (int64_t)(kTabTile / 4) + threadIdx.x * 4;
    uint32_t e[16];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint4 v = t[i];
        e[4 * i] = v.x; e[4 * i + 1] = v.y; e[4 * i + 2] = v.z; e[4 * i + 3] = v.w;
    }
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i) s += e[i];
    uint32_t x = s;
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
        if ((threadIdx.x & 31) >= d) x += y;
    }
    if ((threadIdx.x & 31) == 31) ws[threadIdx.x >> 5] = x;
    __syncthreads();
    uint32_t run = blk[blockIdx.x] + x - s;
    for (int w = 0; w < (int)(threadIdx.x >> 5); ++w) run += ws[w];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const uint32_t v = e[i];
        e[i] = run;
        run += v;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) t[i] = make_uint4(e[4 * i], e[4 * i + 1], e[4 * i + 2], e[4 * i + 3]);
}

// ---- seeding -------------------------------------------------------------

struct SeedScratch {
    unsigned long long *stats;   // table lookups, hits kept, 32-byte sectors the lookups touch
    uint32_t *wstart, *wend;     // windows in reservation order (capacity entries)
    int64_t capacity;
    unsigned long long *n_win;   // windows reserved so far
    int32_t *wcount;             // per read-strand
    int64_t *wbase;              // per read-strand: first scratch slot
    int32_t *ovf;                // read-strands with too many hits for a warp
    unsigned int *n_ovf;
    int32_t *status;
};

struct SeedCfg {
    SeedKParams p;
    int bin_shift;               // bins of 2^bin_shift >= k + merge_dist bases
    uint32_t mask;
    int max_read;                // longest read seeding accepts
    int block_hits;              // hit list of the large-case kernel
};

__device__ __forceinline__ int n_phase(int m, int first, const SeedKParams &p)
{
    return m >= first + p.k ? (m - first - p.k) / p.stride + 1 : 0;
}

// Seed t of a read with ns0 seeds in the first phase.
__device__ __forceinline__ int seed_start(int t, int ns0, const SeedKParams &p)
{
    return t < ns0 ? t * p.stride : p.phase + (t - ns0) * p.stride;
}

// Code of the seed starting at `s` of the read (strand 0) or of its reverse
// complement (strand 1), first base in the low bits.
__device__ __forceinline__ uint32_t seed_code(const uint32_t *reads, int64_t r0, int m, int s, int strand,
                                              const SeedCfg &c)
{
    if (!strand) return load_bases(reads, r0 + s, c.p.k) & c.mask;
    return revcomp_bits(load_bases(reads, r0 + m - s - c.p.k, c.p.k) & c.mask, c.p.k);
}

// 32-byte sectors a lookup of code x reads: table[x - 1 .. x], and the kept
// bucket positions[lo .. lo + cnt).
__device__ __forceinline__ uint32_t lookup_sectors(uint32_t x, uint32_t lo, uint32_t cnt)
{
    uint32_t n = x ? ((x >> 3) - ((x - 1) >> 3) + 1) : 1u;
    if (cnt) n += ((lo + cnt - 1) >> 3) - (lo >> 3) + 1;
    return n;
}

__device__ __forceinline__ void add_stats(unsigned long long *stats, uint64_t a, uint64_t b, uint64_t c)
{
    for (int d = 16; d > 0; d >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, d);
        b += __shfl_xor_sync(0xffffffffu, b, d);
        c += __shfl_xor_sync(0xffffffffu, c, d);
    }
    if ((threadIdx.x & 31) == 0 && (a | b | c)) {
        atomicAdd(stats, (unsigned long long)a);
        atomicAdd(stats + 1, (unsigned long long)b);
        atomicAdd(stats + 2, (unsigned long long)c);
    }
}

// Asynchronous 4-byte copies from global to shared memory: all of a warp's
// bucket reads are in flight together instead of one dependent load (and
// store) after another per lane.
__device__ __forceinline__ void cp_async4(uint32_t *dst_smem, const uint32_t *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// Bucket of a code: [lo, hi) in positions.
__device__ __forceinline__ void bucket(const uint32_t *__restrict__ table, uint32_t code, uint32_t &lo, uint32_t &hi)
{
    lo = code ? __ldg(table + code - 1) : 0u;
    hi = __ldg(table + code);
}

// Copy the hits of seeds tid, tid + nthreads, ... into list[] at slots taken
// from *fill (a shared-memory counter).
__device__ void seed_gather(const uint32_t *reads, int64_t r0, int m, int strand, const uint32_t *table,
                            const uint32_t *__restrict__ positions, const SeedCfg &c, uint32_t *list,
                            int *fill, int tid, int nthreads, uint64_t *st)
{
    const int ns0 = n_phase(m, 0, c.p), ns = ns0 + n_phase(m, c.p.phase, c.p);
    for (int t = tid; t < ns; t += nthreads) {
        uint32_t lo, hi;
        const uint32_t x = seed_code(reads, r0, m, seed_start(t, ns0, c.p), strand, c);
        bucket(table, x, lo, hi);
        const uint32_t cnt = hi - lo <= (uint32_t)c.p.max_hits ? hi - lo : 0u;
        st[0] += 1;
        st[1] += cnt;
        st[2] += lookup_sectors(x, lo, cnt);
        if (cnt == 0) continue;
        const int at = atomicAdd(fill, (int)(hi - lo));
        for (uint32_t j = lo; j < hi; ++j) cp_async4(list + at + (j - lo), positions + j);
    }
    cp_async_wait_all();
}

// Ascending bitonic sort of list[0 .. n) (n a power of two) by the threads
// tid < nthreads; SYNC is the barrier between steps.
template <bool BLOCK>
__device__ void bitonic_sort(uint32_t *list, int n, int tid, int nthreads)
{
    for (int size = 2; size <= n; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = tid; i < (n >> 1); i += nthreads) {
                const int lo = 2 * i - (i & (stride - 1));
                const int hi = lo + stride;
                const bool up = (lo & size) == 0;
                const uint32_t x = list[lo], y = list[hi];
                if ((x > y) == up) {
                    list[lo] = y;
                    list[hi] = x;
                }
            }
            if (BLOCK) __syncthreads(); else __syncwarp();
        }
    }
}

// Ascending bitonic sort of list[0 .. 32 E) held in registers: lane l holds
// elements l + 32 e.  Partners less than 32 apart sit in other lanes
// (shuffles), those 32 or more apart in the same lane.
template <int E>
__device__ void sort_in_registers(uint32_t *list, int H, int lane)
{
    uint32_t x[E];
#pragma unroll
    for (int e = 0; e < E; ++e) x[e] = lane + 32 * e < H ? list[lane + 32 * e] : 0xFFFFFFFFu;
#pragma unroll
    for (int size = 2; size <= 32 * E; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride >= 32) {
                const int d = stride >> 5;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    if (e & d) continue;
                    const bool up = (((lane + 32 * e) & size) == 0);
                    const uint32_t a = x[e], b = x[e | d];
                    x[e] = up ? min(a, b) : max(a, b);
                    x[e | d] = up ? max(a, b) : min(a, b);
                }
            } else {
                const bool lower = (lane & stride) == 0;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const uint32_t y = __shfl_xor_sync(0xffffffffu, x[e], stride);
                    const bool up = (((lane + 32 * e) & size) == 0);
                    x[e] = (lower == up) ? min(x[e], y) : max(x[e], y);
                }
            }
        }
    }
    __syncwarp();
#pragma unroll
    for (int e = 0; e < E; ++e) list[lane + 32 * e] = x[e];
    __syncwarp();
}

// Regions -> merged regions -> CALs -> extended CALs, by one warp over the
// sorted hits list[0 .. H).  Extended CAL c is written to list[2c],
// list[2c + 1] (start, end); a CAL spans more than min_cal_len >= k bases,
// so it holds at least two hits and c < i / 2 for its last hit i: the
// writes never reach a hit still to be read.  Returns the CAL count.
__device__ int cal_pass(uint32_t *list, int H, const int64_t *__restrict__ off, int n_chrom, const SeedCfg &c,
                        int lane)
{
    const SeedKParams &p = c.p;
    int ncal = 0;
    int64_t carry_s = -1;       // last hit of the previous chunk
    int64_t carry_start = -1;   // start of the region open at the end of the previous chunk
    for (int base = 0; base < H; base += 32) {
        const int i = base + lane;
        const bool valid = i < H;
        const int64_t s = valid ? (int64_t)list[i] : 0;
        int64_t prev_s = __shfl_up_sync(0xffffffffu, s, 1);
        if (lane == 0) prev_s = carry_s;
        // a hit close to the one before starts a region only across a
        // chromosome border: the chromosome is looked up only then
        bool starts = false;
        if (valid) {
            starts = i == 0 || s - prev_s - p.k >= p.merge_dist;
            if (!starts) starts = chrom_of(off, n_chrom, s) != chrom_of(off, n_chrom, prev_s);
        }
        const unsigned F = __ballot_sync(0xffffffffu, starts);
        // does the region of hit i end at i?
        bool next_starts = __shfl_down_sync(0xffffffffu, starts, 1);
        if (lane == 31) {
            next_starts = true;
            if (i + 1 < H) {
                const int64_t s1 = (int64_t)list[i + 1];
                next_starts = s1 - s - p.k >= p.merge_dist ||
                              chrom_of(off, n_chrom, s1) != chrom_of(off, n_chrom, s);
            }
        }
        const bool ends = valid && (i == H - 1 || next_starts);
        const unsigned upto = F & (lane == 31 ? 0xffffffffu : ((2u << lane) - 1u));
        const int src = upto ? 31 - __clz(upto) : 0;
        const int64_t s_src = __shfl_sync(0xffffffffu, s, src);
        const int64_t rstart = upto ? s_src : carry_start;
        const int64_t rend = s + p.k - 1;
        const bool is_cal = ends && rend - rstart + 1 > p.min_cal_len;
        int64_t es = 0, ee = 0;
        if (is_cal) {
            const int ch = chrom_of(off, n_chrom, s);
            const int64_t lo = __ldg(off + ch), hi = __ldg(off + ch + 1);
            es = rstart - p.flank < lo ? lo : rstart - p.flank;
            ee = rend + p.flank > hi - 1 ? hi - 1 : rend + p.flank;
        }
        const unsigned C = __ballot_sync(0xffffffffu, is_cal);
        // every lane has read its hits of this chunk (and lane 31 the next
        // one) before any CAL of the chunk is written
        __syncwarp();
        if (is_cal) {
            const int at = ncal + __popc(C & ((1u << lane) - 1u));
            list[2 * at] = (uint32_t)es;
            list[2 * at + 1] = (uint32_t)ee;
        }
        ncal += __popc(C);
        carry_s = __shfl_sync(0xffffffffu, s, 31);
        carry_start = __shfl_sync(0xffffffffu, rstart, 31);
        __syncwarp();
    }
    return ncal;
}

// Join extended CALs (lane 0, in place): windows (start, end) pairs at
// list[0 ..).  Returns the window count.
__device__ int join_pass(uint32_t *list, int ncal, const int64_t *__restrict__ off, int n_chrom, const SeedCfg &c)
{
    const SeedKParams &p = c.p;
    int nw = 0;
    int64_t ja = -1, jb = -1;
    int jc = -1;
    for (int t = 0; t < ncal; ++t) {
        const int64_t a = list[2 * t], b = list[2 * t + 1];
        if (b - a + 1 > p.max_window) continue;
        const int ch = chrom_of(off, n_chrom, a);
        if (ja >= 0) {
            const int64_t nb = b > jb ? b : jb;
            if (ch == jc && a - jb - 1 < p.max_intron && nb - ja + 1 <= p.max_window) {
                jb = nb;
                continue;
            }
            list[2 * nw] = (uint32_t)ja;
            list[2 * nw + 1] = (uint32_t)jb;
            ++nw;
        }
        ja = a;
        jb = b;
        jc = ch;
    }
    if (ja >= 0) {
        list[2 * nw] = (uint32_t)ja;
        list[2 * nw + 1] = (uint32_t)jb;
        ++nw;
    }
    return nw;
}

// The windows of one read-strand from its sorted hit list (one warp).
__device__ void finish_read_strand(uint32_t *list, int H, int64_t rs, const int64_t *__restrict__ off, int n_chrom,
                                   const SeedCfg &c, const SeedScratch &S, int lane)
{
    const int ncal = cal_pass(list, H, off, n_chrom, c, lane);
    int nw = 0;
    if (lane == 0) nw = join_pass(list, ncal, off, n_chrom, c);
    nw = __shfl_sync(0xffffffffu, nw, 0);
    __syncwarp();
    unsigned long long base = 0;
    if (lane == 0 && nw) base = atomicAdd(S.n_win, (unsigned long long)nw);
    base = __shfl_sync(0xffffffffu, base, 0);
    for (int t = lane; t < nw; t += 32) {
        const unsigned long long q = base + t;
        if (q < (unsigned long long)S.capacity) {
            S.wstart[q] = list[2 * t];
            S.wend[q] = list[2 * t + 1];
        }
    }
    if (lane == 0) {
        S.wcount[rs] = nw;
        S.wbase[rs] = (int64_t)base;
        if (base + nw > (unsigned long long)S.capacity) atomicOr(S.status, ST_CAPACITY);
    }
}

__device__ __forceinline__ uint32_t bin_slot(uint32_t b) { return (b * 0x9E3779B1u) >> 22; }

__device__ __forceinline__ uint32_t bin_count(const uint32_t *bins, uint32_t b)
{
    const uint32_t s = bin_slot(b);
    return (bins[s >> 1] >> (16 * (s & 1))) & 0xFFFFu;
}

// Drops, in place, the hits of list[0 .. H) that no other hit lies close
// to, and returns how many remain (in their old order).  Two hits share a
// region only when fewer than k + merge_dist bases separate their starts,
// so they lie in the same or adjacent bins of 2^bin_shift >= k + merge_dist
// bases; a hit alone in its bin and both neighbours forms a region of its
// own, k <= min_cal_len bases long: never a CAL, and it never joins another
// region.  Bins are counted in a hashed table, where a collision can only
// keep a hit that could have gone.  One warp.
__device__ int drop_isolated_hits(uint32_t *list, int H, uint32_t *bins, int sh, int lane)
{
    for (int i = lane; i < kBinWords; i += 32) bins[i] = 0u;
    __syncwarp();
    for (int i = lane; i < H; i += 32) {
        const uint32_t sl = bin_slot(list[i] >> sh);
        atomicAdd(bins + (sl >> 1), 1u << (16 * (sl & 1)));
    }
    __syncwarp();
    int nk = 0;
    for (int base = 0; base < H; base += 32) {
        const int i = base + lane;
        uint32_t v = 0u;
        bool keep = false;
        if (i < H) {
            v = list[i];
            const uint32_t b = v >> sh;
            const uint32_t tot = bin_count(bins, b) + bin_count(bins, b + 1) + (b ? bin_count(bins, b - 1) : 0u);
            keep = tot >= 2;
        }
        const unsigned K = __ballot_sync(0xffffffffu, keep);
        // the chunk is read before any of it is overwritten; earlier chunks
        // kept at most as many hits as they held
        __syncwarp();
        if (keep) list[nk + __popc(K & ((1u << lane) - 1u))] = v;
        nk += __popc(K);
        __syncwarp();
    }
    return nk;
}

__device__ __forceinline__ int pow2_at_least(int h)
{
    int n = 32;
    while (n < h) n <<= 1;
    return n;
}

// Main kernel: one warp per read-strand rs (read rs / 2, strand rs % 2).
__global__ void __launch_bounds__(kSeedWarps * 32)
k_seed(const uint32_t *__restrict__ reads, const int64_t *__restrict__ roff, int64_t n_reads,
       const uint32_t *__restrict__ table, const uint32_t *__restrict__ positions, const int64_t *__restrict__ off,
       int n_chrom, SeedCfg c, SeedScratch S)
{
    __shared__ uint32_t lists[kSeedWarps][kWarpHits];
    __shared__ uint32_t binss[kSeedWarps][kBinWords];
    __shared__ int fills[kSeedWarps];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    if (*(volatile const int32_t *)S.status & ST_BAD_INPUT) return;
    uint32_t *list = lists[wib];
    const int64_t n_rs = 2 * n_reads;
    uint64_t st[3] = {0, 0, 0};  // this lane's lookups, hits kept, sectors read
    for (int64_t rs = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; rs < n_rs;
         rs += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t r = rs >> 1;
        const int strand = (int)(rs & 1);
        const int64_t r0 = roff[r];
        const int64_t m64 = roff[r + 1] - r0;
        if (m64 < 0 || m64 > c.max_read) {
            if (lane == 0) {
                atomicOr(S.status, ST_BAD_INPUT);
                S.wcount[rs] = 0;
                S.wbase[rs] = 0;
            }
            continue;
        }
        const int m = (int)m64;
        // one lookup per seed: the buckets of seeds lane and lane + 32 stay
        // in registers; seeds beyond the 64th (reads over about 390 bases)
        // are looked up again when their hits are copied
        const int ns0 = n_phase(m, 0, c.p), ns = ns0 + n_phase(m, c.p.phase, c.p);
        uint32_t lo0 = 0, n0 = 0, lo1 = 0, n1 = 0;
        int64_t H = 0;
        for (int t = lane; t < ns; t += 32) {
            uint32_t lo, hi;
            const uint32_t x = seed_code(reads, r0, m, seed_start(t, ns0, c.p), strand, c);
            bucket(table, x, lo, hi);
            const uint32_t cnt = hi - lo <= (uint32_t)c.p.max_hits ? hi - lo : 0u;
            if (t < 32) { lo0 = lo; n0 = cnt; } else if (t < 64) { lo1 = lo; n1 = cnt; }
            H += cnt;
            st[0] += 1;
            st[2] += lookup_sectors(x, lo, 0);
        }
        for (int d = 16; d > 0; d >>= 1) H += __shfl_xor_sync(0xffffffffu, H, d);
        if (H == 0) {
            if (lane == 0) {
                S.wcount[rs] = 0;
                S.wbase[rs] = 0;
            }
            continue;
        }
        if (H > kWarpHits) {
            if (lane == 0) S.ovf[atomicAdd(S.n_ovf, 1u)] = (int32_t)rs;
            continue;
        }
        st[1] += n0 + n1;
        st[2] += (n0 ? ((lo0 + n0 - 1) >> 3) - (lo0 >> 3) + 1 : 0) + (n1 ? ((lo1 + n1 - 1) >> 3) - (lo1 >> 3) + 1 : 0);
        uint32_t own = n0 + n1, at = own;
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, at, d);
            if (lane >= d) at += y;
        }
        at -= own;
        for (uint32_t j = 0; j < n0; ++j) cp_async4(list + at + j, positions + lo0 + j);
        for (uint32_t j = 0; j < n1; ++j) cp_async4(list + at + n0 + j, positions + lo1 + j);
        if (ns > 64) {
            if (lane == 31) fills[wib] = (int)(at + own);
            __syncwarp();
            for (int t = 64 + lane; t < ns; t += 32) {
                uint32_t lo, hi;
                const uint32_t x = seed_code(reads, r0, m, seed_start(t, ns0, c.p), strand, c);
                bucket(table, x, lo, hi);
                st[0] += 1;
                if (hi - lo > (uint32_t)c.p.max_hits || hi == lo) {
                    st[2] += lookup_sectors(x, lo, 0);
                    continue;
                }
                st[1] += hi - lo;
                st[2] += lookup_sectors(x, lo, hi - lo);
                const int a = atomicAdd(&fills[wib], (int)(hi - lo));
                for (uint32_t j = lo; j < hi; ++j) cp_async4(list + a + (j - lo), positions + j);
            }
        }
        cp_async_wait_all();
        __syncwarp();
        H = drop_isolated_hits(list, (int)H, binss[wib], c.bin_shift, lane);
        if (H == 0) {
            if (lane == 0) {
                S.wcount[rs] = 0;
                S.wbase[rs] = 0;
            }
            continue;
        }
        const int n = pow2_at_least((int)H);
        if (n == 32) sort_in_registers<1>(list, (int)H, lane);
        else if (n == 64) sort_in_registers<2>(list, (int)H, lane);
        else if (n == 128) sort_in_registers<4>(list, (int)H, lane);
        else if (n == 256) sort_in_registers<8>(list, (int)H, lane);
        else {
            for (int i = (int)H + lane; i < n; i += 32) list[i] = 0xFFFFFFFFu;
            __syncwarp();
            bitonic_sort<false>(list, n, lane, 32);
        }
        finish_read_strand(list, (int)H, rs, off, n_chrom, c, S, lane);
        __syncwarp();
    }
    add_stats(S.stats, st[0], st[1], st[2]);
}

// Large cases: one block per read-strand with a list of c.block_hits
// entries in dynamic shared memory; the block gathers and sorts, warp 0
// finishes.
__global__ void __launch_bounds__(256)
k_seed_large(const uint32_t *__restrict__ reads, const int64_t *__restrict__ roff,
             const uint32_t *__restrict__ table, const uint32_t *__restrict__ positions,
             const int64_t *__restrict__ off, int n_chrom, SeedCfg c, SeedScratch S)
{
    extern __shared__ uint32_t big[];
    __shared__ int fill;
    if (*(volatile const int32_t *)S.status & ST_BAD_INPUT) return;
    uint64_t st[3] = {0, 0, 0};
    const unsigned n_items = *(volatile unsigned *)S.n_ovf;
    for (unsigned it = blockIdx.x; it < n_items; it += gridDim.x) {
        const int64_t rs = S.ovf[it];
        const int64_t r = rs >> 1;
        const int strand = (int)(rs & 1);
        const int64_t r0 = roff[r];
        const int m = (int)(roff[r + 1] - r0);
        if (threadIdx.x == 0) fill = 0;
        __syncthreads();
        seed_gather(reads, r0, m, strand, table, positions, c, big, &fill, threadIdx.x, blockDim.x, st);
        __syncthreads();
        const int H = fill;
        const int n = pow2_at_least(H);
        if (n > c.block_hits) {  // the host bound makes this impossible
            if (threadIdx.x == 0) {
                atomicOr(S.status, ST_INTERNAL);
                S.wcount[rs] = 0;
                S.wbase[rs] = 0;
            }
            __syncthreads();
            continue;
        }
        for (int i = H + threadIdx.x; i < n; i += blockDim.x) big[i] = 0xFFFFFFFFu;
        __syncthreads();
        bitonic_sort<true>(big, n, threadIdx.x, blockDim.x);
        if (threadIdx.x < 32) finish_read_strand(big, H, rs, off, n_chrom, c, S, threadIdx.x);
        __syncthreads();
    }
    add_stats(S.stats, st[0], st[1], st[2]);
}

// Windows from reservation order into (read, strand, reference) order, with
// their chromosome coordinates; one thread per read-strand.
__global__ void k_seed_place(const SeedScratch S, const int64_t *__restrict__ woff, int64_t n_reads,
                             const int64_t *__restrict__ off, int n_chrom, SeedOutPtrs out)
{
    const int64_t n_rs = 2 * n_reads;
    for (int64_t rs = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; rs <= n_rs;
         rs += (int64_t)gridDim.x * blockDim.x) {
        if (rs == n_rs) {
            out.cand_offsets[n_reads] = woff[n_rs];
            *out.count = woff[n_rs];
            continue;
        }
        const int64_t r = rs >> 1;
        const int strand = (int)(rs & 1);
        const int64_t f0 = woff[rs];
        if (!strand) out.cand_offsets[r] = f0;
        const int nw = S.wcount[rs];
        const int64_t b = S.wbase[rs];
        for (int t = 0; t < nw; ++t) {
            const int64_t f = f0 + t, q = b + t;
            if (f >= S.capacity || q >= S.capacity) continue;
            const int64_t a = S.wstart[q], e = S.wend[q];
            const int ch = chrom_of(off, n_chrom, a);
            out.start[f] = a;
            out.length[f] = (int32_t)(e - a + 1);
            out.chrom[f] = ch;
            out.pos[f] = a - __ldg(off + ch);
            out.strand[f] = (int8_t)strand;
            out.pair_read[f] = r + strand * n_reads;
        }
    }
}

// ---- copies of base ranges ----------------------------------------------

// Bases [s0, s0 + L) of src to bases [d0, d0 + L) of dst, reverse
// complemented when rev; a group of kCopyLanes lanes, a destination word per
// lane and step.  Words the range shares with a neighbour are merged with
// atomicOr into a zeroed destination.
constexpr int kCopyLanes = 8;  // a 100-base read spans 7 words

__device__ void copy_range(const uint32_t *__restrict__ src, int64_t s0, int64_t L, uint32_t *dst, int64_t d0,
                           bool rev, int gl)
{
    if (L <= 0) return;
    const int64_t w0 = d0 >> 4, w1 = (d0 + L - 1) >> 4;
    for (int64_t w = w0 + gl; w <= w1; w += kCopyLanes) {
        const int64_t b0 = w << 4 > d0 ? w << 4 : d0;                       // first base of the range in w
        const int64_t b1 = (w << 4) + 16 < d0 + L ? (w << 4) + 16 : d0 + L;  // one past the last
        const int cnt = (int)(b1 - b0);
        uint32_t x;
        if (!rev) {
            x = load_bases(src, s0 + (b0 - d0), cnt);
        } else {
            // destination base b holds the complement of source base
            // s0 + L - 1 - (b - d0): a forward run ending there, reversed
            x = revcomp_bits(load_bases(src, s0 + L - (b1 - d0), cnt), cnt);
        }
        if (cnt < 16) x &= (1u << (2 * cnt)) - 1u;
        x <<= 2 * (int)(b0 - (w << 4));
        if (cnt == 16) dst[w] = x;
        else atomicOr(dst + w, x);
    }
}

// Zero the words holding mult * (*n_bases_dev) bases (at most cap_words).
__global__ void k_zero_words(uint32_t *dst, const int64_t *__restrict__ n_bases_dev, int mult, int64_t cap_words)
{
    int64_t n = (mult * *n_bases_dev + 15) >> 4;
    if (n > cap_words) n = cap_words;
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < n; w += (int64_t)gridDim.x * blockDim.x)
        dst[w] = 0u;
}

__global__ void k_extract(const uint32_t *__restrict__ g, int64_t n_bases, const int64_t *__restrict__ start,
                          const int32_t *__restrict__ len, const int64_t *__restrict__ woff, int64_t n,
                          uint32_t *dst, int64_t cap_bases, int32_t *status)
{
    const int gl = threadIdx.x % kCopyLanes;
    for (int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / kCopyLanes; w < n;
         w += ((int64_t)gridDim.x * blockDim.x) / kCopyLanes) {
        const int64_t d0 = woff[w], L = len[w], s0 = start[w];
        if (L < 0 || s0 < 0 || s0 + L > n_bases) {
            if (gl == 0) atomicOr(status, ST_BAD_INPUT);
            continue;
        }
        if (d0 + L > cap_bases) {
            if (gl == 0) atomicOr(status, ST_CAPACITY);
            continue;
        }
        copy_range(g, s0, L, dst, d0, false, gl);
    }
}

__global__ void k_two_strands(const uint32_t *__restrict__ reads, const int64_t *__restrict__ roff, int64_t n,
                              uint32_t *dst, int64_t cap_bases, int64_t *__restrict__ doff, int32_t *status)
{
    const int gl = threadIdx.x % kCopyLanes;
    if (*(volatile const int32_t *)status & ST_BAD_INPUT) return;
    const int64_t total = roff[n];
    if (2 * total > cap_bases) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, ST_CAPACITY);
        return;
    }
    for (int64_t it = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / kCopyLanes; it < 2 * n;
         it += ((int64_t)gridDim.x * blockDim.x) / kCopyLanes) {
        const int64_t r = it < n ? it : it - n;
        const bool rev = it >= n;
        const int64_t s0 = roff[r], L = roff[r + 1] - s0;
        const int64_t d0 = rev ? total + s0 : s0;
        if (gl == 0) {
            doff[it] = d0;
            if (it == 2 * n - 1) doff[2 * n] = 2 * total;
        }
        copy_range(reads, s0, L, dst, d0, rev, gl);
    }
}

// CSR offsets off[0 .. n]: non-negative and non-decreasing, off[0] == first
// and off[n] == last where those are >= 0.
__global__ void k_check_offsets(const int64_t *__restrict__ off, int64_t n, int64_t first, int64_t last,
                                int32_t *status)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = off[i], b = off[i + 1];
        if (a < 0 || b < a || (i == 0 && first >= 0 && a != first) || (i == n - 1 && last >= 0 && b != last))
            atomicOr(status, ST_BAD_INPUT);
    }
}

int grid_for(int64_t threads, int per_block, int sm_count, int per_sm)
{
    int64_t b = (threads + per_block - 1) / per_block;
    const int64_t cap = (int64_t)sm_count * per_sm;
    if (b > cap) b = cap;
    return b < 1 ? 1 : (int)b;
}

}  // namespace

int seed_count_per_read(int m, const SeedKParams &p)
{
    const int a = m >= p.k ? (m - p.k) / p.stride + 1 : 0;
    const int b = m >= p.phase + p.k ? (m - p.phase - p.k) / p.stride + 1 : 0;
    return a + b;
}

int launch_index_build(const uint32_t *genome, int64_t n_bases, const int64_t *chrom_off, int n_chrom, int k,
                       uint32_t *table, uint32_t *positions, int64_t *out_n, uint32_t *blk, int sm_count,
                       int32_t *status, cudaStream_t st)
{
    const uint64_t n_tab = 1ull << (2 * k);
    if (cuda_failed(cudaMemsetAsync(table, 0, n_tab * sizeof(uint32_t), st))) return SW_ERR_CUDA;
    k_check_offsets<<<grid_for(n_chrom, 256, sm_count, 4), 256, 0, st>>>(chrom_off, n_chrom, 0, n_bases, status);
    const int g = grid_for((n_bases + 15) / 16, 256, sm_count, 8);
    k_index_pass<true><<<g, 256, 0, st>>>(genome, n_bases, chrom_off, n_chrom, k, table, positions, status);
    const int64_t n_blk = (int64_t)(n_tab / kTabTile);
    k_tab_sums<<<(unsigned)n_blk, 256, 0, st>>>((const uint4 *)table, blk);
    k_tab_scan_blocks<<<1, 1024, 0, st>>>(blk, n_blk, out_n);
    k_tab_write<<<(unsigned)n_blk, 256, 0, st>>>((uint4 *)table, blk);
    k_index_pass<false><<<g, 256, 0, st>>>(genome, n_bases, chrom_off, n_chrom, k, table, positions, status);
    count_launch(6);
    return launch_status();
}

size_t seed_scratch_bytes(int64_t n_reads, int64_t capacity)
{
    const int64_t n_rs = 2 * n_reads;
    auto up = [](size_t x) { return (x + 255) / 256 * 256; };
    return up(64) + up(4 * (size_t)n_rs) + up(8 * (size_t)n_rs) + up(4 * (size_t)n_rs) + up(8 * (size_t)(n_rs + 1)) +
           up(8 * (size_t)((n_rs + 255) / 256 + 1)) + 2 * up(4 * (size_t)std::max<int64_t>(capacity, 1));
}

int launch_seed_windows(const uint32_t *reads, const int64_t *roff, int64_t n_reads, const uint32_t *table,
                        const uint32_t *positions, const int64_t *chrom_off, int n_chrom, const SeedKParams &p,
                        int max_read, int block_hits, SeedOutPtrs out, int64_t capacity, uint8_t *scratch,
                        int64_t *stats_host, int sm_count, int32_t *status, cudaStream_t st)
{
    const int64_t n_rs = 2 * n_reads;
    auto up = [](size_t x) { return (x + 255) / 256 * 256; };
    uint8_t *q = scratch;
    SeedScratch S;
    S.n_win = (unsigned long long *)q;
    S.n_ovf = (unsigned int *)(q + 8);
    S.stats = (unsigned long long *)(q + 16);
    q += up(64);
    S.wcount = (int32_t *)q; q += up(4 * (size_t)n_rs);
    S.wbase = (int64_t *)q; q += up(8 * (size_t)n_rs);
    S.ovf = (int32_t *)q; q += up(4 * (size_t)n_rs);
    int64_t *woff = (int64_t *)q; q += up(8 * (size_t)(n_rs + 1));
    int64_t *blk = (int64_t *)q; q += up(8 * (size_t)((n_rs + 255) / 256 + 1));
    S.wstart = (uint32_t *)q; q += up(4 * (size_t)std::max<int64_t>(capacity, 1));
    S.wend = (uint32_t *)q;
    S.capacity = capacity;
    S.status = status;
    SeedCfg c;
    c.p = p;
    c.mask = p.k >= 16 ? 0xFFFFFFFFu : ((1u << (2 * p.k)) - 1u);
    c.max_read = max_read;
    c.block_hits = block_hits;
    c.bin_shift = 0;
    while (((int64_t)1 << c.bin_shift) < (int64_t)p.k + p.merge_dist) ++c.bin_shift;
    if (cuda_failed(cudaMemsetAsync(scratch, 0, 64, st))) return SW_ERR_CUDA;
    if (cuda_failed(cudaFuncSetAttribute(k_seed_large, cudaFuncAttributeMaxDynamicSharedMemorySize, block_hits * 4)))
        return SW_ERR_CUDA;
    k_check_offsets<<<grid_for(n_reads, 256, sm_count, 4), 256, 0, st>>>(roff, n_reads, -1, -1, status);
    k_seed<<<grid_for(n_rs * 32, kSeedWarps * 32, sm_count, 8), kSeedWarps * 32, 0, st>>>(
        reads, roff, n_reads, table, positions, chrom_off, n_chrom, c, S);
    k_seed_large<<<sm_count, 256, (size_t)block_hits * 4, st>>>(reads, roff, table, positions, chrom_off, n_chrom,
                                                                c, S);
    count_launch(3);
    int rc = launch_scan_i32(S.wcount, n_rs, woff, blk, st);
    if (rc) return rc;
    k_seed_place<<<grid_for(n_rs + 1, 256, sm_count, 8), 256, 0, st>>>(S, woff, n_reads, chrom_off, n_chrom, out);
    count_launch();
    if ((rc = launch_status())) return rc;
    // the counters, into a pinned slot that later calls on the stream leave alone
    return cuda_failed(cudaMemcpyAsync(stats_host, S.stats, 3 * sizeof(int64_t), cudaMemcpyDeviceToHost, st))
               ? SW_ERR_CUDA
               : SW_OK;
}

int launch_extract_windows(const uint32_t *genome, int64_t n_bases, const int64_t *start, const int32_t *len,
                           int64_t n, uint32_t *dst, int64_t cap_bases, int64_t *woff, int64_t *blk, int sm_count,
                           int32_t *status, cudaStream_t st)
{
    int rc = launch_scan_i32(len, n, woff, blk, st);
    if (rc) return rc;
    const int64_t cap_words = (cap_bases + 15) / 16;
    k_zero_words<<<grid_for(cap_words, 256, sm_count, 8), 256, 0, st>>>(dst, woff + n, 1, cap_words);
    k_extract<<<grid_for(n * kCopyLanes, 256, sm_count, 8), 256, 0, st>>>(genome, n_bases, start, len, woff, n, dst,
                                                                  cap_bases, status);
    count_launch(2);
    return launch_status();
}

int launch_two_strands(const uint32_t *reads, const int64_t *roff, int64_t n, uint32_t *dst, int64_t cap_bases,
                       int64_t *doff, int sm_count, int32_t *status, cudaStream_t st)
{
    const int64_t cap_words = (cap_bases + 15) / 16;
    k_check_offsets<<<grid_for(n, 256, sm_count, 4), 256, 0, st>>>(roff, n, 0, -1, status);
    k_zero_words<<<grid_for(cap_words, 256, sm_count, 8), 256, 0, st>>>(dst, roff + n, 2, cap_words);
    k_two_strands<<<grid_for(2 * n * kCopyLanes, 256, sm_count, 8), 256, 0, st>>>(reads, roff, n, dst, cap_bases, doff,
                                                                          status);
    count_launch(3);
    return launch_status();
}

}  // namespace swgb
