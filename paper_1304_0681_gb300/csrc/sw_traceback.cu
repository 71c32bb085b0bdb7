// sw_traceback.cu -- CIGAR of the best local alignment of each pair.
//
// The paper's Stage E, task iii returns the alignment itself, not only its
// score; downstream, long runs of deletions in it mark splice junctions.
// The score pass keeps no traceback.  This pass recomputes the DP exactly
// (int32, unfloored E and F) over a rectangle that provably holds every
// optimal alignment ending at the end cell (i_end, j_end):
//
//   rows 0 .. i_end,  window columns j_lo .. j_end,  j_lo = j_end - i_end - D
//
// where D bounds the deletions of any alignment with this score ending on
// read row i_end: with o <= e <= 0 it holds at most i_end+1 aligned read
// bases worth at most `match` each, and D deleted window bases cost at least
// o + (D-1) e, so D <= (match*(i_end+1) + o - score)/(-e) + 1.  Cells outside
// the rectangle can only lower the recomputed values, and every cell on an
// optimal path keeps its value, so every comparison made by the walk comes
// out as in the full matrix and the CIGAR is the full-matrix one.
//
// Each cell stores 4 bits: bits 0-1 the source of H (0: H == 0, 1: diagonal,
// 2: E, 3: F, in that order of preference), bit 2 "E opens here"
// (E == H(i,j-1) + o), bit 3 "F opens here".  Lane k of a T-lane group holds
// 8 rows, so one 32-bit word per lane and column holds its cells.  The words
// go to a per-group slab in global memory; then the group's first lane walks
// back from the end cell, emitting runs in reverse, and reverses them.
#include "sw_device.cuh"
#include "swgb_internal.h"

namespace swgb {

constexpr unsigned FULLMASK = 0xffffffffu;
constexpr int32_t TB_NEG = -(1 << 28);

struct TbPair {
    int64_t rs, ws;
    int32_t m, n, score, ie, je, jlo, W, rows;
    int32_t p;
};

__device__ __forceinline__ TbPair tb_pair(const TracebackLaunch &L, int64_t item, bool on)
{
    TbPair q{0, 0, 0, 0, 0, -1, -1, 0, 0, 0, -1};
    if (!on || item >= L.n_items) return q;
    const int32_t p = L.order[item];
    const int64_t rd = L.ps.pair_read ? L.ps.pair_read[p] : p;
    q.p = p;
    q.rs = L.ps.read_off[rd];
    q.m = (int32_t)(L.ps.read_off[rd + 1] - q.rs);
    q.ws = L.ps.win_off[p];
    q.n = (int32_t)(L.ps.win_off[p + 1] - q.ws);
    q.score = L.score[p];
    if (q.score <= 0) return q;
    q.ie = L.end[2 * p];
    q.je = L.end[2 * p + 1];
    if (q.ie < 0 || q.ie >= q.m || q.je < 0 || q.je >= q.n || q.score > L.sc.ma * min(q.m, q.n)) {
        // an end cell outside the pair: never walk it
        atomicOr(L.status, ST_INTERNAL);
        q.score = 0;
        return q;
    }
    int32_t jlo = 0;
    if (L.sc.ge < 0) {
        const int32_t num = L.sc.ma * (q.ie + 1) + L.sc.go - q.score;
        const int32_t dmax = num < 0 ? 0 : num / (-L.sc.ge) + 1;
        jlo = q.je - q.ie - dmax;
        if (jlo < 0) jlo = 0;
    }
    q.jlo = jlo;
    q.W = q.je - jlo + 1;
    q.rows = q.ie + 1;
    return q;
}

// Run-length writer that emits runs in reverse order into a CSR slot.
struct RevCigar {
    uint32_t *out;
    int64_t cap;
    int32_t n;
    uint32_t op;
    int32_t len;
    bool overflow;
    __device__ void push(uint32_t o, int32_t l)
    {
        if (l <= 0) return;
        if (len > 0 && o == op) { len += l; return; }
        flush();
        op = o;
        len = l;
    }
    __device__ void flush()
    {
        if (len > 0) {
            if (n < cap) out[n] = ((uint32_t)len << 4) | op;
            else overflow = true;
            ++n;
        }
        len = 0;
    }
};

__global__ void __launch_bounds__(128) k_traceback(const TracebackLaunch L)
{
    const int lane = threadIdx.x & 31;
    const int T = L.lanes;
    const int G = 32 / T;
    const int g = lane / T;
    const int k = lane - g * T;
    const bool on = g < G;
    const int64_t warp_global = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint32_t *slab = on ? L.slab + (warp_global * G + g) * L.slab_group_words : nullptr;
    int32_t *bnd = (on && L.boundary) ? L.boundary + (warp_global * G + g) * L.boundary_group_ints : nullptr;
    const int64_t bnd_half = L.boundary_group_ints / 2;
    const int32_t ma = L.sc.ma, mi = L.sc.mi, go = L.sc.go, ge = L.sc.ge;

    for (;;) {
        int base = 0;
        if (lane == 0) base = atomicAdd(L.work_counter, G);
        base = __shfl_sync(FULLMASK, base, 0);
        if (base >= L.n_items) break;
        const int64_t item = base + g;
        const TbPair q = tb_pair(L, item, on);
        const int32_t rows_w = __reduce_max_sync(FULLMASK, (unsigned)q.rows);
        const int32_t W_w = __reduce_max_sync(FULLMASK, (unsigned)q.W);
        const int rpc = T * TB_ROWS;
        const int chunks = (rows_w + rpc - 1) / rpc;
        const int steps = W_w + T - 1;

        for (int c = 0; c < chunks; ++c) {
            const int i0 = c * rpc + k * TB_ROWS;
            uint32_t codes = 0x44444444u;  // 4 bits per row, 4 = no base
            {
                const int cnt = min(TB_ROWS, q.rows - i0);
                if (cnt > 0) {
                    const uint32_t w = load_bases(L.ps.reads, q.rs + i0, cnt);
#pragma unroll
                    for (int r = 0; r < TB_ROWS; ++r)
                        if (r < cnt) codes = (codes & ~(0xFu << (4 * r))) | (((w >> (2 * r)) & 3u) << (4 * r));
                }
            }
            int32_t E[TB_ROWS], Hp[TB_ROWS];
#pragma unroll
            for (int r = 0; r < TB_ROWS; ++r) {
                E[r] = TB_NEG;
                Hp[r] = 0;
            }
            int32_t diag_in = 0, out_h = 0, out_f = TB_NEG;
            uint32_t ww = 0;
            const bool load_bnd = c > 0, store_bnd = c + 1 < chunks;
            const int32_t *bin = load_bnd && bnd ? bnd + (c & 1) * bnd_half : nullptr;
            int32_t *bout = store_bnd && bnd ? bnd + ((c + 1) & 1) * bnd_half : nullptr;

            for (int t = 0; t < steps; ++t) {
                const int j = t - k;
                int32_t up_h = __shfl_up_sync(FULLMASK, out_h, 1);
                int32_t up_f = __shfl_up_sync(FULLMASK, out_f, 1);
                if (k == 0) {
                    if (bin && j < q.W) {
                        up_h = bin[2 * j];
                        up_f = bin[2 * j + 1];
                    } else {
                        up_h = 0;
                        up_f = TB_NEG;
                    }
                }
                if (j >= 0 && j < q.W) {
                    if ((j & 15) == 0) ww = load_bases(L.ps.wins, q.ws + q.jlo + j, min(16, q.W - j));
                    const uint32_t w = ww & 3u;
                    ww >>= 2;
                    int32_t d0 = diag_in, hu = up_h, f = up_f;
                    uint32_t word = 0;
#pragma unroll
                    for (int r = 0; r < TB_ROWS; ++r) {
                        const uint32_t x = (codes >> (4 * r)) & 0xFu;
                        const int32_t s = x == w ? ma : mi;
                        bool eopen, fopen;
                        const int32_t e = __vibmax_s32(Hp[r] + go, E[r] + ge, &eopen);
                        f = __vibmax_s32(hu + go, f + ge, &fopen);
                        const int32_t d = d0 + s;
                        const int32_t h = __vimax3_s32_relu(d, e, f);
                        const uint32_t src = h == 0 ? 0u : (h == d ? 1u : (h == e ? 2u : 3u));
                        word |= (src | ((uint32_t)eopen << 2) | ((uint32_t)fopen << 3)) << (4 * r);
                        d0 = Hp[r];
                        Hp[r] = h;
                        E[r] = e;
                        hu = h;
                        if (i0 + r == q.ie && j == q.W - 1 && h != q.score) atomicOr(L.status, ST_INTERNAL);
                    }
                    slab[((int64_t)c * q.W + j) * T + k] = word;
                    out_h = hu;
                    out_f = f;
                    if (bout && k == T - 1) {
                        bout[2 * j] = out_h;
                        bout[2 * j + 1] = out_f;
                    }
                }
                diag_in = up_h;
            }
            __syncwarp();
        }

        // walk back from the end cell (the group's first lane)
        if (on && k == 0 && q.p >= 0) {
            const int64_t off = L.cig_off[q.p];
            const int64_t cap = L.cig_off[q.p + 1] - off;
            if (q.score <= 0) {
                L.cig_n[q.p] = 0;
            } else {
                RevCigar rc{L.cig_ops + off, cap, 0, 0u, 0, false};
                rc.push(4u, q.m - 1 - q.ie);  // trailing soft clip
                int32_t i = q.ie, jj = q.W - 1;
                int state = 0;
                const int64_t limit = (int64_t)q.rows + q.W + 4;
                int64_t it = 0;
                for (; it < limit; ++it) {
                    if (i < 0 || jj < 0) break;
                    const int cc = i / rpc, kk = (i % rpc) / TB_ROWS, nib = i % TB_ROWS;
                    const uint32_t code = (slab[((int64_t)cc * q.W + jj) * T + kk] >> (4 * nib)) & 0xFu;
                    if (state == 0) {
                        const uint32_t src = code & 3u;
                        if (src == 0u) break;
                        if (src == 1u) { rc.push(0u, 1); --i; --jj; }
                        else state = src == 2u ? 1 : 2;
                    } else if (state == 1) {
                        rc.push(2u, 1);
                        if (code & 4u) state = 0;
                        --jj;
                    } else {
                        rc.push(1u, 1);
                        if (code & 8u) state = 0;
                        --i;
                    }
                }
                if (it >= limit || state != 0) atomicOr(L.status, ST_INTERNAL);
                rc.push(4u, i + 1);  // leading soft clip
                rc.flush();
                if (rc.overflow) {
                    L.cig_n[q.p] = -1;
                    atomicOr(L.status, ST_CAPACITY);
                } else {
                    uint32_t *o = L.cig_ops + off;
                    for (int32_t a = 0, b = rc.n - 1; a < b; ++a, --b) {
                        const uint32_t tmp = o[a];
                        o[a] = o[b];
                        o[b] = tmp;
                    }
                    L.cig_n[q.p] = rc.n;
                }
            }
        }
        __syncwarp();
    }
}

int launch_traceback(const TracebackLaunch &L, int blocks, int threads, cudaStream_t st)
{
    k_traceback<<<blocks, threads, 0, st>>>(L);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? SW_OK : SW_ERR_CUDA;
}

int traceback_kernel_occupancy(int *max_blocks_per_sm, int threads)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(max_blocks_per_sm, k_traceback, threads, 0) == cudaSuccess
               ? SW_OK
               : SW_ERR_CUDA;
}

}  // namespace swgb
