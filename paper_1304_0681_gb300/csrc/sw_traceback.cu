// sw_traceback.cu -- CIGAR of the best local alignment of each pair.
//
// The paper's Stage E, task iii returns the alignment itself, not only its
// score; downstream, long runs of deletions in it mark splice junctions.
// The score pass keeps no traceback.  This pass recomputes the DP exactly
// (int32, unfloored E and F) over a region that provably holds every optimal
// alignment ending at the end cell (i_end, j_end), and walks back through it.
//
// The region.  Any alignment with this score that ends on read row i_end
// holds at most i_end+1 aligned read bases, each worth at most `match`, and
// with o <= e <= 0 one gap run is the cheapest way to spend gap bases, so
//   deletions  D <= (match (i_end+1) + o - score) / (-e) + 1
//   insertions I <= (match (i_end+1) + o - e - score) / (match - e).
// Walking back from the end cell, a deletion lowers the diagonal d = j - i by
// one and an insertion raises it by one, so every optimal path stays in the
// band  j_end - i_end - D <= j - i <= j_end - i_end + I,  rows 0..i_end.
// Cells outside the band are treated as unreachable (H = 0, E = F = -inf);
// that can only lower recomputed values, and cells on optimal paths keep
// theirs, so every comparison of the walk comes out as in the full matrix.
//
// Layout.  A group of T lanes owns one pair; lane k holds 8 rows of a chunk of
// 8T rows and sweeps the chunk's band window of columns with a one-step
// wavefront (shuffles pass the bottom row down); the chunk's last lane hands
// its bottom row to the next chunk through a double-buffered scratch row.
// Each cell stores 4 bits -- bits 0-1 the source of H (0: H == 0, 1: diagonal,
// 2: E, 3: F, in that order of preference), bit 2 "E opens here"
// (E == H(i,j-1) + o), bit 3 "F opens here" -- one 32-bit word per lane and
// column, in a per-group slab.  The group's first lane then walks back from
// the end cell, writes the runs reversed into the pair's CSR slot and
// reverses them in place.
//
// Scheduling.  k_tb_keys gives every pair a cost key (rows x window), a
// counting sort orders each length class by cost so a warp's groups sweep
// similar windows, and pairs whose slab exceeds the per-group slab of the
// main launch form a separate launch with larger slabs.
#include "sw_device.cuh"
#include "swgb_internal.h"

namespace swgb {

constexpr unsigned FULLMASK = 0xffffffffu;
constexpr int32_t TB_NEG = -(1 << 28);

struct TbPair {
    int64_t rs, ws;
    int32_t m, n, score, ie, je;
    int32_t jlo, W, rows;   // rectangle: window columns jlo .. jlo+W-1, rows 0..rows-1
    int32_t a, b;           // band in rectangle columns: row i spans [i + a, i + b]
    int32_t p;
};

__device__ __forceinline__ TbPair tb_pair(const TbParams &P, int32_t p, int32_t *status)
{
    TbPair q{};
    q.p = p;
    q.ie = -1;
    q.je = -1;
    if (p < 0) return q;
    const int64_t rd = P.ps.pair_read ? P.ps.pair_read[p] : p;
    q.rs = P.ps.read_off[rd];
    q.m = (int32_t)(P.ps.read_off[rd + 1] - q.rs);
    q.ws = P.ps.win_off[p];
    q.n = (int32_t)(P.ps.win_off[p + 1] - q.ws);
    q.score = P.score[p];
    if (q.score <= 0) return q;
    q.ie = P.end[2 * p];
    q.je = P.end[2 * p + 1];
    if (q.ie < 0 || q.ie >= q.m || q.je < 0 || q.je >= q.n || q.score > P.sc.ma * min(q.m, q.n)) {
        // an end cell outside the pair: never walk it
        if (status) atomicOr(status, ST_INTERNAL);
        q.score = 0;
        return q;
    }
    const int32_t ma = P.sc.ma, go = P.sc.go, ge = P.sc.ge;
    const int32_t dend = q.je - q.ie;
    int32_t dlo = -q.ie - 1;  // no lower limit when gaps are free
    if (ge < 0) {
        const int32_t num = ma * (q.ie + 1) + go - q.score;
        dlo = dend - (num < 0 ? 0 : num / (-ge) + 1);
    }
    const int32_t inum = ma * (q.ie + 1) + go - ge - q.score;
    const int32_t dhi = dend + (inum < 0 ? 0 : inum / (ma - ge));
    q.jlo = max(0, dlo);
    q.W = q.je - q.jlo + 1;
    q.rows = q.ie + 1;
    q.a = dlo - q.jlo;
    q.b = dhi - q.jlo;
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
        if (len > 0 && o == op) {
            len += l;
            return;
        }
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

__device__ __forceinline__ int64_t lmin(int64_t a, int64_t b) { return a < b ? a : b; }

// Band window of chunk c (rows c*rc .. c*rc+rc-1) in rectangle columns.
__device__ __forceinline__ void chunk_window(const TbPair &q, int c, int rc, int &lo, int &hi)
{
    lo = max(0, c * rc + q.a);
    hi = min(q.W - 1, c * rc + rc - 1 + q.b);
}

// Slab words a pair needs with T lanes: sum over chunks of window x T.
__device__ __forceinline__ int64_t slab_need(const TbPair &q, int T)
{
    if (q.score <= 0) return 0;
    const int rc = T * TB_ROWS;
    const int chunks = (q.rows + rc - 1) / rc;
    const int wcap = min(q.W, rc - 1 + (q.b - q.a) + 1);
    return (int64_t)chunks * wcap * T;
}

// Cost key per pair: class-major, most expensive first within a class.
__global__ void k_tb_keys(TbParams P, const int32_t *__restrict__ order, int64_t n_items,
                          const int32_t *__restrict__ score_keys, int32_t *__restrict__ tb_keys,
                          int32_t *__restrict__ hist, TbClassInfo *__restrict__ info)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n_items;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int32_t p = order[q];
        const int cls = score_keys[p] / N_NBUCKET;
        const int T = P.lanes;
        const TbPair t = tb_pair(P, p, nullptr);
        const int64_t need = slab_need(t, T);
        // big slabs first, then by falling cost (~9% buckets of rows x window)
        int32_t key;
        if (need > P.small_slab_words) {
            key = cls * N_NBUCKET;
        } else {
            const float cost = t.score > 0 ? (float)t.rows * (float)min(t.W, 8 * T + (t.b - t.a)) : 1.f;
            const int cb = min(254, max(0, (int)(8.f * __log2f(cost))));
            key = cls * N_NBUCKET + 1 + (254 - cb);
        }
        tb_keys[p] = key;
        atomicAdd(&hist[key], 1);
        if (need > 0) {
            const bool big = need > P.small_slab_words;
            atomicMax(&info->max_need[cls], (int32_t)(need < (int64_t)INT32_MAX ? need : (int64_t)INT32_MAX));
            atomicMax(&info->max_wcap[big ? 0 : 1][cls], min(t.W, 8 * T + (t.b - t.a)));
            if (big) atomicAdd(&info->n_big[cls], 1);
        }
    }
}

// TILED (one lane per pair only): the warp's slabs and boundary rows are
// interleaved lane-minor -- word (chunk c, column jl) of lane l at
// [(c * WCAP + jl) * 32 + l] -- so that, all lanes being at the same chunk
// and column at every step, each store instruction writes one full line.
// Otherwise every group owns a packed slab of its chunks' windows.
template <bool TILED>
__global__ void __launch_bounds__(128) k_traceback(const TracebackLaunch L)
{
    const TbParams &P = L.P;
    // column tables: s_tab[w] byte x = s(x, w) - o
    __shared__ uint32_t s_tab[4];
    {
        const uint32_t mis4 = ((uint32_t)(uint8_t)(int8_t)(P.sc.mi - P.sc.go)) * 0x01010101u;
        const uint32_t ma4 = ((uint32_t)(uint8_t)(int8_t)(P.sc.ma - P.sc.go)) * 0x01010101u;
        if (threadIdx.x < 4) s_tab[threadIdx.x] = prmt(mis4, ma4, 0x3210u + (4u << (4u * threadIdx.x)));
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    const int T = L.lanes;
    const int G = 32 / T;
    const int g = lane / T;
    const int k = lane - g * T;
    const bool on = g < G;
    const int rc = T * TB_ROWS;
    const int64_t warp_global = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int WCAP = L.wcap;
    // slab: TILED -> the warp's tile, indexed with the lane; else the group's slab
    uint32_t *slab = !on ? nullptr
                         : TILED ? L.slab + warp_global * 32 * L.slab_group_words
                                 : L.slab + (warp_global * G + g) * L.slab_group_words;
    int32_t *bnd = !on ? nullptr
                       : TILED ? L.boundary + warp_global * 32 * L.boundary_group_ints
                               : L.boundary + (warp_global * G + g) * L.boundary_group_ints;
    const int64_t bnd_half = TILED ? 32 * (L.boundary_group_ints / 2) : L.boundary_group_ints / 2;
    const int32_t go = P.sc.go, ge = P.sc.ge;

    for (;;) {
        int base = 0;
        if (lane == 0) base = atomicAdd(L.work_counter, G);
        base = __shfl_sync(FULLMASK, base, 0);
        if (base >= L.n_items) break;
        const int64_t item = base + g;
        const int32_t p = (on && item < L.n_items) ? L.order[item] : -1;
        TbPair q = tb_pair(P, p, L.status);
        const bool over = TILED ? (q.rows > (L.slab_group_words / max(WCAP, 1)) * rc ||
                                   min(q.W, rc + (q.b - q.a)) > WCAP)
                                : (slab_need(q, T) > L.slab_group_words ||
                                   (q.rows > rc && 4 * (int64_t)min(q.W, rc + (q.b - q.a)) > L.boundary_group_ints));
        if (q.score > 0 && over) {
            // the launch was sized from the class maxima; never overrun a slab
            // or a boundary row
            atomicOr(L.status, ST_INTERNAL);
            q.score = 0;
            q.rows = 0;
        }
        const int32_t rows_w = __reduce_max_sync(FULLMASK, (unsigned)(q.score > 0 ? q.rows : 0));
        const int chunks = (rows_w + rc - 1) / rc;
        const int wcap = q.score > 0 ? min(q.W, rc - 1 + (q.b - q.a) + 1) : 0;
        int64_t slab_off = 0;  // words before chunk c in this group's slab

        int prev_lo = 0, prev_hi = -1;
        for (int c = 0; c < chunks; ++c) {
            int lo = 0, hi = -1;
            if (q.score > 0 && c * rc < q.rows) chunk_window(q, c, rc, lo, hi);
            const int width = hi - lo + 1;
            const int steps = __reduce_max_sync(FULLMASK, (unsigned)max(width, 0)) + T - 1;
            const int i0 = c * rc + k * TB_ROWS;
            // per-row selectors into the column table (sign-extended byte);
            // rows past the end row are never read by the walk
            uint32_t sel[TB_ROWS];
            {
                uint32_t codes = 0x44444444u;  // 4 bits per row, 4 = no base
                const int cnt = min(TB_ROWS, q.rows - i0);
                if (q.score > 0 && cnt > 0) {
                    const uint32_t w = load_bases(P.ps.reads, q.rs + i0, cnt);
#pragma unroll
                    for (int r = 0; r < TB_ROWS; ++r)
                        if (r < cnt) codes = (codes & ~(0xFu << (4 * r))) | (((w >> (2 * r)) & 3u) << (4 * r));
                }
#pragma unroll
                for (int r = 0; r < TB_ROWS; ++r) {
                    const uint32_t x = (codes >> (4 * r)) & 0xFu;
                    sel[r] = x < 4u ? x * 0x1111u + 0x8880u : 0x8888u;
                }
            }
            // per row: E - o and H of the previous column.  E - o is floored
            // at 0: since H >= 0 the floor never changes max(H + o, E + e) or
            // which of the two is larger, so E, F and the open bits the walk
            // reads are exact.
            int32_t E[TB_ROWS], Hp[TB_ROWS];
#pragma unroll
            for (int r = 0; r < TB_ROWS; ++r) {
                E[r] = 0;
                Hp[r] = 0;
            }
            // boundary rows are indexed relative to the writing chunk's window
            const int32_t *bin = (bnd && c > 0) ? bnd + (c & 1) * bnd_half : nullptr;
            int32_t *bout = (bnd && c + 1 < chunks) ? bnd + ((c + 1) & 1) * bnd_half : nullptr;
            // diagonal into the chunk's first column: the previous chunk's
            // bottom row one column to the left, if it computed it
            int32_t diag_in = 0;
            // boundary element (column x of the writing chunk, value v)
            auto bidx = [&](int x, int v) -> int64_t { return TILED ? ((int64_t)x * 2 + v) * 32 + lane : 2 * x + v; };
            if (k == 0 && bin && lo - 1 >= prev_lo && lo - 1 <= prev_hi) diag_in = bin[bidx(lo - 1 - prev_lo, 0)];
            int32_t out_h = 0, out_f = 0;
            // the first lane reads the row above from the previous chunk two
            // columns ahead, so the loads are in flight while columns compute
            int32_t nb_h = 0, nb_f = 0, nc_h = 0, nc_f = 0;
            if (k == 0 && bin) {
                if (lo >= prev_lo && lo <= prev_hi) {
                    nb_h = bin[bidx(lo - prev_lo, 0)];
                    nb_f = bin[bidx(lo - prev_lo, 1)];
                }
                if (lo + 1 >= prev_lo && lo + 1 <= prev_hi) {
                    nc_h = bin[bidx(lo + 1 - prev_lo, 0)];
                    nc_f = bin[bidx(lo + 1 - prev_lo, 1)];
                }
            }
            // window bases: ww holds the current word's remaining bases, wn the
            // next 16-base word (requested 16 columns before it is needed)
            const int64_t abs_lo = q.ws + q.jlo + lo, abs_hi = q.ws + q.jlo + hi;
            uint32_t ww = 0, wn = 0;
            int64_t apos = abs_lo;
            if (width > 0) {
                const int64_t a1 = (abs_lo & ~(int64_t)15) + 16;
                ww = load_bases(P.ps.wins, abs_lo, (int)lmin(a1 - abs_lo, abs_hi - abs_lo + 1));
                wn = a1 <= abs_hi ? load_bases(P.ps.wins, a1, (int)lmin(16, abs_hi - a1 + 1)) : 0u;
            }

            for (int t = 0; t < steps; ++t) {
                const int jl = t - k;       // column within the window
                const int jj = lo + jl;     // rectangle column
                int32_t up_h = __shfl_up_sync(FULLMASK, out_h, 1);
                int32_t up_f = __shfl_up_sync(FULLMASK, out_f, 1);
                if (k == 0) {
                    up_h = nb_h;
                    up_f = nb_f;
                    nb_h = nc_h;
                    nb_f = nc_f;
                    const int nx = jj + 2;
                    if (bin && nx >= prev_lo && nx <= prev_hi) {
                        nc_h = bin[bidx(nx - prev_lo, 0)];
                        nc_f = bin[bidx(nx - prev_lo, 1)];
                    } else {
                        nc_h = 0;
                        nc_f = 0;
                    }
                }
                if (jl >= 0 && jl < width) {
                    const uint32_t tw = s_tab[ww & 3u];
                    ww >>= 2;
                    if (((++apos) & 15) == 0) {
                        ww = wn;
                        const int64_t a2 = apos + 16;
                        wn = a2 <= abs_hi ? load_bases(P.ps.wins, a2, (int)lmin(16, abs_hi - a2 + 1)) : 0u;
                    }
                    int32_t d0 = diag_in, hu = up_h, f = up_f;
                    uint32_t word = 0;
#pragma unroll
                    for (int r = 0; r < TB_ROWS; ++r) {
                        const int32_t sp = (int32_t)prmt(tw, 0u, sel[r]);  // s - o
                        const int32_t eext = E[r] + ge;
                        const int32_t e = max(Hp[r], eext);
                        const int32_t fext = f + ge;
                        f = max(hu, fext);
                        const int32_t d = d0 + sp;
                        const int32_t u = __vimax3_s32(d, e, f);
                        const int32_t h = max(u + go, 0);
                        uint32_t code = h == 0 ? 0u : (u == d ? 1u : (u == e ? 2u : 3u));
                        code |= (Hp[r] >= eext ? 4u : 0u) | (hu >= fext ? 8u : 0u);
                        word |= code << (4 * r);
                        d0 = Hp[r];
                        Hp[r] = h;
                        E[r] = e;
                        hu = h;
                    }
                    if (TILED) slab[((int64_t)c * WCAP + jl) * 32 + lane] = word;
                    else slab[slab_off + (int64_t)jl * T + k] = word;
                    out_h = hu;
                    out_f = f;
                    if (bout && k == T - 1) {
                        bout[bidx(jl, 0)] = out_h;
                        bout[bidx(jl, 1)] = out_f;
                    }
                }
                diag_in = up_h;
            }
            slab_off += (int64_t)max(width, 0) * T;
            prev_lo = lo;
            prev_hi = hi;
            __syncwarp();
        }

        // walk back from the end cell (the group's first lane)
        if (on && k == 0 && p >= 0) {
            const int64_t off = P.cig_off[p];
            const int64_t cap = P.cig_off[p + 1] - off;
            if (q.score <= 0) {
                P.cig_n[p] = 0;
            } else {
                RevCigar rcg{P.cig_ops + off, cap, 0, 0u, 0, false};
                rcg.push(4u, q.m - 1 - q.ie);  // trailing soft clip
                int32_t i = q.ie, jj = q.W - 1;
                int state = 0;
                const int64_t limit = (int64_t)q.rows + q.W + 4;
                // words of chunk cc start after the windows of chunks 0..cc-1
                int cc = i / rc, clo, chi;
                int64_t cbase = 0;
                for (int c2 = 0; c2 < cc; ++c2) {
                    int l2, h2;
                    chunk_window(q, c2, rc, l2, h2);
                    cbase += (int64_t)max(h2 - l2 + 1, 0) * T;
                }
                chunk_window(q, cc, rc, clo, chi);
                bool ok = false;
                for (int64_t it = 0; it < limit; ++it) {
                    if (i < 0 || jj < 0) {
                        ok = state == 0;
                        break;
                    }
                    while (i < cc * rc) {  // moved up into the previous chunk
                        --cc;
                        chunk_window(q, cc, rc, clo, chi);
                        cbase -= (int64_t)max(chi - clo + 1, 0) * T;
                    }
                    if (jj < clo || jj > chi) break;  // left the band: inconsistent
                    const int kk = (i - cc * rc) / TB_ROWS, nib = i % TB_ROWS;
                    const int64_t widx = TILED ? ((int64_t)cc * WCAP + (jj - clo)) * 32 + lane
                                               : cbase + (int64_t)(jj - clo) * T + kk;
                    const uint32_t code = (slab[widx] >> (4 * nib)) & 0xFu;
                    if (state == 0) {
                        const uint32_t src = code & 3u;
                        if (src == 0u) {
                            ok = true;
                            break;
                        }
                        if (src == 1u) {
                            rcg.push(0u, 1);
                            --i;
                            --jj;
                        } else {
                            state = src == 2u ? 1 : 2;
                        }
                    } else if (state == 1) {
                        rcg.push(2u, 1);
                        if (code & 4u) state = 0;
                        --jj;
                    } else {
                        rcg.push(1u, 1);
                        if (code & 8u) state = 0;
                        --i;
                    }
                }
                if (!ok) atomicOr(L.status, ST_INTERNAL);
                rcg.push(4u, i + 1);  // leading soft clip
                rcg.flush();
                if (rcg.overflow) {
                    P.cig_n[p] = -1;
                    atomicOr(L.status, ST_CAPACITY);
                } else {
                    uint32_t *o = P.cig_ops + off;
                    for (int32_t a2 = 0, b2 = rcg.n - 1; a2 < b2; ++a2, --b2) {
                        const uint32_t tmp = o[a2];
                        o[a2] = o[b2];
                        o[b2] = tmp;
                    }
                    P.cig_n[p] = rcg.n;
                }
            }
        }
        __syncwarp();
    }
}

int launch_tb_keys(const TbParams &P, const int32_t *order, int64_t n_items, const int32_t *score_keys,
                   int32_t *tb_keys, int32_t *hist, TbClassInfo *info, cudaStream_t st)
{
    const int threads = 256;
    int64_t blocks = (n_items + threads - 1) / threads;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    k_tb_keys<<<(unsigned)blocks, threads, 0, st>>>(P, order, n_items, score_keys, tb_keys, hist, info);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? SW_OK : SW_ERR_CUDA;
}

int launch_traceback(const TracebackLaunch &L, int blocks, int threads, cudaStream_t st)
{
    if (L.tiled) k_traceback<true><<<blocks, threads, 0, st>>>(L);
    else k_traceback<false><<<blocks, threads, 0, st>>>(L);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? SW_OK : SW_ERR_CUDA;
}

int traceback_kernel_occupancy(int *max_blocks_per_sm, int threads)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(max_blocks_per_sm, k_traceback<false>, threads, 0) ==
                   cudaSuccess
               ? SW_OK
               : SW_ERR_CUDA;
}

}  // namespace swgb
