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
// Scheduling.  The score pass's epilogue gives every pair a cost key (rows x
// window), a counting sort orders each length class by cost so a warp's
// groups sweep similar windows, and pairs whose slab exceeds the small slab
// of the main part form a part of their own with larger slabs.  A device
// planner (sw_devplan.cu) sizes every part and assigns it to one of the
// persistent launches below; each warp of a launch owns one scratch slot,
// sized for the largest part of its launch.
#include <algorithm>

#include "sw_band.cuh"
#include "sw_device.cuh"
#include "swgb_internal.h"

namespace swgb {

constexpr unsigned FULLMASK = 0xffffffffu;

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
    const Band bd = band_of(q.score, q.ie, q.je, P.sc);
    q.jlo = bd.jlo;
    q.W = bd.W;
    q.rows = bd.rows;
    q.a = bd.a;
    q.b = bd.b;
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
    const int64_t warp_global = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int32_t go = P.sc.go, ge = P.sc.ge;
    const DevTbPlan &dp = *L.dp;
    const int v = L.variant;
    // warps without a scratch slot, and input already found invalid
    if (warp_global >= dp.var_warps[v]) return;
    // (an unsupported size means some pairs were not scored, so the
    // traceback order is incomplete: do nothing)
    if (*(volatile const int32_t *)L.status & (ST_BAD_INPUT | ST_UNSUPPORTED)) return;
    uint32_t *const slot = L.slab + dp.var_slot_offset[v] + warp_global * dp.var_slot_words[v];

    for (int pi = 0; pi < dp.var_n[v]; ++pi) {
    const TbPartPlan &tp = dp.part[dp.var_part[v][pi]];
    const int T = tp.lanes;
    const int G = 32 / T;
    const int g = lane / T;
    const int k = lane - g * T;
    const bool on = g < G;
    const int rc = T * TB_ROWS;
    const int WCAP = tp.wcap;
    const int64_t slab_words = tp.slab_words, bnd_ints = tp.bnd_ints;
    const int32_t *const order = L.order + tp.start;
    const int64_t n_items = tp.count;
    int32_t *const counter = L.work_counter + 2 * tp.cls + tp.part;
    // the warp's slot: TILED -> one tile indexed with the lane, then the
    // boundary rows; else every group's slab, then every group's boundary row
    uint32_t *slab = !on ? nullptr : TILED ? slot : slot + g * slab_words;
    int32_t *bnd = !on ? nullptr
                       : TILED ? (int32_t *)(slot + 32 * slab_words)
                               : (int32_t *)(slot + G * slab_words + g * bnd_ints);
    const int64_t bnd_half = TILED ? 32 * (bnd_ints / 2) : bnd_ints / 2;

    for (;;) {
        int base = 0;
        if (lane == 0) base = atomicAdd(counter, G);
        base = __shfl_sync(FULLMASK, base, 0);
        if (base >= n_items) break;
        const int64_t item = base + g;
        const int32_t p = (on && item < n_items) ? order[item] : -1;
        TbPair q = tb_pair(P, p, L.status);
        const bool over = TILED ? (q.rows > (slab_words / max(WCAP, 1)) * rc ||
                                   min(q.W, rc + (q.b - q.a)) > WCAP)
                                : (slab_need(q, T) > slab_words ||
                                   (q.rows > rc && 4 * (int64_t)min(q.W, rc + (q.b - q.a)) > bnd_ints));
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
                // every step moves, or switches into a gap state before moving
                const int64_t limit = 2 * ((int64_t)q.rows + q.W) + 4;
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
    }  // parts
}

// ---------------------------------------------------------------------------
// 16x2 traceback.  One lane owns two pairs, A in the low and B in the high
// half of every register, so each DPX instruction recomputes two cells.  It
// serves the classes whose score bound keeps every value below 32768
// (match x min(m, n) <= 32000, match - o <= 127).  A lane stores two 32-bit
// words per window offset (rows 0-3 and rows 4-7; pair A in bits 0-15, pair
// B in bits 16-31), and its words of four consecutive offsets share one
// 32-byte sector: uint2 [((chunk x WCAP4 + t / 4) x 32 + lane) x 4 + t % 4].
// The warp's stores fill each sector over four steps, and a walk moving
// left along a chunk reads one sector per four offsets.
//
// Per cell four bits record which equalities fail (1 = not equal):
//   bit 0  H != H(i-1,j-1) + s    bit 1  H != E
//   bit 2  E != H(i,j-1) + o      bit 3  F != H(i-1,j) + o
// so the walk takes the diagonal where bit 0 is clear, else E where bit 1
// is clear, else F, and a gap run opens where bit 2 (3) is clear -- the same
// preferences as the int32 kernel.  Whether H is 0 is not stored: the walk
// carries the exact value of its current state, starting from the score,
// and stops where H reaches 0.
//
// Each bit is min(x, 1) per half of a difference x that is non-negative in
// both halves (a maximum minus one of its operands), so the differences and
// the packing of the bits are integer multiply-adds on the FMA pipe, next to
// the DPX maxima on the ALU pipe: per two cells 9 ALU and 9 FMA-pipe
// instructions when s - o >= 0 for every substitution (FMA_ADD), else the
// diagonal add and its difference move to the ALU pipe.
//
// Each pair keeps its own chunk windows (the clamped band boxes); both pairs
// of a lane step through window offset t together and the warp steps to its
// widest window.  Offsets past a pair's own window are computed as well:
// they lie right of its box and hold values no larger than the full
// matrix's (past the window end they see an all-(s = o) table, so nothing
// grows there), which changes no cell the walk reads.  Boundary rows hold
// (H | F << 16) per pair and offset, read by the next chunk at its own shift.
//
// A warp sweeps one task (2G pairs) into the tile of its scratch slot and
// then walks the task's pairs, one thread per pair, while the other warps of
// the SM keep sweeping: the walk is a chain of dependent loads, mostly from
// the L2 the sweep just wrote to.

__device__ __forceinline__ uint32_t mad_u32(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

__device__ __forceinline__ uint32_t min_u16x2(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

__device__ __forceinline__ uint32_t splat16(int32_t x) { return ((uint32_t)(uint16_t)(int16_t)x) * 0x10001u; }

// Streams the window bases of one pair, one column per call; past the
// window end it yields table index 4 (all s = o).
struct WinStream {
    uint32_t ww, wn;
    int64_t apos, aend;
    __device__ void start(const uint32_t *__restrict__ wins, int64_t a0, int64_t end)
    {
        apos = a0;
        aend = end;
        ww = wn = 0;
        if (a0 < end) {
            const int64_t a1 = (a0 & ~(int64_t)15) + 16;
            ww = load_bases(wins, a0, (int)lmin(a1 - a0, end - a0));
            wn = a1 < end ? load_bases(wins, a1, (int)lmin(16, end - a1)) : 0u;
        }
    }
    __device__ __forceinline__ uint32_t next(const uint32_t *__restrict__ wins)
    {
        const uint32_t idx = apos < aend ? (ww & 3u) : 4u;
        ww >>= 2;
        if (((++apos) & 15) == 0) {
            ww = wn;
            const int64_t a2 = apos + 16;
            wn = a2 < aend ? load_bases(wins, a2, (int)lmin(16, aend - a2)) : 0u;
        }
        return idx;
    }
};

// Selector nibbles of one row for pair A (bytes 0-1) and pair B (bytes 2-3):
// the row's base picks its byte of the column table and the high byte
// replicates its sign; a row without a base takes the sign of byte 0 (0 or
// -1, never above s = o).
__device__ __forceinline__ uint32_t sel16(uint32_t xa, uint32_t xb)
{
    const uint32_t a = xa < 4u ? (xa | ((8u | xa) << 4)) : 0x88u;
    const uint32_t b = xb < 4u ? ((4u + xb) | ((12u + xb) << 4)) : 0xCCu;
    return a | (b << 8);
}

// Tile geometry of a 16-bit traceback launch: T lanes per group (two pairs),
// G = 32 / T groups and 2G pairs per task.  Word (chunk c, step t, lane)
// of a task's tile: uint2 [((c * S4 + t / 4) * 32 + lane) * 4 + t % 4],
// S4 = ceil((WCAP + T - 1) / 4) groups of four steps per chunk; lane k of a
// group computes window offset t - k at step t.
__device__ __forceinline__ int64_t tb16_word(int c, int t, int lane, int S4)
{
    return ((((int64_t)c * S4 + (t >> 2)) * 32 + lane) << 2) + (t & 3);
}

// Collects a CIGAR as the walk emits it (its last run first) and writes it
// forward into the pair's slot.  The first LB runs emitted -- the whole CIGAR
// in the common case -- stay in a per-thread buffer and are stored at the
// end; runs past those are parked at the end of the slot and moved down in
// batches of loads before stores.  No run is read back from global memory
// unless the CIGAR has more than LB runs.
struct FwdCigar {
    static constexpr int LB = 16;
    uint32_t *out;
    int64_t cap;
    int32_t n;
    uint32_t op;
    int32_t len;
    bool overflow;
    uint32_t buf[LB];
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
            const uint32_t run = ((uint32_t)len << 4) | op;
            if (n >= cap) overflow = true;
            else if (n < LB) buf[n] = run;
            else out[cap - 1 - (n - LB)] = run;
            ++n;
        }
        len = 0;
    }
    // run e (in emission order) goes to position n - 1 - e
    __device__ void finish()
    {
        if (overflow) return;
        const int32_t parked = n - LB;
        if (parked > 0) {
            const int64_t src = cap - n + LB;  // > 0: every source lies above its target
            for (int32_t k = 0; k < parked; k += 4) {
                uint32_t v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (k + u < parked) v[u] = out[src + k + u];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (k + u < parked) out[k + u] = v[u];
            }
        }
        const int32_t nb = n < LB ? n : LB;
        for (int32_t e = 0; e < nb; ++e) out[n - 1 - e] = buf[e];
    }
};

// Walk back from a pair's end cell through the tile of its task (group g,
// 16-bit half `half`), carrying the exact value of the current state (the
// tile does not record where H is 0), and write its CIGAR.  A walk keeps the
// sector of four steps it read last, and the 16-base words of read and
// window that hold its current row and column.  SAME_KERNEL: the tile was
// written by this warp in this launch (ordered by __syncwarp) and is read
// through L2 (ld.global.cg), since the slot is reused by the warp's next
// task; else it was written by an earlier launch and is read through the
// read-only cache, where walks of neighbouring groups share 128-byte lines.
// The walk's CIGAR writer is a separate object (its run buffer is indexed,
// so it lives in local memory, while the walk's own state stays in
// registers).
template <int T, bool SAME_KERNEL>
struct Walk16 {
    const uint2 *tile;
    TbPair qq;
    int32_t p, i, jj, v;
    int g, hs, S4, state, cc, clo, chi;
    int64_t gkey, rkey, wkey, it, limit;
    uint4 ga, gb;
    uint32_t rw, ww;
    bool ok;

    // false when there is nothing to walk (no alignment: 0 runs written)
    __device__ __forceinline__ bool begin(const TbParams &P, FwdCigar &cg, const uint2 *__restrict__ tile_,
                                          int32_t p_, int g_, int half, int WCAP, int64_t lane_chunks)
    {
        constexpr int rc = T * TB_ROWS;
        tile = tile_;
        p = p_;
        g = g_;
        hs = 16 * half;
        S4 = (WCAP + T - 1 + 3) >> 2;
        qq = tb_pair(P, p, nullptr);
        // the sweep skipped (and reported) pairs that overrun the tile
        if ((qq.rows + rc - 1) / rc > lane_chunks || min(qq.W, rc + (qq.b - qq.a)) > WCAP) qq.score = 0;
        if (qq.score <= 0) {
            P.cig_n[p] = 0;
            return false;
        }
        const int64_t off = P.cig_off[p];
        cg.out = P.cig_ops + off;
        cg.cap = P.cig_off[p + 1] - off;
        cg.n = 0;
        cg.op = 0u;
        cg.len = 0;
        cg.overflow = false;
        cg.push(4u, qq.m - 1 - qq.ie);  // trailing soft clip
        i = qq.ie;
        jj = qq.W - 1;
        v = qq.score;  // value of the current state at (i, jj)
        state = 0;
        cc = i / rc;
        chunk_window(qq, cc, rc, clo, chi);
        gkey = rkey = wkey = -1;
        ga = gb = make_uint4(0u, 0u, 0u, 0u);
        rw = ww = 0u;
        ok = false;
        // every step moves, or switches into a gap state before moving
        limit = 2 * ((int64_t)qq.rows + qq.W) + 4;
        it = 0;
        return true;
    }

    // one step; false when the walk is over (done, or inconsistent)
    __device__ __forceinline__ bool step(const TbParams &P, FwdCigar &cg)
    {
        constexpr int rc = T * TB_ROWS;
        if (it++ >= limit) return false;
        if (state == 0 && v == 0) {
            ok = true;
            return false;
        }
        if (i < 0 || jj < 0 || v < 0) return false;
        if (i < cc * rc) {
            cc = i / rc;
            chunk_window(qq, cc, rc, clo, chi);
        }
        if (jj < clo || jj > chi) return false;  // left the band: inconsistent
        const int kk = (i - cc * rc) >> 3, r = i & 7;
        const int t = (jj - clo) + kk;
        const int64_t sector = ((int64_t)cc * S4 + (t >> 2)) * 32 + g * T + kk;
        if (sector != gkey) {
            const uint4 *src = reinterpret_cast<const uint4 *>(tile + (sector << 2));
            if (SAME_KERNEL) {  // written by this warp in this launch: through L2
                ga = __ldcg(src);
                gb = __ldcg(src + 1);
            } else {            // written by an earlier launch: the read-only path
                ga = __ldg(src);
                gb = __ldg(src + 1);
            }
            gkey = sector;
        }
        const int sl = t & 3;
        const uint32_t wlo = sl == 0 ? ga.x : sl == 1 ? ga.z : sl == 2 ? gb.x : gb.z;
        const uint32_t whi = sl == 0 ? ga.y : sl == 1 ? ga.w : sl == 2 ? gb.y : gb.w;
        const uint32_t code = ((r < 4 ? wlo : whi) >> (hs + 4 * (r & 3))) & 0xFu;
        if (state == 0) {
            if (!(code & 1u)) {
                // diagonal: H(i-1, j-1) = H(i, j) - s(r_i, w_j)
                const int64_t rpos = qq.rs + i, wpos = qq.ws + qq.jlo + jj;
                if ((rpos >> 4) != rkey) {
                    rkey = rpos >> 4;
                    rw = __ldg(P.ps.reads + rkey);
                }
                if ((wpos >> 4) != wkey) {
                    wkey = wpos >> 4;
                    ww = __ldg(P.ps.wins + wkey);
                }
                const uint32_t ri = (rw >> (2 * (rpos & 15))) & 3u;
                const uint32_t wj = (ww >> (2 * (wpos & 15))) & 3u;
                v -= ri == wj ? P.sc.ma : P.sc.mi;
                cg.push(0u, 1);
                --i;
                --jj;
            } else {
                state = (code & 2u) ? 2 : 1;
            }
        } else if (state == 1) {
            cg.push(2u, 1);
            if (!(code & 4u)) {
                v -= P.sc.go;  // E(i,j) = H(i,j-1) + o
                state = 0;
            } else {
                v -= P.sc.ge;  // E(i,j) = E(i,j-1) + e
            }
            --jj;
        } else {
            cg.push(1u, 1);
            if (!(code & 8u)) {
                v -= P.sc.go;  // F(i,j) = H(i-1,j) + o
                state = 0;
            } else {
                v -= P.sc.ge;
            }
            --i;
        }
        return true;
    }

    __device__ __forceinline__ void end(const TbParams &P, FwdCigar &cg, int32_t *status)
    {
        if (!ok) atomicOr(status, ST_INTERNAL);
        cg.push(4u, i + 1);  // leading soft clip
        cg.flush();
        if (cg.overflow) {
            P.cig_n[p] = -1;
            atomicOr(status, ST_CAPACITY);
        } else {
            cg.finish();
            P.cig_n[p] = cg.n;
        }
    }
};

template <int T, bool FMA_ADD>
__global__ void __launch_bounds__(128, 4) k_traceback16(const TracebackLaunch L)
{
    constexpr int G = 32 / T;       // groups per warp, two pairs each
    constexpr int PAIRS = 2 * G;    // pairs per task
    const TbParams &P = L.P;
    // s_tab[w] byte x = s(x, w) - o; s_tab[4] = 0 (s = o, past a window end)
    __shared__ uint32_t s_tab[8];
    {
        const uint32_t mis4 = ((uint32_t)(uint8_t)(int8_t)(P.sc.mi - P.sc.go)) * 0x01010101u;
        const uint32_t ma4 = ((uint32_t)(uint8_t)(int8_t)(P.sc.ma - P.sc.go)) * 0x01010101u;
        if (threadIdx.x < 4) s_tab[threadIdx.x] = prmt(mis4, ma4, 0x3210u + (4u << (4u * threadIdx.x)));
        else if (threadIdx.x < 8) s_tab[threadIdx.x] = 0u;
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    const int g = lane / T, k = lane % T;
    const int64_t warp_global = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const DevTbPlan &dp = *L.dp;
    const int v = L.variant;
    // input already found invalid (an unsupported size means some pairs were
    // not scored, so the traceback order is incomplete): do nothing
    if (*(volatile const int32_t *)L.status & (ST_BAD_INPUT | ST_UNSUPPORTED)) return;
    // the warp's boundary row, and its full slot for tasks it also walks
    if (warp_global >= dp.var_run_warps[v]) return;
    uint32_t *const bnd = L.slab + warp_global * dp.var_bnd_words[v];
    const bool has_slot = warp_global < dp.var_warps[v];
    uint2 *const own = (uint2 *)(L.slab + dp.var_slot_offset[v] + warp_global * dp.var_slot_words[v]);
    const int32_t go = P.sc.go, ge = P.sc.ge;
    const uint32_t GE2 = splat16(ge), GO2 = splat16(go);
    const uint32_t one = (uint32_t)L.one;
    const uint32_t m1 = 0u - one, two = one + one, four = two + two, eight = four + four;
    const uint32_t mul1 = eight + eight, mul2 = mul1 * mul1, mul3 = mul2 * mul1;  // 16, 256, 4096
    const uint32_t ONES = 0x00010001u;

    constexpr int rc = T * TB_ROWS;
    // The part's and phase's values live in shared memory, one record per
    // warp, read where they are used (held in registers across the sweep
    // they would crowd out the sweep's own).
    struct PartCtx {
        const int32_t *order;
        int32_t *ctr;        // the phase's work counter
        uint32_t *pool;      // the part's first pooled tile
        int64_t n_items, lo, hi, tile_words, lane_chunks;
        int32_t wcap, s4, pi, phase;
    };
    __shared__ PartCtx s_pc[4];  // 128 threads: 4 warps
    volatile PartCtx *const pc = &s_pc[threadIdx.x >> 5];
    if (lane == 0) pc->pi = 0;
    __syncwarp();
    for (; pc->pi < dp.var_n[v]; __syncwarp(), pc->pi = pc->pi + (lane == 0 ? 1 : 0), __syncwarp()) {
    // tasks 0 .. pool_tasks-1 keep their tiles (32 lanes x slab words) in the
    // pool for k_tb16_walk; the rest are swept into the warp's own slot and
    // walked at once.  The boundary row is updated in place: (H | F << 16) of
    // pair x at offset j in word (j * G + g) * 2 + x.
    if (lane == 0) {
        const TbPartPlan &tp = dp.part[dp.var_part[v][pc->pi]];
        const int32_t s4 = (tp.wcap + T - 1 + 3) >> 2;
        pc->order = L.order + tp.start;
        pc->pool = L.slab + tp.pool_offset;
        pc->n_items = tp.count;
        pc->tile_words = (32 * tp.slab_words + 63) & ~(int64_t)63;
        pc->lane_chunks = tp.slab_words / (8 * (int64_t)max(s4, 1));
        pc->wcap = tp.wcap;
        pc->s4 = s4;
        pc->phase = 0;
    }
    __syncwarp();

    for (; pc->phase < 2; __syncwarp(), pc->phase = pc->phase + (lane == 0 ? 1 : 0), __syncwarp()) {
    if (pc->phase == 1 && !has_slot) break;
    if (lane == 0) {
        const TbPartPlan &tp = dp.part[dp.var_part[v][pc->pi]];
        const int64_t n_pool = min((int64_t)tp.count, (int64_t)tp.pool_tasks * PAIRS);
        const bool ph = pc->phase != 0;
        pc->ctr = L.work_counter + (ph ? CTR_TB_OWN - CTR_TB : 0) + 2 * tp.cls + tp.part;
        pc->lo = ph ? n_pool : 0;
        pc->hi = ph ? (int64_t)tp.count : n_pool;
    }
    __syncwarp();
    const bool own_task = pc->phase != 0;
    for (;;) {
        int bb = 0;
        if (lane == 0) bb = atomicAdd(pc->ctr, PAIRS);
        bb = __shfl_sync(FULLMASK, bb, 0);
        const int64_t base = pc->lo + bb;
        if (base >= pc->hi) break;
        uint2 *const slab = own_task ? own : (uint2 *)(pc->pool + (int64_t)(bb / PAIRS) * pc->tile_words);
        const int WCAP = pc->wcap;
        const int64_t lane_chunks = pc->lane_chunks;
        TbPair q[2];
#pragma unroll
        for (int x = 0; x < 2; ++x) {
            const int64_t item = base + 2 * g + x;
            const int32_t p = item < pc->n_items ? pc->order[item] : -1;
            q[x] = tb_pair(P, p, k == 0 ? L.status : nullptr);
            const bool over = (q[x].rows + rc - 1) / rc > lane_chunks || min(q[x].W, rc + (q[x].b - q[x].a)) > WCAP;
            if (q[x].score > 0 && over) {
                // the launch was sized from the class maxima; never overrun
                if (k == 0) atomicOr(L.status, ST_INTERNAL);
                q[x].score = 0;
                q[x].rows = 0;
            }
        }
        const int32_t rows_l = max(q[0].score > 0 ? q[0].rows : 0, q[1].score > 0 ? q[1].rows : 0);
        const int32_t rows_w = __reduce_max_sync(FULLMASK, (unsigned)rows_l);
        const int chunks = (rows_w + rc - 1) / rc;

        int prev_lo[2] = {0, 0};
        int prev_width = 0;  // offsets the previous chunk's last lanes wrote
        for (int c = 0; c < chunks; ++c) {
            int lo[2], hi[2];
#pragma unroll
            for (int x = 0; x < 2; ++x) {
                lo[x] = 0;
                hi[x] = -1;
                if (q[x].score > 0 && c * rc < q[x].rows) chunk_window(q[x], c, rc, lo[x], hi[x]);
            }
            const int width = __reduce_max_sync(FULLMASK, (unsigned)max(max(hi[0] - lo[0] + 1, hi[1] - lo[1] + 1), 0));
            const int steps = width + T - 1;
            const int i0 = c * rc + k * TB_ROWS;
            uint32_t sel[TB_ROWS];
            {
                uint32_t codes[2];
#pragma unroll
                for (int x = 0; x < 2; ++x) {
                    codes[x] = 0x44444444u;  // 4 bits per row, 4 = no base
                    const int cnt = min(TB_ROWS, q[x].rows - i0);
                    if (q[x].score > 0 && cnt > 0) {
                        const uint32_t w = load_bases(P.ps.reads, q[x].rs + i0, cnt);
#pragma unroll
                        for (int r = 0; r < TB_ROWS; ++r)
                            if (r < cnt) codes[x] = (codes[x] & ~(0xFu << (4 * r))) | (((w >> (2 * r)) & 3u) << (4 * r));
                    }
                }
#pragma unroll
                for (int r = 0; r < TB_ROWS; ++r) sel[r] = sel16((codes[0] >> (4 * r)) & 0xFu, (codes[1] >> (4 * r)) & 0xFu);
            }
            uint32_t E[TB_ROWS], Hp[TB_ROWS];
#pragma unroll
            for (int r = 0; r < TB_ROWS; ++r) {
                E[r] = 0u;
                Hp[r] = 0u;
            }
            // one boundary row, updated in place: the first lane reads offset
            // j (two steps ahead, at j + shift, shift >= 0) at step j - 2, the
            // last lane overwrites it at step j + T - 1
            const uint32_t *bin = (c > 0 && k == 0) ? bnd : nullptr;
            uint32_t *bout = (c + 1 < chunks && k == T - 1) ? bnd : nullptr;
            // a pair's window moves right by shift >= 0 from chunk to chunk; a
            // pair without rows in this chunk reads the row at shift 0 (its
            // values are never used)
            int shift[2];
#pragma unroll
            for (int x = 0; x < 2; ++x) shift[x] = hi[x] >= lo[x] ? max(lo[x] - prev_lo[x], 0) : 0;
            auto bload = [&](int x, int j) -> uint32_t {
                return (bin && j >= 0 && j < prev_width) ? bin[((int64_t)j * G + g) * 2 + x] : 0u;
            };
            // the row above, two offsets ahead: packed (H | F << 16) per pair
            uint32_t nb[2], nc[2], dg[2];
#pragma unroll
            for (int x = 0; x < 2; ++x) {
                dg[x] = bload(x, shift[x] - 1);
                nb[x] = bload(x, shift[x]);
                nc[x] = bload(x, shift[x] + 1);
            }
            uint32_t diag_in = prmt(dg[0], dg[1], 0x5410u);
            WinStream ws[2];
#pragma unroll
            for (int x = 0; x < 2; ++x) {
                const int64_t a0 = q[x].ws + q[x].jlo + lo[x];
                ws[x].start(P.ps.wins, a0, q[x].score > 0 ? q[x].ws + q[x].n : a0);
            }
            uint32_t out_h = 0u, out_f = 0u;
            int64_t widx = tb16_word(c, 0, lane, pc->s4);   // tile word of step t
            int64_t bidx = ((int64_t)(0 - k) * G + g) * 2;  // boundary word of offset t - k

            for (int t = 0; t < steps; ++t) {
                // the row above: from the lane before (its last step), or the
                // previous chunk's boundary row for the group's first lane
                uint32_t up_h = T > 1 ? __shfl_up_sync(FULLMASK, out_h, 1) : 0u;
                uint32_t up_f = T > 1 ? __shfl_up_sync(FULLMASK, out_f, 1) : 0u;
                if (k == 0) {
                    up_h = prmt(nb[0], nb[1], 0x5410u);
                    up_f = prmt(nb[0], nb[1], 0x7632u);
#pragma unroll
                    for (int x = 0; x < 2; ++x) {
                        nb[x] = nc[x];
                        nc[x] = bload(x, t + 2 + shift[x]);
                    }
                }
                const int jl = t - k;  // this lane's window offset
                if (jl >= 0) {
                    const uint32_t tA = s_tab[ws[0].next(P.ps.wins)];
                    const uint32_t tB = s_tab[ws[1].next(P.ps.wins)];
                    uint32_t d0 = diag_in, hu = up_h, f = up_f;
                    uint32_t w0 = 0u, w1 = 0u;
#pragma unroll
                    for (int r = 0; r < TB_ROWS; ++r) {
                        const uint32_t sp = prmt(tA, tB, sel[r]);  // s - o, both pairs
                        const uint32_t e = __viaddmax_s16x2(E[r], GE2, Hp[r]);
                        f = __viaddmax_s16x2(f, GE2, hu);
                        const uint32_t d = FMA_ADD ? mad_u32(d0, one, sp) : __viaddmax_s16x2(d0, sp, 0x80008000u);
                        const uint32_t u = __vimax3_s16x2(d, e, f);
                        const uint32_t h = __viaddmax_s16x2_relu(u, GO2, 0u);
                        const uint32_t nd = FMA_ADD ? min_u16x2(mad_u32(d, m1, u), ONES) : min_u16x2(u ^ d, ONES);
                        const uint32_t ne = min_u16x2(mad_u32(e, m1, u), ONES);
                        const uint32_t nE = min_u16x2(mad_u32(Hp[r], m1, e), ONES);
                        const uint32_t nF = min_u16x2(mad_u32(hu, m1, f), ONES);
                        uint32_t code = mad_u32(ne, two, nd);
                        code = mad_u32(nE, four, code);
                        code = mad_u32(nF, eight, code);
                        if (r == 0) w0 = code;
                        else if (r == 4) w1 = code;
                        else if (r < 4) w0 = mad_u32(code, r == 1 ? mul1 : r == 2 ? mul2 : mul3, w0);
                        else w1 = mad_u32(code, r == 5 ? mul1 : r == 6 ? mul2 : mul3, w1);
                        d0 = Hp[r];
                        Hp[r] = h;
                        E[r] = e;
                        hu = h;
                    }
                    // a lane's four consecutive steps share one 32-byte
                    // sector; pooled tiles stream out (walked much later),
                    // own tiles stay in L2 for the walk right after
                    if (own_task) __stcg(slab + widx, make_uint2(w0, w1));
                    else __stcs(slab + widx, make_uint2(w0, w1));
                    out_h = hu;
                    out_f = f;
                    if (bout) *(uint2 *)(bout + bidx) = make_uint2(prmt(hu, f, 0x5410u), prmt(hu, f, 0x7632u));
                    diag_in = up_h;
                }
                widx += (t & 3) == 3 ? 32 * 4 - 3 : 1;
                bidx += 2 * G;
            }
            prev_lo[0] = lo[0];
            prev_lo[1] = lo[1];
            prev_width = width;
            __syncwarp();
        }
        // a task in the warp's own slot: its walks, one thread per pair,
        // while the other warps of the SM keep sweeping; then the slot is
        // free for the next task
        if (own_task) {
            for (int wi = lane; wi < PAIRS; wi += 32) {
                const int64_t item = base + wi;
                if (item >= pc->n_items) break;
                Walk16<T, true> w;
                FwdCigar cg;
                if (w.begin(P, cg, slab, pc->order[item], wi >> 1, wi & 1, pc->wcap, pc->lane_chunks)) {
                    while (w.step(P, cg)) {
                    }
                    w.end(P, cg, L.status);
                }
            }
            __syncwarp();
        }
    }
    }  // phases
    }  // parts
}

// The walks of a 16-bit launch's pooled tasks: one thread per pair, at full
// occupancy (a walk is a chain of dependent loads from tiles long out of L2,
// so many walks in flight hide the latency).  Item k of a part lives in task
// k / 2G of the part's pool, group (k % 2G) / 2, half k % 2.
template <int T>
__global__ void __launch_bounds__(256, 4) k_tb16_walk(const TracebackLaunch L)
{
    constexpr int PAIRS = 2 * (32 / T);
    const TbParams &P = L.P;
    const DevTbPlan &dp = *L.dp;
    const int v = L.variant;
    if (*(volatile const int32_t *)L.status & (ST_BAD_INPUT | ST_UNSUPPORTED)) return;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    for (int pi = 0; pi < dp.var_n[v]; ++pi) {
        const TbPartPlan &tp = dp.part[dp.var_part[v][pi]];
        const int WCAP = tp.wcap;
        const int S4 = (WCAP + T - 1 + 3) >> 2;
        const int64_t lane_chunks = tp.slab_words / (8 * (int64_t)max(S4, 1));
        const int64_t tile_words = (32 * tp.slab_words + 63) & ~(int64_t)63;
        const int64_t n_pool = min((int64_t)tp.count, (int64_t)tp.pool_tasks * PAIRS);
        const int32_t *const order = L.order + tp.start;
        for (int64_t item = tid; item < n_pool; item += nthreads) {
            const uint2 *tile = (const uint2 *)(L.slab + tp.pool_offset + (item / PAIRS) * tile_words);
            const int wi = (int)(item % PAIRS);
            Walk16<T, false> w;
            FwdCigar cg;
            if (w.begin(P, cg, tile, order[item], wi >> 1, wi & 1, WCAP, lane_chunks)) {
                while (w.step(P, cg)) {
                }
                w.end(P, cg, L.status);
            }
        }
    }
}

// A device-planned launch of traceback variant v: the 16-bit kernel with T =
// 2^v lanes per pair for v < N_TB16_VARIANTS, else the int32 kernel, tiled or
// with T lanes per pair.  fma: every substitution score minus gap_open is
// >= 0, so the 16-bit diagonal add can run on the FMA pipe.
int launch_traceback_variant(int v, bool fma, const TracebackLaunch &L, int blocks, cudaStream_t st)
{
    if (!L.dp || blocks < 1) return SW_ERR_INTERNAL;
    TracebackLaunch V = L;
    V.variant = v;
    switch (v) {
#define SWGB_TB16(VV, TT)                                                                          \
    case VV:                                                                                       \
        if (fma) k_traceback16<TT, true><<<blocks, 128, 0, st>>>(V);                               \
        else k_traceback16<TT, false><<<blocks, 128, 0, st>>>(V);                                  \
        break;
        SWGB_TB16(0, 1)
        SWGB_TB16(1, 2)
        SWGB_TB16(2, 4)
        SWGB_TB16(3, 8)
        SWGB_TB16(4, 16)
        SWGB_TB16(5, 32)
#undef SWGB_TB16
    case TB_VAR_TILED: k_traceback<true><<<blocks, 128, 0, st>>>(V); break;
    case TB_VAR_GROUPED: k_traceback<false><<<blocks, 128, 0, st>>>(V); break;
    default: return SW_ERR_INTERNAL;
    }
    count_launch();
    return launch_status();
}

int launch_tb_walk_variant(int v, const TracebackLaunch &L, int blocks, cudaStream_t st)
{
    if (!L.dp || blocks < 1) return SW_ERR_INTERNAL;
    TracebackLaunch V = L;
    V.variant = v;
    switch (v) {
    case 0: k_tb16_walk<1><<<blocks, 256, 0, st>>>(V); break;
    case 1: k_tb16_walk<2><<<blocks, 256, 0, st>>>(V); break;
    case 2: k_tb16_walk<4><<<blocks, 256, 0, st>>>(V); break;
    case 3: k_tb16_walk<8><<<blocks, 256, 0, st>>>(V); break;
    case 4: k_tb16_walk<16><<<blocks, 256, 0, st>>>(V); break;
    case 5: k_tb16_walk<32><<<blocks, 256, 0, st>>>(V); break;
    default: return SW_ERR_INTERNAL;
    }
    count_launch();
    return launch_status();
}

int tb_walk_variant_blocks(int v, int sm_count, int *blocks)
{
    const void *fn = nullptr;
    switch (v) {
    case 0: fn = (const void *)k_tb16_walk<1>; break;
    case 1: fn = (const void *)k_tb16_walk<2>; break;
    case 2: fn = (const void *)k_tb16_walk<4>; break;
    case 3: fn = (const void *)k_tb16_walk<8>; break;
    case 4: fn = (const void *)k_tb16_walk<16>; break;
    case 5: fn = (const void *)k_tb16_walk<32>; break;
    default: return SW_ERR_INTERNAL;
    }
    int bps = 0;
    if (cuda_failed(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, 256, 0))) return SW_ERR_CUDA;
    *blocks = std::max(bps, 1) * sm_count;
    return SW_OK;
}

// Blocks of a full-occupancy launch of traceback variant v.
int traceback_variant_blocks(int v, int sm_count, int *blocks)
{
    const void *fn = nullptr;
    switch (v) {
    case 0: fn = (const void *)k_traceback16<1, true>; break;
    case 1: fn = (const void *)k_traceback16<2, true>; break;
    case 2: fn = (const void *)k_traceback16<4, true>; break;
    case 3: fn = (const void *)k_traceback16<8, true>; break;
    case 4: fn = (const void *)k_traceback16<16, true>; break;
    case 5: fn = (const void *)k_traceback16<32, true>; break;
    case TB_VAR_TILED: fn = (const void *)k_traceback<true>; break;
    case TB_VAR_GROUPED: fn = (const void *)k_traceback<false>; break;
    default: return SW_ERR_INTERNAL;
    }
    int bps = 0;
    if (cuda_failed(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, 128, 0))) return SW_ERR_CUDA;
    *blocks = std::max(bps, 1) * sm_count;
    return SW_OK;
}

}  // namespace swgb
