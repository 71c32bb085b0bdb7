// sw_score.cu -- the Smith-Waterman score pass (score and end cell).
//
// Stage E, task iii of the paper aligns every read onto each of its extended
// CALs with Smith-Waterman.  This kernel computes, for each (read, window)
// pair, the best local-alignment score of the affine-gap recurrence
//
//   E(i,j) = max(H(i,j-1) + o, E(i,j-1) + e)
//   F(i,j) = max(H(i-1,j) + o, F(i-1,j) + e)
//   H(i,j) = max(0, H(i-1,j-1) + s(r_i, w_j), E(i,j), F(i,j))
//
// and the cell where it is first reached (smallest window index j, then
// smallest read index i).
//
// Work layout.  A group of T consecutive lanes of a warp owns one pair (int32
// mode) or two pairs (int16 modes: pair A in the low and pair B in the high
// half of every register, so each DPX instruction updates two cells).  Lane
// k of a group holds read rows k*R .. k*R+R-1 of the current row chunk in
// registers and sweeps the window columns; lane k works on column t-k at step
// t, receiving the row above its block from lane k-1 with one shuffle per
// value (a wavefront along the anti-diagonal).  The int16 modes take two
// columns per step (2(t-k) and 2(t-k)+1, four shuffles): the second column's
// rows run one row behind the first's, reading the first column's H as its
// previous column while the first reads the second's of the step before
// (two register arrays, no copies), so the two columns' F chains -- each
// row's F, max and ReLU depend on the row above -- overlap.  Reads longer than T*R are
// processed in chunks of T*R rows; the last lane of a chunk stores its bottom
// row (H+o, F per column) to global scratch for the first lane of the next
// chunk.  A warp takes floor(32/T) groups' worth of pairs at a time from a
// length-sorted list with one atomic, and loops until the list is empty.
//
// Arithmetic.  Each lane keeps per row E(i,j) and H(i,j)+o.  E and F are
// floored at 0: max(E, 0) obeys the same recurrence (because e <= 0) and
// never changes H, which is floored at 0 anyway.  The substitution score
// comes from one byte permute: per column a 4-byte table of s(x, w_j) - o for
// the four read bases x, per row a selector that picks the row's read base
// (and sign-replicates, which yields 0 or -1 -- i.e. an effective score of o
// or o-1, below zero -- for rows past the read end).  Window columns past a
// pair's end use an all-zero table, which likewise scores o.  Padded cells can
// therefore only hold values strictly below some real cell's value (o < 0), so
// they never become or tie the best cell and need no masking.
//
// (__vibmax_s16x2 is not used for the running best: the header's inline asm
// writes the max before re-reading its first operand without an early-clobber
// constraint, so with `x = __vibmax_s16x2(x, ...)` the compiler may alias the
// two and the predicates then compare the max with itself.)
//
// Best cell.  Every cell's H is turned into a key (H << TAGB) + (TAGM - r) (r = row in
// the lane's block, so equal H prefers the smaller row); a three-way-max tree
// gives the column's best key, and the lane's running best is replaced only
// when the column's H is strictly larger (so the smallest column wins).  The
// 16-bit keys need (H << TAGB) + TAGM < 32768: H <= 1022 with 5-bit row
// tags (up to 32 rows per lane), H <= 510 with 6-bit tags (up to 64 rows).
// The classifier gives this mode to pairs whose score bound is at most 510;
// with the SW_SCORE_AUTO setting larger bounds take the wide mode below.
//
// Pairs with larger possible scores (up to 32000) keep their two halves
// (MODE_I16W) but build no keys: a three-way-max tree over the rows gives
// each half's column maximum, and when a half's running best strictly rises
// the lane copies the column's R values into one of its two snapshot slots
// (shared memory, four rows per 16-byte store): the slot the other pair does
// not point to, or either when both pairs rise in the same column, so a
// column is stored once.  Each pair points to the slot of the column where
// its best was first reached, and after the chunk the best cell's row is the
// first row of that snapshot holding the best value.  This
// moves the row tracking off the ALU pipe (the kernel's limit) onto the
// shared-memory stores, so the wide mode costs the same ALU operations per
// cell as the 16-bit-key mode.  The int32 mode covers the rest.
#include "sw_band.cuh"
#include "sw_device.cuh"
#include "swgb_internal.h"

namespace swgb {

constexpr unsigned FULL = 0xffffffffu;

struct PairRef {
    int64_t rs, ws;  // first base of read / window
    int32_t m, n;    // lengths (m == 0: no pair)
};

__device__ __forceinline__ PairRef load_pair(const ScoreLaunch &L, const int32_t *order, int64_t n_items,
                                             int64_t item, bool on)
{
    PairRef pr{0, 0, 0, 0};
    if (on && item < n_items) {
        const int64_t p = order[item];
        const int64_t rd = L.ps.pair_read ? L.ps.pair_read[p] : p;
        pr.rs = L.ps.read_off[rd];
        pr.m = (int32_t)(L.ps.read_off[rd + 1] - pr.rs);
        pr.ws = L.ps.win_off[p];
        pr.n = (int32_t)(L.ps.win_off[p + 1] - pr.ws);
    }
    return pr;
}

// Read base codes of rows i0 .. i0+R-1 (4 bits each, 8 per word); rows past
// the read end get code 4 ("no base").
template <int R>
__device__ __forceinline__ void load_rows(const uint32_t *__restrict__ reads, const PairRef &p, int i0,
                                          uint32_t (&codes)[(R + 7) / 8])
{
#pragma unroll
    for (int q = 0; q < (R + 7) / 8; ++q) codes[q] = 0x44444444u;
#pragma unroll
    for (int q16 = 0; q16 < (R + 15) / 16; ++q16) {
        const int row = i0 + 16 * q16;
        const int cnt = min(16, p.m - row);
        if (cnt > 0) {
            uint32_t w = load_bases(reads, p.rs + row, cnt);
#pragma unroll
            for (int b = 0; b < 16; ++b) {
                const int r = 16 * q16 + b;
                if (r < R && b < cnt) {
                    uint32_t &c = codes[r / 8];
                    const int sh = 4 * (r % 8);
                    c = (c & ~(0xFu << sh)) | (((w >> (2 * b)) & 3u) << sh);
                }
            }
        }
    }
}

template <int MODE>
struct Arith;

template <>
struct Arith<MODE_I32> {
    typedef int32_t V;
    static __device__ __forceinline__ V addmax(V a, V b, V c) { return __viaddmax_s32(a, b, c); }
    static __device__ __forceinline__ V addmax_relu(V a, V b, V c) { return __viaddmax_s32_relu(a, b, c); }
    static __device__ __forceinline__ V max3(V a, V b, V c) { return __vimax3_s32(a, b, c); }
    static __device__ __forceinline__ V add(V a, V b) { return a + b; }
    static __device__ __forceinline__ V splat(int32_t x) { return x; }
};

template <>
struct Arith<MODE_I16> {
    typedef uint32_t V;
    static __device__ __forceinline__ V addmax(V a, V b, V c) { return __viaddmax_s16x2(a, b, c); }
    static __device__ __forceinline__ V addmax_relu(V a, V b, V c) { return __viaddmax_s16x2_relu(a, b, c); }
    static __device__ __forceinline__ V max3(V a, V b, V c) { return __vimax3_s16x2(a, b, c); }
    // per-half add (no carry between halves): max(a + b, -32768)
    static __device__ __forceinline__ V add(V a, V b) { return __viaddmax_s16x2(a, b, 0x80008000u); }
    static __device__ __forceinline__ V splat(int32_t x) { return ((uint32_t)(uint16_t)(int16_t)x) * 0x10001u; }
};
template <>
struct Arith<MODE_I16W> : Arith<MODE_I16> {};

// a * one + c on the FMA pipe; `one` is a kernel argument equal to 1, so the
// multiply-add cannot be folded into an ALU add.  With both halves of a and c
// non-negative and their sums below 32768 it is an exact per-half add.
__device__ __forceinline__ uint32_t mad_add(uint32_t a, uint32_t one, uint32_t c)
{
    uint32_t d;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(one), "r"(c));
    return d;
}

// x >> 16 on the FMA pipe (the high word of x * 65536)
__device__ __forceinline__ uint32_t hi16_fma(uint32_t x)
{
    uint32_t d;
    asm("mul.hi.u32 %0, %1, %2;" : "=r"(d) : "r"(x), "r"(0x10000u));
    return d;
}

// Rows 4q .. 4q+3 of a lane's column as one 16-byte word (rows past R: 0,
// which never equals a best value, as bests are >= 1).
template <int R, typename V>
__device__ __forceinline__ uint4 quad_of(const V (&h)[R], int q)
{
    const int r = 4 * q;
    return make_uint4((uint32_t)h[r], r + 1 < R ? (uint32_t)h[r + 1] : 0u, r + 2 < R ? (uint32_t)h[r + 2] : 0u,
                      r + 3 < R ? (uint32_t)h[r + 3] : 0u);
}

// First row of a snapshot whose half (shift 0: low, 16: high) equals best.
template <int R>
__device__ __forceinline__ int snapshot_row(const uint4 *snap, unsigned stride, uint32_t best, int shift)
{
    int row = R - 1;
    for (int q = (R + 3) / 4 - 1; q >= 0; --q) {
        const uint4 v = snap[q * stride];
        if (((v.w >> shift) & 0xFFFFu) == best) row = 4 * q + 3;
        if (((v.z >> shift) & 0xFFFFu) == best) row = 4 * q + 2;
        if (((v.y >> shift) & 0xFFFFu) == best) row = 4 * q + 1;
        if (((v.x >> shift) & 0xFFFFu) == best) row = 4 * q;
    }
    return row;
}

// Dynamic shared memory of a launch: the MODE_I16W snapshot slots.
__host__ __device__ constexpr int score_snapshot_bytes(int rows, int mode, int threads)
{
    return mode == MODE_I16W ? 2 * ((rows + 3) / 4) * 16 * threads : 0;
}

template <int R, int MODE, bool FMA_ADD>
__global__ void __launch_bounds__(128) k_score(const ScoreLaunch L)
{
    typedef Arith<MODE> A;
    typedef typename A::V V;
    constexpr bool PAIR2 = MODE != MODE_I32;
    constexpr int NW = (R + 7) / 8;
    // row tag in the low bits of a key: TAGM - r, so equal H prefers the
    // smaller row; 5 bits cover 32 rows, 6 bits 64
    constexpr uint32_t TAGB = R <= 32 ? 5u : 6u;
    constexpr uint32_t TAGM = (1u << TAGB) - 1u;
    static_assert(R <= 64, "row tags cover at most 64 rows");

    // column tables: s_tab[w] byte x = s(x, w) - o; s_tab[4] = 0 (padding)
    __shared__ uint32_t s_tab[8];
    const int32_t go = L.sc.go, ge = L.sc.ge;
    {
        const uint32_t mis4 = ((uint32_t)(uint8_t)(int8_t)(L.sc.mi - go)) * 0x01010101u;
        const uint32_t ma4 = ((uint32_t)(uint8_t)(int8_t)(L.sc.ma - go)) * 0x01010101u;
        if (threadIdx.x < 8)
            s_tab[threadIdx.x] = threadIdx.x < 4 ? prmt(mis4, ma4, 0x3210u + (4u << (4u * threadIdx.x))) : 0u;
        __syncthreads();
    }

    // MODE_I16W snapshot slots s = 0, 1: quad q of slot s at
    // snap[(s * R4 + q) * blockDim.x] (a warp's stores hit distinct banks)
    constexpr int R4 = (R + 3) / 4;
    extern __shared__ __align__(16) unsigned char s_dyn[];
    uint4 *const snap = reinterpret_cast<uint4 *>(s_dyn) + threadIdx.x;

    const int lane = threadIdx.x & 31;
    const int64_t warp_global = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t one = (uint32_t)L.one;
    const V GO = A::splat(go), GE = A::splat(ge);
    // input already found invalid (or a plan whose shape changed): the
    // scratch may be too small for it, so do nothing
    if (*(volatile const int32_t *)L.status & ST_BAD_INPUT) return;

    // One class given by the host, or every class of this launch's variant
    // in the device plan (longest reads first); the warps of the launch move
    // on to the next class as soon as the current one has no work left.
    // The class's order, count, counter and index live in shared memory, one
    // record per warp, read where they are used: held in registers across
    // the inner loops they would push the largest plans into spills.
    struct ClassCtx {
        const int32_t *order;
        int32_t *work_counter;
        int64_t n_items;
        uint8_t *bnd_warp;       // the warp's boundary slot (nullptr: one row chunk)
        int64_t bnd_group_bytes;
        int32_t cls, ci, n_cls;
    };
    __shared__ ClassCtx s_cc[4];  // 128 threads: 4 warps
    volatile ClassCtx *const cc = &s_cc[threadIdx.x >> 5];
    const bool planned = L.dp != nullptr;
    if (lane == 0) {
        cc->ci = 0;
        cc->n_cls = planned ? L.dp->var_n[L.variant] : 1;
    }
    __syncwarp();
    for (; cc->ci < cc->n_cls; __syncwarp(), cc->ci = cc->ci + (lane == 0 ? 1 : 0), __syncwarp()) {
    const int ci = cc->ci;
    int T = L.lanes, cls = L.cls;
    const int32_t *order = L.order;
    int64_t n_items = L.n_items, bnd_group_bytes = L.boundary_group_bytes;
    int32_t *work_counter = L.work_counter;
    uint8_t *bnd_base = L.boundary;
    int64_t bnd_warp_bytes = 0;  // warp stride of the boundary slots (host-given: G groups of this class)
    if (planned) {
        const DevScorePlan &dp = *L.dp;
        cls = dp.var_cls[L.variant][ci];
        T = dp.cls_lanes[cls];
        order = L.order + dp.cls_start[cls];
        n_items = dp.cls_count[cls];
        work_counter = L.work_counter + cls;
        bnd_group_bytes = dp.cls_bnd_bytes[cls];
        bnd_base = nullptr;
        if (bnd_group_bytes) {
            // reads in several row chunks: only warps with a boundary slot
            if (warp_global >= dp.var_bnd_warps[L.variant]) continue;
            bnd_base = L.boundary + dp.var_bnd_offset[L.variant];
            // every class of the variant uses the same warp stride, so that
            // warps working on different classes never share bytes
            bnd_warp_bytes = dp.var_bnd_slot[L.variant];
        }
    }
    const int G = 32 / T;
    const int g = lane / T;
    const int k = lane - g * T;
    const bool on = g < G;
    const int per_warp = G * (PAIR2 ? 2 : 1);
    if (!planned) bnd_warp_bytes = G * bnd_group_bytes;
    if (lane == 0) {
        cc->order = order;
        cc->work_counter = work_counter;
        cc->n_items = n_items;
        cc->cls = cls;
        cc->bnd_warp = bnd_base ? bnd_base + warp_global * bnd_warp_bytes : nullptr;
        cc->bnd_group_bytes = bnd_group_bytes;
    }
    __syncwarp();

    for (;;) {
        int base = 0;
        if (lane == 0) base = atomicAdd(cc->work_counter, per_warp);
        base = __shfl_sync(FULL, base, 0);
        if (base >= cc->n_items) break;

        const int64_t item = base + (int64_t)g * (PAIR2 ? 2 : 1);
        const PairRef pa = load_pair(L, cc->order, cc->n_items, item, on);
        const PairRef pb = PAIR2 ? load_pair(L, cc->order, cc->n_items, item + 1, on) : PairRef{0, 0, 0, 0};
        const int32_t mg = max(pa.m, pb.m), ng = max(pa.n, pb.n);
        const int32_t mw = __reduce_max_sync(FULL, (unsigned)mg);
        const int32_t nw = __reduce_max_sync(FULL, (unsigned)ng);
        // columns every real pair of the warp has (empty slots never feed a
        // real pair, so they do not limit the fast path)
        const int32_t na = pa.m ? pa.n : INT32_MAX, nbb = pb.m ? pb.n : INT32_MAX;
        const int32_t nmin_w = (int32_t)__reduce_min_sync(FULL, (unsigned)min(na, nbb));
        const int rows_per_chunk = T * R;
        const int chunks = (mw + rows_per_chunk - 1) / rows_per_chunk;
        const int steps = nw + T - 1;

        uint64_t bestA = 0, bestB = 0;

        for (int c = 0; c < chunks; ++c) {
            const int i0 = c * rows_per_chunk + k * R;
            // per-row selectors
            uint32_t sel[R];
            {
                uint32_t ca[NW], cb[NW];
                load_rows<R>(L.ps.reads, pa, i0, ca);
                if (PAIR2) load_rows<R>(L.ps.reads, pb, i0, cb);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const uint32_t xa = (ca[r / 8] >> (4 * (r % 8))) & 0xFu;
                    if (!PAIR2) {
                        sel[r] = xa < 4u ? xa * 0x1111u + 0x8880u : 0x8888u;
                    } else {
                        const uint32_t xb = (cb[r / 8] >> (4 * (r % 8))) & 0xFu;
                        const uint32_t sa = xa < 4u ? xa * 0x11u + 0x80u : 0x88u;
                        const uint32_t sb = xb < 4u ? xb * 0x11u + 0xC4u : 0xCCu;
                        sel[r] = sa | (sb << 8);
                    }
                }
            }
            // per row: E - o and H of the previous column (E floored at o,
            // which never changes H)
            V e[R], h[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                e[r] = 0;
                h[r] = 0;
            }
            V diag_in = 0;             // H(i0-1, j-1)
            V out_h = 0, out_f = 0;    // bottom row (H, F - o) handed to the next lane
            // running best of this chunk
            uint32_t bk0 = PAIR2 && MODE == MODE_I16 ? TAGM * 0x10001u : 0u;
            uint32_t rowA = 0, rowB = 0;
            int slotA = 0, slotB = 1;  // MODE_I16W: the snapshot slot each pair points to
            int32_t jA = 0, jB = 0;
            // window stream: 2-bit codes of the next columns (up to 16)
            uint32_t wwA = 0, wwB = 0;
            const bool load_bnd = c > 0;
            const bool store_bnd = c + 1 < chunks;
            // this group's double-buffered boundary row (bytes per buffer: half)
            uint8_t *const bnd_w = cc->bnd_warp;
            const int64_t bgb = cc->bnd_group_bytes;
            uint8_t *const bnd = (on && bnd_w) ? bnd_w + g * bgb : nullptr;
            const int64_t bnd_half = bgb / 2;
            const V *bin = load_bnd && bnd ? (const V *)(bnd + (c & 1) * bnd_half) : nullptr;
            V *bout = store_bnd && bnd ? (V *)(bnd + ((c + 1) & 1) * bnd_half) : nullptr;

            if constexpr (PAIR2) {
            // two columns per iteration: column j0 = 2(u - k) from h (its
            // previous column in h1) and column j0 + 1 from h1, interleaved
            // one row apart so that their F chains overlap
            V h1[R];
#pragma unroll
            for (int r = 0; r < R; ++r) h1[r] = 0;
            // selectors two rows to a word (prmt reads the low 16 bits; odd
            // rows are shifted down on the FMA pipe where they are used)
            uint32_t sel2[(R + 1) / 2];
#pragma unroll
            for (int r = 0; r < R; r += 2) sel2[r / 2] = sel[r] | (r + 1 < R ? sel[r + 1] << 16 : 0u);
            auto selr = [&](int r) -> uint32_t { return (r & 1) ? hi16_fma(sel2[r / 2]) : sel2[r / 2]; };
            V out_h1 = 0, out_f1 = 0;
            const int iters = (nw + 1) / 2 + T - 1;
            auto col_best = [&](const V (&hv)[R], uint32_t ck, int jj) {
                if constexpr (MODE == MODE_I16) {
                    const uint32_t nb = __vimax_s16x2_relu(bk0, ck | (TAGM * 0x10001u));
                    const uint32_t up = nb ^ bk0;
                    bk0 = nb;
                    if (up & 0xFFFFu) { rowA = ck; jA = jj; }
                    if (up > 0xFFFFu) { rowB = ck; jB = jj; }
                    return;
                }
                const uint32_t nb = __vimax_s16x2_relu(bk0, ck);
                const uint32_t up = nb ^ bk0;
                bk0 = nb;
                const bool upA = (up & 0xFFFFu) != 0, upB = up > 0xFFFFu;
                if (upA || upB) {
                    const int sl = (upA && upB) ? 0 : (upA ? (slotB ^ 1) : (slotA ^ 1));
                    uint4 *const dst = snap + sl * R4 * blockDim.x;
#pragma unroll
                    for (int q = 0; q < R4; ++q) dst[q * blockDim.x] = quad_of<R>(hv, q);
                    if (upA) { slotA = sl; jA = jj; }
                    if (upB) { slotB = sl; jB = jj; }
                }
            };
            for (int u = 0; u < iters; ++u) {
                const int j0 = 2 * (u - k);
                V up_h0 = __shfl_up_sync(FULL, out_h, 1);
                V up_f0 = __shfl_up_sync(FULL, out_f, 1);
                V up_h1 = __shfl_up_sync(FULL, out_h1, 1);
                V up_f1 = __shfl_up_sync(FULL, out_f1, 1);
                if (k == 0) {
                    up_h0 = bin && j0 < ng ? bin[2 * j0] : 0;
                    up_f0 = bin && j0 < ng ? bin[2 * j0 + 1] : 0;
                    up_h1 = bin && j0 + 1 < ng ? bin[2 * j0 + 2] : 0;
                    up_f1 = bin && j0 + 1 < ng ? bin[2 * j0 + 3] : 0;
                }
                uint32_t t0A = 0, t0B = 0, t1A = 0, t1B = 0;
                if (j0 >= 0) {
                    if ((j0 & 15) == 0) {
                        wwA = j0 < pa.n ? load_bases(L.ps.wins, pa.ws + j0, min(16, pa.n - j0)) : 0u;
                        wwB = j0 < pb.n ? load_bases(L.ps.wins, pb.ws + j0, min(16, pb.n - j0)) : 0u;
                    }
                    if (2 * u + 1 < nmin_w) {  // every real pair of the warp has columns j0 and j0 + 1
                        t0A = s_tab[wwA & 3u];
                        t1A = s_tab[(wwA >> 2) & 3u];
                        t0B = s_tab[wwB & 3u];
                        t1B = s_tab[(wwB >> 2) & 3u];
                    } else {
                        t0A = s_tab[j0 < pa.n ? wwA & 3u : 4u];
                        t1A = s_tab[j0 + 1 < pa.n ? (wwA >> 2) & 3u : 4u];
                        t0B = s_tab[j0 < pb.n ? wwB & 3u : 4u];
                        t1B = s_tab[j0 + 1 < pb.n ? (wwB >> 2) & 3u : 4u];
                    }
                    wwA >>= 4;
                    wwB >>= 4;
                }
                V hu0 = up_h0, f0 = up_f0, hu1 = up_h1, f1 = up_f1;
                uint32_t ckA = 0, pkA = 0, ckB = 0, pkB = 0;
                V d0n, d1n;
                uint32_t sprev = selr(0);  // selector of the row the second column needs next
                {
                    const V s0 = (V)prmt(t0A, t0B, sprev);
                    const V s1 = (V)prmt(t1A, t1B, sprev);
                    d0n = FMA_ADD ? (V)mad_add((uint32_t)diag_in, one, (uint32_t)s0) : A::add(diag_in, s0);
                    d1n = FMA_ADD ? (V)mad_add((uint32_t)up_h0, one, (uint32_t)s1) : A::add(up_h0, s1);
                }
#pragma unroll
                for (int r = 0; r <= R; ++r) {
                    const uint32_t snext = r + 1 < R ? selr(r + 1) : 0u;
                    if (r < R) {  // column j0, row r
                        const V d = d0n;
                        e[r] = A::addmax(e[r], GE, h1[r]);
                        if (r + 1 < R) {
                            const V sn = (V)prmt(t0A, t0B, snext);
                            d0n = FMA_ADD ? (V)mad_add((uint32_t)h1[r], one, (uint32_t)sn) : A::add(h1[r], sn);
                        }
                        f0 = A::addmax(f0, GE, hu0);
                        const V hn = A::addmax_relu(A::max3(d, e[r], f0), GO, 0);
                        h[r] = hn;
                        hu0 = hn;
                        const uint32_t k0 = MODE == MODE_I16 ? mad_add((uint32_t)hn, 1u << TAGB, (TAGM - (uint32_t)r) * 0x10001u)
                                                             : (uint32_t)hn;
                        if (r % 2 == 0) pkA = k0;
                        else ckA = r == 1 ? __vimax_s16x2_relu(pkA, k0) : __vimax3_s16x2(ckA, pkA, k0);
                    }
                    if (r >= 1) {  // column j0 + 1, row r - 1
                        const int q = r - 1;
                        const V d = d1n;
                        e[q] = A::addmax(e[q], GE, h[q]);
                        if (q + 1 < R) {
                            const V sn = (V)prmt(t1A, t1B, sprev);  // row q + 1 = r
                            d1n = FMA_ADD ? (V)mad_add((uint32_t)h[q], one, (uint32_t)sn) : A::add(h[q], sn);
                        }
                        f1 = A::addmax(f1, GE, hu1);
                        const V hn = A::addmax_relu(A::max3(d, e[q], f1), GO, 0);
                        h1[q] = hn;
                        hu1 = hn;
                        const uint32_t k1 = MODE == MODE_I16 ? mad_add((uint32_t)hn, 1u << TAGB, (TAGM - (uint32_t)q) * 0x10001u)
                                                             : (uint32_t)hn;
                        if (q % 2 == 0) pkB = k1;
                        else ckB = q == 1 ? __vimax_s16x2_relu(pkB, k1) : __vimax3_s16x2(ckB, pkB, k1);
                    }
                    sprev = snext;
                }
                if (R % 2 == 1) {
                    ckA = R == 1 ? pkA : __vimax_s16x2_relu(ckA, pkA);
                    ckB = R == 1 ? pkB : __vimax_s16x2_relu(ckB, pkB);
                }
                diag_in = up_h1;
                out_h = hu0;
                out_f = f0;
                out_h1 = hu1;
                out_f1 = f1;
                if (bout && k == T - 1 && j0 >= 0) {
                    if (j0 < ng) {
                        bout[2 * j0] = out_h;
                        bout[2 * j0 + 1] = out_f;
                    }
                    if (j0 + 1 < ng) {
                        bout[2 * j0 + 2] = out_h1;
                        bout[2 * j0 + 3] = out_f1;
                    }
                }
                // strict improvement keeps the first column: j0 before j0 + 1
                col_best(h, ckA, j0);
                col_best(h1, ckB, j0 + 1);
            }
            } else {
            // int32: one pair per group, one column per step
            for (int t = 0; t < steps; ++t) {
                const int j = t - k;
                V up_h = __shfl_up_sync(FULL, out_h, 1);
                V up_f = __shfl_up_sync(FULL, out_f, 1);
                if (k == 0) {
                    up_h = bin && j < ng ? bin[2 * j] : 0;
                    up_f = bin && j < ng ? bin[2 * j + 1] : 0;
                }
                // column table
                uint32_t twA = 0;
                if (j >= 0) {
                    if ((j & 15) == 0) wwA = j < pa.n ? load_bases(L.ps.wins, pa.ws + j, min(16, pa.n - j)) : 0u;
                    twA = s_tab[j < pa.n ? wwA & 3u : 4u];
                    wwA >>= 2;
                }
                V hd = diag_in, hu = up_h, f = up_f;
                uint32_t ck0 = 0, pk0 = 0;  // column key, pending key
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const V s = (V)prmt(twA, 0u, sel[r]);
                    e[r] = A::addmax(e[r], GE, h[r]);
                    const V d = (V)mad_add((uint32_t)hd, one, (uint32_t)s);  // exact in int32 for any sign
                    hd = h[r];
                    f = A::addmax(f, GE, hu);
                    const V hn = A::addmax_relu(A::max3(d, e[r], f), GO, 0);
                    h[r] = hn;
                    hu = hn;
                    const uint32_t k0 = mad_add((uint32_t)hn, 1u << TAGB, TAGM - (uint32_t)r);
                    // three-way max over pairs of rows
                    if (r % 2 == 0) pk0 = k0;
                    else ck0 = r == 1 ? max(pk0, k0) : (uint32_t)__vimax3_s32((int)ck0, (int)pk0, (int)k0);
                }
                if (R % 2 == 1) ck0 = R == 1 ? pk0 : max(ck0, pk0);
                diag_in = up_h;
                out_h = h[R - 1];
                out_f = f;
                if (bout && k == T - 1 && j >= 0 && j < ng) {
                    bout[2 * j] = out_h;
                    bout[2 * j + 1] = out_f;
                }
                // strict improvement of H keeps the first (smallest) column
                if (ck0 > (bk0 | TAGM)) {
                    bk0 = ck0;
                    jA = j;
                }
            }
            }
            // fold the chunk's best into the 64-bit per-lane best
            const int rbase = c * rows_per_chunk + k * R;
            if (MODE == MODE_I32) {
                const uint32_t hb = bk0 >> TAGB;
                if (hb) bestA = max(bestA, cell_key(hb, jA, rbase + (int)TAGM - (int)(bk0 & TAGM)));
            } else if (MODE == MODE_I16) {
                const uint32_t ha = (bk0 & 0xFFFFu) >> TAGB, hb = (bk0 >> 16) >> TAGB;
                if (ha) bestA = max(bestA, cell_key(ha, jA, rbase + (int)TAGM - (int)(rowA & TAGM)));
                if (hb) bestB = max(bestB, cell_key(hb, jB, rbase + (int)TAGM - (int)((rowB >> 16) & TAGM)));
            } else {
                const uint32_t ha = bk0 & 0xFFFFu, hb = bk0 >> 16;
                const unsigned bd = blockDim.x;
                if (ha) bestA = max(bestA, cell_key(ha, jA, rbase + snapshot_row<R>(snap + slotA * R4 * bd, bd, ha, 0)));
                if (hb) bestB = max(bestB, cell_key(hb, jB, rbase + snapshot_row<R>(snap + slotB * R4 * bd, bd, hb, 16)));
            }
            __syncwarp();
        }
        // group reduction: lane k = 0 ends with the group's best
        for (int d = 1; d < T; d <<= 1) {
            const int src = (k + d < T) ? lane + d : lane;
            bestA = max(bestA, __shfl_sync(FULL, bestA, src));
            if (PAIR2) bestB = max(bestB, __shfl_sync(FULL, bestB, src));
        }
        // outputs, and with a traceback to follow, each pair's traceback cost
        // key (the key pass folded into this epilogue)
#pragma unroll
        for (int h2 = 0; h2 < (PAIR2 ? 2 : 1); ++h2) {
            const int64_t it = item + h2;
            int32_t tkey = -1, need32 = 0, wc = 0;
            bool big = false;
            if (on && k == 0 && it < cc->n_items) {
                const uint64_t b = h2 ? bestB : bestA;
                const int32_t p = cc->order[it];
                const uint32_t sc = key_h(b);
                const int32_t ie = sc ? key_i(b) : -1, je = sc ? key_j(b) : -1;
                L.out_score[p] = (int32_t)sc;
                L.out_end[2 * p] = ie;
                L.out_end[2 * p + 1] = je;
                if (L.tb_keys) {
                    tb_cost_key(cc->cls, (int32_t)sc, ie, je, L.small_slab_words, L.sc, tkey, need32, wc, big);
                    L.tb_keys[p] = tkey;
                }
            }
            if (L.tb_keys) tb_key_atomics(tkey, cc->cls, need32, wc, big, L.tb_hist, L.tb_info);
        }
    }
    }  // classes
}

const int kScoreRows[N_SCORE_ROWS] = {8, 16, 20, 25, 32, 50};

template <int R>
static int launch_r(int mode, bool fma, const ScoreLaunch &L, int blocks, int threads, cudaStream_t st)
{
    const int smem = score_snapshot_bytes(R, MODE_I16W, threads);
    if (mode == MODE_I32) k_score<R, MODE_I32, true><<<blocks, threads, 0, st>>>(L);
    else if (mode == MODE_I16 && fma) k_score<R, MODE_I16, true><<<blocks, threads, 0, st>>>(L);
    else if (mode == MODE_I16) k_score<R, MODE_I16, false><<<blocks, threads, 0, st>>>(L);
    else if (mode == MODE_I16W && fma) k_score<R, MODE_I16W, true><<<blocks, threads, smem, st>>>(L);
    else if (mode == MODE_I16W) k_score<R, MODE_I16W, false><<<blocks, threads, smem, st>>>(L);
    else return SW_ERR_INTERNAL;
    count_launch();
    return launch_status();
}

// The FMA-pipe diagonal add needs every substitution score minus gap_open
// to be >= 0 in the 16-bit modes (no borrow between halves).
static bool fma_add_ok(const ScoreLaunch &L) { return L.sc.mi - L.sc.go >= 0; }

int launch_score(int rows, int mode, const ScoreLaunch &L, int blocks, int threads, cudaStream_t st)
{
    const bool fma = fma_add_ok(L);
    switch (rows) {
    case 8: return launch_r<8>(mode, fma, L, blocks, threads, st);
    case 16: return launch_r<16>(mode, fma, L, blocks, threads, st);
    case 20: return launch_r<20>(mode, fma, L, blocks, threads, st);
    case 25: return launch_r<25>(mode, fma, L, blocks, threads, st);
    case 32: return launch_r<32>(mode, fma, L, blocks, threads, st);
    case 50: return launch_r<50>(mode, fma, L, blocks, threads, st);
    default: return SW_ERR_INVALID_ARG;
    }
}

// A device-planned launch of variant v = rows index * N_MODES + mode; the
// FMA-pipe diagonal add is chosen from the scoring as for launch_score.
int launch_score_variant(int v, const ScoreLaunch &L, int blocks, cudaStream_t st)
{
    if (v < 0 || v >= N_SCORE_VARIANTS || !L.dp) return SW_ERR_INTERNAL;
    ScoreLaunch V = L;
    V.variant = v;
    return launch_score(score_rows_at(v / N_MODES), v % N_MODES, V, blocks, 128, st);
}

template <int R>
static const void *kernel_ptr(int mode, bool fma)
{
    switch (mode) {
    case MODE_I32: return (const void *)k_score<R, MODE_I32, true>;
    case MODE_I16: return fma ? (const void *)k_score<R, MODE_I16, true> : (const void *)k_score<R, MODE_I16, false>;
    case MODE_I16W:
        return fma ? (const void *)k_score<R, MODE_I16W, true> : (const void *)k_score<R, MODE_I16W, false>;
    default: return nullptr;
    }
}

int score_variant_blocks(int v, int sm_count, int *blocks)
{
    int regs = 0, bps = 0;
    const int rc = score_kernel_regs(score_rows_at(v / N_MODES), v % N_MODES, &regs, &bps, 128);
    if (rc) return rc;
    if (bps < 1) return SW_ERR_INTERNAL;
    *blocks = bps * sm_count;
    return SW_OK;
}

// Registers and resident blocks per SM of the (rows, mode) kernels; also
// lets them take their dynamic shared memory, so it runs before any launch
// of them (both diagonal-add forms; the grid follows the fewer blocks).
int score_kernel_regs(int rows, int mode, int *regs, int *max_blocks_per_sm, int threads)
{
    const int smem = score_snapshot_bytes(rows, mode, threads);
    *regs = 0;
    *max_blocks_per_sm = 0;
    for (int f = 0; f < 2; ++f) {
        const void *fn = nullptr;
        switch (rows) {
        case 8: fn = kernel_ptr<8>(mode, f); break;
        case 16: fn = kernel_ptr<16>(mode, f); break;
        case 20: fn = kernel_ptr<20>(mode, f); break;
        case 25: fn = kernel_ptr<25>(mode, f); break;
        case 32: fn = kernel_ptr<32>(mode, f); break;
        case 50: fn = kernel_ptr<50>(mode, f); break;
        default: return SW_ERR_INVALID_ARG;
        }
        if (!fn) return SW_ERR_INVALID_ARG;
        if (smem > 48 * 1024 &&
            cuda_failed(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)))
            return SW_ERR_CUDA;
        cudaFuncAttributes a;
        if (cuda_failed(cudaFuncGetAttributes(&a, fn))) return SW_ERR_CUDA;
        int bps = 0;
        if (cuda_failed(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, threads, smem))) return SW_ERR_CUDA;
        *regs = std::max(*regs, a.numRegs);
        *max_blocks_per_sm = f == 0 ? bps : std::min(*max_blocks_per_sm, bps);
    }
    return SW_OK;
}

}  // namespace swgb
