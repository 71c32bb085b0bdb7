// sw_band.cuh -- the traceback band of an alignment and its cost key.
//
// An alignment with score S that ends on read row ie holds at most ie + 1
// aligned read bases (each worth at most `match`), and with o <= e one gap
// run is the cheapest way to spend gap bases, so it has at most
//   D = (match (ie + 1) + o - S) / (-e) + 1   deletions and
//   I = (match (ie + 1) + o - e - S) / (match - e)   insertions.
// Walking back from (ie, je), deletions lower the diagonal j - i and
// insertions raise it, so every optimal path lies in the band
// je - ie - D <= j - i <= je - ie + I, rows 0..ie.
#pragma once
#include "sw_device.cuh"
#include "swgb_internal.h"

namespace swgb {

struct Band {
    int32_t jlo, W, rows;  // rectangle: window columns jlo .. jlo + W - 1, rows 0 .. rows - 1
    int32_t a, b;          // band in rectangle columns: row i spans [i + a, i + b]
};

__device__ __forceinline__ Band band_of(int32_t score, int32_t ie, int32_t je, const Scoring &sc)
{
    Band q;
    const int32_t ma = sc.ma, go = sc.go, ge = sc.ge;
    const int32_t dend = je - ie;
    int32_t dlo = -ie - 1;  // no lower limit when gaps are free
    if (ge < 0) {
        const int32_t num = ma * (ie + 1) + go - score;
        dlo = dend - (num < 0 ? 0 : num / (-ge) + 1);
    }
    const int32_t inum = ma * (ie + 1) + go - ge - score;
    const int32_t dhi = dend + (inum < 0 ? 0 : inum / (ma - ge));
    q.jlo = max(0, dlo);
    q.W = je - q.jlo + 1;
    q.rows = ie + 1;
    q.a = dlo - q.jlo;
    q.b = dhi - q.jlo;
    return q;
}

// Traceback sort key of a pair of class cls (class-major): pairs whose
// one-lane slab exceeds small_slab_words first, then the rest, each by
// falling chunk window (~9 % and ~4 % buckets).  A warp sweeps the widest
// window of its pairs at every chunk, so pairs of one task should share the
// width: sorted by it, a task of the 1M-pair batch of 100 x 200 pairs
// sweeps 1.07x the cells of its pairs' own windows, against 1.24x sorted by
// rows x width.  Also the one-lane slab words (need) and chunk window (wc)
// the launch sizing uses.  score <= 0: no alignment (width 0, need 0).
__device__ __forceinline__ void tb_cost_key(int cls, int32_t score, int32_t ie, int32_t je, int32_t small_slab_words,
                                            const Scoring &sc, int32_t &key, int32_t &need32, int32_t &wc, bool &big)
{
    int64_t need = 0;
    wc = 0;
    if (score > 0) {
        const Band t = band_of(score, ie, je, sc);
        const int32_t w = min(t.W, 8 + (t.b - t.a));
        need = (int64_t)((t.rows + 7) / 8) * w;
        wc = w;
    }
    const float lw = __log2f((float)(wc > 1 ? wc : 1));
    big = need > small_slab_words;
    if (big) {
        const int cb = min(63, max(0, (int)(8.f * lw) - 32));
        key = cls * N_NBUCKET + (63 - cb);
    } else {
        const int cb = min(191, max(0, (int)(16.f * lw)));
        key = cls * N_NBUCKET + 64 + (191 - cb);
    }
    need32 = (int32_t)(need < (int64_t)INT32_MAX ? need : (int64_t)INT32_MAX);
}

// Adds a warp's keys to the traceback histogram and class table, one set of
// atomics per distinct key (every lane of the warp calls it; key < 0: none).
__device__ __forceinline__ void tb_key_atomics(int32_t key, int cls, int32_t need32, int32_t wc, bool big,
                                               int32_t *hist, TbClassInfo *info)
{
    const KeyGroup g = key_group(key);
    if (key >= 0) {
        const unsigned mx_need = __reduce_max_sync(g.mask, (unsigned)need32);
        const unsigned mx_wc = __reduce_max_sync(g.mask, (unsigned)wc);
        const unsigned n_big = __reduce_add_sync(g.mask, (unsigned)(big && need32 > 0));
        if (g.rank == 0) {
            atomicAdd(&hist[key], g.size);
            if (mx_need > 0) {
                atomicMax(&info->max_need[cls], (int32_t)mx_need);
                atomicMax(&info->max_wcap[big ? 0 : 1][cls], (int32_t)mx_wc);
            }
            if (n_big) atomicAdd(&info->n_big[cls], (int32_t)n_big);
        }
    }
}

}  // namespace swgb
