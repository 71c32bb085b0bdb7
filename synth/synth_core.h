/*
 * synth_core.h -- the per-read and per-candidate steps of the workload
 * generator, shared by the host generator (synth.c, gcc) and the device
 * generator (synth_gpu.cu, nvcc) so that both write the same workload.
 *
 * This is input generation only; it holds none of the alignment arithmetic.
 *
 * The includer defines, before including this file:
 *   SYNTH_FN       the function qualifiers (static inline, or __device__ ...)
 *   synth_sink_t   a type, and
 *   SYNTH_FN void synth_put(synth_sink_t *o, uint8_t base)
 *                  which receives a window's bases in order, first to last.
 *
 * Floating point: every double expression here must round once per
 * operation on both sides (gcc -ffp-contract=off, nvcc -fmad=false), so that
 * the comparisons against uniforms come out the same.
 */
#ifndef SYNTH_CORE_H
#define SYNTH_CORE_H

#include <stdint.h>

typedef struct {
    uint64_t seed;
    int64_t n_reads;
    int32_t n_len;            /* read length mix: n_len (value, weight) pairs */
    int32_t len_val[8];
    double len_w[8];
    int32_t cand_min, cand_max; /* candidates per read, uniform */
    int32_t win_len;          /* > 0: fixed window length; 0: flanks */
    int32_t flank_min, flank_max;
    double div_lo, div_hi;    /* true window: per-base mutation event probability */
    double indel_share;       /* share of mutation events that are indels */
    double decoy_random;      /* single-candidate reads: P(window is a random decoy) */
    double paralog_share;     /* multi-candidate reads: share of decoys that are paralogs */
    double par_lo, par_hi;    /* paralog divergence */
    double splice_frac;       /* P(read spans a splice junction) */
    int32_t intron_min, intron_max;
    int64_t first_read;       /* local read r is read first_read + r of the seeded set */
} synth_spec_t;

enum { KIND_TRUE = 0, KIND_PARALOG = 1, KIND_RANDOM = 2 };

SYNTH_FN uint64_t mix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

typedef struct { uint64_t key, ctr; uint64_t bits; int nbits; } rng_t;

SYNTH_FN uint64_t rnext(rng_t *g) { return mix64(g->key ^ mix64(g->ctr++)); }
SYNTH_FN double runif(rng_t *g) { return (double)(rnext(g) >> 11) * (1.0 / 9007199254740992.0); }
SYNTH_FN int64_t rint_in(rng_t *g, int64_t lo, int64_t hi) /* inclusive */
{
    return lo + (int64_t)(rnext(g) % (uint64_t)(hi - lo + 1));
}
SYNTH_FN uint8_t rbase(rng_t *g)
{
    if (g->nbits == 0) { g->bits = rnext(g); g->nbits = 32; }
    uint8_t b = (uint8_t)(g->bits & 3u);
    g->bits >>= 2; g->nbits--;
    return b;
}

SYNTH_FN rng_t read_rng(const synth_spec_t *s, int64_t r)
{
    rng_t g = {mix64(s->seed * 0xD1B54A32D192ED03ULL ^ mix64((uint64_t)(s->first_read + r))), 0, 0, 0};
    return g;
}
SYNTH_FN rng_t cand_rng(const rng_t *rg, int64_t k)
{
    rng_t g = {mix64(rg->key + 0x632BE59BD9B4E019ULL * (uint64_t)(k + 1)), 0, 0, 0};
    return g;
}

/* Per-read header draws, in a fixed order. */
typedef struct { int32_t m, c, t, spliced; } read_hdr_t;

SYNTH_FN read_hdr_t read_header(const synth_spec_t *s, rng_t *g)
{
    read_hdr_t h;
    double u = runif(g), tot = 0.0, acc = 0.0;
    for (int k = 0; k < s->n_len; ++k) tot += s->len_w[k];
    h.m = s->len_val[s->n_len - 1];
    for (int k = 0; k < s->n_len; ++k) {
        acc += s->len_w[k] / tot;
        if (u < acc) { h.m = s->len_val[k]; break; }
    }
    h.c = (int32_t)rint_in(g, s->cand_min, s->cand_max);
    h.t = (int32_t)rint_in(g, 0, h.c - 1);
    h.spliced = runif(g) < s->splice_frac;
    return h;
}

SYNTH_FN void read_bases(rng_t *g, int32_t m, uint8_t *out)
{
    for (int32_t i = 0; i < m; ++i) out[i] = rbase(g);
}

/* Mutate read[0..m) at per-base event probability d; returns the length. */
SYNTH_FN int64_t mutate(rng_t *g, const uint8_t *read, int32_t m, double d, double indel_share, uint8_t *out)
{
    int64_t n = 0;
    const double p_indel = d * indel_share;
    for (int32_t i = 0; i < m; ++i) {
        const double u = runif(g);
        if (u < p_indel) {
            const int32_t len = (int32_t)rint_in(g, 1, 3);
            if (rnext(g) & 1u) {               /* insertion after this base */
                out[n++] = read[i];
                for (int32_t k = 0; k < len; ++k) out[n++] = rbase(g);
            } else {                           /* deletion of len read bases */
                i += len - 1;
            }
        } else if (u < d) {
            out[n++] = (uint8_t)((read[i] + 1 + rint_in(g, 0, 2)) & 3);
        } else {
            out[n++] = read[i];
        }
    }
    return n;
}

/* Longest read of a spec, and the longest body (mutated read plus intron)
 * that make_window keeps in its scratch buffer. */
SYNTH_FN int32_t max_read_len(const synth_spec_t *s)
{
    int32_t mx = 0;
    for (int k = 0; k < s->n_len; ++k) if (s->len_val[k] > mx) mx = s->len_val[k];
    return mx;
}
SYNTH_FN int64_t max_body_len(const synth_spec_t *s)
{
    return 4 * (int64_t)max_read_len(s) + s->intron_max + 4;
}

/*
 * Make candidate window k of a read: its bases go to `out` in order, tmp
 * (max_body_len bytes) is scratch.  Returns its length and writes its kind.
 */
SYNTH_FN int64_t make_window(const synth_spec_t *s, const rng_t *rg, const read_hdr_t *h,
                             const uint8_t *read, int64_t k, synth_sink_t *out, uint8_t *tmp, uint8_t *kind)
{
    rng_t g = cand_rng(rg, k);
    int kd;
    if (h->c == 1 && s->cand_max == 1)
        kd = runif(&g) < s->decoy_random ? KIND_RANDOM : KIND_TRUE;
    else if (k == h->t)
        kd = KIND_TRUE;
    else
        kd = runif(&g) < s->paralog_share ? KIND_PARALOG : KIND_RANDOM;
    *kind = (uint8_t)kd;

    int64_t body = 0;
    if (kd != KIND_RANDOM) {
        const double lo = kd == KIND_TRUE ? s->div_lo : s->par_lo;
        const double hi = kd == KIND_TRUE ? s->div_hi : s->par_hi;
        const double d = lo + (hi - lo) * runif(&g);
        body = mutate(&g, read, h->m, d, s->indel_share, tmp);
        if (kd == KIND_TRUE && h->spliced) {
            const int64_t il = rint_in(&g, s->intron_min, s->intron_max);
            const int64_t half = body / 2;
            for (int64_t q = body - 1; q >= half; --q) tmp[q + il] = tmp[q]; /* open the intron gap */
            for (int64_t q = 0; q < il; ++q) tmp[half + q] = rbase(&g);
            tmp[half] = 2; tmp[half + 1] = 3;             /* G T ... */
            tmp[half + il - 2] = 0; tmp[half + il - 1] = 2; /* ... A G */
            body += il;
        }
    }
    int64_t n;
    if (s->win_len > 0) {
        n = s->win_len;
        if (kd == KIND_RANDOM) {
            for (int64_t q = 0; q < n; ++q) synth_put(out, rbase(&g));
        } else if (body >= n) {
            for (int64_t q = 0; q < n; ++q) synth_put(out, tmp[q]);
        } else {
            const int64_t off = rint_in(&g, 0, n - body);
            for (int64_t q = 0; q < off; ++q) synth_put(out, rbase(&g));
            for (int64_t q = 0; q < body; ++q) synth_put(out, tmp[q]);
            for (int64_t q = off + body; q < n; ++q) synth_put(out, rbase(&g));
        }
    } else {
        const int64_t f1 = rint_in(&g, s->flank_min, s->flank_max);
        const int64_t f2 = rint_in(&g, s->flank_min, s->flank_max);
        if (kd == KIND_RANDOM) {
            n = h->m + f1 + f2;
            for (int64_t q = 0; q < n; ++q) synth_put(out, rbase(&g));
        } else {
            n = f1 + body + f2;
            for (int64_t q = 0; q < f1; ++q) synth_put(out, rbase(&g));
            for (int64_t q = 0; q < body; ++q) synth_put(out, tmp[q]);
            for (int64_t q = f1 + body; q < n; ++q) synth_put(out, rbase(&g));
        }
    }
    return n;
}

#endif /* SYNTH_CORE_H */
