/*
 * synth.c -- seeded synthetic (read, candidate window) workloads.
 *
 * This module only makes inputs; it holds none of the alignment arithmetic.
 * Both the oracle and the CUDA path consume what it writes.
 *
 * Shapes follow the paper's Stage E inputs: each read is aligned against its
 * extended candidate alignment locations (CALs) -- the reference region its
 * seeds point to, extended by flanks on both sides -- and, for reads that
 * span a splice junction, against a joined extended CAL that holds both exon
 * halves with the intron between them.  There is no reference genome here, so
 * windows are made directly:
 *
 *   true window     the read, mutated (substitutions + indels of length 1-3),
 *                   embedded in random flanks; for a spliced read the mutated
 *                   read is cut in two halves with a random intron between
 *                   them that starts with GT and ends with AG;
 *   paralog decoy   the read mutated at a higher divergence, in flanks;
 *   random decoy    i.i.d. uniform bases.
 *
 * Randomness: a counter-based generator built from the splitmix64 mixing
 * function (Steele, Lea & Flood 2014; the finaliser constants are those
 * published with it).  Every read r gets a stream keyed by (seed, r), every
 * candidate k of read r a stream keyed by (read key, k), so the output does
 * not depend on the thread count.
 *
 * Base codes: A=0, C=1, G=2, T=3, one byte per base.  synth_pack() writes the
 * 2-bit packed form (4 bases per byte, first base in the low bits).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

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
} synth_spec_t;

enum { KIND_TRUE = 0, KIND_PARALOG = 1, KIND_RANDOM = 2 };

static inline uint64_t mix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

typedef struct { uint64_t key, ctr; uint64_t bits; int nbits; } rng_t;

static inline uint64_t rnext(rng_t *g) { return mix64(g->key ^ mix64(g->ctr++)); }
static inline double runif(rng_t *g) { return (double)(rnext(g) >> 11) * (1.0 / 9007199254740992.0); }
static inline int64_t rint_in(rng_t *g, int64_t lo, int64_t hi) /* inclusive */
{
    return lo + (int64_t)(rnext(g) % (uint64_t)(hi - lo + 1));
}
static inline uint8_t rbase(rng_t *g)
{
    if (g->nbits == 0) { g->bits = rnext(g); g->nbits = 32; }
    uint8_t b = (uint8_t)(g->bits & 3u);
    g->bits >>= 2; g->nbits--;
    return b;
}

static rng_t read_rng(const synth_spec_t *s, int64_t r)
{
    rng_t g = {mix64(s->seed * 0xD1B54A32D192ED03ULL ^ mix64((uint64_t)r)), 0, 0, 0};
    return g;
}
static rng_t cand_rng(const rng_t *rg, int64_t k)
{
    rng_t g = {mix64(rg->key + 0x632BE59BD9B4E019ULL * (uint64_t)(k + 1)), 0, 0, 0};
    return g;
}

/* Per-read header draws, in a fixed order. */
typedef struct { int32_t m, c, t, spliced; } read_hdr_t;

static read_hdr_t read_header(const synth_spec_t *s, rng_t *g)
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

static void read_bases(rng_t *g, int32_t m, uint8_t *out)
{
    for (int32_t i = 0; i < m; ++i) out[i] = rbase(g);
}

/* Mutate read[0..m) at per-base event probability d; returns the length. */
static int64_t mutate(rng_t *g, const uint8_t *read, int32_t m, double d, double indel_share, uint8_t *out)
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

/*
 * Make candidate window k of a read into out (capacity checked by caller).
 * Returns its length and writes its kind.
 */
static int64_t make_window(const synth_spec_t *s, const rng_t *rg, const read_hdr_t *h,
                           const uint8_t *read, int64_t k, uint8_t *out, uint8_t *tmp, uint8_t *kind)
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
            memmove(tmp + half + il, tmp + half, (size_t)(body - half));
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
            for (int64_t q = 0; q < n; ++q) out[q] = rbase(&g);
        } else if (body >= n) {
            memcpy(out, tmp, (size_t)n);
        } else {
            const int64_t off = rint_in(&g, 0, n - body);
            for (int64_t q = 0; q < off; ++q) out[q] = rbase(&g);
            memcpy(out + off, tmp, (size_t)body);
            for (int64_t q = off + body; q < n; ++q) out[q] = rbase(&g);
        }
    } else {
        const int64_t f1 = rint_in(&g, s->flank_min, s->flank_max);
        const int64_t f2 = rint_in(&g, s->flank_min, s->flank_max);
        if (kd == KIND_RANDOM) {
            n = h->m + f1 + f2;
            for (int64_t q = 0; q < n; ++q) out[q] = rbase(&g);
        } else {
            n = f1 + body + f2;
            for (int64_t q = 0; q < f1; ++q) out[q] = rbase(&g);
            memcpy(out + f1, tmp, (size_t)body);
            for (int64_t q = f1 + body; q < n; ++q) out[q] = rbase(&g);
        }
    }
    return n;
}

static int32_t max_read_len(const synth_spec_t *s)
{
    int32_t mx = 0;
    for (int k = 0; k < s->n_len; ++k) if (s->len_val[k] > mx) mx = s->len_val[k];
    return mx;
}
static int64_t max_window_len(const synth_spec_t *s)
{
    const int64_t mm = max_read_len(s);
    int64_t body = 4 * mm + s->intron_max + 4;
    int64_t w = s->win_len > 0 ? s->win_len : body + 2 * (int64_t)s->flank_max + mm;
    return w > body ? w : body;
}

/* ------------------------------------------------------------------------ */

typedef struct {
    const synth_spec_t *s;
    int64_t r0, r1;
    int mode;                 /* 0 headers, 1 window sizes, 2 fill */
    int32_t *read_len, *n_cand;
    const int64_t *cand_off, *read_off, *win_off;
    int32_t *win_len;
    uint8_t *read_codes, *win_codes, *kinds;
    int32_t *true_cand;
    int rc;
} job_t;

static void *worker(void *arg)
{
    job_t *jb = (job_t *)arg;
    const synth_spec_t *s = jb->s;
    const int64_t wmax = max_window_len(s);
    uint8_t *rb = NULL, *wb = NULL, *tb = NULL;
    if (jb->mode >= 1) {
        rb = (uint8_t *)malloc((size_t)max_read_len(s) + 16);
        wb = (uint8_t *)malloc((size_t)wmax + 16);
        tb = (uint8_t *)malloc((size_t)wmax + 16);
        if (!rb || !wb || !tb) { jb->rc = -3; free(rb); free(wb); free(tb); return NULL; }
    }
    for (int64_t r = jb->r0; r < jb->r1; ++r) {
        rng_t g = read_rng(s, r);
        const read_hdr_t h = read_header(s, &g);
        if (jb->mode == 0) { jb->read_len[r] = h.m; jb->n_cand[r] = h.c; continue; }
        uint8_t *rdst = jb->mode == 2 ? jb->read_codes + jb->read_off[r] : rb;
        read_bases(&g, h.m, rdst);
        if (jb->mode == 2) jb->true_cand[r] = (s->cand_max == 1) ? 0 : h.t;
        for (int64_t k = 0; k < h.c; ++k) {
            const int64_t p = jb->cand_off[r] + k;
            uint8_t kind;
            if (jb->mode == 1) {
                jb->win_len[p] = (int32_t)make_window(s, &g, &h, rdst, k, wb, tb, &kind);
            } else {
                const int64_t n = make_window(s, &g, &h, rdst, k, jb->win_codes + jb->win_off[p], tb, &kind);
                if (n != jb->win_off[p + 1] - jb->win_off[p]) jb->rc = -2;
                jb->kinds[p] = kind;
            }
        }
    }
    free(rb); free(wb); free(tb);
    return NULL;
}

static int run_jobs(const synth_spec_t *s, job_t proto, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 128) nthreads = 128;
    pthread_t th[128];
    job_t jobs[128];
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = proto;
        jobs[t].r0 = s->n_reads * t / nthreads;
        jobs[t].r1 = s->n_reads * (t + 1) / nthreads;
        jobs[t].rc = 0;
    }
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, worker, &jobs[t]);
    worker(&jobs[0]);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
    for (int t = 0; t < nthreads; ++t) if (jobs[t].rc) return jobs[t].rc;
    return 0;
}

/* Pass 1: read lengths and candidate counts. */
int synth_headers(const synth_spec_t *s, int32_t *read_len, int32_t *n_cand, int nthreads)
{
    job_t p = {0};
    p.s = s; p.mode = 0; p.read_len = read_len; p.n_cand = n_cand;
    return run_jobs(s, p, nthreads);
}

/* Pass 2: window lengths (cand_off: n_reads+1 CSR of candidates). */
int synth_window_lengths(const synth_spec_t *s, const int64_t *cand_off, int32_t *win_len, int nthreads)
{
    job_t p = {0};
    p.s = s; p.mode = 1; p.cand_off = cand_off; p.win_len = win_len;
    return run_jobs(s, p, nthreads);
}

/* Pass 3: bases, kinds and the true candidate of each read. */
int synth_fill(const synth_spec_t *s, const int64_t *cand_off, const int64_t *read_off,
               const int64_t *win_off, uint8_t *read_codes, uint8_t *win_codes,
               uint8_t *kinds, int32_t *true_cand, int nthreads)
{
    job_t p = {0};
    p.s = s; p.mode = 2; p.cand_off = cand_off; p.read_off = read_off; p.win_off = win_off;
    p.read_codes = read_codes; p.win_codes = win_codes; p.kinds = kinds; p.true_cand = true_cand;
    return run_jobs(s, p, nthreads);
}

/* 2-bit packing: base q goes to byte q/4, bits 2*(q%4)..2*(q%4)+1. */
void synth_pack(const uint8_t *codes, int64_t n_bases, uint8_t *packed)
{
    const int64_t nb = (n_bases + 3) / 4;
    for (int64_t b = 0; b < nb; ++b) {
        uint8_t v = 0;
        for (int q = 0; q < 4; ++q) {
            const int64_t i = 4 * b + q;
            if (i < n_bases) v |= (uint8_t)((codes[i] & 3u) << (2 * q));
        }
        packed[b] = v;
    }
}

/* Inverse of synth_pack. */
void synth_unpack(const uint8_t *packed, int64_t n_bases, uint8_t *codes)
{
    for (int64_t i = 0; i < n_bases; ++i) codes[i] = (uint8_t)((packed[i >> 2] >> (2 * (i & 3))) & 3u);
}
