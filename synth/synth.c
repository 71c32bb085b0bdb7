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

/* Host sink of make_window: stores bases at p (count only when p is NULL). */
struct synth_sink { uint8_t *p; };
#define SYNTH_FN static inline
typedef struct synth_sink synth_sink_t;
SYNTH_FN void synth_put(synth_sink_t *o, uint8_t b)
{
    if (o->p) *o->p++ = b;
}
#include "synth_core.h"

static int64_t max_window_len(const synth_spec_t *s)
{
    const int64_t mm = max_read_len(s);
    const int64_t body = max_body_len(s);
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
    uint8_t *rb = NULL, *tb = NULL;
    if (jb->mode >= 1) {
        rb = (uint8_t *)malloc((size_t)max_read_len(s) + 16);
        tb = (uint8_t *)malloc((size_t)wmax + 16);
        if (!rb || !tb) { jb->rc = -3; free(rb); free(tb); return NULL; }
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
                synth_sink_t count = {NULL};
                jb->win_len[p] = (int32_t)make_window(s, &g, &h, rdst, k, &count, tb, &kind);
            } else {
                synth_sink_t store = {jb->win_codes + jb->win_off[p]};
                const int64_t n = make_window(s, &g, &h, rdst, k, &store, tb, &kind);
                if (n != jb->win_off[p + 1] - jb->win_off[p]) jb->rc = -2;
                jb->kinds[p] = kind;
            }
        }
    }
    free(rb); free(tb);
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

/* ======================================================================== */
/*
 * Reference genomes and reads sampled from them (the inputs of seeding).
 *
 * A genome is n_chrom chromosomes of random bases, back to back, 2-bit
 * packed (base q in byte q/4 at bits 2*(q%4)).  On top of the random bases:
 *
 *   repeat families  a source segment copied to several places with
 *                    per-base substitutions (paralogs: seeds with several
 *                    hits, reads with several candidate locations);
 *   introns          a span starting with GT and ending with AG (gene on the
 *                    forward strand) or CT ... AC (reverse strand), the
 *                    junctions spliced reads are sampled across.
 *
 * Reads follow the paper's simulated datasets: a fixed read length, per-base
 * error probability eps of which a share are indels of length 1..3 (the
 * rest substitutions), half of the reads from the reverse strand (reverse
 * complemented), a fraction spliced across one planted intron.
 */
typedef struct {
    uint64_t seed;
    int32_t n_chrom;
    int32_t pad0;
    double repeat_share;               /* genome share covered by repeat copies */
    int32_t rep_len_min, rep_len_max;
    int32_t rep_copies_min, rep_copies_max;
    double rep_div_lo, rep_div_hi;     /* per-base substitution probability of a copy */
    int64_t n_introns;
    int32_t intron_min, intron_max;
    int32_t margin;                    /* introns keep this far from chromosome ends */
    int32_t pad1;
} genome_spec_t;

static inline uint8_t gget(const uint8_t *pk, int64_t q) { return (uint8_t)((pk[q >> 2] >> (2 * (q & 3))) & 3u); }
static inline void gset(uint8_t *pk, int64_t q, uint8_t b)
{
    const int sh = 2 * (int)(q & 3);
    pk[q >> 2] = (uint8_t)((pk[q >> 2] & ~(3u << sh)) | ((uint32_t)(b & 3u) << sh));
}

typedef struct { const genome_spec_t *s; uint8_t *pk; int64_t b0, b1; } gfill_t;

/* Random bases, 4 per byte, byte range [b0, b1): stream per 1 MiB block. */
static void *gfill_worker(void *arg)
{
    gfill_t *j = (gfill_t *)arg;
    const int64_t BLK = 1 << 20;
    for (int64_t blk = j->b0 / BLK; blk * BLK < j->b1; ++blk) {
        rng_t g = {mix64(j->s->seed * 0x9FB21C651E98DF25ULL ^ mix64((uint64_t)blk + 0x51ED27ULL)), 0, 0, 0};
        const int64_t lo = blk * BLK > j->b0 ? blk * BLK : j->b0;
        const int64_t hi = (blk + 1) * BLK < j->b1 ? (blk + 1) * BLK : j->b1;
        for (int64_t b = blk * BLK; b < hi; b += 8) {
            const uint64_t x = rnext(&g);
            for (int q = 0; q < 8 && b + q < hi; ++q)
                if (b + q >= lo) j->pk[b + q] = (uint8_t)(x >> (8 * q));
        }
    }
    return NULL;
}

static int64_t pick_chrom(rng_t *g, const int64_t *off, int32_t n_chrom, int64_t need)
{
    /* a chromosome by length among those longer than `need`; -1 if none */
    int64_t tot = 0;
    for (int32_t c = 0; c < n_chrom; ++c) if (off[c + 1] - off[c] > need) tot += off[c + 1] - off[c];
    if (tot == 0) return -1;
    int64_t u = (int64_t)(rnext(g) % (uint64_t)tot);
    for (int32_t c = 0; c < n_chrom; ++c) {
        const int64_t L = off[c + 1] - off[c];
        if (L <= need) continue;
        if (u < L) return c;
        u -= L;
    }
    return n_chrom - 1;
}

/*
 * Fill `packed` ((off[n_chrom] + 3) / 4 bytes) and plant the features.
 * introns: n_introns rows of (chrom, global start, length, strand).
 * Returns 0, or -1 when a chromosome is too short for the features.
 */
int synth_genome(const genome_spec_t *s, const int64_t *off, uint8_t *packed, int64_t *introns, int nthreads)
{
    const int64_t G = off[s->n_chrom];
    const int64_t nbytes = (G + 3) / 4;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 128) nthreads = 128;
    pthread_t th[128];
    gfill_t jobs[128];
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].s = s; jobs[t].pk = packed;
        jobs[t].b0 = nbytes * t / nthreads; jobs[t].b1 = nbytes * (t + 1) / nthreads;
    }
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, gfill_worker, &jobs[t]);
    gfill_worker(&jobs[0]);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
    if (G & 3) packed[nbytes - 1] &= (uint8_t)((1u << (2 * (G & 3))) - 1u);

    /* repeat families, until repeat_share of the genome is covered */
    const int64_t target = (int64_t)(s->repeat_share * (double)G);
    uint8_t *src = (uint8_t *)malloc((size_t)s->rep_len_max + 1);
    if (!src) return -3;
    int64_t covered = 0;
    for (uint64_t f = 0; covered < target; ++f) {
        rng_t g = {mix64(s->seed * 0x2545F4914F6CDD1DULL ^ mix64(f + 0xA11CEULL)), 0, 0, 0};
        const int64_t L = rint_in(&g, s->rep_len_min, s->rep_len_max);
        const int64_t c = pick_chrom(&g, off, s->n_chrom, L);
        if (c < 0) { free(src); return -1; }
        const int64_t p = off[c] + rint_in(&g, 0, off[c + 1] - off[c] - L);
        for (int64_t t = 0; t < L; ++t) src[t] = gget(packed, p + t);
        const int64_t copies = rint_in(&g, s->rep_copies_min, s->rep_copies_max);
        for (int64_t k = 0; k < copies; ++k) {
            const double d = s->rep_div_lo + (s->rep_div_hi - s->rep_div_lo) * runif(&g);
            const int64_t c2 = pick_chrom(&g, off, s->n_chrom, L);
            const int64_t q = off[c2] + rint_in(&g, 0, off[c2 + 1] - off[c2] - L);
            for (int64_t t = 0; t < L; ++t) {
                uint8_t b = src[t];
                if (runif(&g) < d) b = (uint8_t)((b + 1 + rint_in(&g, 0, 2)) & 3);
                gset(packed, q + t, b);
            }
            covered += L;
        }
    }
    free(src);

    /* introns with their marks */
    for (int64_t i = 0; i < s->n_introns; ++i) {
        rng_t g = {mix64(s->seed * 0x94D049BB133111EBULL ^ mix64((uint64_t)i + 0x1A7C0ULL)), 0, 0, 0};
        const int64_t L = rint_in(&g, s->intron_min, s->intron_max);
        const int64_t c = pick_chrom(&g, off, s->n_chrom, L + 2 * (int64_t)s->margin);
        if (c < 0) return -1;
        const int64_t st = off[c] + s->margin + rint_in(&g, 0, off[c + 1] - off[c] - L - 2 * (int64_t)s->margin);
        const int strand = (int)(rnext(&g) & 1u);
        /* GT..AG = 2,3 .. 0,2 ; CT..AC = 1,3 .. 0,1 */
        gset(packed, st, strand ? 1 : 2);
        gset(packed, st + 1, 3);
        gset(packed, st + L - 2, 0);
        gset(packed, st + L - 1, strand ? 1 : 2);
        introns[4 * i + 0] = c;
        introns[4 * i + 1] = st;
        introns[4 * i + 2] = L;
        introns[4 * i + 3] = strand;
    }
    return 0;
}

typedef struct {
    uint64_t seed;
    int64_t n_reads;
    int32_t n_len;
    int32_t len_val[8];
    int32_t pad0;
    double len_w[8];
    double eps;            /* per-base error probability */
    double indel_share;    /* share of errors that are indels (length 1..3) */
    double splice_frac;    /* P(read spans one planted intron) */
    int32_t min_exon;      /* bases of the read on each side of the intron */
    int32_t pad1;
} reads_spec_t;

typedef struct {
    const reads_spec_t *rs;
    const int64_t *off;
    int32_t n_chrom;
    const uint8_t *pk;
    const int64_t *introns;
    int64_t n_introns;
    int64_t r0, r1;
    int mode;              /* 0 lengths, 1 fill */
    int32_t *len;
    const int64_t *read_off;
    uint8_t *codes;
    int32_t *t_chrom;
    int64_t *t_pos;
    int8_t *t_strand;
    int32_t *t_intron;
    int rc;
} rjob_t;

static rng_t sample_rng(const reads_spec_t *s, int64_t r)
{
    rng_t g = {mix64(s->seed * 0xE7037ED1A0B428DBULL ^ mix64((uint64_t)r + 0x5EEDULL)), 0, 0, 0};
    return g;
}

static void *reads_worker(void *arg)
{
    rjob_t *j = (rjob_t *)arg;
    const reads_spec_t *s = j->rs;
    for (int64_t r = j->r0; r < j->r1; ++r) {
        rng_t g = sample_rng(s, r);
        double u = runif(&g), tot = 0.0, acc = 0.0;
        for (int k = 0; k < s->n_len; ++k) tot += s->len_w[k];
        int32_t m = s->len_val[s->n_len - 1];
        for (int k = 0; k < s->n_len; ++k) {
            acc += s->len_w[k] / tot;
            if (u < acc) { m = s->len_val[k]; break; }
        }
        if (j->mode == 0) { j->len[r] = m; continue; }
        const int spliced = j->n_introns > 0 && runif(&g) < s->splice_frac && m >= 2 * s->min_exon;
        const int strand = (int)(rnext(&g) & 1u);
        /* template: reference positions pos(t) = a0 + t, jumping over the intron */
        int64_t a0, jump_at = -1, jump_to = 0, chrom;
        int32_t intron = -1;
        if (spliced) {
            intron = (int32_t)rint_in(&g, 0, j->n_introns - 1);
            const int64_t *in = j->introns + 4 * (int64_t)intron;
            const int64_t a = rint_in(&g, s->min_exon, m - s->min_exon);
            chrom = in[0];
            a0 = in[1] - a;
            jump_at = a;
            jump_to = in[1] + in[2];
        } else {
            chrom = pick_chrom(&g, j->off, j->n_chrom, 4 * (int64_t)m + 16);
            if (chrom < 0) { j->rc = -1; return NULL; }
            a0 = j->off[chrom] + rint_in(&g, 0, j->off[chrom + 1] - j->off[chrom] - 4 * (int64_t)m - 16);
        }
        uint8_t *out = j->codes + j->read_off[r];
        const double p_indel = s->eps * s->indel_share;
        int64_t t = 0;
        int32_t n = 0;
        while (n < m) {
            const int64_t q = (jump_at >= 0 && t >= jump_at) ? jump_to + (t - jump_at) : a0 + t;
            const uint8_t b = gget(j->pk, q);
            const double e = runif(&g);
            if (e < p_indel) {
                const int32_t len = (int32_t)rint_in(&g, 1, 3);
                if (rnext(&g) & 1u) {                   /* insertion before this base */
                    for (int32_t k = 0; k < len && n < m; ++k) out[n++] = rbase(&g);
                } else {                                /* deletion of len reference bases */
                    t += len;
                }
            } else if (e < s->eps) {
                out[n++] = (uint8_t)((b + 1 + rint_in(&g, 0, 2)) & 3);
                ++t;
            } else {
                out[n++] = b;
                ++t;
            }
        }
        if (strand) {
            for (int32_t a = 0, b = m - 1; a < b; ++a, --b) {
                const uint8_t x = out[a];
                out[a] = (uint8_t)(3 - out[b]);
                out[b] = (uint8_t)(3 - x);
            }
            if (m & 1) out[m / 2] = (uint8_t)(3 - out[m / 2]);
        }
        j->t_chrom[r] = (int32_t)chrom;
        j->t_pos[r] = a0 - j->off[chrom];
        j->t_strand[r] = (int8_t)strand;
        j->t_intron[r] = intron;
    }
    return NULL;
}

static int run_rjobs(rjob_t proto, int64_t n_reads, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 128) nthreads = 128;
    pthread_t th[128];
    rjob_t jobs[128];
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = proto;
        jobs[t].r0 = n_reads * t / nthreads;
        jobs[t].r1 = n_reads * (t + 1) / nthreads;
        jobs[t].rc = 0;
    }
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, reads_worker, &jobs[t]);
    reads_worker(&jobs[0]);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
    for (int t = 0; t < nthreads; ++t) if (jobs[t].rc) return jobs[t].rc;
    return 0;
}

/* Pass 1: read lengths. */
int synth_read_lengths(const reads_spec_t *s, int32_t *len, int nthreads)
{
    rjob_t p = {0};
    p.rs = s; p.mode = 0; p.len = len;
    return run_rjobs(p, s->n_reads, nthreads);
}

/*
 * Pass 2: read bases (codes at read_off) and the truth of each read: its
 * chromosome, the chromosome position of its first template base on the
 * forward strand, its strand, and the index of the intron it spans (-1).
 */
int synth_sample_reads(const reads_spec_t *s, const int64_t *off, int32_t n_chrom, const uint8_t *packed,
                       const int64_t *introns, int64_t n_introns, const int64_t *read_off, uint8_t *codes,
                       int32_t *t_chrom, int64_t *t_pos, int8_t *t_strand, int32_t *t_intron, int nthreads)
{
    rjob_t p = {0};
    p.rs = s; p.off = off; p.n_chrom = n_chrom; p.pk = packed; p.introns = introns; p.n_introns = n_introns;
    p.mode = 1; p.read_off = read_off; p.codes = codes;
    p.t_chrom = t_chrom; p.t_pos = t_pos; p.t_strand = t_strand; p.t_intron = t_intron;
    return run_rjobs(p, s->n_reads, nthreads);
}
