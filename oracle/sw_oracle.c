/*
 * sw_oracle.c -- plain CPU oracle for affine-gap Smith-Waterman (Gotoh).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * definition that the CUDA path is judged against.  Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * header, table or helper with the CUDA library.
 *
 * What it computes (Stage E, task iii of the paper: the read is aligned onto
 * each extended / joined candidate alignment location (CAL) with the
 * Smith-Waterman algorithm, which returns the alignment, its score and its
 * initial position).  The paper prints no recurrence, so the textbook Gotoh
 * definition is written out here with full int64 matrices:
 *
 *   H(i,0) = H(0,j) = 0,  E(i,0) = F(0,j) = -inf
 *   E(i,j) = max(H(i,j-1) + o, E(i,j-1) + e)          gap in the read  -> 'D'
 *   F(i,j) = max(H(i-1,j) + o, F(i-1,j) + e)          gap in the window-> 'I'
 *   H(i,j) = max(0, H(i-1,j-1) + s(r_i, w_j), E(i,j), F(i,j))
 *
 * so a gap of length k scores o + (k-1) e.  The score is max H (>= 0).
 * Scorings must satisfy match > 0, mismatch <= 0 and o <= e <= 0 (opening a
 * gap costs at least as much as extending it); otherwise the recurrence would
 * not score a gap run as o + (k-1) e.
 *
 * Readings (the paper is silent on all of these):
 *  - end cell: among cells with H == score, the smallest window index j,
 *    then the smallest read index i; score 0 gives end (-1,-1), empty CIGAR.
 *  - traceback from the end cell in state H: stop when H == 0; else prefer
 *    the diagonal (M), then E (D), then F (I).  In state E: if
 *    E(i,j) == H(i,j-1) + o the gap opens here (back to state H), else it
 *    extends.  State F likewise.
 *  - CIGAR: leading soft clip, the M/I/D runs, trailing soft clip; BAM
 *    encoding len << 4 | op with M=0, I=1, D=2, S=4; adjacent equal ops merge.
 *
 * Sequences are plain byte codes 0..3 (A,C,G,T), one byte per base.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define ORC_NEG_INF (INT64_MIN / 4)
#define OP_M 0u
#define OP_I 1u
#define OP_D 2u
#define OP_S 4u

static int64_t max2(int64_t a, int64_t b) { return a > b ? a : b; }

/* Append one op of length len to a CIGAR being built left to right, merging
 * with the previous run when the op is the same. */
static int cigar_push(uint32_t *ops, int64_t cap, int64_t *n, uint32_t op, int64_t len)
{
    if (len <= 0) return 0;
    if (*n > 0 && (ops[*n - 1] & 0xFu) == op) {
        ops[*n - 1] = (uint32_t)((((int64_t)(ops[*n - 1] >> 4)) + len) << 4) | op;
        return 0;
    }
    if (*n >= cap) return -1;
    ops[(*n)++] = (uint32_t)(len << 4) | op;
    return 0;
}

/*
 * Fill the three Gotoh matrices for read r[0..m) against window w[0..n).
 * Matrices are (m+1) x (n+1), row-major, index (i, j) -> i * (n+1) + j.
 */
static void gotoh_fill(const uint8_t *r, int64_t m, const uint8_t *w, int64_t n,
                       int64_t ma, int64_t mi, int64_t go, int64_t ge,
                       int64_t *H, int64_t *E, int64_t *F)
{
    const int64_t ld = n + 1;
    for (int64_t j = 0; j <= n; ++j) { H[j] = 0; E[j] = ORC_NEG_INF; F[j] = ORC_NEG_INF; }
    for (int64_t i = 1; i <= m; ++i) {
        H[i * ld] = 0; E[i * ld] = ORC_NEG_INF; F[i * ld] = ORC_NEG_INF;
        for (int64_t j = 1; j <= n; ++j) {
            const int64_t s = (r[i - 1] == w[j - 1]) ? ma : mi;
            const int64_t e = max2(H[i * ld + j - 1] + go, E[i * ld + j - 1] + ge);
            const int64_t f = max2(H[(i - 1) * ld + j] + go, F[(i - 1) * ld + j] + ge);
            int64_t h = H[(i - 1) * ld + j - 1] + s;
            h = max2(h, e);
            h = max2(h, f);
            h = max2(h, 0);
            E[i * ld + j] = e;
            F[i * ld + j] = f;
            H[i * ld + j] = h;
        }
    }
}

/*
 * Traceback in the filled matrices from cell (ie, je) (1-based matrix
 * coordinates) following the tie-break rules above.  Writes the CIGAR of the
 * whole read (soft clips included) and returns 0, or -1 on capacity overflow,
 * -2 on an inconsistent matrix.  i_end0 is the 0-based read index of the end
 * cell, which fixes the trailing soft clip.
 */
static int gotoh_traceback(const uint8_t *r, int64_t m, const uint8_t *w, int64_t n,
                           int64_t ma, int64_t mi, int64_t go, int64_t ge,
                           const int64_t *H, const int64_t *E, const int64_t *F,
                           int64_t ie, int64_t je, int64_t i_end0,
                           uint32_t *cigar, int64_t cap, int64_t *n_ops)
{
    const int64_t ld = n + 1;
    int64_t i = ie, j = je;
    int state = 0; /* 0 = H, 1 = E, 2 = F */
    /* reversed raw ops, one entry per alignment column */
    uint8_t *rev = (uint8_t *)malloc((size_t)(ie + je + 2));
    int64_t nrev = 0;
    if (!rev) return -2;
    (void)ge;
    for (;;) {
        if (state == 0) {
            const int64_t h = H[i * ld + j];
            if (h == 0) break;
            if (i < 1 || j < 1) { free(rev); return -2; }
            const int64_t s = (r[i - 1] == w[j - 1]) ? ma : mi;
            if (h == H[(i - 1) * ld + j - 1] + s) {
                rev[nrev++] = (uint8_t)OP_M; --i; --j;
            } else if (h == E[i * ld + j]) {
                state = 1;
            } else if (h == F[i * ld + j]) {
                state = 2;
            } else {
                free(rev); return -2;
            }
        } else if (state == 1) {
            if (j < 1) { free(rev); return -2; }
            rev[nrev++] = (uint8_t)OP_D;
            if (E[i * ld + j] == H[i * ld + j - 1] + go) state = 0;
            --j;
        } else {
            if (i < 1) { free(rev); return -2; }
            rev[nrev++] = (uint8_t)OP_I;
            if (F[i * ld + j] == H[(i - 1) * ld + j] + go) state = 0;
            --i;
        }
    }
    /* i is now the number of read bases before the alignment (1-based stop row) */
    int64_t n_out = 0;
    int rc = 0;
    rc |= cigar_push(cigar, cap, &n_out, OP_S, i);
    for (int64_t k = nrev - 1; k >= 0; --k) rc |= cigar_push(cigar, cap, &n_out, rev[k], 1);
    rc |= cigar_push(cigar, cap, &n_out, OP_S, m - 1 - i_end0);
    free(rev);
    *n_ops = n_out;
    return rc ? -1 : 0;
}

/* The three filled matrices, (m+1) x (n+1) row-major, for the pin tests. */
int sw_oracle_matrices(const uint8_t *r, int64_t m, const uint8_t *w, int64_t n,
                       int64_t ma, int64_t mi, int64_t go, int64_t ge,
                       int64_t *H, int64_t *E, int64_t *F)
{
    gotoh_fill(r, m, w, n, ma, mi, go, ge, H, E, F);
    return 0;
}

/*
 * Full-matrix alignment of one (read, window) pair.  Returns 0 on success,
 * -1 if the CIGAR does not fit in cap runs, -2 on an internal inconsistency,
 * -3 on allocation failure.  cigar may be NULL (score and end only).
 */
int sw_oracle_align(const uint8_t *r, int64_t m, const uint8_t *w, int64_t n,
                    int64_t ma, int64_t mi, int64_t go, int64_t ge,
                    int64_t *score, int64_t *i_end, int64_t *j_end,
                    uint32_t *cigar, int64_t cap, int64_t *n_ops)
{
    const int64_t cells = (m + 1) * (n + 1);
    int64_t *H = (int64_t *)malloc((size_t)cells * sizeof(int64_t));
    int64_t *E = (int64_t *)malloc((size_t)cells * sizeof(int64_t));
    int64_t *F = (int64_t *)malloc((size_t)cells * sizeof(int64_t));
    if (!H || !E || !F) { free(H); free(E); free(F); return -3; }
    gotoh_fill(r, m, w, n, ma, mi, go, ge, H, E, F);

    int64_t best = 0;
    for (int64_t i = 1; i <= m; ++i)
        for (int64_t j = 1; j <= n; ++j)
            best = max2(best, H[i * (n + 1) + j]);
    int64_t bi = -1, bj = -1;
    if (best > 0) {
        /* smallest j, then smallest i */
        for (int64_t j = 1; j <= n && bj < 0; ++j)
            for (int64_t i = 1; i <= m; ++i)
                if (H[i * (n + 1) + j] == best) { bi = i; bj = j; break; }
    }
    *score = best;
    *i_end = bi >= 0 ? bi - 1 : -1;
    *j_end = bj >= 0 ? bj - 1 : -1;
    int rc = 0;
    if (n_ops) *n_ops = 0;
    if (cigar && best > 0)
        rc = gotoh_traceback(r, m, w, n, ma, mi, go, ge, H, E, F, bi, bj, bi - 1,
                             cigar, cap, n_ops);
    free(H); free(E); free(F);
    return rc;
}

/*
 * Upper bound on the number of deletions (window bases consumed by gaps) in
 * any alignment with the given score that ends at read row i_end (0-based).
 * Such an alignment holds at most i_end+1 aligned read bases, each worth at
 * most `match`; insertions and mismatches never add score; and with
 * o <= e <= 0 the cheapest way to delete D >= 1 window bases is one run,
 * costing o + (D-1) e.  So score <= match (i_end+1) + o + (D-1) e, which gives
 * D <= (match (i_end+1) + o - score) / (-e) + 1.  Returns -1 when e == 0 (no
 * bound: the caller uses the whole window).
 */
int64_t sw_oracle_deletion_bound(int64_t i_end, int64_t score,
                                 int64_t ma, int64_t go, int64_t ge)
{
    if (ge == 0) return -1;
    const int64_t num = ma * (i_end + 1) + go - score;
    return num < 0 ? 0 : num / (-ge) + 1;
}

/*
 * Rectangle traceback: recompute the DP only over read rows 0..i_end and
 * window columns j_lo..j_end, where j_lo = j_end - i_end - D (D from
 * sw_oracle_deletion_bound), as a fresh local alignment, and trace back from
 * (i_end, j_end).  Every optimal alignment ending at the end cell lies in this
 * rectangle, so the CIGAR equals the full-matrix one; the tests check that.
 * Returns 0, -1 (capacity), -2 (inconsistent: the rectangle does not reach
 * the score), -3 (allocation).
 */
int sw_oracle_rect_traceback(const uint8_t *r, int64_t m, const uint8_t *w, int64_t n,
                             int64_t ma, int64_t mi, int64_t go, int64_t ge,
                             int64_t score, int64_t i_end, int64_t j_end,
                             uint32_t *cigar, int64_t cap, int64_t *n_ops,
                             int64_t *j_lo_out)
{
    *n_ops = 0;
    if (score <= 0) { if (j_lo_out) *j_lo_out = -1; return 0; }
    const int64_t dmax = sw_oracle_deletion_bound(i_end, score, ma, go, ge);
    int64_t j_lo = dmax < 0 ? 0 : j_end - i_end - dmax;
    if (j_lo < 0) j_lo = 0;
    if (j_lo_out) *j_lo_out = j_lo;
    const int64_t rm = i_end + 1, rn = j_end - j_lo + 1;
    (void)n;
    const int64_t cells = (rm + 1) * (rn + 1);
    int64_t *H = (int64_t *)malloc((size_t)cells * sizeof(int64_t));
    int64_t *E = (int64_t *)malloc((size_t)cells * sizeof(int64_t));
    int64_t *F = (int64_t *)malloc((size_t)cells * sizeof(int64_t));
    if (!H || !E || !F) { free(H); free(E); free(F); return -3; }
    gotoh_fill(r, rm, w + j_lo, rn, ma, mi, go, ge, H, E, F);
    int rc;
    if (H[rm * (rn + 1) + rn] != score) rc = -2;
    else rc = gotoh_traceback(r, m, w + j_lo, rn, ma, mi, go, ge, H, E, F, rm, rn, i_end,
                              cigar, cap, n_ops);
    free(H); free(E); free(F);
    return rc;
}

/*
 * Upper bound on the number of insertions (read bases aligned to gaps) in any
 * alignment with the given score that ends at read row i_end: I inserted
 * bases leave at most i_end+1-I aligned ones, and with o <= e <= 0 one run of
 * I costs at least o + (I-1) e, so
 * score <= match (i_end+1-I) + o + (I-1) e, i.e.
 * I <= (match (i_end+1) + o - e - score) / (match - e).
 */
int64_t sw_oracle_insertion_bound(int64_t i_end, int64_t score, int64_t ma, int64_t go, int64_t ge)
{
    const int64_t num = ma * (i_end + 1) + go - ge - score;
    return num < 0 ? 0 : num / (ma - ge);
}

/*
 * Band traceback: like the rectangle traceback, but cells whose diagonal
 * d = j - i lies outside [j_end - i_end - D, j_end - i_end + I] are treated
 * as unreachable (H = 0, E = F = -inf).  Walking back from the end cell, every
 * deletion lowers d by one and every insertion raises it by one, so every
 * optimal alignment ending there stays inside the band.  Returns as
 * sw_oracle_rect_traceback.
 */
int sw_oracle_band_traceback(const uint8_t *r, int64_t m, const uint8_t *w, int64_t n,
                             int64_t ma, int64_t mi, int64_t go, int64_t ge,
                             int64_t score, int64_t i_end, int64_t j_end,
                             uint32_t *cigar, int64_t cap, int64_t *n_ops)
{
    *n_ops = 0;
    if (score <= 0) return 0;
    (void)n;
    const int64_t dmax = sw_oracle_deletion_bound(i_end, score, ma, go, ge);
    const int64_t imax = sw_oracle_insertion_bound(i_end, score, ma, go, ge);
    const int64_t dend = j_end - i_end;
    const int64_t dlo = dmax < 0 ? -(i_end + 1) - 1 : dend - dmax;
    const int64_t dhi = dend + imax;
    const int64_t rm = i_end + 1, rn = j_end + 1;
    const int64_t ld = rn + 1, cells = (rm + 1) * ld;
    int64_t *H = (int64_t *)malloc((size_t)cells * sizeof(int64_t));
    int64_t *E = (int64_t *)malloc((size_t)cells * sizeof(int64_t));
    int64_t *F = (int64_t *)malloc((size_t)cells * sizeof(int64_t));
    if (!H || !E || !F) { free(H); free(E); free(F); return -3; }
    for (int64_t k = 0; k < cells; ++k) { H[k] = 0; E[k] = ORC_NEG_INF; F[k] = ORC_NEG_INF; }
    for (int64_t i = 1; i <= rm; ++i) {
        for (int64_t j = 1; j <= rn; ++j) {
            const int64_t d = (j - 1) - (i - 1);
            if (d < dlo || d > dhi) continue;      /* outside the band */
            const int64_t s = (r[i - 1] == w[j - 1]) ? ma : mi;
            const int64_t e = max2(H[i * ld + j - 1] + go, E[i * ld + j - 1] + ge);
            const int64_t f = max2(H[(i - 1) * ld + j] + go, F[(i - 1) * ld + j] + ge);
            int64_t h = max2(max2(H[(i - 1) * ld + j - 1] + s, e), max2(f, 0));
            E[i * ld + j] = e;
            F[i * ld + j] = f;
            H[i * ld + j] = h;
        }
    }
    int rc;
    if (H[rm * ld + rn] != score) rc = -2;
    else rc = gotoh_traceback(r, m, w, rn, ma, mi, go, ge, H, E, F, rm, rn, i_end, cigar, cap, n_ops);
    free(H); free(E); free(F);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Batch driver: pairs split across pthreads (used for the CPU baseline).    */

typedef struct {
    const uint8_t *reads; const int64_t *roff;
    const uint8_t *wins; const int64_t *woff;
    const int64_t *pair_read;        /* NULL: pair p uses read p */
    int64_t ma, mi, go, ge;
    int64_t *score, *i_end, *j_end;
    uint32_t *cigar; const int64_t *cig_off; int64_t *n_ops;
    int64_t p0, p1;
    int rc;
} batch_job_t;

static void *batch_worker(void *arg)
{
    batch_job_t *jb = (batch_job_t *)arg;
    for (int64_t p = jb->p0; p < jb->p1; ++p) {
        const int64_t rd = jb->pair_read ? jb->pair_read[p] : p;
        const int64_t m = jb->roff[rd + 1] - jb->roff[rd];
        const int64_t n = jb->woff[p + 1] - jb->woff[p];
        int64_t nops = 0;
        uint32_t *cg = jb->cigar ? jb->cigar + jb->cig_off[p] : NULL;
        const int64_t cap = jb->cigar ? jb->cig_off[p + 1] - jb->cig_off[p] : 0;
        int rc = sw_oracle_align(jb->reads + jb->roff[rd], m, jb->wins + jb->woff[p], n,
                                 jb->ma, jb->mi, jb->go, jb->ge,
                                 &jb->score[p], &jb->i_end[p], &jb->j_end[p],
                                 cg, cap, &nops);
        if (jb->n_ops) jb->n_ops[p] = nops;
        if (rc && !jb->rc) jb->rc = rc;
    }
    return NULL;
}

int sw_oracle_batch(const uint8_t *reads, const int64_t *roff,
                    const uint8_t *wins, const int64_t *woff,
                    const int64_t *pair_read, int64_t n_pairs,
                    int64_t ma, int64_t mi, int64_t go, int64_t ge,
                    int64_t *score, int64_t *i_end, int64_t *j_end,
                    uint32_t *cigar, const int64_t *cig_off, int64_t *n_ops,
                    int n_threads)
{
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    pthread_t th[256];
    batch_job_t jobs[256];
    int rc = 0;
    for (int t = 0; t < n_threads; ++t) {
        jobs[t] = (batch_job_t){reads, roff, wins, woff, pair_read, ma, mi, go, ge,
                                score, i_end, j_end, cigar, cig_off, n_ops,
                                n_pairs * t / n_threads, n_pairs * (t + 1) / n_threads, 0};
    }
    for (int t = 1; t < n_threads; ++t) pthread_create(&th[t], NULL, batch_worker, &jobs[t]);
    batch_worker(&jobs[0]);
    for (int t = 1; t < n_threads; ++t) pthread_join(th[t], NULL);
    for (int t = 0; t < n_threads; ++t) if (jobs[t].rc && !rc) rc = jobs[t].rc;
    return rc;
}
