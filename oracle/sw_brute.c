/*
 * sw_brute.c -- exhaustive enumeration of local alignments (tiny inputs).
 *
 * TEST INFRASTRUCTURE ONLY: this is the independent pin for the Gotoh oracle
 * in sw_oracle.c.  It uses no recurrence at all.  It walks every alignment
 * path -- every start cell (i0, j0) of the (m+1) x (n+1) grid, followed by
 * every sequence of M (consume a read and a window base), D (consume a window
 * base) and I (consume a read base) moves -- scores it directly from the
 * definition of the affine gap model (a gap run of length k costs o+(k-1)e,
 * an aligned pair costs match or mismatch), and records, per end cell and per
 * last move, the best score seen.
 *
 * From those three tables the local-alignment quantities follow by their
 * plain definitions: the best score of any alignment ending at (i, j)
 * (floored at 0, the empty alignment), the best ending with a deletion and
 * the best ending with an insertion.  The exhaustive walk is exponential, so
 * it is only used for m, n <= 7.
 */
#include <stdint.h>
#include <string.h>

#define BR_NEG (INT64_MIN / 4)
enum { MV_NONE = 0, MV_M = 1, MV_D = 2, MV_I = 3 };

typedef struct {
    const uint8_t *r, *w;
    int64_t m, n, ma, mi, go, ge;
    int64_t *bm, *bd, *bi; /* (m+1) x (n+1) best score ending with M / D / I */
} brute_ctx_t;

static void walk(const brute_ctx_t *c, int64_t i, int64_t j, int last, int64_t sc)
{
    const int64_t ld = c->n + 1;
    if (last == MV_M && sc > c->bm[i * ld + j]) c->bm[i * ld + j] = sc;
    if (last == MV_D && sc > c->bd[i * ld + j]) c->bd[i * ld + j] = sc;
    if (last == MV_I && sc > c->bi[i * ld + j]) c->bi[i * ld + j] = sc;
    if (i < c->m && j < c->n)
        walk(c, i + 1, j + 1, MV_M, sc + (c->r[i] == c->w[j] ? c->ma : c->mi));
    if (j < c->n)
        walk(c, i, j + 1, MV_D, sc + (last == MV_D ? c->ge : c->go));
    if (i < c->m)
        walk(c, i + 1, j, MV_I, sc + (last == MV_I ? c->ge : c->go));
}

/*
 * Fill best_m / best_d / best_i, each (m+1) x (n+1) int64 row-major, with the
 * best score over all alignment paths that end at that grid point with that
 * last move (BR_NEG where no such path exists).  Returns 0, or -1 if the
 * input is too large for enumeration.
 */
int sw_brute_tables(const uint8_t *r, int64_t m, const uint8_t *w, int64_t n,
                    int64_t ma, int64_t mi, int64_t go, int64_t ge,
                    int64_t *best_m, int64_t *best_d, int64_t *best_i)
{
    if (m < 0 || n < 0 || m > 8 || n > 8) return -1;
    const int64_t cells = (m + 1) * (n + 1);
    for (int64_t k = 0; k < cells; ++k) { best_m[k] = BR_NEG; best_d[k] = BR_NEG; best_i[k] = BR_NEG; }
    brute_ctx_t c = {r, w, m, n, ma, mi, go, ge, best_m, best_d, best_i};
    for (int64_t i0 = 0; i0 <= m; ++i0)
        for (int64_t j0 = 0; j0 <= n; ++j0)
            walk(&c, i0, j0, MV_NONE, 0);
    return 0;
}
