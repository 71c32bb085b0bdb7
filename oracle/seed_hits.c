/*
 * seed_hits.c -- every place a set of k-mers occurs in a reference.
 * TEST INFRASTRUCTURE ONLY (part of the seeding oracle).
 *
 * The definition is direct: position q of the reference is a hit of k-mer x
 * when bases q .. q+k-1 lie in one chromosome and equal x.  The scan walks
 * the reference once, keeping the code of the last k bases; a code is looked
 * up by binary search in the sorted query codes (a small bit filter skips
 * most positions first).  Codes here put the first base in the most
 * significant two bits.  Positions come out in increasing order per query.
 *
 * Reference: 2-bit packed, base q in byte q/4 at bits 2*(q%4).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static int find_code(const uint32_t *codes, int64_t n, uint32_t x)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) / 2;
        if (codes[mid] < x) lo = mid + 1; else hi = mid;
    }
    return (lo < n && codes[lo] == x) ? (int)lo : -1;
}

#define FILTER_BITS 22

static uint32_t filter_slot(uint32_t x) { return (uint32_t)(((uint64_t)x * 0x9E3779B1u) >> (32 - FILTER_BITS)) & ((1u << FILTER_BITS) - 1u); }

/*
 * codes: n_codes distinct k-mer codes, sorted ascending.
 * Pass 1 (positions == NULL): counts[i] = hits of codes[i].
 * Pass 2: positions[offsets[i] ...] = the hits of codes[i], ascending.
 * Returns 0, or -1 for a bad k.
 */
int seed_hits(const uint8_t *packed, const int64_t *chrom_off, int32_t n_chrom, int32_t k,
              const uint32_t *codes, int64_t n_codes, int64_t *counts, const int64_t *offsets, int64_t *positions)
{
    if (k < 1 || k > 16) return -1;
    uint8_t *filter = (uint8_t *)calloc((size_t)1 << (FILTER_BITS - 3), 1);
    int64_t *fill = NULL;
    if (!filter) return -3;
    for (int64_t i = 0; i < n_codes; ++i) {
        const uint32_t s = filter_slot(codes[i]);
        filter[s >> 3] |= (uint8_t)(1u << (s & 7));
    }
    if (positions) {
        fill = (int64_t *)calloc((size_t)(n_codes > 0 ? n_codes : 1), sizeof(int64_t));
        if (!fill) { free(filter); return -3; }
    } else {
        memset(counts, 0, sizeof(int64_t) * (size_t)n_codes);
    }
    const uint32_t mask = (k == 16) ? 0xFFFFFFFFu : ((1u << (2 * k)) - 1u);
    for (int32_t c = 0; c < n_chrom; ++c) {
        uint32_t x = 0;
        int32_t have = 0;   /* bases of the current chromosome in x */
        for (int64_t q = chrom_off[c]; q < chrom_off[c + 1]; ++q) {
            const uint32_t b = (packed[q >> 2] >> (2 * (q & 3))) & 3u;
            x = ((x << 2) | b) & mask;
            if (++have < k) continue;
            const uint32_t s = filter_slot(x);
            if (!(filter[s >> 3] & (1u << (s & 7)))) continue;
            const int i = find_code(codes, n_codes, x);
            if (i < 0) continue;
            const int64_t start = q - k + 1;
            if (positions) positions[offsets[i] + fill[i]++] = start;
            else counts[i]++;
        }
    }
    free(filter);
    free(fill);
    return 0;
}
