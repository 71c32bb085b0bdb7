/*
 * swgb_seed.h -- seeding: reads to the reference windows that sw_batch_align
 * aligns them against (the paper's Stage C region seeker, Stage D CAL
 * seeker, and Stage E tasks i-ii, CAL extension and joining).
 *
 * Part of libswgb (the same library as swgb.h; error codes, sequence packing
 * and streams as documented there).  All pointers are device memory unless
 * stated otherwise.
 *
 * Pipeline of one batch:
 *   sw_index_build        once per reference: the k-mer index
 *   sw_seed_windows       reads -> windows (read, strand, reference span)
 *   sw_reads_two_strands  each read and its reverse complement
 *   sw_extract_windows    windows' bases out of the reference
 *   sw_batch_align_indexed (swgb.h) with pair_read from sw_seed_windows
 *   sw_records, sw_junctions_detect, sw_best_per_read (swgb.h)
 */
#ifndef SWGB_SEED_H
#define SWGB_SEED_H

#include "swgb.h"

#ifdef __cplusplus
extern "C" {
#endif

#define SW_SEED_MAX_READ_LEN 1024   /* longer reads -> SW_ERR_DEVICE_INPUT */
#define SW_SEED_MAX_HITS 1024       /* bound on max_hits (see sw_seed_params_t) */
#define SW_SEED_MAX_LIST 32768      /* hits one read-strand may keep, see below */

/*
 * Reference index.  The reference is n_chrom chromosomes back to back,
 * 2-bit packed (swgb.h packing; the buffer 16-byte aligned and readable
 * through ceil(n_bases / 16) 32-bit words), n_bases < 2^32 - 1;
 * chrom_offsets (device int64[n_chrom + 1]) holds the first base of each
 * chromosome and n_bases at the end (off[0] == 0, non-decreasing).
 *
 * A k-mer's code puts its first base in the two lowest bits (code =
 * sum base_t * 4^t).  The index is a table of 4^k uint32 entries
 * (sw_index_table_words) and a positions array with one uint32 slot per
 * reference position: the bucket of code x is positions[lo .. hi) with
 * lo = x ? table[x - 1] : 0 and hi = table[x]; it holds every position q
 * whose k bases lie in one chromosome and equal x, in no particular order.
 * *out_n_positions (device int64) receives the number of indexed
 * positions.  8 <= k <= 16 (the table of k = 15 takes 4 GiB, k = 16 16 GiB).
 * Offsets that fail the checks above set SW_ERR_DEVICE_INPUT (read with
 * sw_sync_status) and leave the index unspecified.
 */
int64_t sw_index_table_words(int32_t k);
int sw_index_build(const uint8_t *genome, int64_t n_bases, const int64_t *chrom_offsets, int32_t n_chrom,
                   int32_t k, uint32_t *table, uint32_t *positions, int64_t *out_n_positions, sw_stream_t stream);

/*
 * Seeding parameters (host struct).  The paper's defaults where it gives
 * them: k = 15 (§2, Stage C), two phases starting at the first and the
 * eighth base (phase 7) with seeds every `stride` = 12 bases (a 100-base
 * read gives 8 + 7 seeds, as in the paper's example), flank = 30 (Stage E,
 * task i).  The rest are open in the paper:
 *   max_hits     a seed with more hits than this is dropped (repeats)
 *   merge_dist   regions merge when fewer bases than this lie between them
 *   min_cal_len  a merged region is a CAL when it spans more bases than
 *                this; must be >= k (a CAL holds at least two seed hits)
 *   max_intron   extended CALs join when fewer bases than this lie between
 *                them (the longest known intron)
 *   max_window   no window spans more bases; an extended CAL longer than
 *                this on its own is dropped (<= SW_MAX_WINDOW_LEN)
 * Requires 1 <= stride, 0 <= phase <= SW_SEED_MAX_READ_LEN, 1 <= max_hits
 * <= SW_SEED_MAX_HITS, merge_dist, flank, max_intron >= 0, and that a read
 * of SW_SEED_MAX_READ_LEN bases can keep at most SW_SEED_MAX_LIST hits:
 * (seeds of such a read) * max_hits rounded up to a power of two <=
 * SW_SEED_MAX_LIST (SW_ERR_UNSUPPORTED otherwise).
 */
typedef struct {
    int32_t k;
    int32_t stride;
    int32_t phase;
    int32_t max_hits;
    int32_t merge_dist;
    int32_t min_cal_len;
    int32_t flank;
    int32_t max_intron;
    int32_t max_window;
} sw_seed_params_t;

/* Output arrays of sw_seed_windows (a host struct of device pointers, each
 * with `capacity` entries, cand_offsets with n_reads + 1). */
typedef struct {
    int64_t *start;        /* reference position of the window's first base */
    int32_t *length;       /* bases */
    int32_t *chrom;        /* chromosome */
    int64_t *pos;          /* start - chrom_offsets[chrom] */
    int8_t *strand;        /* 0: the read, 1: its reverse complement */
    int64_t *pair_read;    /* read + strand * n_reads (see sw_reads_two_strands) */
    int64_t *cand_offsets; /* windows of read r: cand_offsets[r] .. cand_offsets[r + 1] */
} sw_windows_t;

/*
 * sw_seed_windows -- the windows of every read (Stages C, D, E i-ii).
 *
 * For read r and strand s (s = 1: the steps run on the read's reverse
 * complement), every seed (k bases at 0, stride, 2 stride, ... and at
 * phase, phase + stride, ...) with at most max_hits hits contributes the
 * regions [q, q + k - 1] of its hits; regions in reference order merge when
 * they lie in one chromosome with fewer than merge_dist bases between a
 * region and the merged region before it; a merged region spanning more
 * than min_cal_len bases is a CAL; it is extended by flank bases on both
 * sides within its chromosome; in reference order an extended CAL joins the
 * window before it when they lie in one chromosome, fewer than max_intron
 * bases lie between them and the joined window spans at most max_window
 * bases.  Windows come out per read, strand 0 before strand 1, in reference
 * order; *out_count (device int64) receives their number.
 *
 * reads, read_offsets: packed reads (n_reads + 1 offsets, non-decreasing);
 * reads of more than SW_SEED_MAX_READ_LEN bases set SW_ERR_DEVICE_INPUT.
 * table, positions: an index built with the same k.  When more than
 * `capacity` windows result, SW_ERR_CAPACITY is set, *out_count holds the
 * number needed and the outputs are incomplete.  Device-detected errors are
 * read with sw_sync_status.  Stream-ordered, no host synchronisation.
 */
int sw_seed_windows(const uint32_t *table, const uint32_t *positions, const int64_t *chrom_offsets,
                    int32_t n_chrom, const sw_seed_params_t *params, const uint8_t *reads,
                    const int64_t *read_offsets, int64_t n_reads, const sw_windows_t *out, int64_t capacity,
                    int64_t *out_count, sw_stream_t stream);

/*
 * sw_seed_stats -- after waiting for `stream`: out3[0] = seed lookups,
 * out3[1] = hits kept, out3[2] = 32-byte sectors of the table and the kept
 * buckets those lookups read, in the stream's last sw_seed_windows call
 * (the random reads that bound seeding).  SW_ERR_INVALID_ARG before the
 * stream's first call.
 */
int sw_seed_stats(sw_stream_t stream, int64_t *out3);


/*
 * sw_reads_two_strands -- out holds read r at offsets r and its reverse
 * complement at n_reads + r: out_offsets[i] (int64[2 n_reads + 1]) =
 * read_offsets[i] for i < n_reads, total + read_offsets[i - n_reads] after,
 * with total = read_offsets[n_reads] (read_offsets[0] must be 0).  out
 * holds cap_bases bases (2-bit packed, 16-byte aligned); 2 * total >
 * cap_bases sets SW_ERR_CAPACITY.
 */
int sw_reads_two_strands(const uint8_t *reads, const int64_t *read_offsets, int64_t n_reads, uint8_t *out,
                         int64_t cap_bases, int64_t *out_offsets, sw_stream_t stream);

/*
 * sw_extract_windows -- the bases of windows start[w] .. start[w] +
 * length[w] - 1 of the reference, back to back in `out` (2-bit packed,
 * 16-byte aligned, cap_bases bases), with out_offsets (int64[n_windows + 1])
 * their CSR offsets.  A window that does not fit sets SW_ERR_CAPACITY and is
 * not written.  n_windows is a host count (sw_seed_windows' *out_count).
 */
int sw_extract_windows(const uint8_t *genome, int64_t n_bases, const int64_t *start, const int32_t *length,
                       int64_t n_windows, uint8_t *out, int64_t cap_bases, int64_t *out_offsets,
                       sw_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* SWGB_SEED_H */
