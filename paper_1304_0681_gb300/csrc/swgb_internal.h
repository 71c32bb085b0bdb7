// swgb_internal.h -- declarations shared by the library's translation units.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/swgb.h"

namespace swgb {

// Inputs of one batch as the kernels see them (all device pointers).
struct PairSet {
    const uint32_t *reads;      // packed reads (words)
    const int64_t *read_off;    // n_reads + 1
    const int64_t *pair_read;   // n_pairs, or nullptr: pair p uses read p
    const uint32_t *wins;       // packed windows (words)
    const int64_t *win_off;     // n_pairs + 1
    const uint8_t *mask = nullptr;  // n_pairs, or nullptr: align every pair
};

struct FeatureParams {
    const uint32_t *reads;
    const int64_t *read_off;
    int64_t n_reads;
    const uint32_t *wins;
    const int64_t *win_off;
    const int64_t *cand_off;   // n_reads + 1
    uint16_t *out;             // bf16 [n_pairs][64]
};

struct Scoring {
    int32_t ma, mi, go, ge;
};

// Arithmetic of the score pass.
enum ScoreMode : int32_t {
    MODE_I32 = 0,   // one pair per lane group, int32 cells
    MODE_I16 = 1,   // two pairs per lane group in int16 halves, 16-bit keys
    MODE_I16W = 2,  // two pairs per lane group in int16 halves, 32-bit keys
    N_MODES = 3,
};

// Read-length classes: 16-base steps up to 1024, then 128-base steps.
constexpr int N_MCLASS = 64 + 56;
constexpr int N_NBUCKET = 256;       // window length / 32, clamped
constexpr int N_CLASS = N_MODES * N_MCLASS;

__host__ __device__ inline int mclass_of(int32_t m)
{
    return m <= 1024 ? (m + 15) / 16 - 1 : 64 + (m - 1024 + 127) / 128 - 1;
}
__host__ __device__ inline int32_t mclass_max(int c)
{
    return c < 64 ? 16 * (c + 1) : 1024 + 128 * (c - 64 + 1);
}

// Per-class facts the classify pass reads back to the host.
struct ClassInfo {
    int32_t count[N_CLASS];
    int32_t max_n[N_CLASS];
    int32_t max_m[N_CLASS];
    int32_t status;
    int32_t pad[3];
};

struct TbClassInfo;

struct ScoreLaunch {
    PairSet ps;
    Scoring sc;
    const int32_t *order;    // pair indices of this launch
    int64_t n_items;
    int32_t lanes;           // T: lanes per group
    int32_t *out_score;
    int32_t *out_end;
    uint8_t *boundary;       // per-group chunk boundaries, or nullptr
    int64_t boundary_group_bytes;
    int32_t *work_counter;
    int32_t *status;
    int32_t one = 1;         // a multiplier the compiler cannot fold
    // traceback cost keys from the epilogue (tb_keys == nullptr: none)
    int32_t cls = 0;         // the launch's class
    int32_t *tb_keys = nullptr;
    int32_t *tb_hist = nullptr;
    TbClassInfo *tb_info = nullptr;
    int32_t small_slab_words = 0;
};

// What every traceback kernel needs about the batch.
struct TbParams {
    PairSet ps;
    Scoring sc;
    const int32_t *score;
    const int32_t *end;
    uint32_t *cig_ops;
    const int64_t *cig_off;
    int32_t *cig_n;
    int32_t lanes;            // T lanes per pair
    int32_t small_slab_words; // per-group slab of the main launch
};

// Per-class facts of the traceback sort, read back to size the slabs.
struct TbClassInfo {
    int32_t max_need[N_CLASS];  // largest slab (words) a pair of the class needs
    int32_t n_big[N_CLASS];     // pairs needing more than small_slab_words
    int32_t max_wcap[2][N_CLASS];  // widest chunk window: [0] big-slab launch, [1] main launch
};

struct TracebackLaunch {
    TbParams P;
    const int32_t *order;
    int64_t n_items;
    int32_t lanes;
    uint32_t *slab;          // traceback bit slabs
    int64_t slab_group_words;  // per group; tiled: per lane (chunks x wcap)
    int32_t *boundary;       // chunk boundaries (2 x int32 per column, double-buffered)
    int64_t boundary_group_ints;  // per group; tiled: per lane (2 x 2 x wcap)
    int32_t wcap;            // widest chunk window of the launch
    bool tiled;              // lane-interleaved warp tiles (one lane per pair)
    bool packed16;           // 16x2 kernel: one lane per two pairs (tiled)
    int32_t *work_counter;
    int32_t *status;
    int32_t one = 1;         // a multiplier the compiler cannot fold
};

// Row counts compiled for the score kernels.
constexpr int N_SCORE_ROWS = 6;
extern const int kScoreRows[N_SCORE_ROWS];
constexpr int TB_ROWS = 8;

// force_i32: every pair takes the int32 score mode (else the narrowest
// mode its score bound allows)
int launch_classify(const PairSet &ps, int64_t n_reads, int64_t n_pairs, Scoring sc, bool force_i32,
                    int32_t *keys, int32_t *hist, int32_t *bucket_start, int32_t *cursor,
                    ClassInfo *info, int32_t *order, int32_t *out_score, int32_t *out_end,
                    int32_t *cig_n, cudaStream_t st);
int launch_score(int rows, int mode, const ScoreLaunch &L, int blocks, int threads, cudaStream_t st);
int score_kernel_regs(int rows, int mode, int *regs, int *max_blocks_per_sm, int threads);
int launch_tb_keys(const TbParams &P, int64_t n_pairs, const int32_t *score_keys, int32_t *tb_keys, int32_t *hist,
                   TbClassInfo *info, cudaStream_t st);
int launch_check_counts(const ClassInfo *info, const int32_t *expect, int32_t *status, cudaStream_t st);
int launch_scan_scatter(const int32_t *keys, int64_t n_pairs, const int32_t *class_count, int32_t *hist,
                        int32_t *bucket_start, int32_t *cursor, int32_t *order, cudaStream_t st);
int launch_traceback(const TracebackLaunch &L, int blocks, int threads, cudaStream_t st);
int traceback_kernel_occupancy(int *max_blocks_per_sm, int threads, bool packed16, int lanes);
int launch_alu_probe(int kind, int64_t iters, int blocks, int threads, uint32_t *out, cudaStream_t st);

int launch_features(const FeatureParams &P, cudaStream_t st);
int64_t mlp_floats();
int launch_mlp_init(float *model, uint64_t seed, cudaStream_t st);
int launch_mlp_refresh(float *model, cudaStream_t st);
int launch_mlp_forward(const float *model, const uint16_t *feat, int64_t n, float *out, int sm_count,
                       cudaStream_t st);
int launch_mlp_grad(float *model, const uint16_t *feat, const float *target, const int32_t *idx, int64_t n,
                    int sm_count, cudaStream_t st);
int launch_mlp_adam(float *model, float lr, int32_t step, cudaStream_t st);
int launch_select(const float *pred, const int64_t *cand_off, int64_t n_reads, int32_t k, float tau, uint8_t *mask,
                  cudaStream_t st);
int launch_best_per_read(const int32_t *score, const int64_t *cand_off, int64_t n_reads, const uint8_t *mask,
                         int32_t *best, int32_t *best_cand, cudaStream_t st);

int launch_top_hits(const int32_t *score, const int64_t *cand_off, int64_t n_reads, const uint8_t *mask, int32_t *best,
                    int32_t *best_cand, int32_t *second, int32_t *mapq, cudaStream_t st);
int launch_records(const int32_t *score, const int32_t *end, const sw_cigar_t &cig, int64_t n_pairs,
                   const int32_t *chrom, const int64_t *pos, const int8_t *strand, int32_t min_score,
                   sw_record_t *out, int64_t *out_count, int32_t *blk_count, int64_t *blk_off, cudaStream_t st);
int launch_junctions(const uint32_t *wins, const int64_t *win_off, const int32_t *score, const int32_t *end,
                     const sw_cigar_t &cig, int64_t n_pairs, const int32_t *chrom, const int64_t *pos,
                     int32_t min_score, int32_t min_intron, uint64_t *table, int64_t capacity, int32_t *status,
                     cudaStream_t st);
int launch_table_clear(uint64_t *table, int64_t capacity, cudaStream_t st);
int launch_table_export(const uint64_t *table, int64_t capacity, sw_junction_t *out, int64_t max_out,
                        int64_t *out_count, cudaStream_t st);

int launch_cigar_to_host(const uint32_t *ops, const int64_t *off, const int32_t *n_ops, int64_t n_pairs,
                         uint32_t *host_ops, cudaStream_t st);

int launch_cap_offsets(const int64_t *read_off, int64_t n_pairs, int64_t *cig_off, int64_t *blk, cudaStream_t st);
int launch_cap_offsets_indexed(const int64_t *read_off, const int64_t *pair_read, int64_t n_pairs, int64_t *cig_off,
                               int64_t *blk, cudaStream_t st);
int launch_dense_cigar(const uint32_t *ops, const int64_t *off, const int32_t *n_ops, int64_t n_pairs,
                       int64_t *doff, uint32_t *dense, int64_t dense_cap, int64_t *blk, cudaStream_t st);

int launch_mlp_forward_tc(const float *model, const uint16_t *feat, int64_t n, float *out, int sm_count,
                          int32_t *status, cudaStream_t st);
// A device status word for calls outside the alignment path: cleared on
// `st`, and the word sw_sync_status reads until the next call sets another.
int aux_status_word(cudaStream_t st, int32_t **status);
int filter_scratch(cudaStream_t st, size_t bytes, uint8_t **ptr);
int stream_status_word(cudaStream_t st, int32_t **status);
int launch_or_status(int32_t *dst, const int32_t *src, cudaStream_t st);

// Layout of the filter's model buffer (floats): parameters, Adam moments,
// gradient, step, then bf16 copies of W1 and W2 transposed (K-major).
constexpr int64_t MD_W1 = 0, MD_B1 = 16384, MD_W2 = 16640, MD_B2 = 33024, MD_W3 = 33088, MD_B3 = 33152;
constexpr int64_t MD_NP = 33153;
constexpr int64_t MD_M = MD_NP, MD_V = 2 * MD_NP, MD_G = 3 * MD_NP, MD_STEP = 4 * MD_NP;
constexpr int64_t MD_W1T = 132616;          // bf16 [256][64], 16-byte aligned
constexpr int64_t MD_W2T = MD_W1T + 8192;   // bf16 [64][256]
constexpr int64_t MD_TOTAL = MD_W2T + 8192;

void count_launch(int n = 1);

// The CUDA error behind the last SW_ERR_CUDA of this host thread.
void note_cuda_error(cudaError_t e);
inline bool cuda_failed(cudaError_t e)
{
    if (e == cudaSuccess) return false;
    note_cuda_error(e);
    return true;
}
inline int launch_status() { return cuda_failed(cudaGetLastError()) ? SW_ERR_CUDA : SW_OK; }

// Exclusive scan of int32 values v[0 .. n) into out[0 .. n] (out[n] = the
// total); blk holds (n + 255) / 256 + 1 int64 words.
int launch_scan_i32(const int32_t *v, int64_t n, int64_t *out, int64_t *blk, cudaStream_t st);

// ---- seeding (reads to candidate windows) ----
struct SeedKParams {
    int32_t k, stride, phase, max_hits, merge_dist, min_cal_len, flank, max_intron, max_window;
};
struct SeedOutPtrs {
    int64_t *start;
    int32_t *length;
    int32_t *chrom;
    int64_t *pos;
    int8_t *strand;
    int64_t *pair_read;
    int64_t *cand_offsets;
    int64_t *count;
};
int seed_count_per_read(int m, const SeedKParams &p);
int launch_index_build(const uint32_t *genome, int64_t n_bases, const int64_t *chrom_off, int n_chrom, int k,
                       uint32_t *table, uint32_t *positions, int64_t *out_n, uint32_t *blk, int sm_count,
                       int32_t *status, cudaStream_t st);
size_t seed_scratch_bytes(int64_t n_reads, int64_t capacity);
int launch_seed_windows(const uint32_t *reads, const int64_t *roff, int64_t n_reads, const uint32_t *table,
                        const uint32_t *positions, const int64_t *chrom_off, int n_chrom, const SeedKParams &p,
                        int max_read, int block_hits, SeedOutPtrs out, int64_t capacity, uint8_t *scratch,
                        int64_t *stats_host, int sm_count, int32_t *status, cudaStream_t st);
int launch_gather_probe(const uint32_t *buf, uint64_t mask, int64_t rounds, int blocks, int threads, uint32_t *out,
                        cudaStream_t st);
int launch_extract_windows(const uint32_t *genome, int64_t n_bases, const int64_t *start, const int32_t *len,
                           int64_t n, uint32_t *dst, int64_t cap_bases, int64_t *woff, int64_t *blk, int sm_count,
                           int32_t *status, cudaStream_t st);
int launch_two_strands(const uint32_t *reads, const int64_t *roff, int64_t n, uint32_t *dst, int64_t cap_bases,
                       int64_t *doff, int sm_count, int32_t *status, cudaStream_t st);

}  // namespace swgb
