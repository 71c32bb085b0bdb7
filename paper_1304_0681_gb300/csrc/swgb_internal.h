// swgb_internal.h -- declarations shared by the library's translation units.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/swgb.h"

namespace swgb {

// Status bits written by kernels (atomicOr) and read back by the host.
enum : int32_t {
    ST_BAD_INPUT = 1,
    ST_CAPACITY = 2,
    ST_INTERNAL = 4,
    ST_TIMEOUT = 8,
    ST_UNSUPPORTED = 16,
};

// The error code a call returns for a device status word: invalid input
// first, then an unsupported shape, an exhausted capacity, a device wait
// that ran out (a tensor-core kernel's bounded mbarrier wait), and internal
// errors; SW_OK when no bit is set.
inline int status_to_code(int32_t st)
{
    if (st & ST_BAD_INPUT) return SW_ERR_DEVICE_INPUT;
    if (st & ST_UNSUPPORTED) return SW_ERR_UNSUPPORTED;
    if (st & ST_CAPACITY) return SW_ERR_CAPACITY;
    if (st & ST_TIMEOUT) return SW_ERR_DEVICE_TIMEOUT;
    if (st & ST_INTERNAL) return SW_ERR_INTERNAL;
    return SW_OK;
}

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
struct DevScorePlan;
struct DevTbPlan;

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
    // device-planned launch (dp != nullptr): the launch serves every class
    // of score variant `variant` in the plan; order is then the whole
    // sorted pair order, work_counter the base of the per-class counters and
    // boundary the base of the chunk-boundary scratch
    const DevScorePlan *dp = nullptr;
    int32_t variant = 0;
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

// A persistent traceback launch: every part of traceback variant `variant`
// in the device plan.
struct TracebackLaunch {
    TbParams P;
    const int32_t *order;    // the whole traceback order (parts index into it)
    uint32_t *slab;          // base of the per-warp scratch slots
    int32_t *work_counter;   // base of the per-part counters (2 per class)
    int32_t *status;
    int32_t one = 1;         // a multiplier the compiler cannot fold
    const DevTbPlan *dp = nullptr;
    int32_t variant = 0;
};

// Row counts compiled for the score kernels.
constexpr int N_SCORE_ROWS = 6;
extern const int kScoreRows[N_SCORE_ROWS];
constexpr int TB_ROWS = 8;
__host__ __device__ inline int score_rows_at(int i)
{
    switch (i) {
    case 0: return 8;
    case 1: return 16;
    case 2: return 20;
    case 3: return 25;
    case 4: return 32;
    default: return 50;
    }
}

// ---- device-side launch planning ----
//
// A batch is aligned by a fixed sequence of launches: the host never reads
// anything back.  One-block planner kernels turn the classification's
// per-class facts into the tables below, and every compiled kernel variant
// is launched once, persistent at full occupancy; a launch serves the
// classes (or traceback parts) its variant was given and exits at once when
// it has none.
constexpr int N_SCORE_VARIANTS = N_SCORE_ROWS * N_MODES;  // variant = rows index * N_MODES + mode
constexpr int N_TB16_VARIANTS = 6;                        // 16-bit traceback, T = 1, 2, 4, 8, 16, 32
constexpr int TB_VAR_TILED = 6;                           // int32 traceback, one lane per pair, warp tiles
constexpr int TB_VAR_GROUPED = 7;                         // int32 traceback, T lanes per pair
constexpr int N_TB_VARIANTS = 8;
constexpr int N_TB_PARTS = 2 * N_CLASS;                   // per class: pairs with big slabs, then the rest
constexpr int kMaxPlanOverrides = 16;
constexpr int kPlanThreads = 384;                         // >= N_CLASS

struct PlanOverride {
    int32_t max_read_len, lanes, rows;
};

// What the planners need besides the batch's class tables (by value).
struct PlanParams {
    Scoring sc;
    int32_t n_overrides;
    PlanOverride ov[kMaxPlanOverrides];     // sorted by max_read_len
    int32_t score_warps[N_SCORE_VARIANTS];  // warps each score launch runs
    int32_t tb_warps[N_TB_VARIANTS];        // warps each traceback launch runs
    int64_t score_bnd_bytes;                // chunk-boundary scratch of the score launches
    int64_t tb_bytes;                       // per-warp traceback scratch, shared by the (sequential) launches
    int32_t small_slab_words;
    int32_t allow16;                        // 16-bit traceback allowed (SW_TB_AUTO)
};

struct DevScorePlan {
    int32_t var_n[N_SCORE_VARIANTS];          // classes of each variant
    int32_t var_bnd_warps[N_SCORE_VARIANTS];  // warps with a boundary slot (chunked classes only)
    int64_t var_bnd_offset[N_SCORE_VARIANTS];
    int64_t var_bnd_slot[N_SCORE_VARIANTS];   // bytes of one warp's boundary slot (its largest class)
    int32_t cls_start[N_CLASS];               // first position of the class in the sorted order
    int32_t cls_count[N_CLASS];
    int32_t cls_lanes[N_CLASS];
    int32_t cls_bnd_bytes[N_CLASS];           // per group; 0 when a read fits one row chunk
    int16_t var_cls[N_SCORE_VARIANTS][N_CLASS];  // longest reads first
};

struct TbPartPlan {
    int32_t cls, part, start, count;
    int32_t lanes, wcap;
    int64_t slab_words, bnd_ints;  // per lane (16-bit), per warp tile (tiled) or per group (grouped)
    int32_t variant;
    int32_t pool_tasks;            // 16-bit: tasks whose tiles go to the pool (walked by k_tb16_walk)
    int64_t pool_offset;           // 16-bit: words from the scratch base to the part's first pooled tile
};

// Traceback scratch of one launch (words from the scratch base; the launches
// run one after another and each has the whole budget).  16-bit kernel: the
// boundary rows of the warps that take part, then full per-warp slots for
// tasks swept and walked by the warp itself, then the pool of tiles that the
// separate walk kernel reads.  int32 kernels: per-warp slots only.
struct DevTbPlan {
    int32_t var_n[N_TB_VARIANTS];
    int32_t var_warps[N_TB_VARIANTS];     // warps with a full slot (int32 kernels: the others exit)
    int64_t var_slot_words[N_TB_VARIANTS];
    int64_t var_slot_offset[N_TB_VARIANTS];
    int64_t var_bnd_words[N_TB_VARIANTS];  // 16-bit: boundary row words per warp
    int32_t var_run_warps[N_TB_VARIANTS];  // 16-bit: warps that take part (each with a boundary row)
    int64_t split[2];                     // pairs through the 16-bit and the int32 kernels
    int16_t var_part[N_TB_VARIANTS][N_TB_PARTS];
    TbPartPlan part[N_TB_PARTS];
};

// Score-pass arithmetic of a pair (or class) whose scores are at most hmax
// (match x min(m, n)) under a sw_set_score_mode setting: 16-bit keys up to
// 510, where 6-bit row tags leave every plan (up to 64 rows per lane) open,
// 16-bit halves without keys up to 32000, else 32-bit lanes;
// SW_SCORE_WIDE16 skips the 16-bit keys, SW_SCORE_INT32 takes 32-bit lanes.
// (Keys would fit up to 1022 with 5-bit tags, at most 32 rows per lane; the
// wide mode with 50 rows per lane measured faster on those classes.)
__host__ __device__ inline int score_mode_for(int64_t hmax, int setting)
{
    if (setting == SW_SCORE_INT32) return MODE_I32;
    if (hmax <= 510 && setting != SW_SCORE_WIDE16) return MODE_I16;
    if (hmax <= 32000) return MODE_I16W;
    return MODE_I32;
}

// Score-pass plan of a length class: lanes per group and rows per lane
// (index into score_rows_at) for reads up to m_max in `mode`, hmax the
// class's score bound.  Overrides first (sorted by max_read_len), else a
// cost model: padded rows x ~6.5 ALU operations + ~40 per lane-step (both
// measured), scaled by the share of lanes a warp leaves idle.  In the
// 16-bit-key mode more than 32 rows per lane need 6-bit row tags, which
// hold scores up to 510 only.
__host__ __device__ inline void score_plan_of(int mode, int32_t m_max, int64_t hmax, const PlanOverride *ov,
                                              int n_ov, int &lanes, int &rows_idx)
{
    const int max_rows = (mode == MODE_I16 && hmax > 510) ? 32 : 64;
    for (int i = 0; i < n_ov; ++i)
        if (m_max <= ov[i].max_read_len && ov[i].rows <= max_rows) {
            lanes = ov[i].lanes;
            rows_idx = 0;
            for (int r = 0; r < N_SCORE_ROWS; ++r)
                if (score_rows_at(r) == ov[i].rows) rows_idx = r;
            return;
        }
    // cost = chunks x T x (6.5 R + 40) / (G T / 32) = chunks x (13 R + 80) x 16 / G,
    // compared exactly as the fraction num / G (integers; the first minimum
    // over R ascending, then T ascending, wins).  Plans with one row chunk
    // need T >= ceil(m / R), and G = floor(32 / T) does not grow with T, so
    // for each R the smallest such T is the first minimum (T = 32 with one
    // chunk is never better); reads longer than 32 R take T = 32 in chunks.
    int64_t best_num = -1, best_den = 1;
    lanes = 32;
    rows_idx = 4;
    for (int ri = 0; ri < N_SCORE_ROWS; ++ri) {
        const int R = score_rows_at(ri);
        if (R > max_rows) continue;
        const int t_min = (m_max + R - 1) / R;
        const int T = t_min <= 32 ? (t_min > 0 ? t_min : 1) : 32;
        const int chunks = t_min <= 32 ? 1 : (m_max + 32 * R - 1) / (32 * R);
        const int64_t G = 32 / T;
        const int64_t num = (int64_t)chunks * (13 * R + 80) * 16;
        if (best_num < 0 || num * best_den < best_num * G) {
            best_num = num;
            best_den = G;
            lanes = T;
            rows_idx = ri;
        }
    }
}

// Traceback launch shape of one part of a class (part 0: pairs whose
// one-lane slab exceeds small_slab_words, part 1: the rest).  m_max: the
// class's longest read; max_need: the largest one-lane slab of the class;
// wcap_in: the part's widest chunk window.  The 16-bit kernel serves every
// class with a 16-bit score mode unless allow16 is off.  T lanes share a
// pair: one where a lane's tile (every chunk at the widest window) stays
// small, else the smallest power of two with the longest read in at most 8
// (16-bit) or 4 (int32) chunks of 8T rows -- a chunk sweeps its rows' band
// box, 8T - 1 columns wider than the band, so smaller T wastes fewer cells
// and larger T keeps fewer pairs per warp waiting (measured on the uneven
// batch, 16-bit: 4 chunks 57.0 ms, 8 chunks 49.6 ms, 16 chunks 64.5 ms).
// Also the words one warp's scratch slot needs for this part.
constexpr int kTbChunks16 = 8, kTbChunks32 = 4;
constexpr int64_t kTiledLaneWords = 4096, kTiledLaneWords16 = 8192;
__host__ __device__ inline int64_t tb_part_shape(int mode, bool allow16, int32_t m_max, int64_t max_need,
                                                 int32_t wcap_in, int part, int32_t small_slab_words, TbPartPlan &t,
                                                 int min_lanes16 = 1)
{
    const int64_t chunks = (m_max + TB_ROWS - 1) / TB_ROWS;
    int32_t wcap = wcap_in > 1 ? wcap_in : 1;
    const int64_t wcap4 = (wcap + 3) / 4 * 4;
    const bool packed16 = allow16 && mode != MODE_I32;
    int Tl = 1;
    while (Tl < 32 && (int64_t)Tl * 8 * (packed16 ? kTbChunks16 : kTbChunks32) < m_max) Tl *= 2;
    const bool one_lane16 = chunks * wcap4 * 2 <= kTiledLaneWords16;
    const bool tiled = !packed16 && chunks * wcap <= kTiledLaneWords;
    int T = (packed16 && one_lane16) || tiled ? 1 : Tl;
    if (packed16 && T < min_lanes16) T = min_lanes16;
    t.lanes = T;
    int64_t slot;
    if (packed16) {
        const int64_t chunks_t = (m_max + 8 * T - 1) / (8 * T);
        wcap += 8 * (T - 1);
        const int64_t s4 = (wcap + T - 1 + 3) / 4;
        t.slab_words = chunks_t * s4 * 8;                            // per lane
        t.bnd_ints = chunks_t > 1 ? (int64_t)(32 / T) * 2 * wcap : 0;  // per warp: one row
        int v = 0;
        while ((1 << v) < T) ++v;
        t.variant = v;
        slot = 32 * t.slab_words + t.bnd_ints;
    } else if (tiled) {
        t.slab_words = chunks * wcap;                  // per lane
        t.bnd_ints = chunks > 1 ? (int64_t)4 * wcap : 0;
        t.variant = TB_VAR_TILED;
        slot = 32 * (t.slab_words + t.bnd_ints);
    } else {
        const int64_t chunks_t = (m_max + 8 * T - 1) / (8 * T);
        const int64_t wcap_t = wcap + 8 * (T - 1);
        const int64_t need = max_need > 1 ? max_need : 1;
        t.slab_words = T == 1 ? (part == 0 ? need : (need < small_slab_words ? need : small_slab_words))
                              : chunks_t * wcap_t * T;  // per group
        t.bnd_ints = chunks_t > 1 ? (int64_t)4 * wcap_t : 0;
        t.variant = TB_VAR_GROUPED;
        slot = (int64_t)(32 / T) * (t.slab_words + t.bnd_ints);
    }
    t.wcap = wcap;
    return slot;
}

// score_setting: the sw_set_score_mode value (SW_SCORE_INT32: every pair in
// the int32 mode; SW_SCORE_WIDE16: no 16-bit keys; else the narrowest
// mode its score bound allows)
int launch_classify(const PairSet &ps, int64_t n_reads, int64_t n_pairs, Scoring sc, int score_setting,
                    int32_t *keys, int32_t *hist, int32_t *bucket_start, int32_t *cursor,
                    ClassInfo *info, int32_t *order, int32_t *out_score, int32_t *out_end,
                    int32_t *cig_n, cudaStream_t st);
int launch_score(int rows, int mode, const ScoreLaunch &L, int blocks, int threads, cudaStream_t st);
int score_kernel_regs(int rows, int mode, int *regs, int *max_blocks_per_sm, int threads);
int launch_check_counts(const ClassInfo *info, const int32_t *expect, int32_t *status, cudaStream_t st);
int launch_plan_score(const ClassInfo *info, const PlanParams &pp, DevScorePlan *out, int32_t *status,
                      cudaStream_t st);
int launch_plan_tb(const ClassInfo *info, const TbClassInfo *ti, const DevScorePlan *sp, const PlanParams &pp,
                   DevTbPlan *out, int32_t *status, cudaStream_t st);
// One persistent launch of score variant v (rows index * N_MODES + mode) at
// full occupancy; its grid (blocks) comes from score_variant_blocks.
int launch_score_variant(int v, const ScoreLaunch &L, int blocks, cudaStream_t st);
int score_variant_blocks(int v, int sm_count, int *blocks);
int launch_traceback_variant(int v, bool fma, const TracebackLaunch &L, int blocks, cudaStream_t st);
int traceback_variant_blocks(int v, int sm_count, int *blocks);
// The walks of a 16-bit traceback launch's pooled tasks (v < N_TB16_VARIANTS).
int launch_tb_walk_variant(int v, const TracebackLaunch &L, int blocks, cudaStream_t st);
int tb_walk_variant_blocks(int v, int sm_count, int *blocks);
// Per-class work counters of one batch: score, traceback (pooled tasks),
// traceback (tasks a warp sweeps and walks itself).
constexpr int N_COUNTERS = 6 * N_CLASS;
constexpr int CTR_TB = 2 * N_CLASS, CTR_TB_OWN = 4 * N_CLASS;
int launch_scan_scatter(const int32_t *keys, int64_t n_pairs, const int32_t *class_count, int32_t *hist,
                        int32_t *bucket_start, int32_t *cursor, int32_t *order, cudaStream_t st);

int launch_features(const FeatureParams &P, int sm_count, cudaStream_t st);
int64_t mlp_floats();
int launch_mlp_init(float *model, uint64_t seed, cudaStream_t st);
int launch_mlp_refresh(float *model, cudaStream_t st);
int launch_mlp_forward(const float *model, const uint16_t *feat, int64_t n, float *out, int sm_count,
                       cudaStream_t st);
int launch_mlp_grad(float *model, const uint16_t *feat, const float *target, const int32_t *idx, int64_t n,
                    int sm_count, cudaStream_t st);
int launch_mlp_adam(float *model, float lr, int32_t step, cudaStream_t st);
// The filter's selection rules, by value in the kernel's parameters.
struct SelectRules {
    int32_t n;
    int32_t max_len[SW_FILTER_MAX_RULES];
    int32_t k[SW_FILTER_MAX_RULES];
    float tau[SW_FILTER_MAX_RULES];
    float delta[SW_FILTER_MAX_RULES];
};
int launch_select(const float *pred, const int64_t *cand_off, const int64_t *read_off, int64_t n_reads,
                  const SelectRules &rules, uint8_t *mask, cudaStream_t st);
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
// The gradient on the tensor cores: one partial per CTA (partial: that many
// x MD_NP floats), then their sum in CTA order into the model's gradient.
int mlp_grad_tc_parts(int64_t n, int sm_count);
int launch_mlp_grad_tc(float *model, const uint16_t *feat, const float *target, const int32_t *idx, int64_t n,
                       int sm_count, float *partial, int32_t *status, cudaStream_t st);
// Scratch of sw_mlp_grad on this stream (grown on demand).
int grad_scratch(cudaStream_t st, size_t bytes, float **ptr);
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
int launch_extract_windows(const uint32_t *genome, int64_t n_bases, const int64_t *start, const int32_t *len,
                           int64_t n, uint32_t *dst, int64_t cap_bases, int64_t *woff, int64_t *blk, int sm_count,
                           int32_t *status, cudaStream_t st);
int launch_two_strands(const uint32_t *reads, const int64_t *roff, int64_t n, uint32_t *dst, int64_t cap_bases,
                       int64_t *doff, int sm_count, int32_t *status, cudaStream_t st);

}  // namespace swgb
