/*
 * swgb.h -- C ABI of the GB300 batched Smith-Waterman library (libswgb.so).
 *
 * The library computes Stage E, task iii of "Concurrent and Accurate RNA
 * Sequencing on Multicore Platforms" (Martinez et al., 2013): every read is
 * aligned with the Smith-Waterman algorithm onto each of its extended / joined
 * candidate alignment locations (CALs, "windows" below), returning the
 * alignment, its score and its position (Section 2, Stage E).  The paper does
 * not print the recurrence; the library implements the affine-gap (Gotoh)
 * local alignment
 *
 *   E(i,j) = max(H(i,j-1) + o, E(i,j-1) + e)
 *   F(i,j) = max(H(i-1,j) + o, F(i-1,j) + e)
 *   H(i,j) = max(0, H(i-1,j-1) + s(r_i, w_j), E(i,j), F(i,j))
 *
 * (a gap of length k scores o + (k-1) e), with these tie-breaks:
 *   end cell   among cells with H == score, the smallest window index j,
 *              then the smallest read index i (0-based); score 0 -> (-1,-1);
 *   traceback  from the end cell: stop at H == 0; prefer the diagonal (M),
 *              then a deletion (D, gap in the read), then an insertion (I,
 *              gap in the window); inside a gap, open where E == H + o.
 *
 * Conventions shared by every entry point
 *  - Sequences are 2-bit packed, A=0 C=1 G=2 T=3, four bases per byte, base q
 *    of a buffer in byte q/4 at bits 2*(q%4).  Sequence k of a set occupies
 *    bases [offsets[k], offsets[k+1]) -- sequences are packed back to back
 *    with no alignment padding.  A packed buffer must start on a 16-byte
 *    boundary and hold sw_packed_bytes(total bases) bytes (whole 16-byte
 *    blocks), which the library may read in full.
 *  - Offsets are int64 counts of bases, non-decreasing, offsets[0] >= 0.
 *  - Every pointer named "device" is device memory of the current CUDA device,
 *    owned by the caller; the library keeps no reference after the call's
 *    work completes.  The library owns only its cached scratch memory.
 *  - Calls are stream-ordered on `stream` (NULL = legacy default stream).
 *  - Return value: SW_OK or a negative SW_ERR_* code; no exception crosses the
 *    ABI.  Problems in device-resident inputs (offsets out of order, lengths
 *    out of range) are detected on the device; the call then returns
 *    SW_ERR_DEVICE_INPUT and leaves the outputs unspecified.
 */
#ifndef SWGB_H
#define SWGB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *sw_stream_t; /* same handle as cudaStream_t */

#define SW_OK 0
#define SW_ERR_INVALID_ARG (-1)   /* NULL pointer, negative count, bad scoring */
#define SW_ERR_CAPACITY (-2)      /* a CIGAR did not fit its CSR slot */
#define SW_ERR_CUDA (-3)          /* a CUDA runtime call failed */
#define SW_ERR_DEVICE_TIMEOUT (-4)/* a device-side wait hit its iteration limit */
#define SW_ERR_UNSUPPORTED (-5)   /* a size beyond the documented limits */
#define SW_ERR_DEVICE_INPUT (-6)  /* device-resident input failed validation */
#define SW_ERR_INTERNAL (-7)      /* an internal consistency check failed */
#define SW_ERR_NO_DEVICE (-8)     /* no usable sm_103 device */

#define SW_MAX_READ_LEN 8192      /* bases; longer reads -> SW_ERR_DEVICE_INPUT */
#define SW_MAX_WINDOW_LEN 1048575 /* bases */

/* Scoring.  Requirements: 1 <= match <= 127, -127 <= mismatch <= 0,
 * gap_open <= gap_extend <= 0, gap_open < 0, and match - gap_open <= 127
 * (so every match / mismatch score minus gap_open fits a signed byte).  A gap of length k scores
 * gap_open + (k-1) * gap_extend (pass o + e as gap_open for the o + k e
 * convention). */
typedef struct {
    int32_t match;
    int32_t mismatch;
    int32_t gap_open;
    int32_t gap_extend;
} sw_scoring_t;

/* CIGAR output in CSR form, all device memory owned by the caller.
 * ops[offsets[p] .. offsets[p+1]) receives pair p's runs, BAM-encoded as
 * (length << 4) | op with M=0, I=1, D=2, S=4 (leading and trailing soft clips
 * included, M covering matches and mismatches); n_ops[p] receives the number
 * of runs (0 when the score is 0).  A slot of sw_cigar_capacity(m) runs
 * always suffices for a read of length m; a smaller slot that overflows makes
 * the call return SW_ERR_CAPACITY with n_ops[p] = -1. */
typedef struct {
    uint32_t *ops;
    const int64_t *offsets; /* n_pairs + 1 */
    int32_t *n_ops;         /* n_pairs */
} sw_cigar_t;

/* Upper bound on the CIGAR runs of a read of length m: 2 m + 3 (at most m
 * M/I runs, a D run between or around each, two soft clips). */
int64_t sw_cigar_capacity(int64_t read_len);

/* CSR offsets of CIGAR slots for a batch, on the device: out_offsets[p] =
 * sum over pairs q < p of sw_cigar_capacity(length of q's read), and
 * out_offsets[n_pairs] the total.  read_offsets, pair_read (NULL: pair p
 * uses read p) and out_offsets (int64[n_pairs + 1]) are device memory.
 * Stream-ordered. */
int sw_cigar_offsets(const int64_t *read_offsets, const int64_t *pair_read, int64_t n_pairs, int64_t *out_offsets,
                     sw_stream_t stream);

/* Bytes of a packed buffer holding n_bases: ceil(n_bases / 4) rounded up to
 * a multiple of 16. */
int64_t sw_packed_bytes(int64_t n_bases);

/*
 * sw_batch_align -- align pair p = (read p, window p) for p < n_pairs
 * (Stage E, task iii: the read is mapped onto an extended CAL with SW).
 *
 *  reads, read_offsets        device; packed reads, n_pairs + 1 offsets
 *  windows, window_offsets    device; packed windows, n_pairs + 1 offsets
 *  n_pairs                    >= 0 (0 is a no-op)
 *  scoring                    host pointer, see sw_scoring_t
 *  out_score                  device int32[n_pairs]: the SW score (>= 0)
 *  out_end                    device int32[2 * n_pairs]: (i_end, j_end) of
 *                             pair p at [2p], [2p+1]; (-1, -1) when score 0
 *  out_cigar                  host pointer to a struct of device pointers,
 *                             or NULL for score and end only
 *  stream                     CUDA stream
 *
 * Read length must be 1..SW_MAX_READ_LEN, window length 0..SW_MAX_WINDOW_LEN
 * (an empty window gives score 0).  The call enqueues a fixed sequence of
 * memsets and kernel launches on `stream` and returns without waiting: the
 * batch is classified into length classes on the device, one-block planner
 * kernels size the launches there, and every compiled kernel variant runs
 * once as a persistent launch over the classes planned for it (launches with
 * nothing to do exit at once).  The host never waits for the device, so the
 * call can be captured into a CUDA graph, provided that an uncaptured call on
 * the same stream with at least as many pairs came first: the first call of
 * a size on a stream allocates the library's scratch for it, and a call that
 * would have to grow scratch during a capture returns SW_ERR_UNSUPPORTED.
 * Replays use the bases, offsets and outputs the captured call named.
 * sw_sync_status waits and reports what the kernels found (invalid device
 * input, an overflowing CIGAR slot, ...).  Scratch is bounded per call: a
 * batch whose longest pair needs more than the call's scratch for one warp
 * (far beyond the workloads of the paper, e.g. an 8,000-base read against a
 * window of a million bases) is reported as SW_ERR_UNSUPPORTED.
 */
int sw_batch_align(const uint8_t *reads, const int64_t *read_offsets,
                   const uint8_t *windows, const int64_t *window_offsets,
                   int64_t n_pairs, const sw_scoring_t *scoring,
                   int32_t *out_score, int32_t *out_end, sw_cigar_t *out_cigar,
                   sw_stream_t stream);

/*
 * sw_batch_align_indexed -- as sw_batch_align, but pair p aligns read
 * pair_read[p] (device int64[n_pairs], each in [0, n_reads)) against window p,
 * so the candidate windows of one read share a single copy of it (Stage E
 * maps each read onto all of its extended CALs).  read_offsets has
 * n_reads + 1 entries.
 */
int sw_batch_align_indexed(const uint8_t *reads, const int64_t *read_offsets, int64_t n_reads,
                           const uint8_t *windows, const int64_t *window_offsets,
                           const int64_t *pair_read, int64_t n_pairs,
                           const sw_scoring_t *scoring,
                           int32_t *out_score, int32_t *out_end, sw_cigar_t *out_cigar,
                           sw_stream_t stream);

/*
 * sw_batch_align_host -- the same alignment from HOST buffers: copies the
 * inputs to the device (library-owned staging buffers), aligns, copies
 * score, end and CIGAR back to the host buffers and waits for `stream`.
 * Pointers are host memory (pinned memory makes the copies asynchronous);
 * out_cigar's members are host pointers too.  Returns after the results are
 * in host memory.  Large batches go in two chunks whose copies overlap the
 * other chunk's kernels.  When out_cigar->ops is pinned host memory the
 * device can address, the device writes each pair's used runs straight into
 * its slot and leaves the rest of the slot untouched; otherwise whole slots
 * are copied back.
 */
int sw_batch_align_host(const uint8_t *reads, const int64_t *read_offsets,
                        const uint8_t *windows, const int64_t *window_offsets,
                        int64_t n_pairs, const sw_scoring_t *scoring,
                        int32_t *out_score, int32_t *out_end, sw_cigar_t *out_cigar,
                        sw_stream_t stream);

/*
 * sw_batch_align_masked -- as sw_batch_align_indexed, but only pairs with
 * pair_mask[p] != 0 (device uint8[n_pairs]) are aligned; the others get
 * score -1, end (-1, -1) and 0 CIGAR runs.  This is how the candidates a
 * filter selected are aligned without copying their windows.
 */
int sw_batch_align_masked(const uint8_t *reads, const int64_t *read_offsets, int64_t n_reads,
                          const uint8_t *windows, const int64_t *window_offsets,
                          const int64_t *pair_read, const uint8_t *pair_mask, int64_t n_pairs,
                          const sw_scoring_t *scoring,
                          int32_t *out_score, int32_t *out_end, sw_cigar_t *out_cigar,
                          sw_stream_t stream);

/*
 * Learned candidate filter (an addition to the paper's method: the paper
 * aligns every extended CAL; the filter ranks a read's candidates so that only
 * the top ones are aligned, with exhaustive alignment as the fallback for
 * reads whose ranking is not clear-cut.  It never changes a reported score).
 *
 * Candidates are grouped by read: cand_offsets (device int64[n_reads + 1])
 * gives read r the pairs cand_offsets[r] .. cand_offsets[r+1]-1, and pair p
 * is window p of window_offsets (device int64[n_pairs + 1]).
 *
 * sw_filter_features: per pair 64 bf16 features (device uint16[n_pairs * 64],
 * row-major, 16-byte aligned; SW_ERR_INVALID_ARG otherwise): the 4-mers
 * q = 64 b0 + 16 b1 + 4 b2 + b3 of read and window are counted, and
 * f[k] = sum over b of min(c_read(4k+b), c_window(4k+b)) / (m - 3) for
 * k = 0..63 (0 when the read is shorter than 4).
 */
int sw_filter_features(const uint8_t *reads, const int64_t *read_offsets, int64_t n_reads,
                       const uint8_t *windows, const int64_t *window_offsets,
                       const int64_t *cand_offsets, uint16_t *out_features, sw_stream_t stream);

/*
 * The network: y = w3 . relu(W2^T relu(W1^T f + b1) + b2) + b3, W1 64x256,
 * W2 256x64, w3 64 (33,153 parameters).  A model is one caller-owned device
 * buffer of sw_mlp_bytes() bytes, fp32, laid out as
 *   [0, 33153)         parameters: W1 row-major [64][256], b1[256],
 *                      W2 row-major [256][64], b2[64], w3[64], b3
 *   [33153, 66306)     Adam first moments
 *   [66306, 99459)     Adam second moments
 *   [99459, 132612)    gradient of the last sw_mlp_grad call
 *   [132612]           unused
 *   [132616, 140808)   bf16 W1 transposed [256][64] (serving copy)
 *   [140808, 149000)   bf16 W2 transposed [64][256] (serving copy)
 * sw_mlp_refresh rebuilds the bf16 copies after the caller writes parameters.
 */
int64_t sw_mlp_bytes(void);
int sw_mlp_init(float *model, uint64_t seed, sw_stream_t stream);
int sw_mlp_refresh(float *model, sw_stream_t stream);

/* Predictions for n feature rows on the tensor cores (bf16 inputs and
 * weights, fp32 accumulation): out device float[n].  By default
 * (SW_MLP_AUTO) the 5th-generation tensor cores compute both layers into
 * tensor memory when `features` is 16-byte aligned; SW_MLP_MMA_SYNC (or
 * 4-byte-aligned features) uses warp-level MMA instead.  Both round the
 * hidden layer to bf16 and agree up to fp32 summation order.  A timed-out
 * tensor-core wait is reported as SW_ERR_DEVICE_TIMEOUT by sw_sync_status.
 * sw_set_mlp_kernel is process-wide; SW_ERR_INVALID_ARG for other values. */
#define SW_MLP_AUTO 0
#define SW_MLP_MMA_SYNC 1
int sw_set_mlp_kernel(int32_t kind);
int sw_mlp_forward(const float *model, const uint16_t *features, int64_t n, float *out, sw_stream_t stream);

/* Gradient of mean((y - target)^2) over n samples, written to the model's
 * gradient region.  Sample s uses feature row idx[s] and target[idx[s]] (idx
 * device int32[n], or NULL for s).  By default (SW_GRAD_AUTO), when
 * `features` is 16-byte aligned, the 5th-generation tensor cores compute the
 * five products of the forward and backward pass (bf16 operands: the
 * features, the weights as the serving copies round them, the hidden
 * activation and the two error signals; fp32 accumulation in tensor memory),
 * one partial gradient per CTA, summed in a fixed order (the result does not
 * depend on scheduling).  SW_GRAD_FP32 computes forward and backward in fp32
 * on the CUDA cores instead.  A timed-out tensor-core wait is reported as
 * SW_ERR_DEVICE_TIMEOUT by sw_sync_status.  sw_set_mlp_grad_kernel is
 * process-wide; SW_ERR_INVALID_ARG for other values.  The library keeps the
 * partial gradients in scratch of this stream (33,153 floats per CTA). */
#define SW_GRAD_AUTO 0
#define SW_GRAD_FP32 1
int sw_set_mlp_grad_kernel(int32_t kind);
int sw_mlp_grad(float *model, const uint16_t *features, const float *target, const int32_t *idx, int64_t n,
                sw_stream_t stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) from the stored gradient;
 * step counts from 1.  Also refreshes the bf16 copies. */
int sw_mlp_adam(float *model, float lr, int32_t step, sw_stream_t stream);

/* Per read: mark in pair_mask (device uint8[n_pairs]) its k best-predicted
 * candidates (ties: lower candidate index first) and every other candidate
 * whose prediction is less than delta below the read's best; or all of them
 * when the k-th and (k+1)-th predictions differ by less than tau, or when
 * the read has at most k candidates.  Differences are taken in fp32.  The
 * relative rule (delta) is this library's addition to the top-k filter: it
 * keeps the candidates of reads whose best few predictions are close
 * together without aligning every candidate of those reads; delta = 0
 * turns it off.  1 <= k <= SW_FILTER_MAX_K, delta >= 0, else
 * SW_ERR_INVALID_ARG. */
#define SW_FILTER_MAX_K 16
int sw_filter_select(const float *pred, const int64_t *cand_offsets, int64_t n_reads, int32_t k, float tau,
                     float delta, uint8_t *pair_mask, sw_stream_t stream);

/* One selection rule: reads of length up to max_read_len select as
 * sw_filter_select with this k, tau and delta. */
typedef struct {
    int32_t max_read_len;
    int32_t k;
    float tau;
    float delta;
} sw_select_rule_t;
#define SW_FILTER_MAX_RULES 16

/* sw_filter_select with the rule chosen per read by its length m (from
 * read_offsets, device int64[n_reads + 1] in bases): the first of `rules`
 * (host memory, n_rules of them, max_read_len ascending) with
 * m <= max_read_len, else the last.  The rules let short reads, whose
 * features rank candidates less reliably, keep more candidates than long
 * ones.  read_offsets may be NULL with a single rule.  SW_ERR_INVALID_ARG
 * for n_rules outside 1..SW_FILTER_MAX_RULES, descending bounds, a rule's k
 * outside 1..SW_FILTER_MAX_K or a negative or NaN delta. */
int sw_filter_select_by_length(const float *pred, const int64_t *cand_offsets, const int64_t *read_offsets,
                               int64_t n_reads, const sw_select_rule_t *rules, int32_t n_rules,
                               uint8_t *pair_mask, sw_stream_t stream);

/* Per read: the largest score over its candidates with pair_mask[p] != 0
 * (pair_mask may be NULL: all), and that candidate's index within the read
 * (first on ties); -1 and -1 when none. */
int sw_best_per_read(const int32_t *score, const int64_t *cand_offsets, int64_t n_reads,
                     const uint8_t *pair_mask, int32_t *best_score, int32_t *best_cand, sw_stream_t stream);

/*
 * sw_filter_align -- the filtered search in one call: sw_filter_features,
 * sw_mlp_forward, sw_filter_select_by_length (rules, n_rules: checked as
 * there, before any device work), sw_batch_align_masked (score
 * and end; unselected pairs get score -1 and end (-1, -1)) and
 * sw_best_per_read over the selected pairs.  Reads, windows and offsets as
 * sw_batch_align_indexed; pair_read (device int64[n_pairs]) must agree with
 * cand_offsets (pair p belongs to read r when cand_offsets[r] <= p <
 * cand_offsets[r+1]).  pair_mask (device uint8[n_pairs]) receives the
 * selection, or NULL: the library keeps it in its scratch.  best_score and
 * best_cand: device int32[n_reads] (best_cand may be NULL).  Features and
 * predictions live in library scratch of this stream (132 bytes per pair).
 * A read count of 0 needs n_pairs == 0; with no pairs every read gets -1.
 * Device-detected errors of every step (a timed-out tensor-core wait, an
 * input the alignment rejects) are read with sw_sync_status.
 */
int sw_filter_align(const uint8_t *reads, const int64_t *read_offsets, int64_t n_reads, const uint8_t *windows,
                    const int64_t *window_offsets, const int64_t *pair_read, const int64_t *cand_offsets,
                    int64_t n_pairs, const float *model, const sw_select_rule_t *rules, int32_t n_rules,
                    const sw_scoring_t *scoring, int32_t *out_score, int32_t *out_end, uint8_t *pair_mask,
                    int32_t *best_score, int32_t *best_cand, sw_stream_t stream);

/* One training step: sw_mlp_grad over the n samples (idx may be NULL), then
 * sw_mlp_adam with lr and step (from 1).  SW_ERR_INVALID_ARG for n < 1, a
 * missing array, step < 1 or lr <= 0. */
int sw_filter_train_step(float *model, const uint16_t *features, const float *target, const int32_t *idx, int64_t n,
                         float lr, int32_t step, sw_stream_t stream);

/*
 * Wait for `stream` and report problems the kernels of the last call on
 * `stream` detected on the device (SW_ERR_CAPACITY when a CIGAR slot
 * overflowed, SW_ERR_INTERNAL when a consistency check failed, ...).
 * sw_batch_align returns once its kernels are enqueued, so a caller that
 * wants those errors calls this after it.
 *
 * Streams: the library keeps its scratch, status word and read-back slots
 * per (device, stream).  Calls on one stream run in stream order; calls on
 * different streams share no scratch, so batches on two streams may be in
 * flight at once (each stream's scratch is grown on demand and kept until
 * the process exits).  The queries below that take no stream
 * (sw_last_traceback_split, sw_phase_times) refer to the device's most
 * recent call; sw_phase_timing applies to every stream of the device.
 */
int sw_sync_status(sw_stream_t stream);
/* The same as sw_sync_status. */
int sw_get_status(sw_stream_t stream);

/*
 * Free the library's scratch of `stream` on the current device (after
 * waiting for the stream).  The next call on the stream allocates it again.
 * The caller makes sure no other thread uses the stream meanwhile.
 */
int sw_stream_release(sw_stream_t stream);

/*
 * The CUDA error (cudaError_t value) behind the last SW_ERR_CUDA returned
 * on this host thread, 0 if none; *name (if not NULL) receives its name
 * (static storage).
 */
int sw_last_cuda_error(const char **name);

/*
 * sw_batch_align_noalloc -- score and end cell of pair p = (read p, window p),
 * like sw_batch_align with out_cigar == NULL, without the library allocating
 * any memory.  The paper has no counterpart; this is for callers that cannot
 * let a library call cudaMalloc or cudaFree: applications that give all
 * device memory to their own pool allocator, or latency-sensitive services
 * that cannot afford the device synchronisation those calls imply.
 *
 * Its scratch (work counter, status word, pair order) is one fixed array of
 * 4 * (64 + SW_NOALLOC_MAX_PAIRS) bytes in the library's static device
 * memory, which every GPU that loads the library holds until the process
 * exits.  Limits: n_pairs <= SW_NOALLOC_MAX_PAIRS (else SW_ERR_UNSUPPORTED,
 * checked before any GPU work) and reads of at most SW_NOALLOC_MAX_READ_LEN
 * bases (else SW_ERR_UNSUPPORTED, detected on the device).  Arguments,
 * layouts, scoring requirements and outputs are those of sw_batch_align.
 *
 * Each call looks up the array's device address on the current device (no
 * allocation).  The first call on a device may also load the library's device
 * code there: make it before any stream capture.  Every
 * call on a device uses the same array (it keeps the previous call's
 * contents; the call clears what must start at zero), so calls whose GPU
 * work overlaps -- on different streams or from different threads -- race;
 * serialise them.  Like sw_batch_align, the call waits on `stream` for a
 * validation step, then enqueues the score kernel and returns.
 */
#define SW_NOALLOC_MAX_PAIRS 262144
#define SW_NOALLOC_MAX_READ_LEN 1024
int sw_batch_align_noalloc(const uint8_t *reads, const int64_t *read_offsets,
                           const uint8_t *windows, const int64_t *window_offsets,
                           int64_t n_pairs, const sw_scoring_t *scoring,
                           int32_t *out_score, int32_t *out_end, sw_stream_t stream);

/*
 * sw_batch_align_host_dense -- sw_batch_align_host with the CIGARs packed
 * densely for the host: pair p's runs come back in ops_out[offsets_out[p] ..
 * offsets_out[p+1]), offsets_out has n_pairs + 1 entries and
 * offsets_out[n_pairs] is the total.  The library sizes the device-side
 * CIGAR slots itself (2m + 3 runs per pair) and compacts them on the device,
 * so only the runs cross the host link.  ops_cap is the room in ops_out;
 * when the runs need more, ops_out holds the first ops_cap of them,
 * offsets_out is complete and the call returns SW_ERR_CAPACITY.  All
 * pointers are host memory (pinned for asynchronous copies).  Returns after
 * the results are in host memory.
 */
int sw_batch_align_host_dense(const uint8_t *reads, const int64_t *read_offsets, const uint8_t *windows,
                              const int64_t *window_offsets, int64_t n_pairs, const sw_scoring_t *scoring,
                              int32_t *out_score, int32_t *out_end, uint32_t *ops_out, int64_t ops_cap,
                              int64_t *offsets_out, sw_stream_t stream);

/*
 * Fixed-shape execution with dedicated scratch (pattern: one plan, many
 * replays).  sw_batch_align sizes its scratch from the pair count and grows
 * it on demand; a plan instead owns scratch sized for the worst case of one
 * batch shape, so its executions never allocate, on any stream:
 *
 *   sw_plan_create classifies the batch given by its offsets (device
 *   pointers, as for sw_batch_align_indexed; pair_read may be NULL for one
 *   read per pair), sizes the score boundaries and the traceback for the
 *   worst case of that shape (every window fully inside the band) and
 *   allocates all scratch, auxiliary streams and events the plan will use.
 *   It synchronises `stream` once.  with_cigar = 0 plans score and end
 *   cell only.
 *
 *   sw_plan_align enqueues on `stream` the same fixed sequence of memsets and
 *   launches as sw_batch_align, for the plan's shape and the given packed
 *   bases and outputs: no allocation, no host synchronisation.  So it can be
 *   captured into a CUDA graph and replayed; the bases and outputs may change
 *   between calls or replays (the arrays the captured call named are the
 *   ones a replay uses), the offsets must not.  The device compares the
 *   batch's class counts with the plan's and reports a mismatch as
 *   SW_ERR_DEVICE_INPUT through sw_plan_status.
 *
 *   sw_plan_status waits for `stream` and returns the status the plan's
 *   last execution (or replay) recorded.  sw_plan_destroy waits for the
 *   device and frees the plan.  A plan belongs to the device current at its
 *   creation; executions of one plan must not overlap.
 *
 * The paper has no counterpart: its batches go to OpenMP threads (§3.4).
 */
typedef struct sw_plan sw_plan_t;
int sw_plan_create(const int64_t *read_offsets, int64_t n_reads, const int64_t *window_offsets,
                   const int64_t *pair_read, int64_t n_pairs, const sw_scoring_t *scoring, int32_t with_cigar,
                   sw_stream_t stream, sw_plan_t **out_plan);
int sw_plan_align(sw_plan_t *plan, const uint8_t *reads, const uint8_t *windows, int32_t *out_score,
                  int32_t *out_end, sw_cigar_t *out_cigar, sw_stream_t stream);
int sw_plan_status(sw_plan_t *plan, sw_stream_t stream);
int sw_plan_destroy(sw_plan_t *plan);

/*
 * Stage E, task iv (§2): records and splice junctions from the alignments.
 * All pointers are device pointers; every call is stream-ordered and
 * asynchronous, and device-detected errors are read with sw_sync_status.
 *
 * Records.  A pair whose score is >= min_score (and > 0) becomes a record;
 * records are written in pair order to out_records (room for n_pairs) and
 * their number to *out_count.  The window's reference coordinates come from
 * the caller per pair: window_chrom, window_pos (reference position of the
 * window's first base) and window_strand (copied into the record).  The
 * aligned window columns are j_start..j_end with j_start = j_end + 1 -
 * (M + D bases of the CIGAR); the record holds ref_start = window_pos +
 * j_start, ref_end = window_pos + j_end, read_start = the leading soft clip,
 * read_end = i_end.  Pairs whose CIGAR overflowed (n_ops < 0) are skipped.
 */
typedef struct {
    int64_t pair;
    int64_t ref_start;
    int64_t ref_end;
    int32_t chrom;
    int32_t score;
    int32_t read_start;
    int32_t read_end;
    int32_t strand;
    int32_t n_ops;
} sw_record_t; /* 48 bytes */
int sw_records(const int32_t *score, const int32_t *end, const sw_cigar_t *cigar, int64_t n_pairs,
               const int32_t *window_chrom, const int64_t *window_pos, const int8_t *window_strand,
               int32_t min_score, sw_record_t *out_records, int64_t *out_count, sw_stream_t stream);

/*
 * Top hits.  Among the statistics the SW task reports for an alignment is a
 * quality score, which the paper leaves undefined (§2, Stage E); it is read
 * here as a mapping quality.  Per read r, over its
 * candidates p = cand_offsets[r] .. cand_offsets[r+1]-1 with pair_mask[p] != 0
 * (pair_mask may be NULL: all):
 *   best_score[r]   S1, the largest score
 *   best_cand[r]    its candidate index within the read (first on ties)
 *   second_score[r] S2, the largest score of the other candidates (so a tie
 *                   gives S2 = S1), 0 when there is no other candidate
 *   mapq[r]         min(60, floor(60 (S1 - S2) / S1)), 0 when S1 <= 0
 * A read without candidates gets -1, -1, -1 and 0.  best_cand, second_score
 * and mapq may be NULL.  All arrays are device memory (int32[n_reads];
 * cand_offsets int64[n_reads + 1]).
 */
int sw_top_hits(const int32_t *score, const int64_t *cand_offsets, int64_t n_reads, const uint8_t *pair_mask,
                int32_t *best_score, int32_t *best_cand, int32_t *second_score, int32_t *mapq, sw_stream_t stream);

/*
 * Splice junctions.  Every D run of at least min_intron window bases in the
 * CIGAR of a record (score >= min_score, > 0) is a candidate intron
 * window[j .. j+len-1]; it is a junction when it starts with GT and ends
 * with AG (strand 0) or starts with CT and ends with AC (strand 1).  The
 * junction (chrom, window_pos + j, window_pos + j + len - 1, strand) is
 * counted in a caller-owned open-addressing table that persists across
 * calls (the role of the paper's AVL tree).
 *
 * The table holds `capacity` slots (a power of two, >= 64) in
 * sw_junction_table_words(capacity) 64-bit words: keys, then counts.
 * sw_junction_table_clear empties it.  A full table sets SW_ERR_CAPACITY;
 * a chromosome >= 4096, a position >= 2^32 - 1 or an intron longer than
 * 2^19 bases sets SW_ERR_UNSUPPORTED (those junctions are not counted).
 * sw_junctions_export writes up to max_out junctions (in slot order) and
 * their number to *out_count (the number in the table, which may exceed
 * max_out).  Requires min_intron >= 4.
 */
typedef struct {
    int64_t start;
    int64_t end;
    int64_t count;
    int32_t chrom;
    int32_t strand;
} sw_junction_t; /* 32 bytes */
int64_t sw_junction_table_words(int64_t capacity);
int sw_junction_table_clear(uint64_t *table, int64_t capacity, sw_stream_t stream);
int sw_junctions_detect(const uint8_t *windows, const int64_t *window_offsets, const int32_t *score,
                        const int32_t *end, const sw_cigar_t *cigar, int64_t n_pairs, const int32_t *window_chrom,
                        const int64_t *window_pos, int32_t min_score, int32_t min_intron, uint64_t *table,
                        int64_t capacity, sw_stream_t stream);
int sw_junctions_export(const uint64_t *table, int64_t capacity, sw_junction_t *out, int64_t max_out,
                        int64_t *out_count, sw_stream_t stream);

/* Text of an SW_* code (static storage). */
const char *sw_strerror(int code);

/* Number of kernel launches the library issued since load (all entry points;
 * counts launches, not completions). */
int64_t sw_launch_count(void);

/*
 * Tuning.  The plan for reads of a length class is the number of lanes T
 * that share one pair (or one pair of pairs in the 16-bit path) and the
 * rows R each lane holds in registers.  sw_set_plan overrides the built-in
 * choice for length classes whose longest read is <= max_read_len (0 clears
 * all overrides); r_rows must be one of the compiled row counts (sw_plan_rows
 * lists them), and lanes * r_rows must cover the reads unless lanes == 32
 * (longer reads are then processed in chunks of 32 * r_rows rows).  At most
 * 16 overrides are held (SW_ERR_UNSUPPORTED beyond).  Process-wide; applies
 * to calls made after it, and the planner kernels of a call read the
 * overrides it was enqueued with.
 */
int sw_set_plan(int32_t max_read_len, int32_t lanes, int32_t r_rows);

/*
 * The plan (lanes, rows) the score pass gives a length class whose longest
 * read is max_read_len and longest window max_window_len under a scoring
 * with this match score: the arithmetic mode follows from the score bound
 * match x min(max_read_len, max_window_len) as for a pair, then the
 * overrides of sw_set_plan apply (an override with more than 32 rows is
 * skipped by a 16-bit-key class whose bound exceeds 510), else the built-in
 * cost model.  Without an override, a class whose pairs would give fewer
 * tasks than half the warps of its launch (a small batch) runs with fewer
 * rows per lane on more lanes; the query reports the plan before that
 * adjustment, which depends on the class's pair count.  Host-only;
 * SW_ERR_INVALID_ARG for null outputs or values out of range.
 */
int sw_plan_query(int32_t max_read_len, int32_t max_window_len, int32_t match, int32_t *lanes, int32_t *r_rows);

/*
 * Traceback arithmetic.  SW_TB_AUTO (the default) recomputes two pairs per
 * lane in 16-bit halves for every length class whose score bound
 * (match x min(m, n)) is at most 32000, and uses 32-bit arithmetic for the
 * rest; SW_TB_INT32 uses 32-bit arithmetic for every class.  Both give the
 * same CIGARs.  Returns SW_ERR_INVALID_ARG for any other value.  The setting
 * is process-wide and applies to calls made after it.
 */
#define SW_TB_AUTO 0
#define SW_TB_INT32 1
int sw_set_traceback_mode(int32_t mode);

/*
 * Score-pass arithmetic.  SW_SCORE_AUTO (the default) gives each pair the
 * narrowest exact mode its score bound match x min(m, n) allows: two pairs
 * per lane in 16-bit halves up to 32000 (with 16-bit best-cell keys up to
 * 510, without keys above), 32-bit lanes above.  SW_SCORE_INT32 runs every
 * pair in 32-bit lanes (and so, with a CIGAR, through the 32-bit traceback
 * kernels).  SW_SCORE_WIDE16 runs every pair whose bound is at most 32000 in
 * 16-bit halves without keys (the end row from column snapshots).  All give
 * the same scores, end cells and CIGARs.  Returns SW_ERR_INVALID_ARG for any
 * other value.  Process-wide; applies to calls made after it, and a plan
 * keeps the setting it was created under.
 */
#define SW_SCORE_AUTO 0
#define SW_SCORE_INT32 1
#define SW_SCORE_WIDE16 2
int sw_set_score_mode(int32_t mode);

/*
 * Pairs the most recent sw_batch_align* call with a CIGAR on the current
 * device sent to each traceback kernel: out[0] through the 16-bit kernel,
 * out[1] through the 32-bit kernels (pairs without an alignment included).
 * The split is planned on the device, so this waits for the device.
 * Returns SW_ERR_INVALID_ARG for a null pointer.
 */
int sw_last_traceback_split(int64_t *out2);
int sw_plan_rows(int32_t *rows, int32_t cap);

/*
 * Phase timing (measurement support).  With timing enabled, each call records
 * CUDA events on its stream around its three phases; sw_phase_times waits for
 * the last call and writes the milliseconds of (0) classification and launch
 * planning, (1) the score kernels, (2) the traceback (its sort, planning and
 * kernels).
 * Returns SW_ERR_INVALID_ARG if the last call was not timed.
 */
int sw_phase_timing(int32_t enable);
int sw_phase_times(float *ms3);

#ifdef __cplusplus
}
#endif
#endif /* SWGB_H */
