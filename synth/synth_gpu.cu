/*
 * synth_gpu.cu -- the workload generator on the device: the same steps as
 * synth.c (both include synth_core.h), so a workload generated here equals the
 * host generator's, packed, bit for bit.  It exists for workloads too large to
 * generate on the host in reasonable time (10M reads and 165M candidate
 * windows, about 50 G bases).  Input generation only: none of the alignment
 * arithmetic is here.
 *
 * Compiled with -fmad=false: the generator's double expressions must round
 * once per operation, as gcc's do with -ffp-contract=off.
 *
 * Output layout: reads and windows 2-bit packed back to back (base q in
 * 32-bit word q / 16 at bits 2 (q % 16), the layout of synth_pack), offsets
 * in bases.  The packed buffers must be zeroed before the fill calls: words
 * shared by two neighbouring sequences are merged with atomicOr.
 */
#include <cuda_runtime.h>
#include <stdint.h>

/* Device sink: packs bases into words; counts only when store == 0. */
struct synth_sink {
    uint32_t *words;
    int64_t q, start;
    uint32_t acc;
    int store;
};
typedef struct synth_sink synth_sink_t;
#define SYNTH_FN __device__ static inline
SYNTH_FN void synth_put(synth_sink_t *o, uint8_t b)
{
    if (o->store) {
        o->acc |= (uint32_t)b << (2 * (o->q & 15));
        if ((o->q & 15) == 15) {
            uint32_t *w = o->words + (o->q >> 4);
            if (o->q - 15 >= o->start) *w = o->acc;  /* the whole word is this sequence's */
            else atomicOr(w, o->acc);
            o->acc = 0;
        }
    }
    o->q++;
}
#include "synth_core.h"

__device__ static inline void sink_flush(synth_sink_t *o)
{
    if (o->store && (o->q & 15)) atomicOr(o->words + (o->q >> 4), o->acc);
}

static constexpr int kMaxRead = 1024;        /* longest read a spec may draw */
static constexpr int kMaxBody = 4 * 1024 + 4096 + 16;  /* make_window's scratch */
static constexpr int kThreads = 128;

static int grid_for(int64_t n)
{
    int64_t b = (n + kThreads - 1) / kThreads;
    return (int)(b < 152 * 64 ? (b < 1 ? 1 : b) : 152 * 64);
}

__global__ void __launch_bounds__(kThreads) k_headers(synth_spec_t s, int32_t *read_len, int32_t *n_cand)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < s.n_reads;
         r += (int64_t)gridDim.x * blockDim.x) {
        rng_t g = read_rng(&s, r);
        const read_hdr_t h = read_header(&s, &g);
        read_len[r] = h.m;
        n_cand[r] = h.c;
    }
}

__global__ void __launch_bounds__(kThreads) k_reads(synth_spec_t s, const int64_t *read_off, uint32_t *read_words,
                                                    int32_t *true_cand)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < s.n_reads;
         r += (int64_t)gridDim.x * blockDim.x) {
        rng_t g = read_rng(&s, r);
        const read_hdr_t h = read_header(&s, &g);
        synth_sink_t o = {read_words, read_off[r], read_off[r], 0u, 1};
        for (int32_t i = 0; i < h.m; ++i) synth_put(&o, rbase(&g));
        sink_flush(&o);
        true_cand[r] = s.cand_max == 1 ? 0 : h.t;
    }
}

/* Pair p is candidate p - cand_off[r] of read r = pair_read[p].  With
 * win_off == NULL only the lengths are written. */
__global__ void __launch_bounds__(kThreads) k_windows(synth_spec_t s, int64_t n_pairs, const int64_t *pair_read,
                                                     const int64_t *cand_off, const int64_t *win_off,
                                                     int32_t *win_len, uint32_t *win_words, uint8_t *kinds)
{
    uint8_t read[kMaxRead];
    uint8_t tmp[kMaxBody];
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n_pairs;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = pair_read[p];
        rng_t g = read_rng(&s, r);
        const read_hdr_t h = read_header(&s, &g);
        read_bases(&g, h.m, read);
        const int64_t at = win_off ? win_off[p] : 0;
        synth_sink_t o = {win_words, at, at, 0u, win_off != nullptr};
        uint8_t kind;
        const int64_t n = make_window(&s, &g, &h, read, p - cand_off[r], &o, tmp, &kind);
        sink_flush(&o);
        if (win_len) win_len[p] = (int32_t)n;
        if (kinds) kinds[p] = kind;
    }
}

static int spec_ok(const synth_spec_t *s)
{
    if (!s || s->n_reads < 0 || s->n_len < 1 || s->n_len > 8 || s->cand_min < 1 || s->cand_max < s->cand_min)
        return 0;
    for (int k = 0; k < s->n_len; ++k)
        if (s->len_val[k] < 1 || s->len_val[k] > kMaxRead) return 0;
    if (s->intron_min < 4 || s->intron_max < s->intron_min || s->flank_min < 0 || s->flank_max < s->flank_min)
        return 0;
    int32_t mx = 0;
    for (int k = 0; k < s->n_len; ++k) mx = s->len_val[k] > mx ? s->len_val[k] : mx;
    return 4 * (int64_t)mx + s->intron_max + 4 <= kMaxBody;
}

static int launched()
{
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

extern "C" {

/* read_len, n_cand: device int32[s->n_reads].  0, -1 (spec outside the
 * device generator's limits) or -2 (CUDA error). */
int synth_gpu_headers(const synth_spec_t *s, int32_t *read_len, int32_t *n_cand, void *stream)
{
    if (!spec_ok(s)) return -1;
    if (s->n_reads == 0) return 0;
    k_headers<<<grid_for(s->n_reads), kThreads, 0, (cudaStream_t)stream>>>(*s, read_len, n_cand);
    return launched();
}

/* read_off: device int64[n_reads + 1]; read_words: zeroed packed buffer of
 * read_off[n_reads] bases; true_cand: device int32[n_reads]. */
int synth_gpu_reads(const synth_spec_t *s, const int64_t *read_off, uint32_t *read_words, int32_t *true_cand,
                    void *stream)
{
    if (!spec_ok(s)) return -1;
    if (s->n_reads == 0) return 0;
    k_reads<<<grid_for(s->n_reads), kThreads, 0, (cudaStream_t)stream>>>(*s, read_off, read_words, true_cand);
    return launched();
}

/* pair_read, cand_off: device int64 (n_pairs, n_reads + 1).  Lengths pass:
 * win_off, win_words and kinds NULL, win_len (int32[n_pairs]) written.  Fill
 * pass: win_off (int64[n_pairs + 1]), win_words (zeroed, win_off[n_pairs]
 * bases) and kinds (uint8[n_pairs]); win_len may be NULL. */
int synth_gpu_windows(const synth_spec_t *s, const int64_t *pair_read, const int64_t *cand_off, int64_t n_pairs,
                      const int64_t *win_off, int32_t *win_len, uint32_t *win_words, uint8_t *kinds, void *stream)
{
    if (!spec_ok(s) || n_pairs < 0 || (win_off && !win_words)) return -1;
    if (n_pairs == 0) return 0;
    k_windows<<<grid_for(n_pairs), kThreads, 0, (cudaStream_t)stream>>>(*s, n_pairs, pair_read, cand_off, win_off,
                                                                        win_len, win_words, kinds);
    return launched();
}

}  /* extern "C" */
