// swgb_api.cu -- host side of the C ABI declared in include/swgb.h.
//
// One call = classify (validate, sort pairs by length class) -> read back the
// per-class counts -> per class: score pass, then (when a CIGAR is wanted)
// traceback pass.  Scratch memory is owned by the library, cached per device
// and grown on demand; calls on one device are serialised through an event so
// that two calls never share scratch concurrently.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "sw_device.cuh"
#include "swgb_internal.h"
#include "swgb_seed.h"

namespace swgb {

static std::atomic<int64_t> g_launches{0};
static std::atomic<int32_t> g_tb_mode{SW_TB_AUTO};
static std::atomic<int32_t> g_score_mode{SW_SCORE_AUTO};
void count_launch(int n) { g_launches += n; }

thread_local int g_cuda_error = 0;
void note_cuda_error(cudaError_t e) { g_cuda_error = (int)e; }

namespace {

constexpr int kThreads = 128;
constexpr int kSmallSlabWords = 4096;  // per-group slab of a traceback's main part
constexpr int kMaxDevices = 64;
constexpr int kAuxStreams = 4;
constexpr int kHostChunks = 2;                 // sw_batch_align_host pipelines a batch in this many chunks
constexpr int64_t kHostChunkMin = 65536;       // ... of at least this many pairs
// Scratch budgets of a call, from its pair count (the only size the host
// knows without reading the device): chunk-boundary rows of the score pass,
// and the per-warp slots of the traceback.  A warp's slot is sized on the
// device for its launch's largest part; launches use as many warps as fit.
constexpr int64_t kScoreBndMin = (int64_t)32 << 20, kScoreBndMax = (int64_t)1 << 30, kScoreBndPerPair = 1024;
constexpr int64_t kTbMin = (int64_t)64 << 20, kTbPerPair = (int64_t)32 << 10;
constexpr int64_t kTbCapMax = (int64_t)16 << 30, kTbCapMin = (int64_t)1 << 30;
constexpr double kTbFreeShare = 0.3;

struct Buffer {
    void *ptr = nullptr;
    size_t bytes = 0;
};

// What an execution needs besides scratch: the full-occupancy grid of every
// launch, the auxiliary streams the score launches fork onto (and the events
// of the fork and join), and phase events when timing.
struct ExecCtx {
    int score_blocks[N_SCORE_VARIANTS] = {};
    int tb_blocks[N_TB_VARIANTS] = {};
    int walk_blocks[N_TB16_VARIANTS] = {};
    cudaStream_t aux[kAuxStreams] = {};
    cudaEvent_t fork_ev = nullptr;
    cudaEvent_t join_ev[kAuxStreams] = {};
    bool timing = false;
    cudaEvent_t *phase = nullptr;  // 4 events, when timing
};

int exec_ctx_init(ExecCtx &x, int sm_count)
{
    int rc = SW_OK;
    for (int v = 0; v < N_SCORE_VARIANTS; ++v)
        if ((rc = score_variant_blocks(v, sm_count, &x.score_blocks[v]))) return rc;
    for (int v = 0; v < N_TB_VARIANTS; ++v)
        if ((rc = traceback_variant_blocks(v, sm_count, &x.tb_blocks[v]))) return rc;
    for (int v = 0; v < N_TB16_VARIANTS; ++v)
        if ((rc = tb_walk_variant_blocks(v, sm_count, &x.walk_blocks[v]))) return rc;
    for (int k = 0; k < kAuxStreams; ++k) {
        if (cuda_failed(cudaStreamCreateWithFlags(&x.aux[k], cudaStreamNonBlocking))) return SW_ERR_CUDA;
        if (cuda_failed(cudaEventCreateWithFlags(&x.join_ev[k], cudaEventDisableTiming))) return SW_ERR_CUDA;
    }
    if (cuda_failed(cudaEventCreateWithFlags(&x.fork_ev, cudaEventDisableTiming))) return SW_ERR_CUDA;
    return SW_OK;
}

void exec_ctx_free(ExecCtx &x)
{
    for (int k = 0; k < kAuxStreams; ++k) {
        if (x.aux[k]) cudaStreamDestroy(x.aux[k]);
        if (x.join_ev[k]) cudaEventDestroy(x.join_ev[k]);
        x.aux[k] = nullptr;
        x.join_ev[k] = nullptr;
    }
    if (x.fork_ev) cudaEventDestroy(x.fork_ev);
    x.fork_ev = nullptr;
}

// Library state of one (device, stream): scratch buffers, the status word
// of the stream's last call, events and auxiliary streams.  Calls on one
// stream are ordered by the stream; calls on two streams get two states,
// so their work may overlap on the GPU without sharing scratch.
struct DeviceState {
    bool ready = false;
    int dev = 0;
    int sm_count = 0;
    ExecCtx x;                       // grids, auxiliary streams, fork and join events
    int64_t tb_cap = 0;              // largest traceback budget (set at the first traceback)
    Buffer fixed, dyn;
    Buffer stage;            // sw_batch_align_host device staging
    int32_t *last_status = nullptr;  // device status word of the last call
    const DevTbPlan *last_tplan = nullptr;  // traceback plan of the last call with a CIGAR
    bool timing = false;             // record phase events (sw_phase_times)
    bool timed_cells_valid = false;
    Buffer misc;                     // Stage E task iv: status word and record scan scratch
    Buffer filt;                     // sw_filter_align: features, predictions, selection
    Buffer grad;                     // sw_mlp_grad: per-CTA partial gradients
    int64_t *seed_stats_host = nullptr;  // pinned: counters of the stream's last sw_seed_windows
    cudaEvent_t phase[4] = {nullptr, nullptr, nullptr, nullptr};
    // sw_batch_align_host: copy streams and per-chunk events
    cudaStream_t copy_in = nullptr, copy_out = nullptr;
    cudaEvent_t host_in_ev[kHostChunks] = {};
    cudaEvent_t host_out_ev = nullptr;
    std::mutex mu;
};

std::mutex g_state_mu;
std::vector<std::pair<std::pair<int, cudaStream_t>, DeviceState *>> g_states;  // never freed
DeviceState *g_last_state[kMaxDevices] = {};   // the state of the device's most recent call
bool g_timing[kMaxDevices] = {};               // sw_phase_timing, per device
std::mutex g_plan_mu;
std::vector<PlanOverride> g_plans;

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Fork: the first n auxiliary streams wait for everything enqueued on st so
// far.  Join: st waits for all of their work.  (The pattern is legal under
// stream capture.)
int fork_streams(const ExecCtx &x, cudaStream_t st, int n)
{
    if (cuda_failed(cudaEventRecord(x.fork_ev, st))) return SW_ERR_CUDA;
    for (int k = 0; k < n; ++k)
        if (cuda_failed(cudaStreamWaitEvent(x.aux[k], x.fork_ev, 0))) return SW_ERR_CUDA;
    return SW_OK;
}

int join_streams(const ExecCtx &x, cudaStream_t st, int n)
{
    for (int k = 0; k < n; ++k) {
        if (cuda_failed(cudaEventRecord(x.join_ev[k], x.aux[k]))) return SW_ERR_CUDA;
        if (cuda_failed(cudaStreamWaitEvent(st, x.join_ev[k], 0))) return SW_ERR_CUDA;
    }
    return SW_OK;
}

bool capturing(cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return cs != cudaStreamCaptureStatusNone;
}

int ensure(Buffer &b, size_t bytes)
{
    if (b.bytes >= bytes) return SW_OK;
    // pending work may still use the old buffer
    if (cuda_failed(cudaDeviceSynchronize())) return SW_ERR_CUDA;
    if (b.ptr) cudaFree(b.ptr);
    b.ptr = nullptr;
    b.bytes = 0;
    const size_t want = align_up(bytes + std::min<size_t>(bytes / 4, (size_t)256 << 20), 1 << 20);
    if (cuda_failed(cudaMalloc(&b.ptr, want))) {
        cudaGetLastError();
        return SW_ERR_CUDA;
    }
    b.bytes = want;
    return SW_OK;
}

// As ensure, for a call that may be captured: a buffer cannot grow while
// the stream is capturing (the first call of a size on a stream allocates).
int ensure_on(Buffer &b, size_t bytes, cudaStream_t st)
{
    if (b.bytes >= bytes) return SW_OK;
    if (capturing(st)) return SW_ERR_UNSUPPORTED;
    return ensure(b, bytes);
}

int device_state(DeviceState **out, cudaStream_t st)
{
    int dev = 0;
    if (cuda_failed(cudaGetDevice(&dev)) || dev < 0 || dev >= kMaxDevices) return SW_ERR_NO_DEVICE;
    std::lock_guard<std::mutex> glk(g_state_mu);
    DeviceState *found = nullptr;
    for (auto &e : g_states)
        if (e.first.first == dev && e.first.second == st) found = e.second;
    if (!found) {
        found = new (std::nothrow) DeviceState;
        if (!found) return SW_ERR_CUDA;
        found->dev = dev;
        g_states.push_back({{dev, st}, found});
    }
    DeviceState &s = *found;
    if (!s.ready) {
        cudaDeviceProp prop;
        if (cuda_failed(cudaGetDeviceProperties(&prop, dev))) return SW_ERR_NO_DEVICE;
        s.sm_count = prop.multiProcessorCount;
        const int rc = exec_ctx_init(s.x, s.sm_count);
        if (rc) return rc;
        for (cudaEvent_t &e : s.phase)
            if (cuda_failed(cudaEventCreate(&e))) return SW_ERR_CUDA;
        s.x.phase = s.phase;
        if (cuda_failed(cudaStreamCreateWithFlags(&s.copy_in, cudaStreamNonBlocking))) return SW_ERR_CUDA;
        if (cuda_failed(cudaStreamCreateWithFlags(&s.copy_out, cudaStreamNonBlocking))) return SW_ERR_CUDA;
        for (cudaEvent_t &e : s.host_in_ev)
            if (cuda_failed(cudaEventCreateWithFlags(&e, cudaEventDisableTiming))) return SW_ERR_CUDA;
        if (cuda_failed(cudaEventCreateWithFlags(&s.host_out_ev, cudaEventDisableTiming))) return SW_ERR_CUDA;
        s.ready = true;
    }
    s.timing = g_timing[dev];
    s.x.timing = s.timing;
    g_last_state[dev] = &s;
    *out = &s;
    return SW_OK;
}

void free_state(DeviceState *s)
{
    for (Buffer *b : {&s->fixed, &s->dyn, &s->stage, &s->misc, &s->filt, &s->grad})
        if (b->ptr) {
            cudaFree(b->ptr);
            b->ptr = nullptr;
            b->bytes = 0;
        }
    if (s->seed_stats_host) cudaFreeHost(s->seed_stats_host);
    for (cudaEvent_t e : s->phase)
        if (e) cudaEventDestroy(e);
    exec_ctx_free(s->x);
    if (s->copy_in) cudaStreamDestroy(s->copy_in);
    if (s->copy_out) cudaStreamDestroy(s->copy_out);
    for (cudaEvent_t e : s->host_in_ev)
        if (e) cudaEventDestroy(e);
    if (s->host_out_ev) cudaEventDestroy(s->host_out_ev);
}

// The state of the device's most recent call (for the queries that take no
// stream), or the default stream's.
int last_state(DeviceState **out)
{
    int dev = 0;
    if (cuda_failed(cudaGetDevice(&dev)) || dev < 0 || dev >= kMaxDevices) return SW_ERR_NO_DEVICE;
    {
        std::lock_guard<std::mutex> glk(g_state_mu);
        if (g_last_state[dev]) {
            *out = g_last_state[dev];
            return SW_OK;
        }
    }
    return device_state(out, 0);
}

bool scoring_ok(const sw_scoring_t *s)
{
    return s && s->match >= 1 && s->match <= 127 && s->mismatch >= -127 && s->mismatch <= 0 &&
           s->gap_open <= s->gap_extend && s->gap_extend <= 0 && s->gap_open < 0 &&
           s->match - s->gap_open <= 127;
}

// The scratch of one batch execution: arrays sized by the pair count, the
// class tables and plans, and the dynamic part (score chunk boundaries and
// traceback slots).
struct Scratch {
    int32_t *keys, *order, *hist, *bstart, *cursor, *counters, *tb_keys, *tb_order, *expect;
    ClassInfo *info;
    TbClassInfo *tbinfo;
    DevScorePlan *splan;
    DevTbPlan *tplan;
    uint8_t *score_bnd;
    int64_t score_bnd_bytes;
    uint32_t *tb;
    int64_t tb_bytes;
};

// Lays out the pair-count-sized part at base (nullptr: sizes only); returns
// its bytes.
size_t fixed_layout(int64_t n_pairs, uint8_t *base, Scratch &S)
{
    const size_t nh = (size_t)N_CLASS * N_NBUCKET;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        uint8_t *p = base ? base + off : nullptr;
        off = align_up(off + bytes, 256);
        return p;
    };
    S.keys = (int32_t *)take(sizeof(int32_t) * n_pairs);
    S.order = (int32_t *)take(sizeof(int32_t) * n_pairs);
    S.hist = (int32_t *)take(sizeof(int32_t) * nh);
    S.bstart = (int32_t *)take(sizeof(int32_t) * nh);
    S.cursor = (int32_t *)take(sizeof(int32_t) * nh);
    S.info = (ClassInfo *)take(sizeof(ClassInfo));
    S.counters = (int32_t *)take(sizeof(int32_t) * N_COUNTERS);
    S.tb_keys = (int32_t *)take(sizeof(int32_t) * n_pairs);
    S.tb_order = (int32_t *)take(sizeof(int32_t) * n_pairs);
    S.tbinfo = (TbClassInfo *)take(sizeof(TbClassInfo));
    S.expect = (int32_t *)take(sizeof(int32_t) * 3 * N_CLASS);
    S.splan = (DevScorePlan *)take(sizeof(DevScorePlan));
    S.tplan = (DevTbPlan *)take(sizeof(DevTbPlan));
    return off;
}

PlanParams plan_params(const ExecCtx &x, const Scoring &sc, bool allow16, int64_t score_bnd_bytes,
                       int64_t tb_bytes)
{
    PlanParams pp{};
    pp.sc = sc;
    {
        std::lock_guard<std::mutex> lk(g_plan_mu);
        pp.n_overrides = (int32_t)std::min<size_t>(g_plans.size(), kMaxPlanOverrides);
        for (int i = 0; i < pp.n_overrides; ++i) pp.ov[i] = g_plans[i];
    }
    for (int v = 0; v < N_SCORE_VARIANTS; ++v) pp.score_warps[v] = x.score_blocks[v] * (kThreads / 32);
    for (int v = 0; v < N_TB_VARIANTS; ++v) pp.tb_warps[v] = x.tb_blocks[v] * (kThreads / 32);
    pp.score_bnd_bytes = score_bnd_bytes;
    pp.tb_bytes = tb_bytes;
    pp.small_slab_words = kSmallSlabWords;
    pp.allow16 = allow16 ? 1 : 0;
    return pp;
}

// Enqueues one whole batch on st: classification, the device planners,
// every score variant (forked over the auxiliary streams), and with a CIGAR
// the traceback sort, its planner and every traceback variant.  A fixed
// sequence of memsets and launches: no host synchronisation, no allocation.
// expect (or nullptr): per-class counts and maxima a plan was made for.
int enqueue_core(const PairSet &ps, int64_t n_reads, int64_t n_pairs, const Scoring &sc, int score_setting,
                 bool allow16, int32_t *out_score, int32_t *out_end, const sw_cigar_t *cig, const Scratch &S,
                 const int32_t *expect, const ExecCtx &x, cudaStream_t st)
{
    int rc = SW_OK;
    const size_t nh = (size_t)N_CLASS * N_NBUCKET;
    const PlanParams pp = plan_params(x, sc, allow16, S.score_bnd_bytes, S.tb_bytes);
    const bool timing = x.timing && x.phase;
    if (timing && cuda_failed(cudaEventRecord(x.phase[0], st))) return SW_ERR_CUDA;
    if (cuda_failed(cudaMemsetAsync(S.hist, 0, sizeof(int32_t) * nh, st))) return SW_ERR_CUDA;
    if (cuda_failed(cudaMemsetAsync(S.info, 0, sizeof(ClassInfo), st))) return SW_ERR_CUDA;
    if (cuda_failed(cudaMemsetAsync(S.counters, 0, sizeof(int32_t) * N_COUNTERS, st))) return SW_ERR_CUDA;
    if ((rc = launch_classify(ps, n_reads, n_pairs, sc, score_setting, S.keys, S.hist, S.bstart, S.cursor, S.info,
                              S.order, out_score, out_end, cig ? cig->n_ops : nullptr, st)))
        return rc;
    if (expect && (rc = launch_check_counts(S.info, expect, &S.info->status, st))) return rc;
    if ((rc = launch_plan_score(S.info, pp, S.splan, &S.info->status, st))) return rc;
    if (cig) {
        // the score kernels' epilogue writes each pair's traceback cost key
        // and the class table the traceback planner reads
        if (cuda_failed(cudaMemsetAsync(S.hist, 0, sizeof(int32_t) * nh, st))) return SW_ERR_CUDA;
        if (cuda_failed(cudaMemsetAsync(S.tbinfo, 0, sizeof(TbClassInfo), st))) return SW_ERR_CUDA;
        if (cuda_failed(cudaMemsetAsync(S.tb_keys, 0xFF, sizeof(int32_t) * n_pairs, st))) return SW_ERR_CUDA;
    }
    if (timing && cuda_failed(cudaEventRecord(x.phase[1], st))) return SW_ERR_CUDA;
    if ((rc = fork_streams(x, st, kAuxStreams))) return rc;
    for (int v = 0; v < N_SCORE_VARIANTS; ++v) {
        ScoreLaunch L{};
        L.ps = ps;
        L.sc = sc;
        L.order = S.order;
        L.out_score = out_score;
        L.out_end = out_end;
        L.boundary = S.score_bnd;
        L.work_counter = S.counters;
        L.status = &S.info->status;
        if (cig) {
            L.tb_keys = S.tb_keys;
            L.tb_hist = S.hist;
            L.tb_info = S.tbinfo;
            L.small_slab_words = kSmallSlabWords;
        }
        L.dp = S.splan;
        if ((rc = launch_score_variant(v, L, x.score_blocks[v], x.aux[v % kAuxStreams]))) return rc;
    }
    if ((rc = join_streams(x, st, kAuxStreams))) return rc;
    if (timing && cuda_failed(cudaEventRecord(x.phase[2], st))) return SW_ERR_CUDA;
    if (cig) {
        if ((rc = launch_scan_scatter(S.tb_keys, n_pairs, S.info->count, S.hist, S.bstart, S.cursor, S.tb_order,
                                      st)))
            return rc;
        if ((rc = launch_plan_tb(S.info, S.tbinfo, S.splan, pp, S.tplan, &S.info->status, st))) return rc;
        const TbParams P{ps, sc, out_score, out_end, cig->ops, cig->offsets, cig->n_ops, 1, kSmallSlabWords};
        const bool fma = sc.mi >= sc.go;
        // one after another: each launch has the whole slot budget
        for (int v = 0; v < N_TB_VARIANTS; ++v) {
            TracebackLaunch B{};
            B.P = P;
            B.order = S.tb_order;
            B.slab = S.tb;
            B.work_counter = S.counters + CTR_TB;
            B.status = &S.info->status;
            B.dp = S.tplan;
            if ((rc = launch_traceback_variant(v, fma, B, x.tb_blocks[v], st))) return rc;
            if (v < N_TB16_VARIANTS && (rc = launch_tb_walk_variant(v, B, x.walk_blocks[v], st))) return rc;
        }
    }
    if (timing && cuda_failed(cudaEventRecord(x.phase[3], st))) return SW_ERR_CUDA;
    return SW_OK;
}

int run_batch(const PairSet &ps, int64_t n_reads, int64_t n_pairs, const sw_scoring_t *scoring,
              int32_t *out_score, int32_t *out_end, const sw_cigar_t *cig, cudaStream_t st)
{
    DeviceState *ds = nullptr;
    int rc = device_state(&ds, st);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(ds->mu);
    const Scoring sc{scoring->match, scoring->mismatch, scoring->gap_open, scoring->gap_extend};
    Scratch S{};
    const size_t fixed_bytes = fixed_layout(n_pairs, nullptr, S);
    const int64_t bnd_bytes = std::min(kScoreBndMax, std::max(kScoreBndMin, n_pairs * kScoreBndPerPair));
    int64_t tb_bytes = 0;
    if (cig) {
        if (!ds->tb_cap) {
            // once per stream: a share of the memory free at its first traceback
            size_t free_b = 0, total_b = 0;
            ds->tb_cap = kTbCapMin;
            if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess)
                ds->tb_cap = std::max(kTbCapMin, std::min(kTbCapMax, (int64_t)(kTbFreeShare * (double)free_b)));
        }
        tb_bytes = std::min(ds->tb_cap, std::max(kTbMin, n_pairs * kTbPerPair));
    }
    if ((rc = ensure_on(ds->fixed, fixed_bytes, st))) return rc;
    if ((rc = ensure_on(ds->dyn, (size_t)(bnd_bytes + tb_bytes), st))) return rc;
    fixed_layout(n_pairs, (uint8_t *)ds->fixed.ptr, S);
    S.score_bnd = (uint8_t *)ds->dyn.ptr;
    S.score_bnd_bytes = bnd_bytes;
    S.tb = (uint32_t *)((uint8_t *)ds->dyn.ptr + bnd_bytes);
    S.tb_bytes = tb_bytes;
    ds->last_status = &S.info->status;
    ds->timed_cells_valid = false;
    rc = enqueue_core(ps, n_reads, n_pairs, sc, g_score_mode.load(),
                      g_tb_mode.load() == SW_TB_AUTO, out_score, out_end, cig, S, nullptr, ds->x, st);
    if (rc) return rc;
    if (cig) ds->last_tplan = S.tplan;
    ds->timed_cells_valid = ds->timing;
    return SW_OK;
}

int read_status(DeviceState *ds, cudaStream_t st)
{
    if (cuda_failed(cudaStreamSynchronize(st))) return SW_ERR_CUDA;
    std::lock_guard<std::mutex> lk(ds->mu);
    if (!ds->last_status) return SW_OK;
    int32_t v = 0;
    if (cuda_failed(cudaMemcpy(&v, ds->last_status, sizeof(v), cudaMemcpyDeviceToHost))) return SW_ERR_CUDA;
    return status_to_code(v);
}

int check_common(const void *reads, const int64_t *roff, const void *wins, const int64_t *woff, int64_t n_pairs,
                 const sw_scoring_t *scoring, const int32_t *out_score, const int32_t *out_end,
                 const sw_cigar_t *cig)
{
    if (n_pairs < 0 || !scoring_ok(scoring)) return SW_ERR_INVALID_ARG;
    if (n_pairs == 0) return SW_OK;
    if (!reads || !roff || !wins || !woff || !out_score || !out_end) return SW_ERR_INVALID_ARG;
    if (((uintptr_t)reads & 15u) || ((uintptr_t)wins & 15u)) return SW_ERR_INVALID_ARG;
    if (cig && (!cig->ops || !cig->offsets || !cig->n_ops)) return SW_ERR_INVALID_ARG;
    if (n_pairs > (int64_t)INT32_MAX - 64) return SW_ERR_UNSUPPORTED;
    return SW_OK;
}

// ---------------------------------------------------------------------------
// Plans: one batch shape classified once on the host, its scratch allocated
// for the worst case of that shape, and every execution the same fixed
// sequence as sw_batch_align plus a device check that the batch still has
// the plan's shape.

}  // namespace
}  // namespace swgb

struct sw_plan {
    int device = -1;
    swgb::PairSet ps{};  // offsets and pair map (bases bound per execution)
    int64_t n_reads = 0, n_pairs = 0;
    swgb::Scoring sc{};
    bool cigar = false;
    int score_setting = SW_SCORE_AUTO;  // the score mode setting at creation
    bool allow16 = true;      // the traceback mode setting at creation
    swgb::Buffer fixed, dyn;  // owned: a captured graph keeps pointing here
    swgb::Scratch S{};
    swgb::ExecCtx x;          // owned auxiliary streams and events (a capture creates nothing)
};

namespace swgb {
namespace {

// Worst-case scratch of a shape: every window may lie inside the band, so
// a chunk window is at most the class's longest window (and smaller ones may
// pick other traceback kernels, whose slots are bounded too).
void plan_budgets(const ClassInfo &ci, const PlanParams &pp, bool cigar, int64_t &bnd_bytes, int64_t &tb_bytes)
{
    int64_t slot_s[N_SCORE_VARIANTS] = {};
    for (int c = 0; c < N_CLASS; ++c) {
        if (!ci.count[c]) continue;
        const int mode = c / N_MCLASS;
        const int32_t mm = ci.max_m[c], mn = ci.max_n[c];
        int lanes = 1, ri = 0;
        score_plan_of(mode, mm, (int64_t)pp.sc.ma * std::min(mm, mn), pp.ov, pp.n_overrides, lanes, ri);
        const int rows = score_rows_at(ri);
        if ((mm + lanes * rows - 1) / (lanes * rows) > 1) {
            const int v = ri * N_MODES + mode;
            slot_s[v] = std::max<int64_t>(slot_s[v], (int64_t)(32 / lanes) * 16 * mn);
        }
    }
    int nb = 0;
    int64_t per = 0;
    for (int v = 0; v < N_SCORE_VARIANTS; ++v)
        if (slot_s[v]) {
            ++nb;
            per = std::max(per, slot_s[v] * pp.score_warps[v]);
        }
    bnd_bytes = std::max<int64_t>(nb * (int64_t)align_up(per, 256), 256);
    tb_bytes = 0;
    if (!cigar) return;
    // per traceback launch: its widest boundary row, tile and slot over the
    // classes it may serve, and the pool all of its tasks would fill
    int64_t bnd_v[N_TB_VARIANTS] = {}, slot_v[N_TB_VARIANTS] = {}, pool_v[N_TB_VARIANTS] = {};
    for (int c = 0; c < N_CLASS; ++c) {
        if (!ci.count[c]) continue;
        const int mode = c / N_MCLASS;
        const int32_t mm = ci.max_m[c], mn = std::max(ci.max_n[c], 1);
        const int64_t chunks = (mm + TB_ROWS - 1) / TB_ROWS;
        // the widest window, and the widest below each kernel switch
        const int64_t cand[3] = {mn, std::min<int64_t>(mn, kTiledLaneWords16 / (2 * chunks) / 4 * 4),
                                 std::min<int64_t>(mn, kTiledLaneWords / chunks)};
        for (int64_t w : cand) {
            if (w < 1) continue;
            for (int part = 0; part < 2; ++part) {
                TbPartPlan t{};
                const int64_t slot = tb_part_shape(mode, pp.allow16 != 0, mm, chunks * w, (int32_t)w, part,
                                                   pp.small_slab_words, t);
                const int v = t.variant;
                if (v < N_TB16_VARIANTS) {
                    const int64_t tile = (32 * t.slab_words + 63) & ~(int64_t)63;
                    const int64_t tasks = (ci.count[c] + 2 * (32 >> v) - 1) / (2 * (32 >> v));
                    bnd_v[v] = std::max(bnd_v[v], (t.bnd_ints + 63) & ~(int64_t)63);
                    slot_v[v] = std::max(slot_v[v], tile);
                    pool_v[v] = std::max(pool_v[v], tasks * tile);  // one candidate per class counts
                } else {
                    slot_v[v] = std::max(slot_v[v], (slot + 63) & ~(int64_t)63);
                }
            }
        }
    }
    const int64_t cap = kTbCapMax / 4;  // words
    for (int v = 0; v < N_TB_VARIANTS; ++v) {
        if (!slot_v[v]) continue;
        const int64_t w = pp.tb_warps[v];
        int64_t words;
        if (v < N_TB16_VARIANTS)
            words = std::min(w * bnd_v[v], cap) + std::max({std::min(pool_v[v] + slot_v[v], cap),
                                                            std::min(w * slot_v[v], cap), slot_v[v]});
        else
            words = std::max(std::min(w * slot_v[v], cap), 4 * slot_v[v]);
        tb_bytes = std::max(tb_bytes, 4 * words);
    }
}

int plan_build(sw_plan *pl, DeviceState *ds, cudaStream_t st)
{
    int rc = SW_OK;
    const int64_t n_pairs = pl->n_pairs;
    Scratch &S = pl->S;
    if ((rc = ensure(pl->fixed, fixed_layout(n_pairs, nullptr, S)))) return rc;
    fixed_layout(n_pairs, (uint8_t *)pl->fixed.ptr, S);
    // classify once (it reads offsets only) and read the class table back
    const size_t nh = (size_t)N_CLASS * N_NBUCKET;
    if (cuda_failed(cudaMemsetAsync(S.hist, 0, sizeof(int32_t) * nh, st))) return SW_ERR_CUDA;
    if (cuda_failed(cudaMemsetAsync(S.info, 0, sizeof(ClassInfo), st))) return SW_ERR_CUDA;
    int32_t *tmp_score = S.tb_keys, *tmp_end = nullptr;  // empty-window outputs go to scratch
    if ((rc = ensure(pl->dyn, sizeof(int32_t) * 2 * std::max<int64_t>(n_pairs, 1)))) return rc;
    tmp_end = (int32_t *)pl->dyn.ptr;
    if ((rc = launch_classify(pl->ps, pl->n_reads, n_pairs, pl->sc, pl->score_setting, S.keys, S.hist, S.bstart,
                              S.cursor, S.info, S.order, tmp_score, tmp_end, nullptr, st)))
        return rc;
    ClassInfo ci;
    if (cuda_failed(cudaMemcpyAsync(&ci, S.info, sizeof(ClassInfo), cudaMemcpyDeviceToHost, st)))
        return SW_ERR_CUDA;
    if (cuda_failed(cudaStreamSynchronize(st))) return SW_ERR_CUDA;
    if (ci.status) return status_to_code(ci.status);
    {
        std::vector<int32_t> ex(3 * N_CLASS);
        std::memcpy(ex.data(), ci.count, sizeof(int32_t) * N_CLASS);
        std::memcpy(ex.data() + N_CLASS, ci.max_m, sizeof(int32_t) * N_CLASS);
        std::memcpy(ex.data() + 2 * N_CLASS, ci.max_n, sizeof(int32_t) * N_CLASS);
        if (cuda_failed(cudaMemcpy(S.expect, ex.data(), sizeof(int32_t) * 3 * N_CLASS, cudaMemcpyHostToDevice)))
            return SW_ERR_CUDA;
    }
    if ((rc = exec_ctx_init(pl->x, ds->sm_count))) return rc;
    const PlanParams pp = plan_params(pl->x, pl->sc, pl->allow16, 0, 0);
    int64_t bnd_bytes = 0, tb_bytes = 0;
    plan_budgets(ci, pp, pl->cigar, bnd_bytes, tb_bytes);
    if ((rc = ensure(pl->dyn, (size_t)(bnd_bytes + tb_bytes)))) return rc;
    S.score_bnd = (uint8_t *)pl->dyn.ptr;
    S.score_bnd_bytes = bnd_bytes;
    S.tb = (uint32_t *)((uint8_t *)pl->dyn.ptr + bnd_bytes);
    S.tb_bytes = tb_bytes;
    return SW_OK;
}

int plan_execute(sw_plan *pl, int32_t *out_score, int32_t *out_end, const sw_cigar_t *cig, cudaStream_t st)
{
    return enqueue_core(pl->ps, pl->n_reads, pl->n_pairs, pl->sc, pl->score_setting, pl->allow16, out_score, out_end,
                        pl->cigar ? cig : nullptr, pl->S, pl->S.expect, pl->x, st);
}

}  // namespace
}  // namespace swgb

using namespace swgb;

extern "C" {

int64_t sw_cigar_capacity(int64_t read_len) { return read_len < 0 ? 0 : 2 * read_len + 3; }

int64_t sw_packed_bytes(int64_t n_bases)
{
    if (n_bases < 0) return 0;
    return ((n_bases + 3) / 4 + 15) / 16 * 16;
}

int sw_batch_align(const uint8_t *reads, const int64_t *read_offsets, const uint8_t *windows,
                   const int64_t *window_offsets, int64_t n_pairs, const sw_scoring_t *scoring, int32_t *out_score,
                   int32_t *out_end, sw_cigar_t *out_cigar, sw_stream_t stream)
{
    int rc = check_common(reads, read_offsets, windows, window_offsets, n_pairs, scoring, out_score, out_end,
                          out_cigar);
    if (rc || n_pairs == 0) return rc;
    PairSet ps{(const uint32_t *)reads, read_offsets, nullptr, (const uint32_t *)windows, window_offsets};
    return run_batch(ps, n_pairs, n_pairs, scoring, out_score, out_end, out_cigar, (cudaStream_t)stream);
}

int sw_batch_align_indexed(const uint8_t *reads, const int64_t *read_offsets, int64_t n_reads,
                           const uint8_t *windows, const int64_t *window_offsets, const int64_t *pair_read,
                           int64_t n_pairs, const sw_scoring_t *scoring, int32_t *out_score, int32_t *out_end,
                           sw_cigar_t *out_cigar, sw_stream_t stream)
{
    int rc = check_common(reads, read_offsets, windows, window_offsets, n_pairs, scoring, out_score, out_end,
                          out_cigar);
    if (rc || n_pairs == 0) return rc;
    if (!pair_read || n_reads < 1) return SW_ERR_INVALID_ARG;
    PairSet ps{(const uint32_t *)reads, read_offsets, pair_read, (const uint32_t *)windows, window_offsets};
    return run_batch(ps, n_reads, n_pairs, scoring, out_score, out_end, out_cigar, (cudaStream_t)stream);
}

int sw_batch_align_masked(const uint8_t *reads, const int64_t *read_offsets, int64_t n_reads,
                          const uint8_t *windows, const int64_t *window_offsets, const int64_t *pair_read,
                          const uint8_t *pair_mask, int64_t n_pairs, const sw_scoring_t *scoring, int32_t *out_score,
                          int32_t *out_end, sw_cigar_t *out_cigar, sw_stream_t stream)
{
    int rc = check_common(reads, read_offsets, windows, window_offsets, n_pairs, scoring, out_score, out_end,
                          out_cigar);
    if (rc || n_pairs == 0) return rc;
    if (!pair_read || !pair_mask || n_reads < 1) return SW_ERR_INVALID_ARG;
    PairSet ps{(const uint32_t *)reads, read_offsets, pair_read, (const uint32_t *)windows, window_offsets,
               pair_mask};
    return run_batch(ps, n_reads, n_pairs, scoring, out_score, out_end, out_cigar, (cudaStream_t)stream);
}

int sw_batch_align_host(const uint8_t *reads, const int64_t *read_offsets, const uint8_t *windows,
                        const int64_t *window_offsets, int64_t n_pairs, const sw_scoring_t *scoring,
                        int32_t *out_score, int32_t *out_end, sw_cigar_t *out_cigar, sw_stream_t stream)
{
    int rc = check_common(reads, read_offsets, windows, window_offsets, n_pairs, scoring, out_score, out_end,
                          out_cigar);
    if (rc || n_pairs == 0) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    DeviceState *ds = nullptr;
    if ((rc = device_state(&ds, (cudaStream_t)stream))) return rc;
    const int64_t rb = sw_packed_bytes(read_offsets[n_pairs]);
    const int64_t wb = sw_packed_bytes(window_offsets[n_pairs]);
    const int64_t n_cig = out_cigar ? out_cigar->offsets[n_pairs] : 0;
    size_t off = 0;
    const size_t o_r = off; off = align_up(off + rb, 256);
    const size_t o_w = off; off = align_up(off + wb, 256);
    const size_t o_ro = off; off = align_up(off + 8 * (n_pairs + 1), 256);
    const size_t o_wo = off; off = align_up(off + 8 * (n_pairs + 1), 256);
    const size_t o_s = off; off = align_up(off + 4 * n_pairs, 256);
    const size_t o_e = off; off = align_up(off + 8 * n_pairs, 256);
    const size_t o_co = off; off = align_up(off + (out_cigar ? 8 * (n_pairs + 1) : 0), 256);
    const size_t o_cn = off; off = align_up(off + (out_cigar ? 4 * n_pairs : 0), 256);
    const size_t o_ops = off; off = align_up(off + 4 * n_cig, 256);
    {
        std::lock_guard<std::mutex> lk(ds->mu);
        if ((rc = ensure(ds->stage, off))) return rc;
    }
    uint8_t *b = (uint8_t *)ds->stage.ptr;
    // The batch goes in chunks of pairs through one device copy of it: chunk
    // c+1's inputs are copied in (copy stream) while chunk c computes (the
    // caller's stream) and chunk c-1's outputs are copied out (a second copy
    // stream).  Every chunk uses the batch's own offsets into the shared copy.
    // (with a CIGAR one chunk: measured, the chunks' copies slowed the kernels
    // more than the overlap saved)
    const int64_t n_split = out_cigar ? 1 : kHostChunks;
    const int64_t chunk = std::max<int64_t>(kHostChunkMin, (n_pairs + n_split - 1) / n_split);
    const int64_t n_chunks = (n_pairs + chunk - 1) / chunk;
    auto h2d = [&](size_t o, const void *src, size_t n) {
        return n == 0 || !cuda_failed(cudaMemcpyAsync(b + o, src, n, cudaMemcpyHostToDevice, ds->copy_in));
    };
    auto d2h = [&](void *dst, size_t o, size_t n) {
        return n == 0 || !cuda_failed(cudaMemcpyAsync(dst, b + o, n, cudaMemcpyDeviceToHost, ds->copy_out));
    };
    // the whole words holding bases [q0, q1)
    auto word_bytes = [](int64_t q0, int64_t q1, int64_t total, int64_t &lo, int64_t &n) {
        lo = (q0 >> 4) * 4;
        n = std::min<int64_t>(total, ((q1 + 15) >> 4) * 4) - lo;
        if (n < 0) n = 0;
    };
    auto copy_in = [&](int64_t c) -> bool {
        const int64_t p0 = c * chunk, p1 = std::min<int64_t>(n_pairs, p0 + chunk);
        int64_t lo = 0, n = 0;
        word_bytes(read_offsets[p0], read_offsets[p1], rb, lo, n);
        if (!h2d(o_r + lo, reads + lo, n)) return false;
        word_bytes(window_offsets[p0], window_offsets[p1], wb, lo, n);
        if (!h2d(o_w + lo, windows + lo, n)) return false;
        if (!h2d(o_ro + 8 * p0, read_offsets + p0, 8 * (p1 - p0 + 1))) return false;
        if (!h2d(o_wo + 8 * p0, window_offsets + p0, 8 * (p1 - p0 + 1))) return false;
        if (out_cigar && !h2d(o_co + 8 * p0, out_cigar->offsets + p0, 8 * (p1 - p0 + 1))) return false;
        return !cuda_failed(cudaEventRecord(ds->host_in_ev[c % kHostChunks], ds->copy_in));
    };
    // CIGAR runs go straight into the caller's slots when its op buffer is
    // pinned host memory the device can address; else the slots are copied
    uint32_t *host_ops_dev = nullptr;
    if (out_cigar) {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, out_cigar->ops) == cudaSuccess && at.type == cudaMemoryTypeHost &&
            at.devicePointer)
            host_ops_dev = (uint32_t *)at.devicePointer;
        cudaGetLastError();  // a pageable pointer is not an error here
    }
    // the copy streams start after what the caller enqueued on st
    if (cuda_failed(cudaEventRecord(ds->x.fork_ev, st))) return SW_ERR_CUDA;
    if (cuda_failed(cudaStreamWaitEvent(ds->copy_in, ds->x.fork_ev, 0))) return SW_ERR_CUDA;
    if (cuda_failed(cudaStreamWaitEvent(ds->copy_out, ds->x.fork_ev, 0))) return SW_ERR_CUDA;
    if (!copy_in(0)) return SW_ERR_CUDA;
    for (int64_t c = 0; c < n_chunks; ++c) {
        const int64_t p0 = c * chunk, p1 = std::min<int64_t>(n_pairs, p0 + chunk), np = p1 - p0;
        // the next chunk's inputs, queued before this chunk's host waits
        if (c + 1 < n_chunks) {
            // its event slot must be free: the chunk kHostChunks back has started
            if (!copy_in(c + 1)) return SW_ERR_CUDA;
        }
        if (cuda_failed(cudaStreamWaitEvent(st, ds->host_in_ev[c % kHostChunks], 0))) return SW_ERR_CUDA;
        sw_cigar_t dc{};
        if (out_cigar) {
            dc.ops = (uint32_t *)(b + o_ops);
            dc.offsets = (const int64_t *)(b + o_co) + p0;
            dc.n_ops = (int32_t *)(b + o_cn) + p0;
        }
        PairSet ps{(const uint32_t *)(b + o_r), (const int64_t *)(b + o_ro) + p0, nullptr,
                   (const uint32_t *)(b + o_w), (const int64_t *)(b + o_wo) + p0};
        rc = run_batch(ps, np, np, scoring, (int32_t *)(b + o_s) + p0, (int32_t *)(b + o_e) + 2 * p0,
                       out_cigar ? &dc : nullptr, st);
        if (rc) return rc;
        if (host_ops_dev &&
            (rc = launch_cigar_to_host(dc.ops, dc.offsets, dc.n_ops, np, host_ops_dev, st)))
            return rc;
        // this chunk's outputs, once its kernels are done
        if (cuda_failed(cudaEventRecord(ds->host_out_ev, st))) return SW_ERR_CUDA;
        if (cuda_failed(cudaStreamWaitEvent(ds->copy_out, ds->host_out_ev, 0))) return SW_ERR_CUDA;
        if (!d2h(out_score + p0, o_s + 4 * p0, 4 * np) || !d2h(out_end + 2 * p0, o_e + 8 * p0, 8 * np))
            return SW_ERR_CUDA;
        if (out_cigar) {
            const int64_t c0 = out_cigar->offsets[p0], c1 = out_cigar->offsets[p1];
            if (!d2h(out_cigar->n_ops + p0, o_cn + 4 * p0, 4 * np)) return SW_ERR_CUDA;
            if (!host_ops_dev && !d2h(out_cigar->ops + c0, o_ops + 4 * c0, 4 * (c1 - c0))) return SW_ERR_CUDA;
        }
    }
    // st ends after the last copy out
    if (cuda_failed(cudaEventRecord(ds->host_out_ev, ds->copy_out))) return SW_ERR_CUDA;
    if (cuda_failed(cudaStreamWaitEvent(st, ds->host_out_ev, 0))) return SW_ERR_CUDA;
    return read_status(ds, st);
}

int sw_last_cuda_error(const char **name)
{
    if (name) *name = cudaGetErrorName((cudaError_t)g_cuda_error);
    return g_cuda_error;
}

int sw_stream_release(sw_stream_t stream)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SW_ERR_NO_DEVICE;
    const cudaStream_t st = (cudaStream_t)stream;
    DeviceState *s = nullptr;
    {
        std::lock_guard<std::mutex> glk(g_state_mu);
        for (size_t i = 0; i < g_states.size(); ++i)
            if (g_states[i].first.first == dev && g_states[i].first.second == st) {
                s = g_states[i].second;
                g_states.erase(g_states.begin() + i);
                break;
            }
        if (s && g_last_state[dev] == s) g_last_state[dev] = nullptr;
    }
    if (!s) return SW_OK;
    const int rc = cuda_failed(cudaStreamSynchronize(st)) ? SW_ERR_CUDA : SW_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        free_state(s);
    }
    delete s;
    return rc;
}

int sw_sync_status(sw_stream_t stream)
{
    DeviceState *ds = nullptr;
    int rc = device_state(&ds, (cudaStream_t)stream);
    if (rc) return rc;
    return read_status(ds, (cudaStream_t)stream);
}

int sw_get_status(sw_stream_t stream) { return sw_sync_status(stream); }

const char *sw_strerror(int code)
{
    switch (code) {
    case SW_OK: return "ok";
    case SW_ERR_INVALID_ARG: return "invalid argument";
    case SW_ERR_CAPACITY: return "CIGAR slot too small";
    case SW_ERR_CUDA: return "CUDA runtime error";
    case SW_ERR_DEVICE_TIMEOUT: return "device-side wait timed out";
    case SW_ERR_UNSUPPORTED: return "size beyond supported limits";
    case SW_ERR_DEVICE_INPUT: return "device-resident input failed validation";
    case SW_ERR_INTERNAL: return "internal consistency check failed";
    case SW_ERR_NO_DEVICE: return "no usable CUDA device";
    default: return "unknown error";
    }
}

int64_t sw_launch_count(void) { return g_launches.load(); }

int sw_set_plan(int32_t max_read_len, int32_t lanes, int32_t r_rows)
{
    std::lock_guard<std::mutex> lk(g_plan_mu);
    if (max_read_len <= 0) {
        g_plans.clear();
        return SW_OK;
    }
    if (lanes < 1 || lanes > 32) return SW_ERR_INVALID_ARG;
    bool ok = false;
    for (int i = 0; i < N_SCORE_ROWS; ++i) ok |= kScoreRows[i] == r_rows;
    if (!ok) return SW_ERR_INVALID_ARG;
    if ((max_read_len + lanes * r_rows - 1) / (lanes * r_rows) > 1 && lanes != 32) return SW_ERR_INVALID_ARG;
    if (g_plans.size() >= (size_t)kMaxPlanOverrides) return SW_ERR_UNSUPPORTED;
    g_plans.push_back(PlanOverride{max_read_len, lanes, r_rows});
    std::sort(g_plans.begin(), g_plans.end(),
              [](const PlanOverride &a, const PlanOverride &b) { return a.max_read_len < b.max_read_len; });
    return SW_OK;
}

int sw_plan_query(int32_t max_read_len, int32_t max_window_len, int32_t match, int32_t *lanes, int32_t *r_rows)
{
    if (!lanes || !r_rows || max_read_len < 1 || max_read_len > SW_MAX_READ_LEN || max_window_len < 1 ||
        match < 1 || match > 127)
        return SW_ERR_INVALID_ARG;
    const int64_t hmax = (int64_t)match * std::min(max_read_len, max_window_len);
    const int mode = score_mode_for(hmax, g_score_mode.load());
    PlanOverride ov[kMaxPlanOverrides];
    int n_ov = 0;
    {
        std::lock_guard<std::mutex> lk(g_plan_mu);
        n_ov = (int)std::min<size_t>(g_plans.size(), kMaxPlanOverrides);
        for (int i = 0; i < n_ov; ++i) ov[i] = g_plans[i];
    }
    int l = 0, ri = 0;
    score_plan_of(mode, max_read_len, hmax, ov, n_ov, l, ri);
    *lanes = l;
    *r_rows = score_rows_at(ri);
    return SW_OK;
}

int sw_set_traceback_mode(int32_t mode)
{
    if (mode != SW_TB_AUTO && mode != SW_TB_INT32) return SW_ERR_INVALID_ARG;
    g_tb_mode.store(mode);
    return SW_OK;
}

int sw_set_score_mode(int32_t mode)
{
    if (mode != SW_SCORE_AUTO && mode != SW_SCORE_INT32 && mode != SW_SCORE_WIDE16) return SW_ERR_INVALID_ARG;
    g_score_mode.store(mode);
    return SW_OK;
}

int sw_plan_rows(int32_t *rows, int32_t cap)
{
    if (!rows) return N_SCORE_ROWS;
    for (int i = 0; i < N_SCORE_ROWS && i < cap; ++i) rows[i] = kScoreRows[i];
    return N_SCORE_ROWS;
}

int sw_last_traceback_split(int64_t *out2)
{
    if (!out2) return SW_ERR_INVALID_ARG;
    DeviceState *ds = nullptr;
    const int rc = last_state(&ds);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(ds->mu);
    out2[0] = out2[1] = 0;
    if (!ds->last_tplan) return SW_OK;
    // the split is planned on the device: wait for it
    if (cuda_failed(cudaDeviceSynchronize())) return SW_ERR_CUDA;
    if (cuda_failed(cudaMemcpy(out2, ds->last_tplan->split, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost)))
        return SW_ERR_CUDA;
    return SW_OK;
}

int sw_phase_timing(int32_t enable)
{
    int dev = 0;
    if (cuda_failed(cudaGetDevice(&dev)) || dev < 0 || dev >= kMaxDevices) return SW_ERR_NO_DEVICE;
    std::lock_guard<std::mutex> glk(g_state_mu);
    g_timing[dev] = enable != 0;
    return SW_OK;
}

int sw_phase_times(float *ms3)
{
    if (!ms3) return SW_ERR_INVALID_ARG;
    DeviceState *ds = nullptr;
    int rc = last_state(&ds);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(ds->mu);
    if (!ds->timed_cells_valid) return SW_ERR_INVALID_ARG;
    if (cuda_failed(cudaEventSynchronize(ds->phase[3]))) return SW_ERR_CUDA;
    for (int i = 0; i < 3; ++i)
        if (cuda_failed(cudaEventElapsedTime(&ms3[i], ds->phase[i], ds->phase[i + 1]))) return SW_ERR_CUDA;
    return SW_OK;
}

int sw_plan_create(const int64_t *read_offsets, int64_t n_reads, const int64_t *window_offsets,
                   const int64_t *pair_read, int64_t n_pairs, const sw_scoring_t *scoring, int32_t with_cigar,
                   sw_stream_t stream, sw_plan_t **out_plan)
{
    if (!out_plan) return SW_ERR_INVALID_ARG;
    *out_plan = nullptr;
    if (!read_offsets || !window_offsets || n_pairs < 1 || !scoring_ok(scoring)) return SW_ERR_INVALID_ARG;
    if (pair_read && n_reads < 1) return SW_ERR_INVALID_ARG;
    if (n_pairs > (int64_t)INT32_MAX - 64) return SW_ERR_UNSUPPORTED;
    DeviceState *ds = nullptr;
    int rc = device_state(&ds, (cudaStream_t)stream);
    if (rc) return rc;
    sw_plan *pl = new (std::nothrow) sw_plan();
    if (!pl) return SW_ERR_INVALID_ARG;
    cudaGetDevice(&pl->device);
    pl->ps = PairSet{nullptr, read_offsets, pair_read, nullptr, window_offsets};
    pl->n_reads = pair_read ? n_reads : n_pairs;
    pl->n_pairs = n_pairs;
    pl->sc = Scoring{scoring->match, scoring->mismatch, scoring->gap_open, scoring->gap_extend};
    pl->cigar = with_cigar != 0;
    pl->score_setting = g_score_mode.load();
    pl->allow16 = g_tb_mode.load() == SW_TB_AUTO;
    {
        std::lock_guard<std::mutex> lk(ds->mu);
        rc = plan_build(pl, ds, (cudaStream_t)stream);
    }
    if (rc) {
        sw_plan_destroy(pl);
        return rc;
    }
    *out_plan = pl;
    return SW_OK;
}

int sw_plan_align(sw_plan_t *plan, const uint8_t *reads, const uint8_t *windows, int32_t *out_score,
                  int32_t *out_end, sw_cigar_t *out_cigar, sw_stream_t stream)
{
    if (!plan || !reads || !windows || !out_score || !out_end) return SW_ERR_INVALID_ARG;
    if (((uintptr_t)reads & 15u) || ((uintptr_t)windows & 15u)) return SW_ERR_INVALID_ARG;
    if (out_cigar && (!out_cigar->ops || !out_cigar->offsets || !out_cigar->n_ops)) return SW_ERR_INVALID_ARG;
    if (out_cigar && !plan->cigar) return SW_ERR_INVALID_ARG;
    int dev = -1;
    if (cuda_failed(cudaGetDevice(&dev)) || dev != plan->device) return SW_ERR_INVALID_ARG;
    plan->ps.reads = (const uint32_t *)reads;
    plan->ps.wins = (const uint32_t *)windows;
    return plan_execute(plan, out_score, out_end, out_cigar, (cudaStream_t)stream);
}

int sw_plan_status(sw_plan_t *plan, sw_stream_t stream)
{
    if (!plan) return SW_ERR_INVALID_ARG;
    if (cuda_failed(cudaStreamSynchronize((cudaStream_t)stream))) return SW_ERR_CUDA;
    int32_t v = 0;
    if (cuda_failed(cudaMemcpy(&v, &plan->S.info->status, sizeof(v), cudaMemcpyDeviceToHost))) return SW_ERR_CUDA;
    return status_to_code(v);
}

int sw_plan_destroy(sw_plan_t *plan)
{
    if (!plan) return SW_OK;
    int prev = -1;
    cudaGetDevice(&prev);
    if (plan->device >= 0) cudaSetDevice(plan->device);
    cudaDeviceSynchronize();
    if (plan->fixed.ptr) cudaFree(plan->fixed.ptr);
    if (plan->dyn.ptr) cudaFree(plan->dyn.ptr);
    exec_ctx_free(plan->x);
    if (prev >= 0) cudaSetDevice(prev);
    delete plan;
    return SW_OK;
}

int sw_batch_align_host_dense(const uint8_t *reads, const int64_t *read_offsets, const uint8_t *windows,
                              const int64_t *window_offsets, int64_t n_pairs, const sw_scoring_t *scoring,
                              int32_t *out_score, int32_t *out_end, uint32_t *ops_out, int64_t ops_cap,
                              int64_t *offsets_out, sw_stream_t stream)
{
    int rc = check_common(reads, read_offsets, windows, window_offsets, n_pairs, scoring, out_score, out_end,
                          nullptr);
    if (rc) return rc;
    if (!offsets_out || ops_cap < 0 || (ops_cap > 0 && !ops_out)) return SW_ERR_INVALID_ARG;
    if (n_pairs == 0) {
        offsets_out[0] = 0;
        return SW_OK;
    }
    cudaStream_t st = (cudaStream_t)stream;
    DeviceState *ds = nullptr;
    if ((rc = device_state(&ds, (cudaStream_t)stream))) return rc;
    const int64_t rb = sw_packed_bytes(read_offsets[n_pairs]);
    const int64_t wb = sw_packed_bytes(window_offsets[n_pairs]);
    // device slots of 2m + 3 runs per pair
    const int64_t n_slots = 2 * (read_offsets[n_pairs] - read_offsets[0]) + 3 * n_pairs;
    const int64_t dense_cap = std::min<int64_t>(std::max<int64_t>(ops_cap, 1), n_slots);
    const int64_t n_blk = (n_pairs + 255) / 256;
    size_t off = 0;
    const size_t o_r = off; off = align_up(off + rb, 256);
    const size_t o_w = off; off = align_up(off + wb, 256);
    const size_t o_ro = off; off = align_up(off + 8 * (n_pairs + 1), 256);
    const size_t o_wo = off; off = align_up(off + 8 * (n_pairs + 1), 256);
    const size_t o_s = off; off = align_up(off + 4 * n_pairs, 256);
    const size_t o_e = off; off = align_up(off + 8 * n_pairs, 256);
    const size_t o_co = off; off = align_up(off + 8 * (n_pairs + 1), 256);
    const size_t o_cn = off; off = align_up(off + 4 * n_pairs, 256);
    const size_t o_ops = off; off = align_up(off + 4 * n_slots, 256);
    const size_t o_do = off; off = align_up(off + 8 * (n_pairs + 1), 256);
    const size_t o_dense = off; off = align_up(off + 4 * dense_cap, 256);
    const size_t o_blk = off; off = align_up(off + 8 * n_blk, 256);
    {
        std::lock_guard<std::mutex> lk(ds->mu);
        if ((rc = ensure(ds->stage, off))) return rc;
    }
    uint8_t *b = (uint8_t *)ds->stage.ptr;
    auto h2d = [&](size_t o, const void *src, size_t n) {
        return n == 0 || !cuda_failed(cudaMemcpyAsync(b + o, src, n, cudaMemcpyHostToDevice, st));
    };
    auto d2h = [&](void *dst, size_t o, size_t n) {
        return n == 0 || !cuda_failed(cudaMemcpyAsync(dst, b + o, n, cudaMemcpyDeviceToHost, st));
    };
    if (!h2d(o_r, reads, rb) || !h2d(o_w, windows, wb) || !h2d(o_ro, read_offsets, 8 * (n_pairs + 1)) ||
        !h2d(o_wo, window_offsets, 8 * (n_pairs + 1)))
        return SW_ERR_CUDA;
    int64_t *cig_off = (int64_t *)(b + o_co), *blk = (int64_t *)(b + o_blk);
    if ((rc = launch_cap_offsets((const int64_t *)(b + o_ro), n_pairs, cig_off, blk, st))) return rc;
    // the slots are counted from the first read's start
    sw_cigar_t dc{(uint32_t *)(b + o_ops), cig_off, (int32_t *)(b + o_cn)};
    PairSet ps{(const uint32_t *)(b + o_r), (const int64_t *)(b + o_ro), nullptr, (const uint32_t *)(b + o_w),
               (const int64_t *)(b + o_wo)};
    if ((rc = run_batch(ps, n_pairs, n_pairs, scoring, (int32_t *)(b + o_s), (int32_t *)(b + o_e), &dc, st)))
        return rc;
    int64_t *doff = (int64_t *)(b + o_do);
    if ((rc = launch_dense_cigar(dc.ops, cig_off, dc.n_ops, n_pairs, doff, (uint32_t *)(b + o_dense), dense_cap, blk,
                                 st)))
        return rc;
    if (!d2h(out_score, o_s, 4 * n_pairs) || !d2h(out_end, o_e, 8 * n_pairs) ||
        !d2h(offsets_out, o_do, 8 * (n_pairs + 1)))
        return SW_ERR_CUDA;
    if (cuda_failed(cudaStreamSynchronize(st))) return SW_ERR_CUDA;
    const int64_t total = offsets_out[n_pairs];
    const int64_t n_copy = std::min<int64_t>(total, ops_cap);
    if (!d2h(ops_out, o_dense, 4 * n_copy)) return SW_ERR_CUDA;
    rc = read_status(ds, st);
    if (rc) return rc;
    return total > ops_cap ? SW_ERR_CAPACITY : SW_OK;
}

// ---- Stage E, task iv ---------------------------------------------------

}  // extern "C"

namespace swgb {
int aux_status_word(cudaStream_t st, int32_t **status)
{
    DeviceState *ds = nullptr;
    int rc = device_state(&ds, st);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(ds->mu);
    if ((rc = ensure(ds->misc, 256))) return rc;
    *status = (int32_t *)ds->misc.ptr;
    if (cuda_failed(cudaMemsetAsync(*status, 0, sizeof(int32_t), st))) return SW_ERR_CUDA;
    ds->last_status = *status;
    return SW_OK;
}
// Scratch of sw_filter_align on this stream (grown on demand).
int filter_scratch(cudaStream_t st, size_t bytes, uint8_t **ptr)
{
    DeviceState *ds = nullptr;
    int rc = device_state(&ds, st);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(ds->mu);
    if ((rc = ensure(ds->filt, bytes))) return rc;
    *ptr = (uint8_t *)ds->filt.ptr;
    return SW_OK;
}

int grad_scratch(cudaStream_t st, size_t bytes, float **ptr)
{
    DeviceState *ds = nullptr;
    int rc = device_state(&ds, st);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(ds->mu);
    if ((rc = ensure(ds->grad, bytes))) return rc;
    *ptr = (float *)ds->grad.ptr;
    return SW_OK;
}

// The status word sw_sync_status will read for this stream's last call.
int stream_status_word(cudaStream_t st, int32_t **status)
{
    DeviceState *ds = nullptr;
    int rc = device_state(&ds, st);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(ds->mu);
    *status = ds->last_status;
    return SW_OK;
}
}  // namespace swgb

extern "C" {

static int stage_e_status(DeviceState *ds, size_t extra, cudaStream_t st, int32_t **status, uint8_t **scratch)
{
    // a status word in front of the scratch, cleared by each call
    int rc = ensure(ds->misc, 256 + extra);
    if (rc) return rc;
    *status = (int32_t *)ds->misc.ptr;
    *scratch = (uint8_t *)ds->misc.ptr + 256;
    if (cuda_failed(cudaMemsetAsync(*status, 0, sizeof(int32_t), st))) return SW_ERR_CUDA;
    ds->last_status = *status;
    return SW_OK;
}

int sw_records(const int32_t *score, const int32_t *end, const sw_cigar_t *cigar, int64_t n_pairs,
               const int32_t *window_chrom, const int64_t *window_pos, const int8_t *window_strand,
               int32_t min_score, sw_record_t *out_records, int64_t *out_count, sw_stream_t stream)
{
    if (n_pairs < 0 || !out_count) return SW_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (n_pairs == 0) return !cuda_failed(cudaMemsetAsync(out_count, 0, sizeof(int64_t), st)) ? SW_OK : SW_ERR_CUDA;
    if (!score || !end || !cigar || !cigar->ops || !cigar->offsets || !cigar->n_ops || !window_chrom ||
        !window_pos || !window_strand || !out_records)
        return SW_ERR_INVALID_ARG;
    if (n_pairs > (int64_t)INT32_MAX - 64) return SW_ERR_UNSUPPORTED;
    DeviceState *ds = nullptr;
    int rc = device_state(&ds, (cudaStream_t)stream);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(ds->mu);
    const int64_t n_blk = (n_pairs + 255) / 256;
    int32_t *status = nullptr;
    uint8_t *scratch = nullptr;
    if ((rc = stage_e_status(ds, align_up(4 * n_blk, 256) + 8 * n_blk, st, &status, &scratch))) return rc;
    int32_t *blk_count = (int32_t *)scratch;
    int64_t *blk_off = (int64_t *)(scratch + align_up(4 * n_blk, 256));
    return launch_records(score, end, *cigar, n_pairs, window_chrom, window_pos, window_strand, min_score,
                          out_records, out_count, blk_count, blk_off, st);
}

int sw_top_hits(const int32_t *score, const int64_t *cand_offsets, int64_t n_reads, const uint8_t *pair_mask,
                int32_t *best_score, int32_t *best_cand, int32_t *second_score, int32_t *mapq, sw_stream_t stream)
{
    if (n_reads < 0) return SW_ERR_INVALID_ARG;
    if (n_reads == 0) return SW_OK;
    if (!score || !cand_offsets || !best_score) return SW_ERR_INVALID_ARG;
    return launch_top_hits(score, cand_offsets, n_reads, pair_mask, best_score, best_cand, second_score, mapq,
                           (cudaStream_t)stream);
}

int64_t sw_junction_table_words(int64_t capacity) { return capacity < 0 ? 0 : 2 * capacity; }

static bool table_ok(const uint64_t *table, int64_t capacity)
{
    return table && capacity >= 64 && (capacity & (capacity - 1)) == 0 && capacity <= ((int64_t)1 << 40);
}

int sw_junction_table_clear(uint64_t *table, int64_t capacity, sw_stream_t stream)
{
    if (!table_ok(table, capacity)) return SW_ERR_INVALID_ARG;
    return launch_table_clear(table, capacity, (cudaStream_t)stream);
}

int sw_junctions_detect(const uint8_t *windows, const int64_t *window_offsets, const int32_t *score,
                        const int32_t *end, const sw_cigar_t *cigar, int64_t n_pairs, const int32_t *window_chrom,
                        const int64_t *window_pos, int32_t min_score, int32_t min_intron, uint64_t *table,
                        int64_t capacity, sw_stream_t stream)
{
    if (n_pairs < 0 || min_intron < 4 || !table_ok(table, capacity)) return SW_ERR_INVALID_ARG;
    if (n_pairs == 0) return SW_OK;
    if (!windows || ((uintptr_t)windows & 15u) || !window_offsets || !score || !end || !cigar || !cigar->ops ||
        !cigar->offsets || !cigar->n_ops || !window_chrom || !window_pos)
        return SW_ERR_INVALID_ARG;
    DeviceState *ds = nullptr;
    int rc = device_state(&ds, (cudaStream_t)stream);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(ds->mu);
    cudaStream_t st = (cudaStream_t)stream;
    int32_t *status = nullptr;
    uint8_t *scratch = nullptr;
    if ((rc = stage_e_status(ds, 0, st, &status, &scratch))) return rc;
    return launch_junctions((const uint32_t *)windows, window_offsets, score, end, *cigar, n_pairs, window_chrom,
                            window_pos, min_score, min_intron, table, capacity, status, st);
}

int sw_junctions_export(const uint64_t *table, int64_t capacity, sw_junction_t *out, int64_t max_out,
                        int64_t *out_count, sw_stream_t stream)
{
    if (!table_ok(table, capacity) || max_out < 0 || !out_count || (max_out > 0 && !out)) return SW_ERR_INVALID_ARG;
    return launch_table_export(table, capacity, out, max_out, out_count, (cudaStream_t)stream);
}

}  // extern "C"

// ---- seeding (Stages C, D, E i-ii) ----------------------------------------

extern "C" {

int64_t sw_index_table_words(int32_t k) { return (k < 8 || k > 16) ? 0 : (int64_t)1 << (2 * k); }

int sw_index_build(const uint8_t *genome, int64_t n_bases, const int64_t *chrom_offsets, int32_t n_chrom,
                   int32_t k, uint32_t *table, uint32_t *positions, int64_t *out_n_positions, sw_stream_t stream)
{
    if (!genome || ((uintptr_t)genome & 15u) || !chrom_offsets || !table || !positions || !out_n_positions ||
        k < 8 || k > 16 || n_chrom < 1 || n_bases < 0)
        return SW_ERR_INVALID_ARG;
    if (n_bases >= (int64_t)UINT32_MAX) return SW_ERR_UNSUPPORTED;
    DeviceState *ds = nullptr;
    int rc = device_state(&ds, (cudaStream_t)stream);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(ds->mu);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n_blk = ((size_t)1 << (2 * k)) / 4096;
    int32_t *status = nullptr;
    uint8_t *scratch = nullptr;
    if ((rc = stage_e_status(ds, 4 * n_blk, st, &status, &scratch))) return rc;
    return launch_index_build((const uint32_t *)genome, n_bases, chrom_offsets, n_chrom, k, table, positions,
                              out_n_positions, (uint32_t *)scratch, ds->sm_count, status, st);
}

static int seed_params_check(const sw_seed_params_t *p, SeedKParams *kp, int *block_hits)
{
    if (!p || p->k < 8 || p->k > 16 || p->stride < 1 || p->phase < 0 || p->phase > SW_SEED_MAX_READ_LEN ||
        p->max_hits < 1 || p->max_hits > SW_SEED_MAX_HITS || p->merge_dist < 0 || p->min_cal_len < p->k ||
        p->flank < 0 || p->max_intron < 0 || p->max_window < 1 || p->max_window > SW_MAX_WINDOW_LEN)
        return SW_ERR_INVALID_ARG;
    *kp = SeedKParams{p->k, p->stride, p->phase, p->max_hits, p->merge_dist, p->min_cal_len, p->flank,
                      p->max_intron, p->max_window};
    const int64_t bound = (int64_t)seed_count_per_read(SW_SEED_MAX_READ_LEN, *kp) * p->max_hits;
    int64_t n = 32;
    while (n < bound) n <<= 1;
    if (n > SW_SEED_MAX_LIST) return SW_ERR_UNSUPPORTED;
    *block_hits = (int)n;
    return SW_OK;
}

int sw_seed_windows(const uint32_t *table, const uint32_t *positions, const int64_t *chrom_offsets,
                    int32_t n_chrom, const sw_seed_params_t *params, const uint8_t *reads,
                    const int64_t *read_offsets, int64_t n_reads, const sw_windows_t *out, int64_t capacity,
                    int64_t *out_count, sw_stream_t stream)
{
    SeedKParams kp;
    int block_hits = 0;
    int rc = seed_params_check(params, &kp, &block_hits);
    if (rc) return rc;
    if (n_reads < 0 || capacity < 0 || !out || !out_count || !out->cand_offsets || !table || !positions ||
        !chrom_offsets || n_chrom < 1)
        return SW_ERR_INVALID_ARG;
    if (n_reads > (int64_t)INT32_MAX / 2 - 1 || capacity >= (int64_t)UINT32_MAX) return SW_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    if (n_reads == 0) {
        if (cuda_failed(cudaMemsetAsync(out_count, 0, sizeof(int64_t), st)) ||
            cuda_failed(cudaMemsetAsync(out->cand_offsets, 0, sizeof(int64_t), st)))
            return SW_ERR_CUDA;
        return SW_OK;
    }
    if (!reads || ((uintptr_t)reads & 15u) || !read_offsets || !out->start || !out->length || !out->chrom ||
        !out->pos || !out->strand || !out->pair_read)
        return SW_ERR_INVALID_ARG;
    DeviceState *ds = nullptr;
    if ((rc = device_state(&ds, (cudaStream_t)stream))) return rc;
    std::lock_guard<std::mutex> lk(ds->mu);
    int32_t *status = nullptr;
    uint8_t *scratch = nullptr;
    if ((rc = stage_e_status(ds, seed_scratch_bytes(n_reads, capacity), st, &status, &scratch))) return rc;
    if (!ds->seed_stats_host && cuda_failed(cudaMallocHost(&ds->seed_stats_host, 4 * sizeof(int64_t))))
        return SW_ERR_CUDA;
    SeedOutPtrs o{out->start, out->length, out->chrom, out->pos, out->strand, out->pair_read, out->cand_offsets,
                  out_count};
    return launch_seed_windows((const uint32_t *)reads, read_offsets, n_reads, table, positions, chrom_offsets,
                               n_chrom, kp, SW_SEED_MAX_READ_LEN, block_hits, o, capacity, scratch,
                               ds->seed_stats_host, ds->sm_count, status, st);
}

int sw_reads_two_strands(const uint8_t *reads, const int64_t *read_offsets, int64_t n_reads, uint8_t *out,
                         int64_t cap_bases, int64_t *out_offsets, sw_stream_t stream)
{
    if (n_reads < 0 || cap_bases < 0 || !out_offsets) return SW_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (n_reads == 0)
        return !cuda_failed(cudaMemsetAsync(out_offsets, 0, sizeof(int64_t), st)) ? SW_OK : SW_ERR_CUDA;
    if (!reads || ((uintptr_t)reads & 15u) || !read_offsets || !out || ((uintptr_t)out & 15u))
        return SW_ERR_INVALID_ARG;
    DeviceState *ds = nullptr;
    int rc = device_state(&ds, (cudaStream_t)stream);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(ds->mu);
    int32_t *status = nullptr;
    uint8_t *scratch = nullptr;
    if ((rc = stage_e_status(ds, 0, st, &status, &scratch))) return rc;
    return launch_two_strands((const uint32_t *)reads, read_offsets, n_reads, (uint32_t *)out, cap_bases,
                              out_offsets, ds->sm_count, status, st);
}

int sw_extract_windows(const uint8_t *genome, int64_t n_bases, const int64_t *start, const int32_t *length,
                       int64_t n_windows, uint8_t *out, int64_t cap_bases, int64_t *out_offsets,
                       sw_stream_t stream)
{
    if (n_windows < 0 || cap_bases < 0 || n_bases < 0 || !out_offsets) return SW_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (n_windows == 0)
        return !cuda_failed(cudaMemsetAsync(out_offsets, 0, sizeof(int64_t), st)) ? SW_OK : SW_ERR_CUDA;
    if (!genome || ((uintptr_t)genome & 15u) || !start || !length || !out || ((uintptr_t)out & 15u))
        return SW_ERR_INVALID_ARG;
    DeviceState *ds = nullptr;
    int rc = device_state(&ds, (cudaStream_t)stream);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(ds->mu);
    int32_t *status = nullptr;
    uint8_t *scratch = nullptr;
    if ((rc = stage_e_status(ds, 8 * ((size_t)(n_windows + 255) / 256 + 1), st, &status, &scratch))) return rc;
    return launch_extract_windows((const uint32_t *)genome, n_bases, start, length, n_windows, (uint32_t *)out,
                                  cap_bases, out_offsets, (int64_t *)scratch, ds->sm_count, status, st);
}

}  // extern "C"

extern "C" {

int sw_seed_stats(sw_stream_t stream, int64_t *out3)
{
    if (!out3) return SW_ERR_INVALID_ARG;
    DeviceState *ds = nullptr;
    int rc = device_state(&ds, (cudaStream_t)stream);
    if (rc) return rc;
    if (cuda_failed(cudaStreamSynchronize((cudaStream_t)stream))) return SW_ERR_CUDA;
    std::lock_guard<std::mutex> lk(ds->mu);
    if (!ds->seed_stats_host) return SW_ERR_INVALID_ARG;
    for (int i = 0; i < 3; ++i) out3[i] = ds->seed_stats_host[i];
    return SW_OK;
}

}  // extern "C"

extern "C" {

int sw_cigar_offsets(const int64_t *read_offsets, const int64_t *pair_read, int64_t n_pairs, int64_t *out_offsets,
                     sw_stream_t stream)
{
    if (n_pairs < 0 || !out_offsets || (n_pairs > 0 && !read_offsets)) return SW_ERR_INVALID_ARG;
    DeviceState *ds = nullptr;
    int rc = device_state(&ds, (cudaStream_t)stream);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(ds->mu);
    cudaStream_t st = (cudaStream_t)stream;
    int32_t *status = nullptr;
    uint8_t *scratch = nullptr;
    if ((rc = stage_e_status(ds, 8 * ((size_t)(n_pairs + 255) / 256 + 1), st, &status, &scratch))) return rc;
    return launch_cap_offsets_indexed(read_offsets, pair_read, n_pairs, out_offsets, (int64_t *)scratch, st);
}

}  // extern "C"
