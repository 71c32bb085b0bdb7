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
constexpr int kTbLanes = 1;            // lanes per pair in the traceback
constexpr int kSmallSlabWords = 4096;  // per-pair slab of the main traceback launch
constexpr size_t kSlabBudget = (size_t)4 << 30;
constexpr int64_t kTiledLaneWords = 4096;  // largest lane tile of a lane-interleaved traceback
constexpr int64_t kTiledLaneWords16 = 8192;  // the same for the 16-bit traceback (two pairs per lane)
// Lanes per pair of a multi-lane traceback: the smallest power of two T with
// the class's longest read in at most this many chunks of 8T rows.  A chunk
// sweeps its rows' band box, 8T - 1 columns wider than the band, so smaller T
// wastes fewer cells per pair and larger T keeps fewer pairs per warp waiting.
// Measured on the uneven batch (2M pairs, reads 75-800 bp), 16-bit sweep:
// 4 chunks 57.0 ms, 8 chunks 49.6 ms, 16 chunks 64.5 ms of traceback.
constexpr int kTbChunks32 = 4;
constexpr int kTbChunks16 = 8;
// 16-bit traceback tiles kept for the walk: up to this share of the free
// device memory, at most kTile16Cap; larger batches go in rounds
constexpr double kTile16FreeShare = 0.4;
constexpr size_t kTile16Cap = (size_t)64 << 30;
constexpr int kMaxDevices = 64;
constexpr int kAuxStreams = 4;
constexpr int kHostChunks = 2;                 // sw_batch_align_host pipelines a batch in this many chunks
constexpr int64_t kHostChunkMin = 65536;       // ... of at least this many pairs
constexpr bool kConcurrentTbParts = false;

struct Buffer {
    void *ptr = nullptr;
    size_t bytes = 0;
};

struct PlanOverride {
    int32_t max_read_len, lanes, rows;
};

// Library state of one (device, stream): scratch buffers, the status word
// of the stream's last call, pinned read-back slots, events and auxiliary
// streams.  Calls on one stream are ordered by the stream; calls on two
// streams get two states, so their work may overlap on the GPU without
// sharing scratch.
struct DeviceState {
    bool ready = false;
    int dev = 0;
    int sm_count = 0;
    int cc_major = 0, cc_minor = 0;
    Buffer fixed, dyn;
    Buffer stage;            // sw_batch_align_host device staging
    ClassInfo *info_host = nullptr;  // pinned
    TbClassInfo *tbinfo_host = nullptr;  // pinned
    cudaEvent_t last_done = nullptr;
    bool last_recorded = false;
    int32_t *last_status = nullptr;  // device status word of the last call
    bool timing = false;             // record phase events (sw_phase_times)
    bool timed_cells_valid = false;
    int64_t tb_split[2] = {0, 0};    // pairs per traceback kernel (16-bit, 32-bit) of the last call
    size_t tile16_budget = 0;        // 16-bit traceback tile budget (set at the first traceback)
    Buffer misc;                     // Stage E task iv: status word and record scan scratch
    Buffer filt;                     // sw_filter_align: features, predictions, selection
    int64_t *seed_stats_host = nullptr;  // pinned: counters of the stream's last sw_seed_windows
    cudaEvent_t phase[4] = {nullptr, nullptr, nullptr, nullptr};
    // independent launches (length classes, traceback parts) fork onto these
    // streams and join back, so one launch's tail overlaps the next
    cudaStream_t aux[kAuxStreams] = {};
    cudaEvent_t fork_ev = nullptr;
    cudaEvent_t join_ev[kAuxStreams] = {};
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
int fork_streams(DeviceState *ds, cudaStream_t st, int n)
{
    if (cuda_failed(cudaEventRecord(ds->fork_ev, st))) return SW_ERR_CUDA;
    for (int k = 0; k < n; ++k)
        if (cuda_failed(cudaStreamWaitEvent(ds->aux[k], ds->fork_ev, 0))) return SW_ERR_CUDA;
    return SW_OK;
}

int join_streams(DeviceState *ds, cudaStream_t st, int n)
{
    for (int k = 0; k < n; ++k) {
        if (cuda_failed(cudaEventRecord(ds->join_ev[k], ds->aux[k]))) return SW_ERR_CUDA;
        if (cuda_failed(cudaStreamWaitEvent(st, ds->join_ev[k], 0))) return SW_ERR_CUDA;
    }
    return SW_OK;
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
        s.cc_major = prop.major;
        s.cc_minor = prop.minor;
        if (cuda_failed(cudaMallocHost(&s.info_host, sizeof(ClassInfo)))) return SW_ERR_CUDA;
        if (cuda_failed(cudaMallocHost(&s.tbinfo_host, sizeof(TbClassInfo)))) return SW_ERR_CUDA;
        if (cuda_failed(cudaEventCreateWithFlags(&s.last_done, cudaEventDisableTiming))) return SW_ERR_CUDA;
        for (cudaEvent_t &e : s.phase)
            if (cuda_failed(cudaEventCreate(&e))) return SW_ERR_CUDA;
        for (int k = 0; k < kAuxStreams; ++k) {
            if (cuda_failed(cudaStreamCreateWithFlags(&s.aux[k], cudaStreamNonBlocking))) return SW_ERR_CUDA;
            if (cuda_failed(cudaEventCreateWithFlags(&s.join_ev[k], cudaEventDisableTiming))) return SW_ERR_CUDA;
        }
        if (cuda_failed(cudaEventCreateWithFlags(&s.fork_ev, cudaEventDisableTiming))) return SW_ERR_CUDA;
        if (cuda_failed(cudaStreamCreateWithFlags(&s.copy_in, cudaStreamNonBlocking))) return SW_ERR_CUDA;
        if (cuda_failed(cudaStreamCreateWithFlags(&s.copy_out, cudaStreamNonBlocking))) return SW_ERR_CUDA;
        for (cudaEvent_t &e : s.host_in_ev)
            if (cuda_failed(cudaEventCreateWithFlags(&e, cudaEventDisableTiming))) return SW_ERR_CUDA;
        if (cuda_failed(cudaEventCreateWithFlags(&s.host_out_ev, cudaEventDisableTiming))) return SW_ERR_CUDA;
        s.ready = true;
    }
    s.timing = g_timing[dev];
    g_last_state[dev] = &s;
    *out = &s;
    return SW_OK;
}

void free_state(DeviceState *s)
{
    for (Buffer *b : {&s->fixed, &s->dyn, &s->stage, &s->misc, &s->filt})
        if (b->ptr) {
            cudaFree(b->ptr);
            b->ptr = nullptr;
            b->bytes = 0;
        }
    if (s->info_host) cudaFreeHost(s->info_host);
    if (s->seed_stats_host) cudaFreeHost(s->seed_stats_host);
    if (s->tbinfo_host) cudaFreeHost(s->tbinfo_host);
    if (s->last_done) cudaEventDestroy(s->last_done);
    for (cudaEvent_t e : s->phase)
        if (e) cudaEventDestroy(e);
    for (int k = 0; k < kAuxStreams; ++k) {
        if (s->aux[k]) cudaStreamDestroy(s->aux[k]);
        if (s->join_ev[k]) cudaEventDestroy(s->join_ev[k]);
    }
    if (s->fork_ev) cudaEventDestroy(s->fork_ev);
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

int status_to_code(int32_t st)
{
    if (st & ST_BAD_INPUT) return SW_ERR_DEVICE_INPUT;
    if (st & ST_UNSUPPORTED) return SW_ERR_UNSUPPORTED;
    if (st & ST_CAPACITY) return SW_ERR_CAPACITY;
    if (st & ST_TIMEOUT) return SW_ERR_DEVICE_TIMEOUT;
    if (st & ST_INTERNAL) return SW_ERR_INTERNAL;
    return SW_OK;
}

struct Plan {
    int lanes, rows;
};

// Lanes per group and rows per lane for reads up to m_max in a mode.  In
// the 16-bit-key mode a lane block of more than 32 rows needs 6-bit row tags,
// which leave room for scores up to 510 only (hmax: the class's score bound).
Plan choose_plan(int mode, int32_t m_max, int64_t hmax)
{
    const int max_rows = (mode == MODE_I16 && hmax > 510) ? 32 : 64;
    {
        std::lock_guard<std::mutex> lk(g_plan_mu);
        for (const PlanOverride &o : g_plans)
            if (m_max <= o.max_read_len && o.rows <= max_rows) return Plan{o.lanes, o.rows};
    }
    // estimated issue cost per pair-column: padded rows x ~6.5 ALU ops + ~40
    // ops per lane-step (both measured), scaled by the fraction of lanes a
    // warp leaves idle
    double best = 1e300;
    Plan bp{32, 32};
    for (int ri = 0; ri < N_SCORE_ROWS; ++ri) {
        const int R = kScoreRows[ri];
        if (R > max_rows) continue;
        for (int T = 1; T <= 32; ++T) {
            const int chunks = (m_max + T * R - 1) / (T * R);
            if (chunks > 1 && T < 32) continue;
            const int G = 32 / T;
            const double lane_util = (double)(G * T) / 32.0;
            const double cost = chunks * (double)T * (R * 6.5 + 40.0) / lane_util;
            if (cost < best - 1e-9) {
                best = cost;
                bp = Plan{T, R};
            }
        }
    }
    return bp;
}

int run_batch(const PairSet &ps, int64_t n_reads, int64_t n_pairs, const sw_scoring_t *scoring,
              int32_t *out_score, int32_t *out_end, const sw_cigar_t *cig, cudaStream_t st)
{
    DeviceState *ds = nullptr;
    int rc = device_state(&ds, st);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(ds->mu);
    if (ds->last_recorded && cuda_failed(cudaStreamWaitEvent(st, ds->last_done, 0))) return SW_ERR_CUDA;

    const Scoring sc{scoring->match, scoring->mismatch, scoring->gap_open, scoring->gap_extend};
    const size_t nh = (size_t)N_CLASS * N_NBUCKET;
    size_t off = 0;
    const size_t o_keys = off; off = align_up(off + sizeof(int32_t) * n_pairs, 256);
    const size_t o_order = off; off = align_up(off + sizeof(int32_t) * n_pairs, 256);
    const size_t o_hist = off; off = align_up(off + sizeof(int32_t) * nh, 256);
    const size_t o_bstart = off; off = align_up(off + sizeof(int32_t) * nh, 256);
    const size_t o_cursor = off; off = align_up(off + sizeof(int32_t) * nh, 256);
    const size_t o_info = off; off = align_up(off + sizeof(ClassInfo), 256);
    const size_t o_counters = off; off = align_up(off + sizeof(int32_t) * 4 * N_CLASS, 256);
    const size_t o_tbkeys = off; off = align_up(off + sizeof(int32_t) * n_pairs, 256);
    const size_t o_tborder = off; off = align_up(off + sizeof(int32_t) * n_pairs, 256);
    const size_t o_tbinfo = off; off = align_up(off + sizeof(TbClassInfo), 256);
    if ((rc = ensure(ds->fixed, off))) return rc;
    uint8_t *fx = (uint8_t *)ds->fixed.ptr;
    int32_t *keys = (int32_t *)(fx + o_keys), *order = (int32_t *)(fx + o_order);
    int32_t *hist = (int32_t *)(fx + o_hist), *bstart = (int32_t *)(fx + o_bstart);
    int32_t *cursor = (int32_t *)(fx + o_cursor), *counters = (int32_t *)(fx + o_counters);
    ClassInfo *info = (ClassInfo *)(fx + o_info);
    int32_t *tb_keys = (int32_t *)(fx + o_tbkeys), *tb_order = (int32_t *)(fx + o_tborder);
    TbClassInfo *tbinfo = (TbClassInfo *)(fx + o_tbinfo);
    ds->last_status = &info->status;

    ds->timed_cells_valid = false;
    if (ds->timing && cuda_failed(cudaEventRecord(ds->phase[0], st))) return SW_ERR_CUDA;
    if (cuda_failed(cudaMemsetAsync(hist, 0, sizeof(int32_t) * nh, st))) return SW_ERR_CUDA;
    if (cuda_failed(cudaMemsetAsync(info, 0, sizeof(ClassInfo), st))) return SW_ERR_CUDA;
    if (cuda_failed(cudaMemsetAsync(counters, 0, sizeof(int32_t) * 4 * N_CLASS, st))) return SW_ERR_CUDA;
    if ((rc = launch_classify(ps, n_reads, n_pairs, sc, g_score_mode.load() == SW_SCORE_INT32, keys, hist, bstart,
                              cursor, info, order, out_score,
                              out_end, cig ? cig->n_ops : nullptr, st)))
        return rc;
    if (cuda_failed(cudaMemcpyAsync(ds->info_host, info, sizeof(ClassInfo), cudaMemcpyDeviceToHost, st)))
        return SW_ERR_CUDA;
    if (cuda_failed(cudaStreamSynchronize(st))) return SW_ERR_CUDA;
    const ClassInfo ci = *ds->info_host;
    if (ci.status) return status_to_code(ci.status);

    // class ranges in the sorted order, plans and scratch needs
    struct ClassRun {
        int cls, mode;
        int64_t start, count;
        int32_t max_m, max_n;
        Plan plan;
        int score_blocks;
        size_t bnd_bytes_group;
        size_t bnd_offset;  // of this class's boundary scratch in the dynamic buffer
    };
    std::vector<ClassRun> runs;
    int64_t pos = 0;
    size_t need_dyn = 0;
    for (int cls = 0; cls < N_CLASS; ++cls) {
        const int32_t cnt = ci.count[cls];
        if (!cnt) continue;
        ClassRun r{};
        r.cls = cls;
        r.mode = cls / N_MCLASS;
        r.start = pos;
        r.count = cnt;
        r.max_m = ci.max_m[cls];
        r.max_n = ci.max_n[cls];
        pos += cnt;
        r.plan = choose_plan(r.mode, r.max_m, (int64_t)sc.ma * std::min(r.max_m, r.max_n));
        int regs = 0, bps = 0;
        if ((rc = score_kernel_regs(r.plan.rows, r.mode, &regs, &bps, kThreads))) return rc;
        if (bps < 1) return SW_ERR_INTERNAL;
        const int G = 32 / r.plan.lanes;
        const int per_warp = G * (r.mode == MODE_I32 ? 1 : 2);
        const int64_t warps_needed = (cnt + per_warp - 1) / per_warp;
        const int64_t wpb = kThreads / 32;
        int64_t blocks = std::min<int64_t>((warps_needed + wpb - 1) / wpb, (int64_t)bps * ds->sm_count);
        r.score_blocks = (int)std::max<int64_t>(blocks, 1);
        const int chunks = (r.max_m + r.plan.lanes * r.plan.rows - 1) / (r.plan.lanes * r.plan.rows);
        r.bnd_bytes_group = chunks > 1 ? (size_t)2 * r.max_n * 2 * sizeof(uint32_t) : 0;
        // classes run concurrently: each gets its own boundary scratch
        r.bnd_offset = need_dyn;
        need_dyn += align_up(r.bnd_bytes_group * (size_t)r.score_blocks * wpb * G, 256);
        runs.push_back(r);
    }
    if ((rc = ensure(ds->dyn, std::max<size_t>(need_dyn, 256)))) return rc;

    if (ds->timing && cuda_failed(cudaEventRecord(ds->phase[1], st))) return SW_ERR_CUDA;
    // with a CIGAR, the score kernels' epilogue also writes the traceback
    // cost keys and the class table the traceback is sized from
    if (cig) {
        if (cuda_failed(cudaMemsetAsync(hist, 0, sizeof(int32_t) * nh, st))) return SW_ERR_CUDA;
        if (cuda_failed(cudaMemsetAsync(tbinfo, 0, sizeof(TbClassInfo), st))) return SW_ERR_CUDA;
        if (cuda_failed(cudaMemsetAsync(tb_keys, 0xFF, sizeof(int32_t) * n_pairs, st))) return SW_ERR_CUDA;
    }
    // one launch per class; several classes fork onto the auxiliary streams
    const int n_aux_score = runs.size() > 1 ? (int)std::min<size_t>(runs.size(), kAuxStreams) : 0;
    if (n_aux_score && (rc = fork_streams(ds, st, n_aux_score))) return rc;
    for (size_t ri = 0; ri < runs.size(); ++ri) {
        const ClassRun &r = runs[ri];
        const cudaStream_t cs = n_aux_score ? ds->aux[ri % n_aux_score] : st;
        ScoreLaunch L{};
        L.ps = ps;
        L.sc = sc;
        L.order = order + r.start;
        L.n_items = r.count;
        L.lanes = r.plan.lanes;
        L.out_score = out_score;
        L.out_end = out_end;
        L.boundary = r.bnd_bytes_group ? (uint8_t *)ds->dyn.ptr + r.bnd_offset : nullptr;
        L.boundary_group_bytes = (int64_t)r.bnd_bytes_group;
        L.work_counter = counters + r.cls;
        L.status = &info->status;
        if (cig) {
            L.cls = r.cls;
            L.tb_keys = tb_keys;
            L.tb_hist = hist;
            L.tb_info = tbinfo;
            L.small_slab_words = kSmallSlabWords;
        }
        if ((rc = launch_score(r.plan.rows, r.mode, L, r.score_blocks, kThreads, cs))) return rc;
    }
    if (n_aux_score && (rc = join_streams(ds, st, n_aux_score))) return rc;
    if (ds->timing && cuda_failed(cudaEventRecord(ds->phase[2], st))) return SW_ERR_CUDA;
    if (cig) {
        // order each class by traceback cost, then size the slabs from the
        // per-class maxima (a second, small read-back)
        TbParams P{ps, sc, out_score, out_end, cig->ops, cig->offsets, cig->n_ops, kTbLanes, kSmallSlabWords};
        if ((rc = launch_scan_scatter(tb_keys, n_pairs, info->count, hist, bstart, cursor, tb_order, st))) return rc;
        if (cuda_failed(cudaMemcpyAsync(ds->tbinfo_host, tbinfo, sizeof(TbClassInfo), cudaMemcpyDeviceToHost, st)))
            return SW_ERR_CUDA;
        if (cuda_failed(cudaStreamSynchronize(st))) return SW_ERR_CUDA;
        const TbClassInfo ti = *ds->tbinfo_host;
        int tbps = 0;
        if ((rc = traceback_kernel_occupancy(&tbps, kThreads, false, 1))) return rc;
        const bool allow16 = g_tb_mode.load() == SW_TB_AUTO;
        if (!ds->tile16_budget) {
            // once per device: a share of the memory free at the first call
            // (plus what the dynamic buffer already holds)
            size_t free_b = 0, total_b = 0;
            ds->tile16_budget = (size_t)4 << 30;
            if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess)
                ds->tile16_budget = std::max(ds->tile16_budget,
                                             std::min(kTile16Cap, (size_t)(kTile16FreeShare * (free_b + ds->dyn.bytes))));
        }
        const size_t tile16_budget = ds->tile16_budget;
        const int64_t wpb = kThreads / 32;
        struct TbRun {
            int64_t start, count;
            int64_t slab_words, bnd_ints;  // per group, or per lane when tiled
            int32_t wcap;
            bool tiled, packed16;
            int blocks;
            int64_t round_tasks;  // 16-bit kernel: tasks (64 pairs) per round
            int lanes;            // int32 kernels: lanes per pair
            size_t need;          // scratch bytes of one round
            size_t offset;        // of its scratch in the dynamic buffer
            bool one_round;
            int cls, part;
        };
        std::vector<TbRun> tbr;
        size_t need = 0;
        for (const ClassRun &r : runs) {
            const int64_t big = ti.n_big[r.cls];
            const int64_t max_need = std::max<int64_t>(ti.max_need[r.cls], 1);
            const int64_t parts[2][2] = {{r.start, big}, {r.start + big, r.count - big}};
            for (int part = 0; part < 2; ++part) {
                const int64_t cnt = parts[part][1];
                if (cnt <= 0) continue;
                TbRun t{};
                t.start = parts[part][0];
                t.count = cnt;
                const int rc = kTbLanes * TB_ROWS;
                const int64_t chunks = (r.max_m + rc - 1) / rc;
                t.wcap = (int32_t)std::max<int64_t>(ti.max_wcap[part][r.cls], 1);
                // 16-bit halves (two pairs per lane group) wherever the class's
                // score bound allows it; else int32 lanes.  T lanes share a
                // pair: one where a lane's tile (every chunk at the widest
                // window) stays small, else a power of two covering the
                // longest read in a few chunks (kTbChunks16, kTbChunks32), so
                // that one pair's cells do not run on a single lane.  A T-lane
                // chunk window is at most 8 (T - 1) wider than the one-lane
                // windows the key pass measured.
                const int64_t wcap4 = (t.wcap + 3) / 4 * 4;
                t.packed16 = allow16 && r.mode != MODE_I32;
                int Tl = 1;
                while (Tl < 32 && (int64_t)Tl * 8 * (t.packed16 ? kTbChunks16 : kTbChunks32) < r.max_m) Tl *= 2;
                const bool one_lane16 = chunks * wcap4 * 2 <= kTiledLaneWords16;
                t.tiled = !t.packed16 && chunks * t.wcap <= kTiledLaneWords;
                t.lanes = (t.packed16 && one_lane16) || t.tiled ? 1 : Tl;
                if (t.packed16) {
                    const int T = t.lanes;
                    const int64_t chunks_t = (r.max_m + 8 * T - 1) / (8 * T);
                    t.wcap = (int32_t)(t.wcap + 8 * (T - 1));
                    const int64_t s4 = (t.wcap + T - 1 + 3) / 4;
                    t.slab_words = chunks_t * s4 * 8;                                      // per lane
                    t.bnd_ints = chunks_t > 1 ? (int64_t)(32 / T) * 2 * t.wcap : 0;  // per warp: one row
                } else if (t.tiled) {
                    t.slab_words = chunks * t.wcap;
                    t.bnd_ints = chunks > 1 ? (int64_t)2 * 2 * t.wcap : 0;
                } else {
                    const int T = t.lanes;
                    const int64_t chunks_t = (r.max_m + 8 * T - 1) / (8 * T);
                    const int64_t wcap_t = t.wcap + 8 * (T - 1);
                    t.slab_words = T == 1 ? (part == 0 ? max_need : std::min<int64_t>(max_need, kSmallSlabWords))
                                          : chunks_t * wcap_t * T;
                    t.bnd_ints = chunks_t > 1 ? (int64_t)2 * 2 * wcap_t : 0;
                }
                const int per_warp = t.packed16 ? 64 / t.lanes : 32 / t.lanes;
                if (t.packed16) {
                    // a tile per task, kept until the walk: tasks go in rounds
                    // that fit the tile budget
                    int occ = 0;
                    const int orc = traceback_kernel_occupancy(&occ, kThreads, true, t.lanes);
                    if (orc) return orc;
                    const size_t tile_bytes = (size_t)32 * t.slab_words * 4;
                    const int64_t tasks = (cnt + per_warp - 1) / per_warp;
                    t.round_tasks = std::max<int64_t>(1, std::min<int64_t>(tasks, (int64_t)(tile16_budget / tile_bytes)));
                    const size_t bnd_per_block = (size_t)wpb * t.bnd_ints * 4;
                    int64_t blocks = std::min<int64_t>((t.round_tasks + wpb - 1) / wpb, (int64_t)std::max(occ, 1) * ds->sm_count);
                    t.blocks = (int)std::max<int64_t>(blocks, 1);
                    t.need = tile_bytes * (size_t)t.round_tasks + bnd_per_block * (size_t)t.blocks;
                    t.one_round = t.round_tasks == tasks;
                } else {
                    const size_t per_block = (size_t)wpb * (32 / t.lanes) * (t.slab_words + t.bnd_ints) * 4;
                    int64_t blocks = std::min<int64_t>(((cnt + per_warp - 1) / per_warp + wpb - 1) / wpb,
                                                       (int64_t)std::max(tbps, 1) * ds->sm_count);
                    blocks = std::min<int64_t>(blocks, (int64_t)(kSlabBudget / std::max<size_t>(per_block, 1)));
                    t.blocks = (int)std::max<int64_t>(blocks, 1);
                    t.need = per_block * (size_t)t.blocks;
                    t.one_round = true;
                }
                t.cls = r.cls;
                t.part = part;
                tbr.push_back(t);
            }
        }
        // Parts run concurrently on the auxiliary streams, each in its own
        // scratch region, when all of them fit one round of the budget;
        // otherwise one after another, each from the start of the buffer.
        size_t total = 0;
        bool all_one_round = true;
        for (TbRun &t : tbr) {
            t.offset = total;
            total += align_up(t.need, 256);
            all_one_round = all_one_round && t.one_round;
            need = std::max(need, t.need);
        }
        // (measured: on a one-class batch the big and main parts slowed each
        // other down, on the uneven batch it gained 0.1 %, so parts run in order)
        const bool concurrent = kConcurrentTbParts && tbr.size() > 1 && all_one_round &&
                                total <= std::max(tile16_budget, need);
        if (!concurrent)
            for (TbRun &t : tbr) t.offset = 0;
        if ((rc = ensure(ds->dyn, std::max<size_t>(concurrent ? total : need, 256)))) return rc;
        ds->tb_split[0] = ds->tb_split[1] = 0;
        for (const TbRun &t : tbr) ds->tb_split[t.packed16 ? 0 : 1] += t.count;
        const int n_aux_tb = concurrent ? (int)std::min<size_t>(tbr.size(), kAuxStreams) : 0;
        if (n_aux_tb && (rc = fork_streams(ds, st, n_aux_tb))) return rc;
        for (size_t ti2 = 0; ti2 < tbr.size(); ++ti2) {
            const TbRun &t = tbr[ti2];
            const cudaStream_t ts = n_aux_tb ? ds->aux[ti2 % std::max(n_aux_tb, 1)] : st;
            uint8_t *region = (uint8_t *)ds->dyn.ptr + t.offset;
            TracebackLaunch B{};
            B.P = P;
            B.P.lanes = t.lanes;
            B.lanes = t.lanes;
            B.slab = (uint32_t *)region;
            B.slab_group_words = t.slab_words;
            B.boundary_group_ints = t.bnd_ints;
            B.wcap = t.wcap;
            B.tiled = t.tiled;
            B.packed16 = t.packed16;
            B.work_counter = counters + 2 * N_CLASS + 2 * t.cls + t.part;
            B.status = &info->status;
            if (t.packed16) {
                const int64_t round_items = t.round_tasks * (64 / t.lanes);
                const size_t tiles = (size_t)t.round_tasks * 32 * t.slab_words;
                B.boundary = (int32_t *)region + tiles;
                for (int64_t r0 = 0; r0 < t.count; r0 += round_items) {
                    B.order = tb_order + t.start + r0;
                    B.n_items = std::min<int64_t>(round_items, t.count - r0);
                    if (r0 > 0 && cuda_failed(cudaMemsetAsync(B.work_counter, 0, sizeof(int32_t), ts)))
                        return SW_ERR_CUDA;
                    if ((rc = launch_traceback(B, t.blocks, kThreads, ts))) return rc;
                }
            } else {
                B.order = tb_order + t.start;
                B.n_items = t.count;
                const size_t slab_total = (size_t)t.blocks * wpb * (32 / t.lanes) * t.slab_words;
                B.boundary = (int32_t *)region + slab_total;
                if ((rc = launch_traceback(B, t.blocks, kThreads, ts))) return rc;
            }
        }
        if (n_aux_tb && (rc = join_streams(ds, st, n_aux_tb))) return rc;
    }
    if (ds->timing && cuda_failed(cudaEventRecord(ds->phase[3], st))) return SW_ERR_CUDA;
    ds->timed_cells_valid = ds->timing;
    if (cuda_failed(cudaEventRecord(ds->last_done, st))) return SW_ERR_CUDA;
    ds->last_recorded = true;
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
// Plans: the launch decisions of one batch shape, taken once, so that the
// execution itself is a fixed sequence of launches (capturable).

struct PlanScoreRun {
    int cls, mode, rows, lanes, blocks;
    int64_t start, count;
    size_t bnd_bytes_group, bnd_offset;
};

struct PlanTbRun {
    int cls, lanes, blocks;
    bool packed16, tiled;
    int64_t start, count, slab_words, bnd_ints, round_tasks;
    int32_t wcap;
};

}  // namespace
}  // namespace swgb

struct sw_plan {
    int device = -1;
    swgb::PairSet ps{};  // offsets and pair map (bases bound per execution)
    int64_t n_reads = 0, n_pairs = 0;
    swgb::Scoring sc{};
    bool cigar = false;
    bool force_i32 = false;   // the score mode setting at creation
    swgb::Buffer fixed, dyn;  // owned: a captured graph keeps pointing here
    int32_t *keys = nullptr, *order = nullptr, *hist = nullptr, *bstart = nullptr, *cursor = nullptr;
    int32_t *counters = nullptr, *tb_keys = nullptr, *tb_order = nullptr, *expect = nullptr;
    swgb::ClassInfo *info = nullptr;
    swgb::TbClassInfo *tbinfo = nullptr;
    std::vector<swgb::PlanScoreRun> sruns;
    std::vector<swgb::PlanTbRun> truns;
    size_t tb_tiles_bytes = 0;  // offset of the traceback boundary rows in dyn
};

namespace swgb {
namespace {

int plan_build(sw_plan *pl, DeviceState *ds, cudaStream_t st)
{
    int rc = SW_OK;
    const size_t nh = (size_t)N_CLASS * N_NBUCKET;
    const int64_t n_pairs = pl->n_pairs;
    size_t off = 0;
    const size_t o_keys = off; off = align_up(off + sizeof(int32_t) * n_pairs, 256);
    const size_t o_order = off; off = align_up(off + sizeof(int32_t) * n_pairs, 256);
    const size_t o_hist = off; off = align_up(off + sizeof(int32_t) * nh, 256);
    const size_t o_bstart = off; off = align_up(off + sizeof(int32_t) * nh, 256);
    const size_t o_cursor = off; off = align_up(off + sizeof(int32_t) * nh, 256);
    const size_t o_info = off; off = align_up(off + sizeof(ClassInfo), 256);
    const size_t o_counters = off; off = align_up(off + sizeof(int32_t) * 4 * N_CLASS, 256);
    const size_t o_tbkeys = off; off = align_up(off + sizeof(int32_t) * n_pairs, 256);
    const size_t o_tborder = off; off = align_up(off + sizeof(int32_t) * n_pairs, 256);
    const size_t o_tbinfo = off; off = align_up(off + sizeof(TbClassInfo), 256);
    const size_t o_expect = off; off = align_up(off + sizeof(int32_t) * 3 * N_CLASS, 256);
    if ((rc = ensure(pl->fixed, off))) return rc;
    uint8_t *fx = (uint8_t *)pl->fixed.ptr;
    pl->keys = (int32_t *)(fx + o_keys);
    pl->order = (int32_t *)(fx + o_order);
    pl->hist = (int32_t *)(fx + o_hist);
    pl->bstart = (int32_t *)(fx + o_bstart);
    pl->cursor = (int32_t *)(fx + o_cursor);
    pl->info = (ClassInfo *)(fx + o_info);
    pl->counters = (int32_t *)(fx + o_counters);
    pl->tb_keys = (int32_t *)(fx + o_tbkeys);
    pl->tb_order = (int32_t *)(fx + o_tborder);
    pl->tbinfo = (TbClassInfo *)(fx + o_tbinfo);
    pl->expect = (int32_t *)(fx + o_expect);

    // classify once (it reads offsets only) and read the class table back
    if (cuda_failed(cudaMemsetAsync(pl->hist, 0, sizeof(int32_t) * nh, st))) return SW_ERR_CUDA;
    if (cuda_failed(cudaMemsetAsync(pl->info, 0, sizeof(ClassInfo), st))) return SW_ERR_CUDA;
    int32_t *tmp_score = pl->tb_keys, *tmp_end = nullptr;  // empty-window outputs go to scratch
    if ((rc = ensure(pl->dyn, sizeof(int32_t) * 2 * std::max<int64_t>(n_pairs, 1)))) return rc;
    tmp_end = (int32_t *)pl->dyn.ptr;
    if ((rc = launch_classify(pl->ps, pl->n_reads, n_pairs, pl->sc, pl->force_i32, pl->keys, pl->hist, pl->bstart,
                              pl->cursor,
                              pl->info, pl->order, tmp_score, tmp_end, nullptr, st)))
        return rc;
    ClassInfo ci;
    if (cuda_failed(cudaMemcpyAsync(&ci, pl->info, sizeof(ClassInfo), cudaMemcpyDeviceToHost, st)))
        return SW_ERR_CUDA;
    if (cuda_failed(cudaStreamSynchronize(st))) return SW_ERR_CUDA;
    if (ci.status) return status_to_code(ci.status);
    {
        std::vector<int32_t> ex(3 * N_CLASS);
        std::memcpy(ex.data(), ci.count, sizeof(int32_t) * N_CLASS);
        std::memcpy(ex.data() + N_CLASS, ci.max_m, sizeof(int32_t) * N_CLASS);
        std::memcpy(ex.data() + 2 * N_CLASS, ci.max_n, sizeof(int32_t) * N_CLASS);
        if (cuda_failed(cudaMemcpy(pl->expect, ex.data(), sizeof(int32_t) * 3 * N_CLASS, cudaMemcpyHostToDevice)))
            return SW_ERR_CUDA;
    }

    // score launches, as sw_batch_align plans them
    const int64_t wpb = kThreads / 32;
    int64_t pos = 0;
    size_t score_scratch = 0;
    for (int cls = 0; cls < N_CLASS; ++cls) {
        const int32_t cnt = ci.count[cls];
        if (!cnt) continue;
        PlanScoreRun r{};
        r.cls = cls;
        r.mode = cls / N_MCLASS;
        r.start = pos;
        r.count = cnt;
        pos += cnt;
        const int32_t max_m = ci.max_m[cls], max_n = ci.max_n[cls];
        const Plan plan = choose_plan(r.mode, max_m, (int64_t)pl->sc.ma * std::min(max_m, max_n));
        r.rows = plan.rows;
        r.lanes = plan.lanes;
        int regs = 0, bps = 0;
        if ((rc = score_kernel_regs(r.rows, r.mode, &regs, &bps, kThreads))) return rc;
        if (bps < 1) return SW_ERR_INTERNAL;
        const int G = 32 / r.lanes;
        const int per_warp = G * (r.mode == MODE_I32 ? 1 : 2);
        const int64_t warps_needed = (cnt + per_warp - 1) / per_warp;
        r.blocks = (int)std::max<int64_t>(1, std::min<int64_t>((warps_needed + wpb - 1) / wpb, (int64_t)bps * ds->sm_count));
        const int chunks = (max_m + r.lanes * r.rows - 1) / (r.lanes * r.rows);
        r.bnd_bytes_group = chunks > 1 ? (size_t)2 * max_n * 2 * sizeof(uint32_t) : 0;
        r.bnd_offset = score_scratch;
        score_scratch += align_up(r.bnd_bytes_group * (size_t)r.blocks * wpb * G, 256);
        pl->sruns.push_back(r);
    }

    // traceback launches for the worst case: any window may be inside the
    // band, so a chunk window is at most the class's longest window
    size_t tb_need = 0;
    if (pl->cigar) {
        if (!ds->tile16_budget) {
            size_t free_b = 0, total_b = 0;
            ds->tile16_budget = (size_t)4 << 30;
            if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess)
                ds->tile16_budget = std::max(ds->tile16_budget,
                                             std::min(kTile16Cap, (size_t)(kTile16FreeShare * (free_b + ds->dyn.bytes))));
        }
        int tbps = 0;
        if ((rc = traceback_kernel_occupancy(&tbps, kThreads, false, 1))) return rc;
        const bool allow16 = g_tb_mode.load() == SW_TB_AUTO;
        for (const PlanScoreRun &r : pl->sruns) {
            PlanTbRun t{};
            t.cls = r.cls;
            t.start = r.start;
            t.count = r.count;
            const int32_t max_m = ci.max_m[r.cls], max_n = ci.max_n[r.cls];
            const int64_t chunks = (max_m + TB_ROWS - 1) / TB_ROWS;
            const int64_t wcap1 = max_n;
            const int64_t wcap4 = (wcap1 + 3) / 4 * 4;
            t.packed16 = allow16 && r.mode != MODE_I32;
            int Tl = 1;
            while (Tl < 32 && (int64_t)Tl * 8 * (t.packed16 ? kTbChunks16 : kTbChunks32) < max_m) Tl *= 2;
            t.tiled = !t.packed16 && chunks * wcap1 <= kTiledLaneWords;
            t.lanes = (t.packed16 && chunks * wcap4 * 2 <= kTiledLaneWords16) || t.tiled ? 1 : Tl;
            const int T = t.lanes;
            const int64_t chunks_t = (max_m + 8 * T - 1) / (8 * T);
            const int64_t wcap_t = wcap1 + 8 * (T - 1);
            t.wcap = (int32_t)(t.packed16 ? wcap_t : wcap1);
            if (t.packed16) {
                const int64_t s4 = (wcap_t + T - 1 + 3) / 4;
                t.slab_words = chunks_t * s4 * 8;
                t.bnd_ints = chunks_t > 1 ? (int64_t)(32 / T) * 2 * wcap_t : 0;
                int occ = 0;
                if ((rc = traceback_kernel_occupancy(&occ, kThreads, true, T))) return rc;
                const size_t tile_bytes = (size_t)32 * t.slab_words * 4;
                const int per_warp = 64 / T;
                const int64_t tasks = (t.count + per_warp - 1) / per_warp;
                t.round_tasks = std::max<int64_t>(1, std::min<int64_t>(tasks, (int64_t)(ds->tile16_budget / tile_bytes)));
                t.blocks = (int)std::max<int64_t>(1, std::min<int64_t>((t.round_tasks + wpb - 1) / wpb, (int64_t)std::max(occ, 1) * ds->sm_count));
                tb_need = std::max(tb_need, tile_bytes * (size_t)t.round_tasks + (size_t)wpb * t.bnd_ints * 4 * t.blocks);
            } else {
                if (t.tiled) {
                    t.slab_words = chunks * wcap1;
                    t.bnd_ints = chunks > 1 ? 4 * wcap1 : 0;
                } else {
                    t.slab_words = chunks_t * wcap_t * T;
                    t.bnd_ints = chunks_t > 1 ? 4 * wcap_t : 0;
                }
                const int per_warp = 32 / T;
                const size_t per_block = (size_t)wpb * per_warp * (t.slab_words + t.bnd_ints) * 4;
                int64_t blocks = std::min<int64_t>(((t.count + per_warp - 1) / per_warp + wpb - 1) / wpb,
                                                   (int64_t)std::max(tbps, 1) * ds->sm_count);
                blocks = std::min<int64_t>(blocks, (int64_t)(kSlabBudget / std::max<size_t>(per_block, 1)));
                t.blocks = (int)std::max<int64_t>(blocks, 1);
                t.round_tasks = 0;
                tb_need = std::max(tb_need, per_block * (size_t)t.blocks);
            }
            pl->truns.push_back(t);
        }
    }
    return ensure(pl->dyn, std::max<size_t>(std::max(score_scratch, tb_need), 256));
}

int plan_execute(sw_plan *pl, int32_t *out_score, int32_t *out_end, const sw_cigar_t *cig, cudaStream_t st)
{
    int rc = SW_OK;
    const size_t nh = (size_t)N_CLASS * N_NBUCKET;
    const PairSet &ps = pl->ps;
    if (cuda_failed(cudaMemsetAsync(pl->hist, 0, sizeof(int32_t) * nh, st))) return SW_ERR_CUDA;
    if (cuda_failed(cudaMemsetAsync(pl->info, 0, sizeof(ClassInfo), st))) return SW_ERR_CUDA;
    if (cuda_failed(cudaMemsetAsync(pl->counters, 0, sizeof(int32_t) * 4 * N_CLASS, st))) return SW_ERR_CUDA;
    if ((rc = launch_classify(ps, pl->n_reads, pl->n_pairs, pl->sc, pl->force_i32, pl->keys, pl->hist, pl->bstart,
                              pl->cursor,
                              pl->info, pl->order, out_score, out_end, cig ? cig->n_ops : nullptr, st)))
        return rc;
    if ((rc = launch_check_counts(pl->info, pl->expect, &pl->info->status, st))) return rc;
    for (const PlanScoreRun &r : pl->sruns) {
        ScoreLaunch L{};
        L.ps = ps;
        L.sc = pl->sc;
        L.order = pl->order + r.start;
        L.n_items = r.count;
        L.lanes = r.lanes;
        L.out_score = out_score;
        L.out_end = out_end;
        L.boundary = r.bnd_bytes_group ? (uint8_t *)pl->dyn.ptr + r.bnd_offset : nullptr;
        L.boundary_group_bytes = (int64_t)r.bnd_bytes_group;
        L.work_counter = pl->counters + r.cls;
        L.status = &pl->info->status;
        if ((rc = launch_score(r.rows, r.mode, L, r.blocks, kThreads, st))) return rc;
    }
    if (!pl->cigar || !cig) return SW_OK;
    TbParams P{ps, pl->sc, out_score, out_end, cig->ops, cig->offsets, cig->n_ops, 1, kSmallSlabWords};
    if (cuda_failed(cudaMemsetAsync(pl->hist, 0, sizeof(int32_t) * nh, st))) return SW_ERR_CUDA;
    if (cuda_failed(cudaMemsetAsync(pl->tbinfo, 0, sizeof(TbClassInfo), st))) return SW_ERR_CUDA;
    if ((rc = launch_tb_keys(P, pl->n_pairs, pl->keys, pl->tb_keys, pl->hist, pl->tbinfo, st))) return rc;
    if ((rc = launch_scan_scatter(pl->tb_keys, pl->n_pairs, pl->info->count, pl->hist, pl->bstart, pl->cursor,
                                  pl->tb_order, st)))
        return rc;
    const int64_t wpb = kThreads / 32;
    for (const PlanTbRun &t : pl->truns) {
        TracebackLaunch B{};
        B.P = P;
        B.P.lanes = t.lanes;
        B.lanes = t.lanes;
        B.slab = (uint32_t *)pl->dyn.ptr;
        B.slab_group_words = t.slab_words;
        B.boundary_group_ints = t.bnd_ints;
        B.wcap = t.wcap;
        B.tiled = t.tiled;
        B.packed16 = t.packed16;
        B.work_counter = pl->counters + 2 * N_CLASS + 2 * t.cls;
        B.status = &pl->info->status;
        if (t.packed16) {
            const int64_t round_items = t.round_tasks * (64 / t.lanes);
            B.boundary = (int32_t *)pl->dyn.ptr + (size_t)t.round_tasks * 32 * t.slab_words;
            for (int64_t r0 = 0; r0 < t.count; r0 += round_items) {
                B.order = pl->tb_order + t.start + r0;
                B.n_items = std::min<int64_t>(round_items, t.count - r0);
                if (r0 > 0 && cuda_failed(cudaMemsetAsync(B.work_counter, 0, sizeof(int32_t), st)))
                    return SW_ERR_CUDA;
                if ((rc = launch_traceback(B, t.blocks, kThreads, st))) return rc;
            }
        } else {
            B.order = pl->tb_order + t.start;
            B.n_items = t.count;
            B.boundary = (int32_t *)pl->dyn.ptr + (size_t)t.blocks * wpb * (32 / t.lanes) * t.slab_words;
            if ((rc = launch_traceback(B, t.blocks, kThreads, st))) return rc;
        }
    }
    return SW_OK;
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
    if (cuda_failed(cudaEventRecord(ds->fork_ev, st))) return SW_ERR_CUDA;
    if (cuda_failed(cudaStreamWaitEvent(ds->copy_in, ds->fork_ev, 0))) return SW_ERR_CUDA;
    if (cuda_failed(cudaStreamWaitEvent(ds->copy_out, ds->fork_ev, 0))) return SW_ERR_CUDA;
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
    g_plans.push_back(PlanOverride{max_read_len, lanes, r_rows});
    std::sort(g_plans.begin(), g_plans.end(),
              [](const PlanOverride &a, const PlanOverride &b) { return a.max_read_len < b.max_read_len; });
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
    if (mode != SW_SCORE_AUTO && mode != SW_SCORE_INT32) return SW_ERR_INVALID_ARG;
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
    out2[0] = ds->tb_split[0];
    out2[1] = ds->tb_split[1];
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

int sw_alu_probe(int32_t kind, int64_t iters, double *ops_per_s, sw_stream_t stream)
{
    if (!ops_per_s || iters < 1 || kind < 0 || kind > 6) return SW_ERR_INVALID_ARG;
    DeviceState *ds = nullptr;
    int rc = device_state(&ds, (cudaStream_t)stream);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int threads = 256, blocks = ds->sm_count * 8;
    uint32_t *out = nullptr;
    if (cuda_failed(cudaMalloc(&out, sizeof(uint32_t) * threads * blocks))) return SW_ERR_CUDA;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    rc = launch_alu_probe(kind, iters / 8 + 1, blocks, threads, out, st);  // warm-up
    cudaEventRecord(e0, st);
    if (!rc) rc = launch_alu_probe(kind, iters, blocks, threads, out, st);
    cudaEventRecord(e1, st);
    float ms = 0.f;
    if (!rc && (cuda_failed(cudaEventSynchronize(e1)) || cuda_failed(cudaEventElapsedTime(&ms, e0, e1))))
        rc = SW_ERR_CUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (rc) return rc;
    *ops_per_s = (double)blocks * threads * 8.0 * (double)iters / (ms * 1e-3);
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
    pl->force_i32 = g_score_mode.load() == SW_SCORE_INT32;
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
    if (cuda_failed(cudaMemcpy(&v, &plan->info->status, sizeof(v), cudaMemcpyDeviceToHost))) return SW_ERR_CUDA;
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

int sw_gather_probe(int32_t log2_words, int64_t rounds, double *loads_per_s, sw_stream_t stream)
{
    if (!loads_per_s || log2_words < 20 || log2_words > 34 || rounds < 1) return SW_ERR_INVALID_ARG;
    DeviceState *ds = nullptr;
    int rc = device_state(&ds, (cudaStream_t)stream);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t words = (size_t)1 << log2_words;
    const int threads = 256, blocks = ds->sm_count * 8;
    uint32_t *buf = nullptr, *out = nullptr;
    if (cuda_failed(cudaMalloc(&buf, words * sizeof(uint32_t)))) return SW_ERR_CUDA;
    if (cuda_failed(cudaMalloc(&out, sizeof(uint32_t) * threads * blocks))) {
        cudaFree(buf);
        return SW_ERR_CUDA;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms = 0.f;
    rc = cuda_failed(cudaMemsetAsync(buf, 0x5A, words * sizeof(uint32_t), st)) ? SW_ERR_CUDA : SW_OK;
    if (!rc && (cuda_failed(cudaEventCreate(&e0)) || cuda_failed(cudaEventCreate(&e1)))) rc = SW_ERR_CUDA;
    if (!rc) rc = launch_gather_probe(buf, words - 1, rounds / 8 + 1, blocks, threads, out, st);  // warm-up
    if (!rc && cuda_failed(cudaEventRecord(e0, st))) rc = SW_ERR_CUDA;
    if (!rc) rc = launch_gather_probe(buf, words - 1, rounds, blocks, threads, out, st);
    if (!rc && cuda_failed(cudaEventRecord(e1, st))) rc = SW_ERR_CUDA;
    if (!rc && (cuda_failed(cudaEventSynchronize(e1)) || cuda_failed(cudaEventElapsedTime(&ms, e0, e1))))
        rc = SW_ERR_CUDA;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    cudaFree(buf);
    if (rc) return rc;
    *loads_per_s = (double)blocks * threads * 8.0 * (double)rounds / (ms * 1e-3);
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
