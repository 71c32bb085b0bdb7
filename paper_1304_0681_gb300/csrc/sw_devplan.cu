// sw_devplan.cu -- launch planning on the device.
//
// The paper hands whole batches to OpenMP threads and balances the thread
// counts of its stages by hand (Section 3.4, Section 4.3).  Here a batch is
// sorted into length classes on the GPU, and two one-block kernels plan the
// launches from the classification's per-class facts, so that the host
// enqueues a fixed sequence of launches and never waits for the device:
//
//   k_plan_score  per class the lanes per pair and rows per lane (the cost
//                 model of score_plan_of), the class's place in the sorted
//                 order, its score variant (compiled rows x arithmetic
//                 mode), and the chunk-boundary scratch of classes whose
//                 reads need several row chunks;
//   k_plan_tb     per class and part (pairs with big slabs, the rest) the
//                 traceback kernel, its lanes per pair and slab sizes
//                 (tb_part_shape), and per traceback variant the size of a
//                 warp's scratch slot and how many warps fit the budget.
//
// Each variant's list is ordered longest reads first, so the persistent
// launches end on short work.
#include "sw_device.cuh"
#include "swgb_internal.h"

namespace swgb {

__global__ void __launch_bounds__(kPlanThreads) k_plan_score(const ClassInfo *__restrict__ info, const PlanParams pp,
                                                             DevScorePlan *__restrict__ out,
                                                             int32_t *__restrict__ status)
{
    __shared__ int32_t s_var[N_CLASS], s_cnt[N_CLASS], s_bnd[N_CLASS], s_lanes[N_CLASS];
    for (int c = threadIdx.x; c < N_CLASS; c += blockDim.x) {
        const int32_t cnt = info->count[c];
        int32_t var = -1, bnd = 0, lanes = 1;
        if (cnt > 0) {
            const int mode = c / N_MCLASS;
            const int32_t mm = info->max_m[c], mn = info->max_n[c];
            int ri = 0;
            const int64_t hmax = (int64_t)pp.sc.ma * min(mm, mn);
            score_plan_of(mode, mm, hmax, pp.ov, pp.n_overrides, lanes, ri);
            // a class with fewer tasks than half its launch's warps (a small
            // batch) finishes when one task does: fewer rows per lane, on
            // more lanes, shorten the task while it still fits one row chunk
            // (not when an override chose the plan)
            bool chosen = false;
            for (int i = 0; i < pp.n_overrides; ++i) chosen |= mm <= pp.ov[i].max_read_len;
            while (!chosen && ri > 0) {
                const int64_t per_warp = (int64_t)(32 / lanes) * (mode != MODE_I32 ? 2 : 1);
                const int64_t tasks = (cnt + per_warp - 1) / per_warp;
                if (2 * tasks >= pp.score_warps[ri * N_MODES + mode]) break;
                const int t2 = (mm + score_rows_at(ri - 1) - 1) / score_rows_at(ri - 1);
                if (t2 > 32) break;
                --ri;
                lanes = t2;
            }
            const int rows = score_rows_at(ri);
            const int chunks = (mm + lanes * rows - 1) / (lanes * rows);
            // per group: two buffers x longest window x (H, F) x 4 bytes
            bnd = chunks > 1 ? 16 * mn : 0;
            var = ri * N_MODES + mode;
        }
        s_var[c] = var;
        s_cnt[c] = cnt;
        s_bnd[c] = bnd;
        s_lanes[c] = lanes;
        out->cls_count[c] = cnt;
        out->cls_lanes[c] = lanes;
        out->cls_bnd_bytes[c] = bnd;
    }
    __syncthreads();
    // the first warp finishes: class starts (a warp scan over the counts),
    // then each variant's class list, longest reads first (classes are
    // mode-major, so within a variant -- one mode -- a larger class index is
    // a longer read class), built with ballots
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    const unsigned lt = (1u << lane) - 1u;
    {
        constexpr int PER = (N_CLASS + 31) / 32;
        int32_t sum = 0;
        for (int i = 0; i < PER; ++i) {
            const int c = lane * PER + i;
            if (c < N_CLASS) sum += s_cnt[c];
        }
        int32_t x = sum;
        for (int d = 1; d < 32; d <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += y;
        }
        int32_t run = x - sum;
        for (int i = 0; i < PER; ++i) {
            const int c = lane * PER + i;
            if (c < N_CLASS) {
                out->cls_start[c] = run;
                run += s_cnt[c];
            }
        }
    }
    int nb = 0;
    int32_t n_v[N_SCORE_VARIANTS];
    int64_t slot_v[N_SCORE_VARIANTS];
    for (int v = 0; v < N_SCORE_VARIANTS; ++v) {
        int32_t n = 0;
        int64_t slot = 0;
        for (int c0 = N_CLASS - 1; c0 >= 0; c0 -= 32) {
            const int c = c0 - lane;
            const bool hit = c >= 0 && s_var[c] == v;
            const unsigned m = __ballot_sync(0xffffffffu, hit);
            if (hit) {
                out->var_cls[v][n + __popc(m & lt)] = (int16_t)c;
                slot = max(slot, (int64_t)(32 / s_lanes[c]) * s_bnd[c]);  // a warp's groups
            }
            n += __popc(m);
        }
        for (int d = 16; d; d >>= 1) slot = max(slot, __shfl_xor_sync(0xffffffffu, slot, d));
        n_v[v] = n;
        slot_v[v] = slot;
        nb += slot > 0;
    }
    if (lane != 0) return;
    const int64_t share = nb ? (pp.score_bnd_bytes / nb) & ~(int64_t)255 : 0;
    int64_t off = 0;
    for (int v = 0; v < N_SCORE_VARIANTS; ++v) {
        out->var_n[v] = n_v[v];
        out->var_bnd_warps[v] = 0;
        out->var_bnd_offset[v] = 0;
        out->var_bnd_slot[v] = slot_v[v];
        if (slot_v[v] > 0) {
            const int64_t w = min((int64_t)pp.score_warps[v], share / slot_v[v]);
            if (w < 1) atomicOr(status, ST_UNSUPPORTED);  // one warp's rows do not fit the scratch
            out->var_bnd_warps[v] = (int32_t)w;
            out->var_bnd_offset[v] = off;
            off += share;
        }
    }
}

__global__ void __launch_bounds__(kPlanThreads) k_plan_tb(const ClassInfo *__restrict__ info,
                                                          const TbClassInfo *__restrict__ ti,
                                                          const DevScorePlan *__restrict__ sp, const PlanParams pp,
                                                          DevTbPlan *__restrict__ out, int32_t *__restrict__ status)
{
    __shared__ int64_t s_slot[N_TB_PARTS];
    __shared__ int8_t s_pv[N_TB_PARTS];  // each part's variant (-1: none)
    for (int c = threadIdx.x; c < N_CLASS; c += blockDim.x) {
        const int32_t cnt = info->count[c];
        const int32_t big = ti->n_big[c];
        const int32_t counts[2] = {big, cnt - big};
        const int32_t starts[2] = {sp->cls_start[c], sp->cls_start[c] + big};
        for (int part = 0; part < 2; ++part) {
            TbPartPlan t{};
            t.cls = c;
            t.part = part;
            t.start = starts[part];
            t.count = counts[part];
            t.variant = -1;
            int64_t slot = 0;
            if (t.count > 0) {
                const int64_t need = ti->max_need[c] > 1 ? ti->max_need[c] : 1;
                // a part too small to give a task (64 / T pairs) to a quarter
                // of the warps of a launch spreads each pair over more lanes
                // (at most 8): the tasks then finish sooner, which is what a
                // small batch waits for
                int min_lanes = 1;
                while (min_lanes < 8 && (int64_t)t.count * min_lanes < (int64_t)pp.tb_warps[0] * 16) min_lanes *= 2;
                slot = tb_part_shape(c / N_MCLASS, pp.allow16 != 0, info->max_m[c], need, ti->max_wcap[part][c],
                                     part, pp.small_slab_words, t, min_lanes);
            }
            out->part[2 * c + part] = t;
            s_slot[2 * c + part] = slot;
            s_pv[2 * c + part] = (int8_t)t.variant;
        }
    }
    __syncthreads();
    // the first warp finishes: each variant's part list (longest reads
    // first, big-slab part first), its slot and pool sizes, and the split
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    const unsigned lt = (1u << lane) - 1u;
    const int PAIRS_OF[N_TB16_VARIANTS] = {64, 32, 16, 8, 4, 2};
    int32_t n_v[N_TB_VARIANTS];
    int64_t slot_v[N_TB_VARIANTS], bnd_v[N_TB_VARIANTS], need_v[N_TB_VARIANTS];
    int64_t split16 = 0, split32 = 0;
    for (int v = 0; v < N_TB_VARIANTS; ++v) {
        int32_t n = 0;
        int64_t slot = 0, bnd = 0, need = 0;
        for (int q0 = N_TB_PARTS - 1; q0 >= 0; q0 -= 32) {
            // parts 2c (big) and 2c + 1 of class c, classes descending
            const int qi = q0 - lane;
            const int q = qi >= 0 ? (qi ^ 1) : -1;
            const bool hit = q >= 0 && s_pv[q] == v;
            const TbPartPlan *t = hit ? &out->part[q] : nullptr;
            const unsigned m = __ballot_sync(0xffffffffu, hit);
            if (hit) {
                out->var_part[v][n + __popc(m & lt)] = (int16_t)q;
                slot = max(slot, s_slot[q]);
                if (v < N_TB16_VARIANTS) {
                    bnd = max(bnd, t->bnd_ints);
                    need += (int64_t)((t->count + PAIRS_OF[v] - 1) / PAIRS_OF[v]) * 32 * t->slab_words;
                    split16 += t->count;
                } else {
                    split32 += t->count;
                }
            }
            n += __popc(m);
        }
        for (int d = 16; d; d >>= 1) {
            slot = max(slot, __shfl_xor_sync(0xffffffffu, slot, d));
            bnd = max(bnd, __shfl_xor_sync(0xffffffffu, bnd, d));
            need += __shfl_xor_sync(0xffffffffu, need, d);
        }
        n_v[v] = n;
        slot_v[v] = slot;
        bnd_v[v] = bnd;
        need_v[v] = need;
    }
    for (int d = 16; d; d >>= 1) {
        split16 += __shfl_xor_sync(0xffffffffu, split16, d);
        split32 += __shfl_xor_sync(0xffffffffu, split32, d);
    }
    if (lane != 0) return;
    out->split[0] = split16;
    out->split[1] = split32;
    // the launches run one after another, each with the whole budget
    const int64_t total = pp.tb_bytes / 4;
    auto r64 = [](int64_t x) { return (x + 63) & ~(int64_t)63; };  // 256-byte alignment
    for (int v = 0; v < N_TB_VARIANTS; ++v) {
        out->var_n[v] = n_v[v];
        out->var_slot_offset[v] = 0;
        out->var_bnd_words[v] = 0;
        out->var_warps[v] = 0;
        out->var_run_warps[v] = 0;
        out->var_slot_words[v] = 0;
        if (!n_v[v]) continue;
        if (v >= N_TB16_VARIANTS) {
            // int32 kernels: a slot per warp, as many warps as fit
            const int64_t words = r64(slot_v[v]);
            const int64_t w = min((int64_t)pp.tb_warps[v], total / max(words, (int64_t)1));
            if (w < 1) atomicOr(status, ST_UNSUPPORTED);  // one warp's slot does not fit the scratch
            out->var_slot_words[v] = words;
            out->var_warps[v] = (int32_t)w;
            continue;
        }
        // 16-bit kernel: boundary rows of the warps that take part, full
        // slots, then the pool; tiles go to the pool (walked later at full
        // occupancy) or are swept and walked by warps that hold a full slot
        int64_t tile = 0;
        for (int i = 0; i < n_v[v]; ++i) tile = max(tile, 32 * out->part[out->var_part[v][i]].slab_words);
        const int64_t bnd = r64(bnd_v[v]), need = need_v[v];
        tile = r64(tile);
        if (bnd + tile > total) {
            atomicOr(status, ST_UNSUPPORTED);  // not even one warp's row and slot fit the scratch
            continue;
        }
        // as many warps as fit take part (each with a boundary row), at
        // least one of them with a full slot
        const int64_t run = bnd ? min((int64_t)pp.tb_warps[v], (total - tile) / bnd) : (int64_t)pp.tb_warps[v];
        const int64_t avail = total - run * bnd;  // >= tile
        // T >= 4: a task has at most 16 walks, cheap next to its sweep, so
        // every running warp gets a slot if it can and the pool takes the
        // rest; T <= 2: 32 or 64 walks per task run best in the separate walk
        // kernel, so the pool comes first (half the space when it cannot
        // hold every task)
        int64_t slots;
        if (v >= 2) slots = max((int64_t)1, min(run, avail / tile));
        else if (need + tile <= avail) slots = max((int64_t)1, min(run, (avail - need) / tile));
        else slots = max((int64_t)1, min(run, (avail / 2) / tile));
        out->var_bnd_words[v] = bnd;
        out->var_slot_words[v] = tile;
        out->var_slot_offset[v] = run * bnd;
        out->var_run_warps[v] = (int32_t)run;
        out->var_warps[v] = (int32_t)slots;
        int64_t pool = out->var_slot_offset[v] + slots * tile;
        for (int i = 0; i < n_v[v]; ++i) {
            TbPartPlan &t = out->part[out->var_part[v][i]];
            const int64_t tw = r64(32 * t.slab_words);
            const int64_t tasks = (t.count + PAIRS_OF[v] - 1) / PAIRS_OF[v];
            const int64_t fit = min(tasks, (total - pool) / tw);
            t.pool_tasks = (int32_t)fit;
            t.pool_offset = pool;
            pool += fit * tw;
        }
    }
}

int launch_plan_score(const ClassInfo *info, const PlanParams &pp, DevScorePlan *out, int32_t *status,
                      cudaStream_t st)
{
    k_plan_score<<<1, kPlanThreads, 0, st>>>(info, pp, out, status);
    count_launch();
    return launch_status();
}

int launch_plan_tb(const ClassInfo *info, const TbClassInfo *ti, const DevScorePlan *sp, const PlanParams &pp,
                   DevTbPlan *out, int32_t *status, cudaStream_t st)
{
    k_plan_tb<<<1, kPlanThreads, 0, st>>>(info, ti, sp, pp, out, status);
    count_launch();
    return launch_status();
}

}  // namespace swgb
