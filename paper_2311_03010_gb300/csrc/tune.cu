// tune.cu -- partition parameters of the level solves and their autotuner
// (C ABI).
//
// The parameters decide how a level solve is split over the GPU: how many
// blocks a grid-mode solve uses (pixels per block, blocks per SM) and which
// levels run on one thread-block cluster instead.  They are process-wide and
// change only while no plan owns a workspace and no server exists, so every
// solve of the process is partitioned the same way alone, batched or served.
// eecmg_autotune times candidate settings on the caller's own workload (one
// batched restoration of the given plans) by coordinate search and keeps the
// fastest (a change must gain at least 3 %).
#include <string>
#include <vector>

#include "level_solve.hpp"
#include "plan.hpp"

using namespace eecmg;

namespace {

eecmg_tuning to_c(const Tuning& t) {
    eecmg_tuning c;
    c.cluster_max_px = t.cluster_max_px;
    c.px_per_block = t.px_per_block;
    c.blocks_per_sm = t.blocks_per_sm;
    c.resident_max_tiles = t.resident_max_tiles;
    c.psd_tile_h = t.psd_tile_h;
    return c;
}

Tuning from_c(const eecmg_tuning& c) {
    Tuning t;
    t.cluster_max_px = c.cluster_max_px;
    t.px_per_block = c.px_per_block;
    t.blocks_per_sm = c.blocks_per_sm;
    t.resident_max_tiles = c.resident_max_tiles;
    t.psd_tile_h = c.psd_tile_h;
    return t;
}

struct TuneRun {
    std::vector<eecmg_plan_s*> plans;
    std::vector<float*> u;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~TuneRun() {
        for (auto* P : plans) eecmg_plan_destroy(P);
        for (float* x : u) cudaFree(x);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
};

// Mean milliseconds of one batched restoration of the plans under t.
eecmg_status time_tuning(TuneRun& R, const float* const* g, int reps, cudaStream_t s, const Tuning& t,
                         float* ms) {
    set_tuning_raw(t);
    for (auto* P : R.plans) {  // launch shapes were baked into graphs and job tables
        forget_plan_batches(P);
        if (P->gexec) {
            cudaGraphExecDestroy(P->gexec);
            P->gexec = nullptr;
        }
    }
    const int n = (int)R.plans.size();
    for (int w = 0; w < 2; ++w) {
        eecmg_status st = restore_batched_impl(R.plans.data(), g, R.u.data(), n, s);
        if (st != EECMG_OK) return st;
    }
    cudaEventRecord(R.e0, s);
    for (int r = 0; r < reps; ++r) {
        eecmg_status st = restore_batched_impl(R.plans.data(), g, R.u.data(), n, s);
        if (st != EECMG_OK) return st;
    }
    cudaEventRecord(R.e1, s);
    cudaError_t e = cudaEventSynchronize(R.e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, R.e0, R.e1);
    if (e != cudaSuccess) return set_error(EECMG_ERR_CUDA, std::string("eecmg_autotune: ") + cudaGetErrorString(e));
    *ms /= (float)reps;
    return EECMG_OK;
}

}  // namespace

extern "C" {

eecmg_status eecmg_get_tuning(eecmg_tuning* out) {
    if (!out) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_get_tuning: out is NULL");
    *out = to_c(get_tuning());
    return EECMG_OK;
}

eecmg_status eecmg_set_tuning(const eecmg_tuning* t) {
    if (!t) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_set_tuning: NULL tuning");
    const Tuning x = from_c(*t);
    if (!tuning_valid(x))
        return set_error(EECMG_ERR_INVALID_ARG,
                         "eecmg_set_tuning: need 1024 <= px_per_block <= 4194304, cluster_max_px >= 0, "
                         "1 <= blocks_per_sm <= 3, 0 <= resident_max_tiles <= 32");
    if (g_live_owners.load() > 0)
        return set_error(EECMG_ERR_BUSY,
                         "eecmg_set_tuning: destroy every plan with a workspace and every server first");
    set_tuning_raw(x);
    return EECMG_OK;
}

eecmg_status eecmg_autotune(const eecmg_plan_t* plans, const float* const* g, int n, int reps,
                            cudaStream_t s, eecmg_tuning* best) {
    if (!plans || !g || n < 1 || reps < 1)
        return set_error(EECMG_ERR_INVALID_ARG, "eecmg_autotune: bad arguments");
    for (int i = 0; i < n; ++i)
        if (!plans[i] || !g[i] || !plans[i]->opt.persistent)
            return set_error(EECMG_ERR_INVALID_ARG,
                             "eecmg_autotune: NULL plan or input, or a plan without the persistent solve");
    if (g_live_owners.load() > 0)
        return set_error(EECMG_ERR_BUSY,
                         "eecmg_autotune: destroy every plan with a workspace and every server first "
                         "(describe the workload with workspace = 0 plans)");
    const Tuning start = get_tuning();
    eecmg_status st = EECMG_OK;
    Tuning cur = start;
    {
        TuneRun R;
        for (int i = 0; i < n && st == EECMG_OK; ++i) {
            eecmg_plan_s* P = nullptr;
            st = plan_materialize(plans[i], &P);
            if (st == EECMG_OK) R.plans.push_back(P);
            float* u = nullptr;
            if (st == EECMG_OK && cudaMalloc((void**)&u, sizeof(float) * (size_t)P->W * P->H) != cudaSuccess) {
                cudaGetLastError();
                st = set_error(EECMG_ERR_OOM, "eecmg_autotune: output buffers");
            }
            if (u) R.u.push_back(u);
        }
        if (st == EECMG_OK && (cudaEventCreate(&R.e0) != cudaSuccess || cudaEventCreate(&R.e1) != cudaSuccess))
            st = set_error(EECMG_ERR_CUDA, "eecmg_autotune: events");
        float best_ms = 0.f;
        if (st == EECMG_OK) st = time_tuning(R, g, reps, s, cur, &best_ms);
        // coordinate search: resident threshold, cluster threshold, pixels per
        // block, blocks per SM, then the rows of the fused level start's tiles
        const int rmt[] = {0, 16, 32};
        const long long cmax[] = {0, 4096, 16384, 65536, 262144};
        const int ppb[] = {1024, 2048, 4096};
        const int bps[] = {1, 2, 3};
        const int pth[] = {16, 32};
        for (int axis = 0; axis < 5 && st == EECMG_OK; ++axis) {
            const int nc = axis == 1 ? 5 : (axis == 4 ? 2 : 3);
            Tuning base = cur;
            for (int c = 0; c < nc && st == EECMG_OK; ++c) {
                Tuning t = base;
                if (axis == 0) t.resident_max_tiles = rmt[c];
                if (axis == 1) t.cluster_max_px = cmax[c];
                if (axis == 2) t.px_per_block = ppb[c];
                if (axis == 3) t.blocks_per_sm = bps[c];
                if (axis == 4) t.psd_tile_h = pth[c];
                if (t.cluster_max_px == base.cluster_max_px && t.px_per_block == base.px_per_block &&
                    t.blocks_per_sm == base.blocks_per_sm && t.resident_max_tiles == base.resident_max_tiles &&
                    t.psd_tile_h == base.psd_tile_h)
                    continue;  // already timed
                float ms = 0.f;
                st = time_tuning(R, g, reps, s, t, &ms);
                // a candidate must beat the incumbent by 3 %: timing noise does
                // not move the partition between runs
                if (st == EECMG_OK && ms < 0.97f * best_ms) {
                    best_ms = ms;
                    cur = t;
                }
            }
        }
        for (auto* P : R.plans) forget_plan_batches(P);
    }  // the private plans are destroyed here
    if (st != EECMG_OK) {
        set_tuning_raw(start);
        return st;
    }
    set_tuning_raw(cur);
    if (best) *best = to_c(cur);
    return EECMG_OK;
}

}  // extern "C"
