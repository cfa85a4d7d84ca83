// batch.cu -- batched restoration: many images of different sizes and PSFs,
// one persistent cooperative launch per cascade step covering all of them.
//
// Each image keeps its own plan (workspace, level pyramid, scalars).  Per
// cascade step s (levels counted from the coarsest, so every image's level s
// is at the same depth of Algorithm 2), the level solves of all images are
// jobs of one persistent launch: image i's job owns a range of blocks with its
// own group barrier, reduction partials and scalars, so the images never
// wait for one another inside the launch.  Jobs are grouped by solver,
// separability, precision and storage type (one kernel instantiation each)
// and, within a
// group, share the largest PSF radius (smaller PSFs are zero-padded).  The
// restriction and the prolongation chain run before each step as one launch
// per kind of operation over all images (k_ops_batch).
// The whole batch is captured once as a CUDA graph per set of plans and
// replayed.  The graph's kernels read their buffers from device job tables, so
// each image's finest level runs in the caller's g and u: the table fields that
// name them are rebound when the caller's buffers change (see BatchCtx).
#include <algorithm>
#include <cstddef>
#include <cstring>
#include <cstdint>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "batch.hpp"
#include "launch.hpp"

namespace eecmg {

LevelJob make_job(eecmg_plan_s* P, int l) {
    LevelPlan& L = P->lv[l];
    LevelJob J;
    J.g = L.g;
    J.u = L.u;
    for (int i = 0; i < 2; ++i) {
        J.v[i] = P->vec[0 + i];
        J.aw[i] = P->vec[2 + i];
        J.d[i] = P->vec[4 + i];
        J.hd[i] = P->vec[6 + i];
    }
    J.r = P->vec[8];
    J.taps = P->dtaps + 2 * l;
    J.tapsT = P->dtaps + 2 * l + 1;
    J.sc = P->sc + l;
    J.partials = P->partials;
    J.gs = P->gsync + l;
    J.conv_tol2 = P->conv_tol2;
    J.disc2 = L.disc2;
    J.early = P->opt.early_check;
    J.h = L.h;
    J.w = L.w;
    J.m = L.m;
    const int nzero = P->opt.prolong == EECMG_PROLONG_EECMG ? 2 : 1;
    J.zero_start = l < nzero ? 1 : 0;
    set_level_start(P, l, J);
    return J;
}

eecmg_status plan_waves(const std::vector<std::pair<eecmg_plan_s*, int>>& items,
                        std::vector<HostWave>& waves) {
    waves.clear();
    // (cluster size, resident tiles, instantiation) -> indices of items
    std::map<std::tuple<int, int, int, int, int, int>, std::vector<int>> groups;
    for (int i = 0; i < (int)items.size(); ++i) {
        eecmg_plan_s* P = items[i].first;
        const int l = items[i].second;
        const int cg = P->opt.smoother == EECMG_SMOOTHER_CGLS ? 1 : 0;
        const int bf = P->opt.storage == EECMG_STORAGE_BF16 ? 1 : 0;
        const LevelShape sh = level_shape(P->lv[l].h, P->lv[l].w, P->lv[l].rt, cg, bf);
        groups[{sh.cluster, sh.resident, cg, P->lv[l].sepH, P->opt.precise_conv, bf}].push_back(i);
    }
    for (auto& kv : groups) {
        const int cl = std::get<0>(kv.first), res = std::get<1>(kv.first), cg = std::get<2>(kv.first),
                  sep = std::get<3>(kv.first), prec = std::get<4>(kv.first),
                  bf = std::get<5>(kv.first);
        int rt = 0;
        for (int i : kv.second) rt = std::max(rt, items[i].first->lv[items[i].second].rt);
        // clusters are independent: one launch holds them all
        const int cap = cl > 0 ? INT32_MAX : level_capacity(rt, sep, prec, cg, bf);
        if (cap <= 0) return set_error(EECMG_ERR_CUDA, "batched level solve: occupancy query failed");
        HostWave cur;
        cur.rt = rt;
        cur.sep = sep;
        cur.prec = prec;
        cur.cgls = cg;
        cur.bf16 = bf;
        cur.cluster = cl;
        cur.resident = res;
        for (int i : kv.second) {
            const LevelPlan& Lp = items[i].first->lv[items[i].second];
            const int nb = cl > 0 ? cl : std::max(1, std::min(cap, level_shape(Lp.h, Lp.w, Lp.rt, cg, bf).blocks));
            if ((long long)cur.blocks + nb > cap && !cur.jobs.empty()) {  // next wave
                waves.push_back(cur);
                cur.jobs.clear();
                cur.block_job.clear();
                cur.blocks = 0;
            }
            LevelJob J = make_job(items[i].first, items[i].second);
            J.block0 = cur.blocks;
            J.nblocks = nb;
            for (int b = 0; b < nb; ++b) cur.block_job.push_back((unsigned short)cur.jobs.size());
            cur.jobs.push_back(J);
            cur.blocks += nb;
        }
        if (!cur.jobs.empty()) waves.push_back(cur);
    }
    return EECMG_OK;
}

void add_op(std::vector<OpGroup>& groups, size_t gi, int op, OpItem it) {
    if (groups.size() <= gi) groups.resize(gi + 1);
    groups[gi].op = op;
    it.bx = op_blocks_x(op, it.w);
    if (op == OP_PSD) it.th = psd_tile_rows();
    groups[gi].items.push_back(it);
}

int place_items(OpGroup& g) {
    int blocks = 0;
    for (auto& it : g.items) {
        it.block0 = blocks;
        blocks += op_blocks(g.op, it.h, it.w);
    }
    return blocks;
}

// Every coarse level straight from the finest, g_l(a, b) = g_{L-1}(2^j a, 2^j b)
// with j = L-1-l (the restrictions compose; pure copies, so bitwise the
// level-by-level chain): one launch for the whole pyramid of every plan.
void restrict_ops(const std::vector<eecmg_plan_s*>& plans, std::vector<OpGroup>& groups) {
    const size_t base = groups.size();
    for (eecmg_plan_s* P : plans)
        for (int l = P->L - 2; l >= 0; --l) {
            const LevelPlan& F = P->lv[P->L - 1];
            OpItem rs;
            rs.a = F.g;
            rs.w1 = F.w;
            rs.h2 = 1 << (P->L - 1 - l);  // stride into the finest level
            rs.out = P->lv[l].g;
            rs.h = P->lv[l].h;
            rs.w = P->lv[l].w;
            add_op(groups, base, OP_RESTRICT, rs);
        }
}

void step_ops(const std::vector<std::pair<eecmg_plan_s*, int>>& items, std::vector<OpGroup>& groups) {
    const size_t base = groups.size();
    const size_t G_PSD = base, G_EXTRA = base + 1, G_QUAD = base + 2, G_LIN = base + 3,
                 G_SMOOTH = base + 4, G_STEP0 = base + 5;  // + diffusion step
    for (auto& itm : items) {
        eecmg_plan_s& P = *itm.first;
        const int st = itm.second;
        const int nzero = P.opt.prolong == EECMG_PROLONG_EECMG ? 2 : 1;
        LevelPlan& L = P.lv[st];
        // the persistent solve writes its zero start, or runs the fused start, itself
        if (st < nzero || level_fused_start(&P, st)) continue;
        LevelPlan& L1 = P.lv[st - 1];
        float* up = P.vec[0];
        float* sm = P.vec[1];
        const int steps = P.opt.diffusion_steps;
        const float kpm = (float)P.kpm;
        if (P.opt.prolong == EECMG_PROLONG_EECMG && steps >= 1) {  // fused D(S(P(Pi))), then D steps 2..
            LevelPlan& L2 = P.lv[st - 2];
            OpItem x;
            x.a = L1.u;
            x.b = L2.u;
            x.out = steps == 1 ? L.u : sm;
            x.h = L.h;
            x.w = L.w;
            x.h1 = L1.h;
            x.w1 = L1.w;
            x.h2 = L2.h;
            x.w2 = L2.w;
            x.s0 = (float)P.opt.s_scale;
            x.p0 = (float)P.tau;
            x.p1 = 1.f / (kpm * kpm);
            add_op(groups, G_PSD, OP_PSD, x);
            const float* cur = x.out;
            for (int d = 1; d < steps; ++d) {
                float* nxt = (d == steps - 1) ? L.u : (cur == sm ? up : sm);
                OpItem dn;
                dn.a = cur;
                dn.out = nxt;
                dn.h = L.h;
                dn.w = L.w;
                dn.p0 = (float)P.tau;
                dn.p1 = 1.f / (kpm * kpm);
                add_op(groups, G_STEP0 + 1 + (size_t)d, OP_DENOISE, dn);
                cur = nxt;
            }
            continue;
        }
        if (P.opt.prolong == EECMG_PROLONG_EECMG) {  // fused P(Pi)
            LevelPlan& L2 = P.lv[st - 2];
            OpItem x;
            x.a = L1.u;
            x.b = L2.u;
            x.out = up;
            x.h = L.h;
            x.w = L.w;
            x.h1 = L1.h;
            x.w1 = L1.w;
            x.h2 = L2.h;
            x.w2 = L2.w;
            add_op(groups, G_EXTRA, OP_PROLONG, x);
        } else {
            OpItem q;
            q.a = L1.u;
            q.out = up;
            q.h = L.h;
            q.w = L.w;
            q.h1 = L1.h;
            q.w1 = L1.w;
            const bool quad = P.opt.prolong == EECMG_PROLONG_IECMG_P;
            add_op(groups, quad ? G_QUAD : G_LIN, quad ? OP_QUADRATIC : OP_LINEAR, q);
        }
        OpItem sms;
        sms.a = up;
        sms.out = sm;
        sms.h = L.h;
        sms.w = L.w;
        sms.p0 = (float)P.opt.s_scale;
        add_op(groups, G_SMOOTH, OP_SMOOTH, sms);
        if (steps <= 0) {
            OpItem c;
            c.a = sm;
            c.out = L.u;
            c.h = L.h;
            c.w = L.w;
            add_op(groups, G_STEP0, OP_COPY, c);
            continue;
        }
        const float* cur = sm;
        for (int d = 0; d < steps; ++d) {
            float* nxt = (d == steps - 1) ? L.u : (cur == sm ? up : sm);
            OpItem dn;
            dn.a = cur;
            dn.out = nxt;
            dn.h = L.h;
            dn.w = L.w;
            dn.p0 = (float)P.tau;
            dn.p1 = 1.f / (kpm * kpm);
            add_op(groups, G_STEP0 + 1 + (size_t)d, OP_DENOISE, dn);  // never in the copy group
            cur = nxt;
        }
    }
}

namespace {

struct Wave {
    const LevelJob* d_jobs = nullptr;
    const unsigned short* d_block_job = nullptr;
    int njobs = 0, blocks = 0, rt = 0, sep = 0, prec = 0, cgls = 0, bf16 = 0, cluster = 0, resident = 0;
};

struct OpLaunch {
    int op = -1;
    const OpItem* d_items = nullptr;
    int n = 0, blocks = 0;
};

struct BatchCtx {
    std::vector<eecmg_plan_s*> plans;
    std::vector<std::vector<Wave>> steps;  // per cascade step
    std::vector<OpLaunch> restrict_ops;    // the data pyramids
    std::vector<std::vector<OpLaunch>> step_ops;  // per cascade step, before its waves
    void* dmem = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    size_t graph_nodes = 0;  // kernel nodes of one batched restoration
    // Steps 0 and 1 (the two levels solved from zero, Algorithm 2) run as two
    // branches of the graph when every job of both is a resident solve: such
    // a solve touches only its own level's g, u, scalars and sync words.
    bool fork01 = false;
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // Measurement hook: event-record nodes around the level-solve launches of
    // cascade step timed_step (-1: none).
    int timed_step = -1;
    cudaEvent_t tev[2] = {nullptr, nullptr};
    // Image binding: the finest level of plan i reads bound_g[i] and writes bound_u[i] (its
    // workspace's own buffers, or the caller's).  sites: where the tables hold those two
    // pointers (byte offset of the 8-byte field in the table image, found at build time,
    // when every such field still holds its plan's own workspace buffer).  h_img: a pinned
    // copy of the table image, patched and uploaded when a binding changes.
    struct Site {
        size_t off;
        int plan;
        bool isu;
    };
    std::vector<Site> sites;
    std::vector<const float*> bound_g;
    std::vector<float*> bound_u;
    char* h_img = nullptr;
    size_t img_bytes = 0;
    cudaEvent_t ev_up = nullptr;
    ~BatchCtx() {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        if (side) cudaStreamDestroy(side);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        for (cudaEvent_t e : tev)
            if (e) cudaEventDestroy(e);
        if (dmem) cudaFree(dmem);
        if (h_img) cudaFreeHost(h_img);
        if (ev_up) cudaEventDestroy(ev_up);
    }
};

std::mutex g_batch_mu;
std::map<std::vector<eecmg_plan_s*>, std::unique_ptr<BatchCtx>> g_batches;
std::vector<std::vector<eecmg_plan_s*>> g_batch_lru;  // least recently used first
constexpr size_t BATCH_CACHE_MAX = 64;                // cached plan sets (graph + job tables)

void touch_batch(const std::vector<eecmg_plan_s*>& key) {
    auto it = std::find(g_batch_lru.begin(), g_batch_lru.end(), key);
    if (it != g_batch_lru.end()) g_batch_lru.erase(it);
    g_batch_lru.push_back(key);
}

// Builds the job tables of every step (one device allocation).
eecmg_status build_ctx(BatchCtx& C) {
    int maxL = 0;
    for (auto* P : C.plans) maxL = std::max(maxL, P->L);
    std::vector<std::vector<HostWave>> hsteps(maxL);
    for (int s = 0; s < maxL; ++s) {
        std::vector<std::pair<eecmg_plan_s*, int>> items;
        for (auto* P : C.plans)
            if (s < P->L) items.push_back({P, s});
        eecmg_status st = plan_waves(items, hsteps[s]);
        if (st != EECMG_OK) return st;
    }
    // per-level operations: one launch per kind over all images
    std::vector<OpGroup> rgroups;
    restrict_ops(C.plans, rgroups);
    std::vector<std::vector<OpGroup>> sgroups(maxL);
    for (int s = 0; s < maxL; ++s) {
        std::vector<std::pair<eecmg_plan_s*, int>> items;
        for (auto* P : C.plans)
            if (s < P->L) items.push_back({P, s});
        step_ops(items, sgroups[s]);
    }
    size_t bytes = 0;
    auto group_bytes = [](std::vector<OpGroup>& gs) {
        size_t b = 0;
        for (auto& g : gs) b += (sizeof(OpItem) * g.items.size() + 255) / 256 * 256;
        return b;
    };
    bytes += group_bytes(rgroups);
    for (auto& gs : sgroups) bytes += group_bytes(gs);
    for (auto& st : hsteps)
        for (auto& w : st) {
            bytes += (sizeof(LevelJob) * w.jobs.size() + 255) / 256 * 256;
            bytes += (sizeof(unsigned short) * w.block_job.size() + 255) / 256 * 256;
        }
    const size_t img = bytes ? bytes : 256;
    cudaError_t e = cudaMalloc(&C.dmem, img);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&C.h_img, img);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&C.ev_up, cudaEventDisableTiming);
    if (e != cudaSuccess) return set_error(EECMG_ERR_OOM, "eecmg_restore_batched: job tables");
    C.img_bytes = img;
    std::memset(C.h_img, 0, img);
    char* p = (char*)C.dmem;
    const size_t np = C.plans.size();
    C.bound_g.resize(np);
    C.bound_u.resize(np);
    for (size_t i = 0; i < np; ++i) {
        const LevelPlan& F = C.plans[i]->lv[C.plans[i]->L - 1];
        C.bound_g[i] = F.g;
        C.bound_u[i] = F.u;
    }
    // a pointer field at image offset off that holds some plan's finest g or u is a site
    auto note = [&](size_t off, const void* v) {
        for (size_t i = 0; i < np; ++i) {
            if (v == C.bound_g[i]) C.sites.push_back({off, (int)i, false});
            if (v == C.bound_u[i]) C.sites.push_back({off, (int)i, true});
        }
    };
    auto upload_groups = [&](std::vector<OpGroup>& gs, std::vector<OpLaunch>& out) -> cudaError_t {
        for (auto& g : gs) {
            if (g.items.empty() || g.op < 0) continue;
            OpLaunch L;
            L.op = g.op;
            L.blocks = place_items(g);
            L.n = (int)g.items.size();
            L.d_items = (const OpItem*)p;
            const size_t base = (size_t)(p - (char*)C.dmem);
            std::memcpy(C.h_img + base, g.items.data(), sizeof(OpItem) * g.items.size());
            for (size_t k = 0; k < g.items.size(); ++k) {
                const size_t o = base + k * sizeof(OpItem);
                note(o + offsetof(OpItem, a), g.items[k].a);
                note(o + offsetof(OpItem, b), g.items[k].b);
                note(o + offsetof(OpItem, out), g.items[k].out);
            }
            p += (sizeof(OpItem) * g.items.size() + 255) / 256 * 256;
            out.push_back(L);
        }
        return cudaSuccess;
    };
    e = upload_groups(rgroups, C.restrict_ops);
    C.step_ops.assign(maxL, {});
    for (int s = 0; s < maxL && e == cudaSuccess; ++s) e = upload_groups(sgroups[s], C.step_ops[s]);
    C.steps.assign(maxL, {});
    for (int s = 0; s < maxL; ++s)
        for (auto& w : hsteps[s]) {
            Wave dw;
            dw.d_jobs = (const LevelJob*)p;
            size_t base = (size_t)(p - (char*)C.dmem);
            std::memcpy(C.h_img + base, w.jobs.data(), sizeof(LevelJob) * w.jobs.size());
            for (size_t k = 0; k < w.jobs.size(); ++k) {
                const size_t o = base + k * sizeof(LevelJob);
                note(o + offsetof(LevelJob, g), w.jobs[k].g);
                note(o + offsetof(LevelJob, u), w.jobs[k].u);
                note(o + offsetof(LevelJob, s_u1), w.jobs[k].s_u1);
                note(o + offsetof(LevelJob, s_u2), w.jobs[k].s_u2);
            }
            p += (sizeof(LevelJob) * w.jobs.size() + 255) / 256 * 256;
            dw.d_block_job = (const unsigned short*)p;
            base = (size_t)(p - (char*)C.dmem);
            std::memcpy(C.h_img + base, w.block_job.data(), sizeof(unsigned short) * w.block_job.size());
            p += (sizeof(unsigned short) * w.block_job.size() + 255) / 256 * 256;
            dw.njobs = (int)w.jobs.size();
            dw.blocks = w.blocks;
            dw.rt = w.rt;
            dw.sep = w.sep;
            dw.prec = w.prec;
            dw.cgls = w.cgls;
            dw.bf16 = w.bf16;
            dw.cluster = w.cluster;
            dw.resident = w.resident;
            C.steps[s].push_back(dw);
        }
    e = cudaMemcpy(C.dmem, C.h_img, img, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return set_error(EECMG_ERR_CUDA, "eecmg_restore_batched: table upload");
    e = cudaStreamCreateWithFlags(&C.cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return set_error(EECMG_ERR_CUDA, "eecmg_restore_batched: stream");
    C.fork01 = maxL >= 2;
    for (auto* P : C.plans) {
        const int cg = P->opt.smoother == EECMG_SMOOTHER_CGLS ? 1 : 0;
        const int bf = P->opt.storage == EECMG_STORAGE_BF16 ? 1 : 0;
        bool ok = P->L >= 2 && P->opt.prolong == EECMG_PROLONG_EECMG;
        for (int l = 0; l < 2 && ok; ++l)
            ok = level_shape(P->lv[l].h, P->lv[l].w, P->lv[l].rt, cg, bf).resident > 0;
        C.fork01 = C.fork01 && ok;
    }
    if (C.fork01 &&
        (cudaStreamCreateWithFlags(&C.side, cudaStreamNonBlocking) != cudaSuccess ||
         cudaEventCreateWithFlags(&C.ev_fork, cudaEventDisableTiming) != cudaSuccess ||
         cudaEventCreateWithFlags(&C.ev_join, cudaEventDisableTiming) != cudaSuccess))
        return set_error(EECMG_ERR_CUDA, "eecmg_restore_batched: side stream");
    return EECMG_OK;
}

#define BCK(call)                                                                              \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return set_error(EECMG_ERR_CUDA, std::string("eecmg_restore_batched: ") + #call + \
                                                 ": " + cudaGetErrorString(e_));               \
    } while (0)

eecmg_status enqueue_step(BatchCtx& C, int st, cudaStream_t s) {
    for (const OpLaunch& L : C.step_ops[st]) BCK(launch_ops_batch(L.op, L.d_items, L.n, L.blocks, s));
    const bool timed = st == C.timed_step && !C.steps[st].empty();
    if (timed) BCK(cudaEventRecordWithFlags(C.tev[0], s, cudaEventRecordExternal));
    for (auto& w : C.steps[st])
        BCK(launch_level_batch(w.d_jobs, w.d_block_job, w.njobs, w.blocks, w.rt, w.sep, w.prec, w.cgls,
                               w.bf16, w.cluster, w.resident, s));
    if (timed) BCK(cudaEventRecordWithFlags(C.tev[1], s, cudaEventRecordExternal));
    return EECMG_OK;
}

eecmg_status enqueue_batch(BatchCtx& C, cudaStream_t s) {
    for (const OpLaunch& L : C.restrict_ops) BCK(launch_ops_batch(L.op, L.d_items, L.n, L.blocks, s));
    int st = 0;
    if (C.fork01) {  // step 0 on the side branch, step 1 on the main one
        BCK(cudaEventRecord(C.ev_fork, s));
        BCK(cudaStreamWaitEvent(C.side, C.ev_fork, 0));
        eecmg_status e0 = enqueue_step(C, 0, C.side);
        eecmg_status e1 = e0 == EECMG_OK ? enqueue_step(C, 1, s) : e0;
        BCK(cudaEventRecord(C.ev_join, C.side));  // always join the branch back
        BCK(cudaStreamWaitEvent(s, C.ev_join, 0));
        if (e1 != EECMG_OK) return e1;
        st = 2;
    }
    for (; st < (int)C.steps.size(); ++st) {
        eecmg_status e = enqueue_step(C, st, s);
        if (e != EECMG_OK) return e;
    }
    return EECMG_OK;
}

}  // namespace

eecmg_status restore_batched_impl(const eecmg_plan_t* plans, const float* const* g, float* const* u,
                                  int n, cudaStream_t s) {
    std::vector<eecmg_plan_s*> key(plans, plans + n);
    {
        std::vector<eecmg_plan_s*> sorted = key;
        std::sort(sorted.begin(), sorted.end());
        if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end())
            return set_error(EECMG_ERR_INVALID_ARG, "eecmg_restore_batched: plans must be distinct");
    }
    for (int i = 0; i < n; ++i) {
        if (!plans[i] || !g[i] || !u[i])
            return set_error(EECMG_ERR_INVALID_ARG, "eecmg_restore_batched: NULL plan or buffer");
        if (!plans[i]->opt.persistent)
            return set_error(EECMG_ERR_INVALID_ARG,
                             "eecmg_restore_batched: plans must use the persistent level solve");
    }
    std::lock_guard<std::mutex> lock(g_batch_mu);
    auto it = g_batches.find(key);
    if (it == g_batches.end()) {
        if (g_batches.size() >= BATCH_CACHE_MAX && !g_batch_lru.empty()) {
            // drop the least recently used plan set (cudaFree of its tables
            // waits for work in flight)
            g_batches.erase(g_batch_lru.front());
            g_batch_lru.erase(g_batch_lru.begin());
        }
        auto C = std::make_unique<BatchCtx>();
        C->plans = key;
        eecmg_status st = build_ctx(*C);
        if (st != EECMG_OK) return st;
        it = g_batches.emplace(key, std::move(C)).first;
    }
    touch_batch(key);
    BatchCtx& C = *it->second;
    // Each finest level works in the caller's g and u directly when its u overlaps no image's
    // g and no other image's u (the solvers never write g); otherwise it goes through the
    // workspace's own level buffers, with a copy in and a copy out.
    std::vector<char> inplace(n);
    auto span = [&](const void* ptr, int i) {
        const uintptr_t a0 = reinterpret_cast<uintptr_t>(ptr);
        return std::make_pair(a0, a0 + sizeof(float) * (uintptr_t)plans[i]->W * (uintptr_t)plans[i]->H);
    };
    auto overlap = [](std::pair<uintptr_t, uintptr_t> x, std::pair<uintptr_t, uintptr_t> y) {
        return x.first < y.second && y.first < x.second;
    };
    for (int i = 0; i < n; ++i) {
        bool ok = true;
        for (int j = 0; j < n && ok; ++j)
            ok = !overlap(span(u[i], i), span(g[j], j)) && (j == i || !overlap(span(u[i], i), span(u[j], j)));
        inplace[i] = ok;
    }
    bool rebind = false;
    for (int i = 0; i < n; ++i) {
        eecmg_plan_s* P = plans[i];
        LevelPlan& F = P->lv[P->L - 1];
        const float* bg = inplace[i] ? g[i] : F.g;
        float* bu = inplace[i] ? u[i] : F.u;
        if (bg != C.bound_g[i] || bu != C.bound_u[i]) rebind = true;
        C.bound_g[i] = bg;
        C.bound_u[i] = bu;
        if (!inplace[i])
            BCK(cudaMemcpyAsync(F.g, g[i], sizeof(float) * P->W * P->H, cudaMemcpyDeviceToDevice, s));
    }
    if (rebind) {  // patch the pointer sites and upload the tables ahead of this launch
        BCK(cudaEventSynchronize(C.ev_up));  // the previous upload has read the pinned image
        for (const BatchCtx::Site& st : C.sites) {
            const void* v = st.isu ? (const void*)C.bound_u[st.plan] : (const void*)C.bound_g[st.plan];
            std::memcpy(C.h_img + st.off, &v, sizeof(v));
        }
        BCK(cudaMemcpyAsync(C.dmem, C.h_img, C.img_bytes, cudaMemcpyHostToDevice, s));
        BCK(cudaEventRecord(C.ev_up, s));
    }
    if (!C.gexec) {
        BCK(cudaStreamBeginCapture(C.cap_stream, cudaStreamCaptureModeThreadLocal));
        eecmg_status st = enqueue_batch(C, C.cap_stream);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(C.cap_stream, &graph);
        if (st != EECMG_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e != cudaSuccess)
            return set_error(EECMG_ERR_CUDA, std::string("eecmg_restore_batched: capture: ") + cudaGetErrorString(e));
        {  // count the kernel nodes: one device launch each per restoration
            size_t nn = 0;
            cudaGraphGetNodes(graph, nullptr, &nn);
            std::vector<cudaGraphNode_t> nodes(nn);
            if (nn) cudaGraphGetNodes(graph, nodes.data(), &nn);
            C.graph_nodes = 0;
            for (auto nd : nodes) {
                cudaGraphNodeType t;
                if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++C.graph_nodes;
            }
        }
        e = cudaGraphInstantiate(&C.gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            C.gexec = nullptr;
            return set_error(EECMG_ERR_CUDA, std::string("eecmg_restore_batched: instantiate: ") + cudaGetErrorString(e));
        }
    }
    BCK(cudaGraphLaunch(C.gexec, s));
    for (int i = 0; i < n; ++i) {
        eecmg_plan_s* P = plans[i];
        LevelPlan& F = P->lv[P->L - 1];
        if (!inplace[i] && u[i] != F.u)
            BCK(cudaMemcpyAsync(u[i], F.u, sizeof(float) * P->W * P->H, cudaMemcpyDeviceToDevice, s));
        P->last_stream = s;
    }
    return EECMG_OK;
}

eecmg_status batch_graph_nodes(const eecmg_plan_t* plans, int n, int* nodes) {
    std::vector<eecmg_plan_s*> key(plans, plans + n);
    std::lock_guard<std::mutex> lock(g_batch_mu);
    auto it = g_batches.find(key);
    if (it == g_batches.end() || !it->second->gexec)
        return set_error(EECMG_ERR_INVALID_ARG, "eecmg_batch_info: no batched restoration of these plans yet");
    *nodes = (int)it->second->graph_nodes;
    return EECMG_OK;
}

eecmg_status batch_time_step(const eecmg_plan_t* plans, int n, int step, int enable) {
    std::vector<eecmg_plan_s*> key(plans, plans + n);
    std::lock_guard<std::mutex> lock(g_batch_mu);
    auto it = g_batches.find(key);
    if (it == g_batches.end())
        return set_error(EECMG_ERR_INVALID_ARG,
                         "eecmg_batch_time_step: no batched restoration of these plans yet");
    BatchCtx& C = *it->second;
    if (enable && (step < 0 || step >= (int)C.steps.size()))
        return set_error(EECMG_ERR_INVALID_ARG, "eecmg_batch_time_step: step out of range");
    const int want = enable ? step : -1;
    if (want == C.timed_step) return EECMG_OK;
    for (int i = 0; i < 2 && enable; ++i)
        if (!C.tev[i]) BCK(cudaEventCreate(&C.tev[i]));
    // the graph is captured again, with or without the event nodes, at the next replay
    if (C.gexec) {
        BCK(cudaDeviceSynchronize());
        cudaGraphExecDestroy(C.gexec);
        C.gexec = nullptr;
    }
    C.timed_step = want;
    return EECMG_OK;
}

eecmg_status batch_step_time(const eecmg_plan_t* plans, int n, float* ms, int* launches,
                             double* bytes) {
    std::vector<eecmg_plan_s*> key(plans, plans + n);
    std::lock_guard<std::mutex> lock(g_batch_mu);
    auto it = g_batches.find(key);
    if (it == g_batches.end() || it->second->timed_step < 0 || !it->second->gexec)
        return set_error(EECMG_ERR_INVALID_ARG,
                         "eecmg_batch_step_time: no timed replay (eecmg_batch_time_step, then "
                         "eecmg_restore_batched)");
    BatchCtx& C = *it->second;
    const int st = C.timed_step;
    BCK(cudaEventSynchronize(C.tev[1]));
    float t = 0.f;
    BCK(cudaEventElapsedTime(&t, C.tev[0], C.tev[1]));
    if (ms) *ms = t;
    if (launches) *launches = (int)C.steps[st].size();
    if (bytes) {
        double b = 0.0;
        for (eecmg_plan_s* P : C.plans) {
            if (st >= P->L) continue;
            Scalars sc;
            BCK(cudaMemcpy(&sc, P->sc + st, sizeof(Scalars), cudaMemcpyDeviceToHost));
            const int nzero = P->opt.prolong == EECMG_PROLONG_EECMG ? 2 : 1;
            b += level_solve_bytes(P, st, sc, st < nzero);
        }
        *bytes = b;
    }
    return EECMG_OK;
}

// A destroyed plan invalidates every cached batch that contains it.
void forget_plan_batches(eecmg_plan_s* P) {
    std::lock_guard<std::mutex> lock(g_batch_mu);
    for (auto it = g_batches.begin(); it != g_batches.end();) {
        if (std::find(it->first.begin(), it->first.end(), P) != it->first.end()) {
            auto l = std::find(g_batch_lru.begin(), g_batch_lru.end(), it->first);
            if (l != g_batch_lru.end()) g_batch_lru.erase(l);
            it = g_batches.erase(it);
        } else {
            ++it;
        }
    }
}

}  // namespace eecmg
