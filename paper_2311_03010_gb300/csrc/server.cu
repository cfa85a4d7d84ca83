// server.cu -- continuous-batching restoration server (C ABI).
//
// Requests are admitted first come, first served while their workspace fits
// in the server's device arena (one allocation of mem_budget_bytes made at
// creation, carved first-fit) and at most max_slots are active.  An admitted
// request gets its plan's workspace layout inside the arena: data and
// solution pyramids, solver vectors, taps, scalars and barrier state stay
// resident on the device until it completes.
//
// A scheduler thread advances every active request together.  One tick runs
// at least one cascade step (Algorithm 2) of each active request: for a
// request just admitted, the copy of its data and the restriction of the data
// pyramid; then per request the start of its current level (the prolongation
// chain, or the zero start); then the level solves of all of them as jobs of
// persistent cooperative launches (one per kernel instantiation, see
// batch.hpp).  Requests whose next level is small go on to it in further
// rounds of the same tick (at most MAX_ROUNDS steps per tick).
// Requests admitted at different times therefore share launches while they
// sit at different levels.  Each job keeps the block count of the same solve
// launched alone, so a served result is bitwise the result of eecmg_restore
// on the request's plan.  Two ticks may be in flight; a request completes
// with the tick that ran its finest level, and its latency runs from
// submission to the end of its result's copy (right after the round of the
// tick that ran that level) on the device clock.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "batch.hpp"
#include "launch.hpp"

using namespace eecmg;

namespace {

using Clock = std::chrono::steady_clock;

constexpr int RING = 2;              // ticks in flight
// An idle scheduler spins this long on the submission counter before it sleeps,
// so that a request arriving meanwhile starts without the thread's wake-up
// latency (one host core stays busy while requests keep arriving).
constexpr auto IDLE_SPIN = std::chrono::milliseconds(10);
constexpr size_t QUEUE_CAP = 65536;  // queued (not yet admitted) requests
constexpr int MAX_LEVELS = 30;
constexpr int MAX_DIFFUSION = 16;    // Perona-Malik steps per level of a served request
// A tick runs up to MAX_ROUNDS rounds: round 0 advances every active request by
// one cascade step; a request takes part in the next round while its next
// level has at most SMALL_LEVEL_PX pixels.  The coarse steps of a request are
// short on the GPU (a level is a quarter of the next) and a tick's host work
// is not: with one step per tick the GPU idled between the ticks of a lone
// request (GB300: +38 us on a 256^2 request, +176 us on a 4096^2 one against
// the plain loop).  Levels above 1024^2 still get a tick each, so requests
// admitted meanwhile join at the next tick.
constexpr int MAX_ROUNDS = 5;
constexpr long long SMALL_LEVEL_PX = 1LL << 20;

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

// Upper bound of one tick's job tables and operation items (enqueue_tick), so
// that the tick ring is allocated once, at creation.  Every active request
// adds at most MAX_LEVELS + 1 admission items (the copy of its data, the
// restriction to each coarser level, the reset of its scalars), per round at
// most 3 + MAX_DIFFUSION items (the start of its cascade step: zero start, or
// the fused prolongation chain or prolongation, smoothing and the diffusion
// steps) and one level-solve job of at most max(16, 3 x SMs) blocks, and one
// item for the copy of its result; there are at most 4 + MAX_ROUNDS x (8 +
// MAX_DIFFUSION) operation groups (a round's result copies are a group of their
// own) and one wave per job, each table rounded up to 256 bytes.
size_t tick_table_bound(int max_slots, int nsm) {
    const size_t slots = (size_t)max_slots;
    const size_t items = slots * (MAX_LEVELS + 2 + (size_t)MAX_ROUNDS * (3 + MAX_DIFFUSION));
    const size_t groups = 4 + (size_t)MAX_ROUNDS * (8 + MAX_DIFFUSION);
    const size_t jobs = slots * MAX_ROUNDS;
    const size_t job_blocks = std::max<size_t>(16, 3 * (size_t)nsm);
    return items * sizeof(OpItem) + 256 * groups + jobs * (sizeof(LevelJob) + 256) +
           jobs * (sizeof(unsigned short) * job_blocks + 256);
}

// First-fit allocator over [0, cap): free ranges by offset, coalesced on
// release.
class Arena {
public:
    void reset(size_t cap) {
        free_.clear();
        if (cap) free_[0] = cap;
        used_ = 0;
    }
    bool alloc(size_t bytes, size_t* off) {
        bytes = round256(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            *off = it->first;
            const size_t rest = it->second - bytes, start = it->first + bytes;
            free_.erase(it);
            if (rest) free_[start] = rest;
            used_ += bytes;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = round256(bytes);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
private:
    std::map<size_t, size_t> free_;
    size_t used_ = 0;
};

struct Request {
    uint64_t ticket = 0;
    const eecmg_plan_s* tmpl = nullptr;
    const float* g = nullptr;
    float* u = nullptr;
    Clock::time_point t_submit;
    eecmg_plan_s slot;  // the request's resident state (workspace in the arena)
    size_t off = 0, bytes = 0;
    int sidx = -1;      // status area
    int step = 0;       // next cascade step
    int fin_round = 0;  // the round of its last tick that ran its finest level
    bool direct = false;  // the finest level works in the caller's g and u (no copies)
};

struct Result {
    int done = 0;
    eecmg_status st = EECMG_OK;
    double latency_ms = 0.0;
};

}  // namespace

struct eecmg_server_s {
    int device = 0, nsm = 0, max_slots = 0;
    size_t budget = 0;
    char* arena_mem = nullptr;
    Arena arena;
    cudaStream_t stream = nullptr;
    // job tables of the ticks in flight
    size_t ring_bytes = 0;
    char* d_ring = nullptr;  // RING x ring_bytes, device
    char* h_ring = nullptr;  // RING x ring_bytes, pinned host
    cudaEvent_t ev[RING] = {};
    cudaEvent_t rev[RING][MAX_ROUNDS] = {};  // end of each round's finishing requests' copies
    bool busy[RING] = {};
    std::vector<Request*> fin[RING];
    // per-slot status areas (pinned): every level's Scalars, then GroupSync
    char* h_stat = nullptr;
    size_t stat_stride = 0;
    std::vector<int> free_sidx;
    cudaEvent_t base_ev = nullptr;
    Clock::time_point base_host;
    // shared state (mu)
    std::mutex mu;
    std::condition_variable cv, cv_done;
    std::deque<Request*> queue;
    std::vector<Request*> active;
    std::unordered_map<uint64_t, Result> results;
    uint64_t next_ticket = 1;
    size_t outstanding = 0;
    bool stop = false;
    std::atomic<uint64_t> submitted{0};  // requests queued so far (read while spinning)
    std::atomic<bool> stopping{false};
    eecmg_status fatal = EECMG_OK;
    std::string fatal_msg;
    std::thread th;
    uint64_t tick = 0;  // scheduler thread only
};

namespace {

#define SCK(call)                                                                          \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return set_error(EECMG_ERR_CUDA, std::string("eecmg_server: ") + #call + ": " + \
                                                 cudaGetErrorString(e_));                  \
    } while (0)

// Gives the request its plan's layout at ws (host-side only).
void bind_slot(Request* r, char* ws) {
    eecmg_plan_s& S = r->slot;
    const eecmg_plan_s& T = *r->tmpl;
    S.W = T.W;
    S.H = T.H;
    S.L = T.L;
    S.tau = T.tau;
    S.kpm = T.kpm;
    S.conv_tol2 = T.conv_tol2;
    S.opt = T.opt;
    S.device = T.device;
    S.lv = T.lv;
    S.layout = T.layout;
    S.ws_bytes = T.ws_bytes;
    S.max_blocks = T.max_blocks;
    S.owns_ws = false;
    bind_workspace(&S, ws);
    // The finest level reads the caller's data and writes the caller's result in place (both
    // stay valid until the request completes; the solver never writes g): no copy in, no
    // copy out.  Overlapping buffers keep the workspace's own level and the two copies.
    const uintptr_t g0 = reinterpret_cast<uintptr_t>(r->g), u0 = reinterpret_cast<uintptr_t>(r->u);
    const uintptr_t nb = sizeof(float) * (uintptr_t)S.W * (uintptr_t)S.H;
    r->direct = g0 + nb <= u0 || u0 + nb <= g0;
    if (r->direct) {
        S.lv[S.L - 1].g = const_cast<float*>(r->g);
        S.lv[S.L - 1].u = r->u;
    }
}

char* stat_area(eecmg_server_s* S, int sidx) { return S->h_stat + (size_t)sidx * S->stat_stride; }

// Enqueues tick k's work on the server stream: the admissions, then up to
// MAX_ROUNDS rounds of cascade steps, each round one batched launch per kind
// of per-level operation (k_ops_batch) followed by the level solves of that
// round as the persistent launches of plan_waves.  `finishing` receives the
// requests whose finest level ran in it; every other active request's step
// advances by the rounds it took part in (when the tick is committed).
eecmg_status enqueue_tick(eecmg_server_s* S, const std::vector<Request*>& admitted, int k,
                          std::vector<Request*>& finishing, std::vector<int>& advance) {
    cudaStream_t s = S->stream;
    std::vector<OpGroup> pre;  // launch groups before the rounds
    // per round, the result copies of the requests whose finest level ran in it: they are
    // launched right after that round, so a request's result does not wait for the rounds
    // the tick runs after it for other requests' small levels
    std::vector<std::vector<OpGroup>> rpost;
    // admissions: the data copied in, its pyramid restricted, scalars zeroed
    std::vector<eecmg_plan_s*> adm;
    for (Request* r : admitted) {
        eecmg_plan_s& P = r->slot;
        SCK(cudaMemcpyAsync(P.dtaps, r->tmpl->htaps.data(), sizeof(Taps) * 2 * P.L,
                            cudaMemcpyHostToDevice, s));
        LevelPlan& F = P.lv[P.L - 1];
        if (!r->direct) {
            OpItem in;
            in.a = r->g;
            in.out = F.g;
            in.h = F.h;
            in.w = F.w;
            add_op(pre, 0, OP_COPY, in);
        }
        adm.push_back(&P);
    }
    restrict_ops(adm, pre);
    const size_t gz = pre.size();
    for (eecmg_plan_s* P : adm) {  // scalars, barrier state and partials, as in a new plan
        const PlanLayout& Y = P->layout;
        OpItem z;
        z.out = (float*)(P->ws + Y.sc_off);
        z.h = 1;
        z.w = (int)((Y.bytes - Y.sc_off) / sizeof(float));
        add_op(pre, gz, OP_ZERO, z);
    }
    // the rounds: every active request in round 0, then those whose next level is small
    std::vector<std::vector<OpGroup>> rops;
    std::vector<std::vector<HostWave>> rwaves;
    advance.assign(S->active.size(), 0);
    std::vector<int> cur(S->active.size());
    for (size_t i = 0; i < cur.size(); ++i) cur[(size_t)i] = (int)i;
    for (int round = 0; round < MAX_ROUNDS && !cur.empty(); ++round) {
        std::vector<std::pair<eecmg_plan_s*, int>> items;
        items.reserve(cur.size());
        for (int i : cur) items.push_back({&S->active[i]->slot, S->active[i]->step + round});
        rops.emplace_back();
        rpost.emplace_back();
        step_ops(items, rops.back());
        rwaves.emplace_back();
        eecmg_status e = plan_waves(items, rwaves.back());
        if (e != EECMG_OK) return e;
        std::vector<int> next;
        for (int i : cur) {
            Request* r = S->active[i];
            eecmg_plan_s& P = r->slot;
            const int st = r->step + round;
            advance[i] += 1;
            if (st == P.L - 1) {
                if (!r->direct) {
                    LevelPlan& F = P.lv[P.L - 1];
                    OpItem c;
                    c.a = F.u;
                    c.out = r->u;
                    c.h = F.h;
                    c.w = F.w;
                    add_op(rpost.back(), 0, OP_COPY, c);
                }
                r->fin_round = round;
                finishing.push_back(r);
            } else if ((long long)P.lv[st + 1].h * P.lv[st + 1].w <= SMALL_LEVEL_PX) {
                next.push_back(i);
            }
        }
        cur.swap(next);
    }
    // pack job tables and op items into the tick's ring slot: one upload
    size_t need = 0;
    auto groups_need = [&](const std::vector<OpGroup>& gs) {
        for (auto& g : gs) need += round256(sizeof(OpItem) * g.items.size());
    };
    groups_need(pre);
    for (auto& rp : rpost) groups_need(rp);
    for (auto& ro : rops) groups_need(ro);
    for (auto& ws : rwaves)
        for (auto& w : ws)
            need += round256(sizeof(LevelJob) * w.jobs.size()) +
                    round256(sizeof(unsigned short) * w.block_job.size());
    if (need > S->ring_bytes)
        return set_error(EECMG_ERR_INVALID_ARG, "eecmg_server: tick tables exceed the ring slot");
    char* h = S->h_ring + (size_t)k * S->ring_bytes;
    char* d = S->d_ring + (size_t)k * S->ring_bytes;
    size_t off = 0;
    auto put = [&](const void* src, size_t bytes, size_t* at) -> bool {
        if (off + round256(bytes) > S->ring_bytes) return false;
        *at = off;
        if (bytes) std::memcpy(h + off, src, bytes);
        off += round256(bytes);
        return true;
    };
    struct Placed {
        int op;
        size_t at;
        int n, blocks;
    };
    auto place_groups = [&](std::vector<OpGroup>& groups, std::vector<Placed>& out) -> bool {
        for (auto& g : groups) {
            if (g.items.empty() || g.op < 0) continue;
            const int blocks = place_items(g);
            size_t at = 0;
            if (!put(g.items.data(), sizeof(OpItem) * g.items.size(), &at)) return false;
            out.push_back(Placed{g.op, at, (int)g.items.size(), blocks});
        }
        return true;
    };
    std::vector<Placed> pre_l;
    std::vector<std::vector<Placed>> rpost_l(rpost.size());
    std::vector<std::vector<Placed>> rops_l(rops.size());
    std::vector<std::vector<size_t>> jo(rwaves.size()), bo(rwaves.size());
    bool fits = place_groups(pre, pre_l);
    for (size_t r = 0; r < rpost.size() && fits; ++r) fits = place_groups(rpost[r], rpost_l[r]);
    for (size_t r = 0; r < rops.size() && fits; ++r) fits = place_groups(rops[r], rops_l[r]);
    for (size_t r = 0; r < rwaves.size() && fits; ++r) {
        const auto& waves = rwaves[r];
        jo[r].resize(waves.size());
        bo[r].resize(waves.size());
        for (size_t w = 0; w < waves.size() && fits; ++w)
            fits = put(waves[w].jobs.data(), sizeof(LevelJob) * waves[w].jobs.size(), &jo[r][w]) &&
                   put(waves[w].block_job.data(), sizeof(unsigned short) * waves[w].block_job.size(),
                       &bo[r][w]);
    }
    if (!fits) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_server: tick tables exceed the ring slot");
    if (off) SCK(cudaMemcpyAsync(d, h, off, cudaMemcpyHostToDevice, s));
    for (const Placed& p : pre_l)
        SCK(launch_ops_batch(p.op, (const OpItem*)(d + p.at), p.n, p.blocks, s));
    for (size_t r = 0; r < rops.size(); ++r) {
        for (const Placed& p : rops_l[r])
            SCK(launch_ops_batch(p.op, (const OpItem*)(d + p.at), p.n, p.blocks, s));
        const auto& waves = rwaves[r];
        for (size_t w = 0; w < waves.size(); ++w) {
            const HostWave& W = waves[w];
            SCK(launch_level_batch((const LevelJob*)(d + jo[r][w]), (const unsigned short*)(d + bo[r][w]),
                                   (int)W.jobs.size(), W.blocks, W.rt, W.sep, W.prec, W.cgls, W.bf16,
                                   W.cluster, W.resident, s));
        }
        bool any = false;
        for (const Placed& p : rpost_l[r])
            SCK(launch_ops_batch(p.op, (const OpItem*)(d + p.at), p.n, p.blocks, s));
        for (Request* q : finishing) {
            if (q->fin_round != (int)r) continue;
            any = true;
            eecmg_plan_s& P = q->slot;
            char* a = stat_area(S, q->sidx);
            SCK(cudaMemcpyAsync(a, P.sc, sizeof(Scalars) * P.L, cudaMemcpyDeviceToHost, s));
            SCK(cudaMemcpyAsync(a + sizeof(Scalars) * MAX_LEVELS, P.gsync, sizeof(GroupSync) * P.L,
                                cudaMemcpyDeviceToHost, s));
        }
        if (any) SCK(cudaEventRecord(S->rev[k][r], s));
    }
    SCK(cudaEventRecord(S->ev[k], s));
    return EECMG_OK;
}

// The request's status from its copied scalars and barrier state.
eecmg_status request_status(eecmg_server_s* S, const Request* r) {
    const char* a = stat_area(S, r->sidx);
    const Scalars* sc = (const Scalars*)a;
    const GroupSync* gs = (const GroupSync*)(a + sizeof(Scalars) * MAX_LEVELS);
    for (int l = 0; l < r->slot.L; ++l)
        if (gs[l].err) return EECMG_ERR_TIMEOUT;
    for (int l = 0; l < r->slot.L; ++l)
        if (sc[l].stopped == 3) return EECMG_ERR_NUMERIC;
    return EECMG_OK;
}

// Waits for tick slot k and completes the requests that finished in it.
void complete(eecmg_server_s* S, int k) {
    const cudaError_t e = cudaEventSynchronize(S->ev[k]);
    // a request's result is ready at the end of its round's copies
    auto done_at = [&](const Request* r, cudaError_t* err) {
        float ms = 0.f;
        *err = cudaEventElapsedTime(&ms, S->base_ev, S->rev[k][r->fin_round]);
        return S->base_host +
               std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double, std::milli>(ms));
    };
    {
        std::lock_guard<std::mutex> lk(S->mu);
        for (Request* r : S->fin[k]) {
            cudaError_t er = e;
            Clock::time_point t_done = S->base_host;
            if (er == cudaSuccess) t_done = done_at(r, &er);
            Result& res = S->results[r->ticket];
            res.done = 1;
            res.st = er == cudaSuccess ? request_status(S, r) : EECMG_ERR_CUDA;
            res.latency_ms = std::chrono::duration<double, std::milli>(t_done - r->t_submit).count();
            S->arena.release(r->off, r->bytes);
            S->free_sidx.push_back(r->sidx);
            --S->outstanding;
            delete r;
        }
    }
    S->fin[k].clear();
    S->busy[k] = false;
    S->cv_done.notify_all();
}

bool any_busy(const eecmg_server_s* S) {
    for (int k = 0; k < RING; ++k)
        if (S->busy[k]) return true;
    return false;
}

void complete_oldest(eecmg_server_s* S) {
    for (int i = 0; i < RING; ++i) {
        const int k = (int)((S->tick + i) % RING);
        if (S->busy[k]) {
            complete(S, k);
            return;
        }
    }
}

// A CUDA error on the server stream: every request in the server fails.
void fail_all(eecmg_server_s* S, eecmg_status st) {
    cudaStreamSynchronize(S->stream);
    std::lock_guard<std::mutex> lk(S->mu);
    S->fatal = st;
    S->fatal_msg = eecmg_last_error();
    auto fail = [&](Request* r) {
        Result& res = S->results[r->ticket];
        res.done = 1;
        res.st = st;
        if (r->sidx >= 0) {
            S->arena.release(r->off, r->bytes);
            S->free_sidx.push_back(r->sidx);
        }
        --S->outstanding;
        delete r;
    };
    for (int k = 0; k < RING; ++k) {
        for (Request* r : S->fin[k]) fail(r);
        S->fin[k].clear();
        S->busy[k] = false;
    }
    for (Request* r : S->active) fail(r);
    S->active.clear();
    for (Request* r : S->queue) fail(r);
    S->queue.clear();
    S->cv_done.notify_all();
}

void scheduler(eecmg_server_s* S) {
    cudaSetDevice(S->device);
    for (;;) {
        std::vector<Request*> admitted;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            auto ready = [&] { return S->stop || !S->queue.empty() || !S->active.empty() || any_busy(S); };
            if (!ready()) {
                const uint64_t seen = S->submitted.load(std::memory_order_relaxed);
                lk.unlock();
                const auto t0 = Clock::now();
                while (S->submitted.load(std::memory_order_acquire) == seen &&
                       !S->stopping.load(std::memory_order_acquire) && Clock::now() - t0 < IDLE_SPIN)
                    std::this_thread::yield();
                lk.lock();
            }
            S->cv.wait(lk, ready);
            if (S->queue.empty() && S->active.empty() && !any_busy(S)) {
                if (S->stop) break;
                continue;
            }
            // a slot (status area) stays taken until its request's tick completes
            while (!S->queue.empty() && (int)S->active.size() < S->max_slots &&
                   !S->free_sidx.empty()) {
                Request* r = S->queue.front();
                size_t off = 0;
                if (!S->arena.alloc(r->bytes, &off)) break;  // first come, first served
                S->queue.pop_front();
                r->off = off;
                r->sidx = S->free_sidx.back();
                S->free_sidx.pop_back();
                bind_slot(r, S->arena_mem + off);
                S->active.push_back(r);
                admitted.push_back(r);
            }
        }
        if (admitted.empty() && S->active.empty()) {
            // memory is held by requests finishing in flight: wait for them
            complete_oldest(S);
            continue;
        }
        const int k = (int)(S->tick % RING);
        if (S->busy[k]) complete(S, k);
        std::vector<Request*> finishing;
        std::vector<int> advance;
        eecmg_status st = enqueue_tick(S, admitted, k, finishing, advance);
        if (st != EECMG_OK) {
            fail_all(S, st);
            continue;
        }
        S->busy[k] = true;
        S->fin[k] = finishing;
        // advance[i] belongs to S->active[i] as enqueued (only this thread changes active)
        for (size_t i = 0; i < advance.size(); ++i) S->active[i]->step += advance[i];
        {
            std::lock_guard<std::mutex> lk(S->mu);
            auto done = [&](Request* r) {
                return std::find(finishing.begin(), finishing.end(), r) != finishing.end();
            };
            S->active.erase(std::remove_if(S->active.begin(), S->active.end(), done), S->active.end());
        }
        ++S->tick;
    }
}

void free_server(eecmg_server_s* S) {
    if (S->stream) cudaStreamSynchronize(S->stream);
    for (int k = 0; k < RING; ++k)
        if (S->ev[k]) cudaEventDestroy(S->ev[k]);
    for (int k = 0; k < RING; ++k)
        for (int r = 0; r < MAX_ROUNDS; ++r)
            if (S->rev[k][r]) cudaEventDestroy(S->rev[k][r]);
    if (S->base_ev) cudaEventDestroy(S->base_ev);
    if (S->stream) cudaStreamDestroy(S->stream);
    if (S->d_ring) cudaFree(S->d_ring);
    if (S->h_ring) cudaFreeHost(S->h_ring);
    if (S->h_stat) cudaFreeHost(S->h_stat);
    if (S->arena_mem) cudaFree(S->arena_mem);
    delete S;
}

}  // namespace

extern "C" {

eecmg_status eecmg_server_create(size_t mem_budget_bytes, int max_slots, eecmg_server_t* out) {
    if (!out) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_server_create: out is NULL");
    *out = nullptr;
    if (mem_budget_bytes == 0 || max_slots < 1 || max_slots > 4096)
        return set_error(EECMG_ERR_INVALID_ARG,
                         "eecmg_server_create: need mem_budget_bytes > 0 and 1 <= max_slots <= 4096");
    auto* S = new (std::nothrow) eecmg_server_s();
    if (!S) return set_error(EECMG_ERR_OOM, "eecmg_server_create: host allocation failed");
    S->budget = round256(mem_budget_bytes);
    S->max_slots = max_slots;
    auto fail = [&](eecmg_status st, const std::string& msg) {
        cudaGetLastError();
        free_server(S);
        return set_error(st, "eecmg_server_create: " + msg);
    };
    cudaError_t e = cudaGetDevice(&S->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&S->nsm, cudaDevAttrMultiProcessorCount, S->device);
    if (e != cudaSuccess) return fail(EECMG_ERR_CUDA, cudaGetErrorString(e));
    e = cudaMalloc((void**)&S->arena_mem, S->budget);
    if (e != cudaSuccess) {
        S->arena_mem = nullptr;
        return fail(EECMG_ERR_OOM, std::string("arena: ") + cudaGetErrorString(e));
    }
    S->arena.reset(S->budget);
    // sized once for the largest tick admission allows (no allocation while serving)
    S->ring_bytes = round256(tick_table_bound(max_slots, S->nsm));
    S->stat_stride = round256((sizeof(Scalars) + sizeof(GroupSync)) * MAX_LEVELS);
    e = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc((void**)&S->d_ring, RING * S->ring_bytes);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&S->h_ring, RING * S->ring_bytes);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&S->h_stat, S->stat_stride * max_slots);
    for (int k = 0; k < RING && e == cudaSuccess; ++k) e = cudaEventCreate(&S->ev[k]);
    for (int k = 0; k < RING && e == cudaSuccess; ++k)
        for (int r = 0; r < MAX_ROUNDS && e == cudaSuccess; ++r) e = cudaEventCreate(&S->rev[k][r]);
    if (e == cudaSuccess) e = cudaEventCreate(&S->base_ev);
    if (e == cudaSuccess) e = cudaEventRecord(S->base_ev, S->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(S->base_ev);
    if (e != cudaSuccess) return fail(EECMG_ERR_CUDA, cudaGetErrorString(e));
    S->base_host = Clock::now();
    for (int i = max_slots - 1; i >= 0; --i) S->free_sidx.push_back(i);
    try {
        S->th = std::thread(scheduler, S);
    } catch (...) {
        return fail(EECMG_ERR_OOM, "scheduler thread");
    }
    g_live_owners.fetch_add(1);  // the partition parameters stay fixed while it exists
    *out = S;
    return EECMG_OK;
}

eecmg_status eecmg_server_submit(eecmg_server_t S, eecmg_plan_t P, const float* g, float* u,
                                 uint64_t* ticket) {
    if (!S || !P || !g || !u || !ticket)
        return set_error(EECMG_ERR_INVALID_ARG, "eecmg_server_submit: NULL argument");
    *ticket = 0;
    if (P->L > MAX_LEVELS || P->opt.diffusion_steps > MAX_DIFFUSION || !P->opt.persistent ||
        P->device != S->device)
        return set_error(EECMG_ERR_INVALID_ARG,
                         "eecmg_server_submit: the plan must use the persistent level solve, at most "
                         "30 levels and 16 diffusion steps, on the server's device");
    if (round256(P->ws_bytes) > S->budget)
        return set_error(EECMG_ERR_OOM, "eecmg_server_submit: the request alone exceeds the memory budget");
    auto* r = new (std::nothrow) Request();
    if (!r) return set_error(EECMG_ERR_OOM, "eecmg_server_submit: host allocation failed");
    r->tmpl = P;
    r->g = g;
    r->u = u;
    r->bytes = P->ws_bytes;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->fatal != EECMG_OK) {
            delete r;
            return set_error(S->fatal, "eecmg_server_submit: server failed earlier: " + S->fatal_msg);
        }
        if (S->queue.size() >= QUEUE_CAP) {
            delete r;
            return set_error(EECMG_ERR_BUSY, "eecmg_server_submit: queue full");
        }
        r->ticket = S->next_ticket++;
        r->t_submit = Clock::now();
        S->results[r->ticket] = Result();
        S->queue.push_back(r);
        ++S->outstanding;
        *ticket = r->ticket;
        S->submitted.fetch_add(1, std::memory_order_release);
    }
    S->cv.notify_one();
    return EECMG_OK;
}

eecmg_status eecmg_server_poll(eecmg_server_t S, uint64_t ticket, int* done, double* latency_ms) {
    if (!S || !done) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_server_poll: NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->results.find(ticket);
    if (it == S->results.end()) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_server_poll: unknown ticket");
    *done = it->second.done;
    if (latency_ms) *latency_ms = it->second.done ? it->second.latency_ms : 0.0;
    if (it->second.done && it->second.st != EECMG_OK)
        return set_error(it->second.st, "eecmg_server_poll: the request failed");
    return EECMG_OK;
}

eecmg_status eecmg_server_drain(eecmg_server_t S) {
    if (!S) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_server_drain: NULL server");
    std::unique_lock<std::mutex> lk(S->mu);
    S->cv_done.wait(lk, [&] { return S->outstanding == 0; });
    if (S->fatal != EECMG_OK) return set_error(S->fatal, "eecmg_server_drain: " + S->fatal_msg);
    return EECMG_OK;
}

eecmg_status eecmg_server_destroy(eecmg_server_t S) {
    if (!S) return EECMG_OK;
    {
        std::unique_lock<std::mutex> lk(S->mu);
        S->cv_done.wait(lk, [&] { return S->outstanding == 0; });
        S->stop = true;
        S->stopping.store(true, std::memory_order_release);
    }
    S->cv.notify_all();
    if (S->th.joinable()) S->th.join();
    free_server(S);
    g_live_owners.fetch_sub(1);
    return EECMG_OK;
}

}  // extern "C"
