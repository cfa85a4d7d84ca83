// plan.hpp -- the plan object behind eecmg_plan_t (internal).
#pragma once

#include <string>
#include <vector>

#include "common.cuh"
#include "level_solve.hpp"
#include "persistent.cuh"

namespace eecmg {

struct LevelPlan {
    int h = 0, w = 0;   // rows, cols
    int m = 0;          // scheduled iterations
    int rt = 0;         // kernel template radius
    int sepH = 0, sepHT = 0;
    double disc2 = 0.0; // (c delta)^2 N_l, discrepancy rule
    float* g = nullptr; // data pyramid (workspace)
    float* u = nullptr; // level solution (workspace)
};

// Kernel classes of the optional per-launch profiler.
enum KernelClass : int {
    KC_CONV = 0, KC_MR_B, KC_MR_FINAL, KC_CG_STEP, KC_CG_P, KC_RESTRICT, KC_PROLONG,
    KC_SMOOTH, KC_DENOISE, KC_COPY, KC_LEVEL, KC_COUNT
};

// Eager-mode profiler: an event pair around every launch of a restoration,
// with the launch's algorithmic bytes (reads + writes the operator must do).
struct Profiler {
    bool on = false;
    struct Rec {
        int cls;
        double bytes;
        cudaEvent_t e0, e1;
        int level = -1;   // persistent level solve: bytes counted from the iterations run
    };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> free_events;
    double ms[KC_COUNT] = {};
    double bytes[KC_COUNT] = {};
    long long launches[KC_COUNT] = {};
};

eecmg_status set_error(eecmg_status st, const std::string& msg);
int schedule_m(int L, int l);

}  // namespace eecmg

// Byte offsets of a plan's workspace regions (the layout is fixed by the
// plan's description; a workspace can be bound anywhere 256-byte aligned).
struct PlanLayout {
    std::vector<size_t> g_off, u_off;  // per level
    size_t vec_off[9] = {};
    size_t taps_off = 0, sc_off = 0, gs_off = 0, part_off = 0;
    size_t bytes = 0;                  // total
};

struct eecmg_plan_s {
    int W = 0, H = 0, L = 0;
    double tau = 0.2, kpm = 10.0;
    double conv_tol2 = 0.0;
    eecmg_options opt{};
    int device = 0;
    std::vector<eecmg::LevelPlan> lv;
    std::vector<eecmg::Taps> htaps;     // host copy of the level taps
    PlanLayout layout;
    bool owns_ws = false;
    char* ws = nullptr;
    size_t ws_bytes = 0;
    size_t max_blocks = 0;
    eecmg::Taps* dtaps = nullptr;     // [2l] = H_l, [2l+1] = H_l^T
    eecmg::Scalars* sc = nullptr;     // one per level
    eecmg::GroupSync* gsync = nullptr; // one per level (persistent solves)
    double* partials = nullptr;
    static constexpr int NVEC = 9;
    float* vec[NVEC] = {};              // solver vectors, each max level size
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t last_stream = nullptr;
    eecmg::Profiler prof;
};

#include <atomic>

namespace eecmg {
// Points the plan's level and solver buffers into ws (P->layout.bytes long).
void bind_workspace(eecmg_plan_s* P, char* ws);
// Plans owning a workspace plus live servers: the partition parameters may
// change only while this is zero.
extern std::atomic<int> g_live_owners;
eecmg_status plan_allocate(eecmg_plan_s* P, const char* who);
eecmg_status plan_materialize(const eecmg_plan_s* D, eecmg_plan_s** out);
eecmg_status solve_level_enqueue(eecmg_plan_s* P, int l, const float* g, float* u, int m,
                                 bool zero_start, cudaStream_t s, bool own_start = false);
// Whether the persistent solve of level l starts the level itself (Algorithm 2,
// Step 2: the fused D(S(P(Pi))) of a plan with fuse_start and one Perona-Malik
// step, l >= 2); the two coarsest levels write their zero start themselves in
// any case.
bool level_fused_start(const eecmg_plan_s* P, int l);
// Fills the start fields of level l's job (zero start or fused start).
void set_level_start(const eecmg_plan_s* P, int l, LevelJob& J);
eecmg_status prolong_enqueue(eecmg_plan_s* P, int l, cudaStream_t s);
eecmg_status cascade_enqueue(eecmg_plan_s* P, cudaStream_t s);
eecmg_status run_cascade(eecmg_plan_s* P, cudaStream_t s);
eecmg_status restore_batched_impl(const eecmg_plan_t* plans, const float* const* g, float* const* u,
                                  int n, cudaStream_t s);
void forget_plan_batches(eecmg_plan_s* P);
eecmg_status batch_graph_nodes(const eecmg_plan_t* plans, int n, int* nodes);
eecmg_status batch_time_step(const eecmg_plan_t* plans, int n, int step, int enable);
eecmg_status batch_step_time(const eecmg_plan_t* plans, int n, float* ms, int* launches,
                             double* bytes);
// Algorithmic bytes of a persistent level solve from the iterations it ran.
double level_solve_bytes(const eecmg_plan_s* P, int l, const Scalars& sc, bool zero_start);
}  // namespace eecmg
