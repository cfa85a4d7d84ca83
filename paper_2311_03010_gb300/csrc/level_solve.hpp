// level_solve.hpp -- persistent level solve (one cooperative launch per level).
#pragma once

#include "persistent.cuh"

namespace eecmg {

// One level solve.  MR-II uses v[2], aw[2], d[2], hd[2], r; CGLS uses
// v[0] = s, v[1] = p, aw[0] = q, r.  The job's GroupSync must be zero at
// the first launch (every launch leaves it zero again); partials holds
// 2 x NPART doubles per block.
struct LevelJob {
    const float* g = nullptr;
    float* u = nullptr;
    float* v[2] = {};
    float* aw[2] = {};
    float* d[2] = {};
    float* hd[2] = {};
    float* r = nullptr;
    const Taps* taps = nullptr;
    const Taps* tapsT = nullptr;
    Scalars* sc = nullptr;
    double* partials = nullptr;
    GroupSync* gs = nullptr;
    double conv_tol2 = 0.0, disc2 = 0.0;
    int early = 1;  // MR-II early stop check: 0 off, 1 near the limit, 2 before every step
    int h = 0, w = 0, m = 0, zero_start = 0;
    int block0 = 0, nblocks = 0;  // this job's blocks within a batched launch
    // The start of the level, run by the solve as its first phase (Algorithm 2,
    // Step 2): start = 1 writes u = D(S(P(Pi(s_u1, s_u2)))) (one Perona-Malik
    // step) before r_0 is formed; 0 leaves u as given.  With zero_start the r_0
    // phase also writes the zero start into u.
    int start = 0;
    const float* s_u1 = nullptr;  // level-1 solution, s_h1 x s_w1
    const float* s_u2 = nullptr;  // level-2 solution, s_h2 x s_w2
    int s_h1 = 0, s_w1 = 0, s_h2 = 0, s_w2 = 0;
    float s_scale = 1.f, s_tau = 0.f, s_ik2 = 0.f;  // S weight scale, D step and 1 / k^2
};

// Kernel parameter: one job by value, or (jobs != nullptr) a device table of
// njobs jobs, block b serving job block_job[b].  cluster > 0: every job runs
// on one thread-block cluster of that many blocks (cluster mode); 0: the
// jobs' blocks form one cooperative grid.
struct LevelLaunch {
    LevelJob job;
    const LevelJob* jobs = nullptr;
    const unsigned short* block_job = nullptr;
    int njobs = 1;
    int cluster = 0;
    int resident = 0;  // > 0: shared-memory resident MR-II, this many tiles per block
};

enum LevelOp {
    LS_COOP = 0,
    LS_CLUSTER = 1,
    LS_CAPACITY = 2,
    LS_CLUSTER_MAX = 3,
    LS_RESIDENT = 4,      // cluster launch of the resident solver (L.cluster, L.resident)
    LS_RESIDENT_MAX = 5,  // largest cluster of the resident solver with L.resident tiles per block
};

// How a level solve of h x w pixels is partitioned: one cluster of `cluster`
// blocks (small levels; resident > 0: the shared-memory resident MR-II with
// that many tiles per block), or a cooperative grid of `blocks` blocks.
// Depends only on the level size, the kernel radius rt, the solver, the
// storage type and the device, so a solve of a plan is partitioned (and its
// sums rounded) the same way alone, batched or served.
struct LevelShape {
    int cluster = 0;
    int blocks = 0;
    int resident = 0;
};
LevelShape level_shape(int h, int w, int rt, int cgls, int bf16);

// Partition parameters of the level solves (process-wide).
struct Tuning {
    int px_per_block = 2048;           // grid mode: at least one block per this many pixels (>= 1024)
    long long cluster_max_px = 16384;  // levels with at most this many pixels run in cluster mode
    int blocks_per_sm = 2;             // grid mode: at most this many blocks per SM (1..3)
    int resident_max_tiles = 32;       // FP32 levels of at most this many 32 x 64 tiles
                                       // run shared-memory resident (0 = never, <= 32)
    int psd_tile_h = 32;               // rows of the fused level start's 64-column tiles (16, 32)
};
Tuning get_tuning();
void set_tuning_raw(const Tuning& t);  // no liveness check (see eecmg_set_tuning)
bool tuning_valid(const Tuning& t);

// Launches a device job table: one cooperative grid of total_blocks blocks
// (cluster == 0; the caller sized the jobs' block ranges to fit
// co-residency, see level_capacity), or clusters of `cluster` blocks, one per
// job (resident > 0: the resident MR-II solver, that many tiles per block).
// All jobs share the kernel radius rt (>= each job's own), separability,
// precision, solver and storage.
cudaError_t launch_level_batch(const LevelJob* d_jobs, const unsigned short* d_block_job, int njobs,
                               int total_blocks, int rt, int sep, int prec, int cgls, int bf16,
                               int cluster, int resident, cudaStream_t s);
// Co-resident block capacity of the solver instantiation (0 on error).
int level_capacity(int rt, int sep, int prec, int cgls, int bf16);

// Blocks a level solve of h x w pixels can use.
int level_want_blocks(int h, int w);

// Launches the persistent solver with as many co-resident blocks as useful
// (capped by occupancy); *blocks_used receives the grid size.
// bf16: the streamed Krylov direction vectors are stored as BF16.
cudaError_t launch_level_solve(const LevelJob& J, int rt, int sep, int prec, int cgls, int bf16,
                               cudaStream_t s, int* blocks_used);

}  // namespace eecmg
