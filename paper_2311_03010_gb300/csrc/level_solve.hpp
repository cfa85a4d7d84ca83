// level_solve.hpp -- persistent level solve (one cooperative launch per level).
#pragma once

#include "persistent.cuh"

namespace eecmg {

// One level solve.  MR-II uses v[2], aw[2], d[2], hd[2], r; CGLS uses
// v[0] = s, v[1] = p, aw[0] = q, r.  The group's GroupSync must be zero at
// the first launch (every barrier leaves it zero again).
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
    int h = 0, w = 0, m = 0, zero_start = 0;
};

// Launches the persistent solver with as many co-resident blocks as useful
// (capped by occupancy); *blocks_used receives the grid size.
cudaError_t launch_level_solve(const LevelJob& J, int rt, int sep, int prec, int cgls,
                               cudaStream_t s, int* blocks_used);

}  // namespace eecmg
