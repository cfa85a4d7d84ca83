// batch.hpp -- grouping of many level solves into persistent cooperative
// launches (shared by the batched restoration and the server).
#pragma once

#include <utility>
#include <vector>

#include "launch.hpp"
#include "level_solve.hpp"
#include "plan.hpp"

namespace eecmg {

// One cooperative launch: a table of jobs, block b of the grid serving job
// block_job[b].  All jobs share the kernel instantiation (solver,
// separability, precision, storage) and the radius rt (the largest of them).
struct HostWave {
    std::vector<LevelJob> jobs;
    std::vector<unsigned short> block_job;
    int blocks = 0, rt = 0, sep = 0, prec = 0, cgls = 0, bf16 = 0;
    int cluster = 0;  // > 0: one cluster of this many blocks per job
    int resident = 0; // > 0: the resident MR-II solver, this many tiles per block
};

// The level-l solve of plan P as a job (buffers from P's workspace).
LevelJob make_job(eecmg_plan_s* P, int l);

// Groups the level solves items[i] = (plan, level) into waves.  Every job
// gets the partition of the same solve launched alone (level_shape), so each
// result is bitwise that of the plan's own restoration.  Cluster-mode jobs of
// one instantiation share one launch; cooperative jobs that do not fit the
// co-resident capacity of their instantiation start a new wave.  Groups come
// out in a fixed order (by cluster size and instantiation, then item order).
eecmg_status plan_waves(const std::vector<std::pair<eecmg_plan_s*, int>>& items,
                        std::vector<HostWave>& waves);

// Per-level operations of many images, one launch per group (a group holds
// one kind of operation, k_ops_batch).
struct OpGroup {
    int op = -1;
    std::vector<OpItem> items;
};

// Appends an operation to group gi.
void add_op(std::vector<OpGroup>& groups, size_t gi, int op, OpItem it);

// Restriction of the data pyramids of `plans` (each finest g in place):
// groups appended in execution order, one per depth.
void restrict_ops(const std::vector<eecmg_plan_s*>& plans, std::vector<OpGroup>& groups);

// The start of cascade step items[i] = (plan, level) before its level solve:
// the zero start (Algorithm 2's first levels) or the prolongation chain of
// prolong_enqueue (the fused D(S(P(Pi))) pass and any further D steps; or Pi
// or not, P or L, S, the D steps), with the same buffers and per-pixel code.
// Groups appended in execution order.
void step_ops(const std::vector<std::pair<eecmg_plan_s*, int>>& items, std::vector<OpGroup>& groups);

// Sets each item's block0 within its group; returns the group's blocks.
int place_items(OpGroup& g);

}  // namespace eecmg
