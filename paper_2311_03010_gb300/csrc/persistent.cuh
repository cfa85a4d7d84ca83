// persistent.cuh -- phase barriers with a fused deterministic reduction, for
// the persistent (one launch per level solve) kernels.
//
// Grid mode: all blocks of a job are co-resident (cooperative launch).  At
// the end of a phase every block writes its double-float block sums into its slot of
// the phase's partials (double-buffered by phase parity), then adds one to
// the job's arrival counter with release semantics.  Every block waits until
// the counter reaches (phase + 1) x blocks, then sums all blocks' partials in
// a fixed order and runs the phase's scalar update on its own replica of the
// scalars: all replicas stay identical, so no block has to broadcast.  The
// wait spins on an acquire load with a clock64 limit: a wait that runs out
// sets the job's error flag and every block returns, so a kernel can never
// hang the GPU; the host reports the flag as a timeout.  The counter starts
// at zero; the last block to leave the kernel resets it for the next launch.
#pragma once

#include "common.cuh"

namespace eecmg {


struct alignas(64) GroupSync {
    unsigned int count;   // arrivals in this launch (phases x blocks)
    unsigned int exits;   // blocks that have left this launch
    int err;              // 1 after a wait ran out (sticky)
    int pad[13];
};

// ~2 s at the GB300's maximum SM clock: far beyond any phase of a level solve.
constexpr long long GROUP_WAIT_LIMIT_CYCLES = 4000000000LL;

template <typename T>
__device__ __forceinline__ T ldcg(const T* p) {
    return __ldcg(p);
}

__device__ __forceinline__ void red_release_add(unsigned int* p, unsigned int v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Every thread of every block of the job calls this with its NV FP32 values
// in v (thread-local contributions).  partials holds 2 x nb x NPART
// double-float slots (8 bytes each).  All sums run in double-float on the FP32
// pipes, and finish receives the job totals as double-float pairs.  Returns false if the
// job is in error (the caller returns).
template <int NV, class Finish>
__device__ __forceinline__ bool grid_reduce(const float (&v)[NV], double* partials, GroupSync* gs,
                                            unsigned int nb, unsigned int bid, unsigned int phase,
                                            Finish&& finish,
                                            long long limit = GROUP_WAIT_LIMIT_CYCLES) {
    DF in[NV], out[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) in[j] = DF{v[j], 0.f};
    block_sum_df<NV>(in, out);  // ends with __syncthreads()
    __shared__ int s_ok;
    float2* slot = reinterpret_cast<float2*>(partials) + (size_t)(phase & 1u) * nb * NPART;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) slot[(size_t)bid * NPART + j] = make_float2(out[j].hi, out[j].lo);
        red_release_add(&gs->count, 1u);  // orders this block's phase writes before the arrival
        const unsigned int target = (phase + 1u) * nb;
        int ok = 1;
        const long long t0 = clock64();
        while (ld_acquire(&gs->count) < target) {
            if (*(volatile int*)&gs->err) {
                ok = 0;
                break;
            }
            if (clock64() - t0 > limit) {
                atomicExch(&gs->err, 1);
                ok = 0;
                break;
            }
            __nanosleep(20);
        }
        s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) return false;
    // every block: the blocks' partials in a fixed order, then the update
    if (nb <= 32) {  // one warp: lane b holds block b's partial, a butterfly sums them
        if (threadIdx.x < 32) {
            DF acc[NV];
#pragma unroll
            for (int j = 0; j < NV; ++j) {
                acc[j] = DF{0.f, 0.f};
                if (threadIdx.x < nb) {
                    const float2 p = __ldcg(slot + (size_t)threadIdx.x * NPART + j);
                    acc[j] = DF{p.x, p.y};
                }
            }
            warp_sum_df_n<NV>(acc);
            if (threadIdx.x == 0) finish(acc);
        }
    } else {
        DF acc[NV];
#pragma unroll
        for (int j = 0; j < NV; ++j) acc[j] = DF{0.f, 0.f};
        for (unsigned int b = threadIdx.x; b < nb; b += NTHREADS) {
#pragma unroll
            for (int j = 0; j < NV; ++j) {
                const float2 p = __ldcg(slot + (size_t)b * NPART + j);
                acc[j] = df_add(acc[j], DF{p.x, p.y});
            }
        }
        DF tot[NV];
        block_sum_df<NV>(acc, tot);
        if (threadIdx.x == 0) finish(tot);
    }
    __syncthreads();
    return true;
}

// Called by all threads of every block at the end of a grid-mode solve.
__device__ __forceinline__ void grid_exit(GroupSync* gs, unsigned int nb) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int t = atomicAdd(&gs->exits, 1u);
        if (t == nb - 1) {  // every block has passed its last wait
            gs->count = 0u;
            gs->exits = 0u;
            __threadfence();
        }
    }
}

// ---------------------------------------------------------------------------
// Cluster mode: a small level solve runs on one thread-block cluster (up to
// CLUSTER_MAX blocks, one per SM of a GPC) instead of a cooperative grid.
// A reduction then never leaves the GPC: every block writes its double-float
// block sums into a slot of every block's shared memory (distributed shared
// memory) and arrives on each block's mbarrier; each block waits on its own
// mbarrier (bounded), sums the slots in a fixed order (rank order up to 4
// blocks, a butterfly beyond) and runs the scalar update itself.  All blocks hold identical scalar state (the same sums in
// the same order), so no broadcast is needed and one barrier ends a phase.
// ---------------------------------------------------------------------------

constexpr int CLUSTER_MAX = 16;

// Per-block shared state of a level solve: the block's replica of the
// solve's scalars (both modes) and, in cluster mode, the exchange slots.
struct ClusterState {
    double slots[2][CLUSTER_MAX][NPART];  // [phase parity][source rank][value], double-float pairs
    unsigned long long mbar[2];  // phases alternate between the two barriers
    int err;
    Scalars sc;                           // this block's replica of the solve's scalars
};

__device__ __forceinline__ unsigned int smem_u32(const void* p) {
    return (unsigned int)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned int cluster_map(unsigned int addr, unsigned int rank) {
    unsigned int r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;"
                 ::: "memory");
}

__device__ __forceinline__ bool mbar_test_parity(unsigned int addr, unsigned int parity) {
    unsigned int ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    return ok != 0;
}

// Called by all threads of every block of the cluster at kernel start, after
// the job is in shared memory: loads the scalar replica, initialises the two
// mbarriers for nb arrivals per phase and makes them visible cluster-wide.
__device__ __forceinline__ void cluster_begin(ClusterState& cs, const Scalars* gsc, unsigned int nb) {
    if (threadIdx.x == 0) {
        cs.sc = *gsc;
        cs.err = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&cs.mbar[0])), "r"(nb)
                     : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&cs.mbar[1])), "r"(nb)
                     : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    cluster_sync_all();
}

// Called by all threads at kernel end: block 0 writes the scalars back and no
// block leaves while another may still write into its shared memory.
__device__ __forceinline__ void cluster_end(ClusterState& cs, Scalars* gsc, unsigned int rank) {
    __syncthreads();
    if (rank == 0 && threadIdx.x == 0) *gsc = cs.sc;
    cluster_sync_all();
}

template <int NV, class Finish>
__device__ __forceinline__ bool cluster_reduce(const float (&v)[NV], ClusterState& cs,
                                               unsigned int phase, unsigned int nb,
                                               unsigned int rank, GroupSync* gs, Finish&& finish,
                                               long long limit = GROUP_WAIT_LIMIT_CYCLES) {
    DF in[NV], out[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) in[j] = DF{v[j], 0.f};
    block_sum_df<NV>(in, out);  // warp 0 holds lane 0's sums; ends with __syncthreads()
    // phase k uses slots[k & 1] and mbar[k & 1], whose own phase parity is (k >> 1) & 1.  A block
    // arrives for phase k + 1 only after it has seen every block's phase-k arrival, and for phase
    // k + 2 only after every block has arrived for k + 1, i.e. has finished waiting on phase k:
    // so no arrival can land on a barrier that is still collecting an earlier phase.
    const unsigned int par = phase & 1u, bpar = (phase >> 1) & 1u;
    if (threadIdx.x < nb) {  // lane t delivers this block's sums to block t
        const unsigned int t = threadIdx.x;
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            const unsigned int dst = cluster_map(smem_u32(&cs.slots[par][rank][j]), t);
            asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(dst), "f"(out[j].hi),
                         "f"(out[j].lo)
                         : "memory");
        }
        const unsigned int bar = cluster_map(smem_u32(&cs.mbar[par]), t);
        asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar)
                     : "memory");
    }
    if (threadIdx.x < 32) {  // warp 0: every lane waits (bounded) and acquires, lane q reads block q's sums
        const unsigned int bar = smem_u32(&cs.mbar[par]);
        const long long t0 = clock64();
        bool ok = true;
        while (!mbar_test_parity(bar, bpar)) {
            if (clock64() - t0 > limit) {
                ok = false;
                break;
            }
        }
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) {
            if (threadIdx.x == 0) {
                cs.err = 1;
                atomicExch(&gs->err, 1);
            }
        } else if (nb <= 4) {  // a few slots: lane 0 adds them in rank order
            if (threadIdx.x == 0) {
                DF acc[NV];
#pragma unroll
                for (int j = 0; j < NV; ++j) acc[j] = DF{0.f, 0.f};
                for (unsigned int q = 0; q < nb; ++q) {
#pragma unroll
                    for (int j = 0; j < NV; ++j) {
                        const float2 p = *reinterpret_cast<const float2*>(&cs.slots[par][q][j]);
                        acc[j] = df_add(acc[j], DF{p.x, p.y});
                    }
                }
                finish(acc);
            }
        } else {  // lane q holds block q's sums; a 16-lane butterfly adds them
            DF acc[NV];
#pragma unroll
            for (int j = 0; j < NV; ++j) {
                acc[j] = DF{0.f, 0.f};
                if (threadIdx.x < nb) {
                    const float2 p = *reinterpret_cast<const float2*>(&cs.slots[par][threadIdx.x][j]);
                    acc[j] = DF{p.x, p.y};
                }
            }
            warp_sum_df_n<NV, CLUSTER_MAX>(acc);  // lanes >= nb add zeros
            if (threadIdx.x == 0) finish(acc);
        }
    }
    __syncthreads();
    return cs.err == 0;
}

// The reduction + barrier of one phase, in grid or cluster mode.
struct LevelSync {
    double* partials;
    GroupSync* gs;
    unsigned int nb, bid;
    ClusterState* cs;
    bool cluster;
    unsigned int phase;
    template <int NV, class Finish>
    __device__ __forceinline__ bool reduce(const float (&v)[NV], Finish&& finish) {
        if (cluster) return cluster_reduce<NV>(v, *cs, phase++, nb, bid, gs, finish);
        return grid_reduce<NV>(v, partials, gs, nb, bid, phase++, finish);
    }
};

}  // namespace eecmg
