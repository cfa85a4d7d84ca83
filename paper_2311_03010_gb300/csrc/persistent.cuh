// persistent.cuh -- group barrier with a fused deterministic reduction, for
// the persistent (one launch per level solve) kernels.
//
// All blocks of a group are co-resident (cooperative launch).  At the end of
// a phase every block publishes its FP64 block sums; the last block to
// arrive sums all blocks' partials in a fixed order, runs the phase's scalar
// update on one thread and releases the others by bumping a generation
// counter.  Waits spin on that counter with a clock64 limit: a wait that
// runs out sets the group's error flag and every block returns, so a kernel
// can never hang the GPU; the host reports the flag as a timeout.
#pragma once

#include "common.cuh"

namespace eecmg {

#ifdef EECMG_TRACE
extern __device__ unsigned long long g_eecmg_trace[1 << 16];
extern __device__ unsigned int g_eecmg_trace_n;
__device__ __forceinline__ void trace_any(unsigned int tag) {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    const unsigned int i = atomicAdd(&g_eecmg_trace_n, 2u);
    if (i + 1 < (1u << 16)) {
        g_eecmg_trace[i] = tag;
        g_eecmg_trace[i + 1] = t;
    }
}
#define GTRACE(cond, tag) \
    do {                  \
        if (cond) trace_any(tag); \
    } while (0)
#else
#define GTRACE(cond, tag) ((void)0)
#endif

struct alignas(64) GroupSync {
    unsigned int count;   // arrivals in the current phase
    unsigned int gen;     // phase generation (bumped by the last arrival)
    int err;              // 1 after a wait ran out
    int pad[13];
};

// ~2 s at the GB300's maximum SM clock: far beyond any phase of a level solve.
constexpr long long GROUP_WAIT_LIMIT_CYCLES = 4000000000LL;

template <typename T>
__device__ __forceinline__ T ldcg(const T* p) {
    return __ldcg(p);
}

// Every thread of every block in the group calls this with its block's NV
// values in v (thread-local contributions; reduced here).  Returns false if
// the group is in error (the caller returns).
//
// Memory ordering: each thread's phase writes are ordered before the
// arrival by __syncthreads() and thread 0's GPU-scope fence (fences are
// cumulative); waiters fence after seeing the new generation and then
// release their block with __syncthreads().  Vectors written in the phase
// are read afterwards through L2 (ld.global.cg).
template <int NV, class Finish>
__device__ __forceinline__ bool group_reduce(const double (&v)[NV], double* partials,
                                             GroupSync* gs, unsigned int nb, unsigned int bid,
                                             Finish&& finish) {
    double out[NV];
    block_sum<NV>(v, out);  // ends with __syncthreads()
    __shared__ int s_last, s_ok;
    GTRACE(bid == 0 && threadIdx.x == 0, 20);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) partials[(size_t)bid * NPART + j] = out[j];
        const unsigned int gen = *(volatile unsigned int*)&gs->gen;
        __threadfence();
        const unsigned int t = atomicAdd(&gs->count, 1u);
        GTRACE(bid == 0, 21);
        s_last = (t == nb - 1);
        s_ok = 1;
        if (!s_last) {
            const long long t0 = clock64();
            while (*(volatile unsigned int*)&gs->gen == gen) {
                if (*(volatile int*)&gs->err) {
                    s_ok = 0;
                    break;
                }
                if (clock64() - t0 > GROUP_WAIT_LIMIT_CYCLES) {
                    atomicExch(&gs->err, 1);
                    s_ok = 0;
                    break;
                }
                __nanosleep(32);
            }
            GTRACE(bid == 0, 22);
        }
        __threadfence();
    }
    __syncthreads();
    if (s_last) {
        // the last block sums the blocks' partials in a fixed order, runs the
        // scalar update and releases the group
        GTRACE(threadIdx.x == 0, 30);
        double acc[NV];
#pragma unroll
        for (int j = 0; j < NV; ++j) acc[j] = 0.0;
        for (unsigned int b = threadIdx.x; b < nb; b += NTHREADS) {
#pragma unroll
            for (int j = 0; j < NV; ++j) acc[j] += __ldcg(partials + (size_t)b * NPART + j);
        }
        double tot[NV];
        block_sum<NV>(acc, tot);
        GTRACE(threadIdx.x == 0, 31);
        if (threadIdx.x == 0) {
            finish(tot);
            GTRACE(true, 32);
            gs->count = 0u;
            __threadfence();
            atomicAdd(&gs->gen, 1u);
            GTRACE(true, 33);
        }
        __syncthreads();
    }
    return s_ok != 0 && *(volatile int*)&gs->err == 0;
}

}  // namespace eecmg
