// selftest.cu -- diagnostics: the bounded waits of the level-solve barriers,
// and a probe of the GPU's FP32 FMA rate (the compute half of the roofline).
//
// One block runs one reduction barrier whose arrival count can never be
// reached (it claims to be one of two blocks, or expects two arrivals on its
// cluster mbarrier while only itself delivers), with a wait limit of about
// 10 microseconds.  The wait must give up, set the job's error flag and let
// the block return; nothing faults or hangs, and the context stays usable.
#include <algorithm>
#include <string>

#include "launch.hpp"
#include "persistent.cuh"
#include "plan.hpp"

using namespace eecmg;

namespace {

constexpr long long SELFTEST_LIMIT_CYCLES = 20000;

struct SelftestScratch {
    GroupSync gs;
    Scalars sc;
    double partials[2 * 2 * NPART];
};

__global__ void __launch_bounds__(NTHREADS) k_wait_timeout_grid(SelftestScratch* x) {
    const float v[1] = {1.f};
    // one block, but the barrier waits for two arrivals
    grid_reduce<1>(v, x->partials, &x->gs, 2u, 0u, 0u, [&](DF*) {}, SELFTEST_LIMIT_CYCLES);
}

__global__ void __launch_bounds__(NTHREADS) k_wait_timeout_cluster(SelftestScratch* x) {
    __shared__ ClusterState CS;
    cluster_begin(CS, &x->sc, 2u);  // mbarrier expects two arrivals per phase
    const float v[1] = {1.f};
    // a cluster of one block delivers only to itself (nb = 1): one arrival
    cluster_reduce<1>(v, CS, 0u, 1u, 0u, &x->gs, [&](DF*) {}, SELFTEST_LIMIT_CYCLES);
    cluster_end(CS, &x->sc, 0u);
}

}  // namespace

extern "C" eecmg_status eecmg_selftest_bounded_wait(int cluster, cudaStream_t s) {
    SelftestScratch* x = nullptr;
    cudaError_t e = cudaMalloc((void**)&x, sizeof(SelftestScratch));
    if (e != cudaSuccess) return set_error(EECMG_ERR_OOM, "eecmg_selftest_bounded_wait: scratch");
    e = cudaMemsetAsync(x, 0, sizeof(SelftestScratch), s);
    if (e == cudaSuccess) {
        if (cluster) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(1);
            cfg.blockDim = dim3(NTHREADS);
            cfg.stream = s;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = 1;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            e = cudaLaunchKernelEx(&cfg, k_wait_timeout_cluster, x);
        } else {
            k_wait_timeout_grid<<<1, NTHREADS, 0, s>>>(x);
            e = cudaGetLastError();
        }
    }
    int err = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, &x->gs.err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(x);
    if (e != cudaSuccess)
        return set_error(EECMG_ERR_CUDA, std::string("eecmg_selftest_bounded_wait: ") + cudaGetErrorString(e));
    if (err) return set_error(EECMG_ERR_TIMEOUT, "eecmg_selftest_bounded_wait: the wait gave up as designed");
    return EECMG_OK;
}

namespace {

// Independent fmaf chains: 8 per thread, 16 rounds per loop trip, so every
// SM sub-partition always has FMAs ready to issue.  The chains stay bounded
// (|x| -> b / (1 - a)); the store is only there to keep them alive.
constexpr int PROBE_CHAINS = 8, PROBE_UNROLL = 16, PROBE_THREADS = 256;

__global__ void __launch_bounds__(PROBE_THREADS) k_fma_probe(float* sink, int iters, float a, float b) {
    float x[PROBE_CHAINS];
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) x[i] = 1e-3f * (float)threadIdx.x + (float)i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < PROBE_UNROLL; ++u)
#pragma unroll
            for (int i = 0; i < PROBE_CHAINS; ++i) x[i] = fmaf(x[i], a, b);
    }
    float t = 0.f;
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) t += x[i];
    if (t == -1.0f) sink[threadIdx.x] = t;  // never true for these inputs
}

}  // namespace

extern "C" eecmg_status eecmg_probe_fp32_fma(int reps, cudaStream_t s, double* tflops) {
    if (reps < 1 || !tflops) return set_error(EECMG_ERR_INVALID_ARG, "eecmg_probe_fp32_fma: bad arguments");
    int dev = 0, nsm = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_probe, PROBE_THREADS, 0);
    if (e != cudaSuccess || per_sm < 1)
        return set_error(EECMG_ERR_CUDA, "eecmg_probe_fp32_fma: device query failed");
    float* sink = nullptr;
    e = cudaMalloc((void**)&sink, sizeof(float) * PROBE_THREADS);
    if (e != cudaSuccess) return set_error(EECMG_ERR_OOM, "eecmg_probe_fp32_fma: scratch");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int blocks = nsm * per_sm, iters = 4096;
    const double fmas = (double)blocks * PROBE_THREADS * iters * PROBE_UNROLL * PROBE_CHAINS;
    double best = 0.0;
    for (int r = 0; r <= reps && e == cudaSuccess; ++r) {  // launch 0 warms up
        e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) {
            k_fma_probe<<<blocks, PROBE_THREADS, 0, s>>>(sink, iters, 0.9999999f, 1e-7f);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && r > 0 && ms > 0.f) best = std::max(best, 2.0 * fmas / (ms * 1e-3) / 1e12);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess)
        return set_error(EECMG_ERR_CUDA, std::string("eecmg_probe_fp32_fma: ") + cudaGetErrorString(e));
    *tflops = best;
    return EECMG_OK;
}
