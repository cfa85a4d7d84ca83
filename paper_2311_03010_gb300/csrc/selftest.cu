// selftest.cu -- diagnostic: the bounded waits of the level-solve barriers.
//
// One block runs one reduction barrier whose arrival count can never be
// reached (it claims to be one of two blocks, or expects two arrivals on its
// cluster mbarrier while only itself delivers), with a wait limit of about
// 10 microseconds.  The wait must give up, set the job's error flag and let
// the block return; nothing faults or hangs, and the context stays usable.
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
