// level_solve.cu -- dispatch of the persistent level solve (kernels in
// level_solve_impl.cuh, instantiated in the ls_*.cu translation units).
#include "level_solve_impl.cuh"

namespace eecmg {

#ifdef EECMG_TRACE
__device__ unsigned long long g_eecmg_trace[1 << 16];
__device__ unsigned int g_eecmg_trace_n;
#endif

namespace {

cudaError_t dispatch(const LevelLaunch& L, int rt, int sep, int prec, int cgls, int bf16, int want,
                     cudaStream_t s, int* used) {
    if (rt < 0 || rt > RMAX) return cudaErrorInvalidValue;
    const bool lo = rt < 6;
    if (cgls) {
        if (bf16)
            return lo ? launch_level_cgls_bf16_lo(L, rt, sep, prec, want, s, used)
                      : launch_level_cgls_bf16_hi(L, rt, sep, prec, want, s, used);
        return lo ? launch_level_cgls_f32_lo(L, rt, sep, prec, want, s, used)
                  : launch_level_cgls_f32_hi(L, rt, sep, prec, want, s, used);
    }
    if (bf16)
        return lo ? launch_level_mr2_bf16_lo(L, rt, sep, prec, want, s, used)
                  : launch_level_mr2_bf16_hi(L, rt, sep, prec, want, s, used);
    return lo ? launch_level_mr2_f32_lo(L, rt, sep, prec, want, s, used)
              : launch_level_mr2_f32_hi(L, rt, sep, prec, want, s, used);
}

}  // namespace

// Blocks of a level solve: one per 32 x 64 tile or per 1024 pixels, at most
// two per SM.  The count depends only on the level's size, so a solve is
// partitioned (and its reductions rounded) the same way alone or in a batch.
int level_want_blocks(int h, int w) {
    static int cap = 0;
    if (cap == 0) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cap = 2 * (sms > 0 ? sms : 1);
    }
    const size_t n = (size_t)h * w;
    const int tiles = (int)conv_blocks(h, w);
    const int elem = (int)((n + 4 * NTHREADS - 1) / (4 * NTHREADS));
    const int want = tiles > elem ? tiles : elem;
    return want < cap ? want : cap;
}

cudaError_t launch_level_solve(const LevelJob& J, int rt, int sep, int prec, int cgls, int bf16,
                               cudaStream_t s, int* blocks_used) {
    if (J.h <= 0 || J.w <= 0) return cudaSuccess;
    LevelLaunch L;
    L.job = J;
    return dispatch(L, rt, sep, prec, cgls, bf16, level_want_blocks(J.h, J.w), s, blocks_used);
}

cudaError_t launch_level_batch(const LevelJob* d_jobs, const unsigned short* d_block_job, int njobs,
                               int total_blocks, int rt, int sep, int prec, int cgls, int bf16,
                               cudaStream_t s) {
    if (njobs <= 0 || total_blocks <= 0) return cudaSuccess;
    LevelLaunch L;
    L.jobs = d_jobs;
    L.block_job = d_block_job;
    L.njobs = njobs;
    return dispatch(L, rt, sep, prec, cgls, bf16, -total_blocks, s, nullptr);
}

int level_capacity(int rt, int sep, int prec, int cgls, int bf16) {
    LevelLaunch L;
    int cap = 0;
    if (dispatch(L, rt, sep, prec, cgls, bf16, 0, nullptr, &cap) != cudaSuccess) return 0;
    return cap;
}

}  // namespace eecmg

#ifdef EECMG_TRACE
// Tracing builds only: copies the phase timestamps out and resets them.
extern "C" int eecmg_trace_dump(unsigned long long* out, int max) {
    unsigned int n = 0;
    cudaDeviceSynchronize();
    cudaMemcpyFromSymbol(&n, eecmg::g_eecmg_trace_n, sizeof(n));
    if (n > (1u << 16)) n = 1u << 16;
    if ((int)n > max) n = (unsigned int)max;
    cudaMemcpyFromSymbol(out, eecmg::g_eecmg_trace, sizeof(unsigned long long) * n);
    const unsigned int z = 0;
    cudaMemcpyToSymbol(eecmg::g_eecmg_trace_n, &z, sizeof(z));
    return (int)n;
}
#endif
