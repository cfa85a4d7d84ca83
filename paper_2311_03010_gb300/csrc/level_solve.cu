// level_solve.cu -- dispatch of the persistent level solve (kernels in
// level_solve_impl.cuh, instantiated in the ls_*.cu translation units).
#include "level_solve_impl.cuh"

namespace eecmg {

cudaError_t launch_level_solve(const LevelJob& J, int rt, int sep, int prec, int cgls,
                               cudaStream_t s, int* blocks_used) {
    if (J.h <= 0 || J.w <= 0) return cudaSuccess;
    const size_t n = (size_t)J.h * J.w;
    const int tiles = (int)conv_blocks(J.h, J.w);
    const int elem = (int)((n + 4 * NTHREADS - 1) / (4 * NTHREADS));
    const int want = tiles > elem ? tiles : elem;
    if (rt < 0 || rt > RMAX) return cudaErrorInvalidValue;
    if (cgls)
        return rt < 6 ? launch_level_cgls_lo(J, rt, sep, prec, want, s, blocks_used)
                      : launch_level_cgls_hi(J, rt, sep, prec, want, s, blocks_used);
    return rt < 6 ? launch_level_mr2_lo(J, rt, sep, prec, want, s, blocks_used)
                  : launch_level_mr2_hi(J, rt, sep, prec, want, s, blocks_used);
}

}  // namespace eecmg
