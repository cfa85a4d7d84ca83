// Instantiations of the persistent level solver: CGLS, BF16 storage, radii 6..12.
#include "level_solve_impl.cuh"

namespace eecmg {

cudaError_t launch_level_cgls_bf16_hi(const LevelLaunch& L, int rt, int sep, int prec, int op,
                                      int blocks, cudaStream_t s, int* out) {
    switch (rt) {
        case 6: return launch_level_r<6, true, __nv_bfloat16>(L, sep, prec, op, blocks, s, out);
        case 7: return launch_level_r<7, true, __nv_bfloat16>(L, sep, prec, op, blocks, s, out);
        case 8: return launch_level_r<8, true, __nv_bfloat16>(L, sep, prec, op, blocks, s, out);
        case 9: return launch_level_r<9, true, __nv_bfloat16>(L, sep, prec, op, blocks, s, out);
        case 10: return launch_level_r<10, true, __nv_bfloat16>(L, sep, prec, op, blocks, s, out);
        case 11: return launch_level_r<11, true, __nv_bfloat16>(L, sep, prec, op, blocks, s, out);
        case 12: return launch_level_r<12, true, __nv_bfloat16>(L, sep, prec, op, blocks, s, out);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace eecmg
