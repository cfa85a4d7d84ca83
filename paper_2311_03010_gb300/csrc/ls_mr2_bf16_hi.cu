// Instantiations of the persistent level solver: MR-II, BF16 storage, radii 6..12.
#include "level_solve_impl.cuh"

namespace eecmg {

cudaError_t launch_level_mr2_bf16_hi(const LevelLaunch& L, int rt, int sep, int prec, int op,
                                     int blocks, cudaStream_t s, int* out) {
    switch (rt) {
        case 6: return launch_level_r<6, false, __nv_bfloat16>(L, sep, prec, op, blocks, s, out);
        case 7: return launch_level_r<7, false, __nv_bfloat16>(L, sep, prec, op, blocks, s, out);
        case 8: return launch_level_r<8, false, __nv_bfloat16>(L, sep, prec, op, blocks, s, out);
        case 9: return launch_level_r<9, false, __nv_bfloat16>(L, sep, prec, op, blocks, s, out);
        case 10: return launch_level_r<10, false, __nv_bfloat16>(L, sep, prec, op, blocks, s, out);
        case 11: return launch_level_r<11, false, __nv_bfloat16>(L, sep, prec, op, blocks, s, out);
        case 12: return launch_level_r<12, false, __nv_bfloat16>(L, sep, prec, op, blocks, s, out);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace eecmg
