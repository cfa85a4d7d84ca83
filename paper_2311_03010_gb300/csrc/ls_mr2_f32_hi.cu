// Instantiations of the persistent level solver: MR-II, FP32 storage, radii 6..12.
#include "level_solve_impl.cuh"

namespace eecmg {

cudaError_t launch_level_mr2_f32_hi(const LevelLaunch& L, int rt, int sep, int prec, int op,
                                    int blocks, cudaStream_t s, int* out) {
    switch (rt) {
        case 6: return launch_level_r<6, false, float>(L, sep, prec, op, blocks, s, out);
        case 7: return launch_level_r<7, false, float>(L, sep, prec, op, blocks, s, out);
        case 8: return launch_level_r<8, false, float>(L, sep, prec, op, blocks, s, out);
        case 9: return launch_level_r<9, false, float>(L, sep, prec, op, blocks, s, out);
        case 10: return launch_level_r<10, false, float>(L, sep, prec, op, blocks, s, out);
        case 11: return launch_level_r<11, false, float>(L, sep, prec, op, blocks, s, out);
        case 12: return launch_level_r<12, false, float>(L, sep, prec, op, blocks, s, out);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace eecmg
