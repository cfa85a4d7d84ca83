// Instantiations of the persistent level solver: MR-II, FP32 storage, radii 0..5 (also the
// shared-memory resident form).
#include "level_solve_impl.cuh"

namespace eecmg {

cudaError_t launch_level_mr2_f32_lo(const LevelLaunch& L, int rt, int sep, int prec, int op,
                                    int blocks, cudaStream_t s, int* out) {
    switch (rt) {
        case 0: return launch_level_r<0, false, float>(L, sep, prec, op, blocks, s, out);
        case 1: return launch_level_r<1, false, float>(L, sep, prec, op, blocks, s, out);
        case 2: return launch_level_r<2, false, float>(L, sep, prec, op, blocks, s, out);
        case 3: return launch_level_r<3, false, float>(L, sep, prec, op, blocks, s, out);
        case 4: return launch_level_r<4, false, float>(L, sep, prec, op, blocks, s, out);
        case 5: return launch_level_r<5, false, float>(L, sep, prec, op, blocks, s, out);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace eecmg
