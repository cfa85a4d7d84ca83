// Instantiations of the volume level solve and apply kernels, radii 3, 4.
#include "volume_impl.cuh"

namespace eecmg {
namespace vol {

bool vol_kernels_r34(int r, const void** solve, const void** apply) {
    switch (r) {
        case 3:
            *solve = (const void*)k_vol_mr2<3>;
            *apply = (const void*)k_vol_apply<3>;
            return true;
        case 4:
            *solve = (const void*)k_vol_mr2<4>;
            *apply = (const void*)k_vol_apply<4>;
            return true;
        default:
            return false;
    }
}

}  // namespace vol
}  // namespace eecmg
