// Instantiations of the volume level solve and apply kernels, radii 5, 6.
#include "volume_impl.cuh"

namespace eecmg {
namespace vol {

bool vol_kernels_r56(int r, const void** solve, const void** apply) {
    switch (r) {
        case 5:
            *solve = (const void*)k_vol_mr2<5>;
            *apply = (const void*)k_vol_apply<5>;
            return true;
        case 6:
            *solve = (const void*)k_vol_mr2<6>;
            *apply = (const void*)k_vol_apply<6>;
            return true;
        default:
            return false;
    }
}

}  // namespace vol
}  // namespace eecmg
