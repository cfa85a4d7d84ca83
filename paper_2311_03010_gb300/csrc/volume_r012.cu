// Instantiations of the volume level solve and apply kernels, radii 0, 1, 2.
#include "volume_impl.cuh"

namespace eecmg {
namespace vol {

bool vol_kernels_r012(int r, const void** solve, const void** apply) {
    switch (r) {
        case 0:
            *solve = (const void*)k_vol_mr2<0>;
            *apply = (const void*)k_vol_apply<0>;
            return true;
        case 1:
            *solve = (const void*)k_vol_mr2<1>;
            *apply = (const void*)k_vol_apply<1>;
            return true;
        case 2:
            *solve = (const void*)k_vol_mr2<2>;
            *apply = (const void*)k_vol_apply<2>;
            return true;
        default:
            return false;
    }
}

}  // namespace vol
}  // namespace eecmg
