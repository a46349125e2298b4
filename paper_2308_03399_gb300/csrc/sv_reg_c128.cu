// Instantiations of the register pass kernel: complex128, stage by stage.
#include "sv_pass_reg.cuh"

namespace sv {

template <class R, int WP, int PAIRED, int VAR> const void* reg_fn() {
    return (const void*)k_pass_reg<R, WP, PAIRED, VAR>;
}

const void* reg_kernel_c128(int wp) {
    switch (wp) {
    case 1: return reg_fn<double, 1, 0, REG_PLAIN>();
    case 2: return reg_fn<double, 2, 0, REG_PLAIN>();
    case 3: return reg_fn<double, 3, 0, REG_PLAIN>();
    default: return reg_fn<double, 4, 0, REG_PLAIN>();
    }
}

}  // namespace sv
