// Instantiations of the register pass kernel: complex64, stage by stage.
#include "sv_pass_reg.cuh"

namespace sv {

template <class R, int WP, int PAIRED, int VAR> const void* reg_fn() {
    return (const void*)k_pass_reg<R, WP, PAIRED, VAR>;
}

template <int PAIRED, int VAR> const void* reg_fn_c64(int wp) {
    switch (wp) {
    case 1: return reg_fn<float, 1, PAIRED, VAR>();
    case 2: return reg_fn<float, 2, PAIRED, VAR>();
    case 3: return reg_fn<float, 3, PAIRED, VAR>();
    default: return reg_fn<float, 4, PAIRED, VAR>();
    }
}

const void* reg_kernel_plain_c64(int wp, int paired) {
    return paired ? reg_fn_c64<1, REG_PLAIN>(wp) : reg_fn_c64<0, REG_PLAIN>(wp);
}

}  // namespace sv
