// Instantiations of the register pass kernel: complex64 folded passes (any
// group width) and passes reducing measurement bins (4-qubit groups).
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

const void* reg_kernel_fold_c64(int wp, int paired) {
    return paired ? reg_fn_c64<1, REG_FOLD>(wp) : reg_fn_c64<0, REG_FOLD>(wp);
}

const void* reg_kernel_bins_c64(int paired) {
    return paired ? reg_fn<float, 4, 1, REG_BINS>() : reg_fn<float, 4, 0, REG_BINS>();
}

}  // namespace sv
