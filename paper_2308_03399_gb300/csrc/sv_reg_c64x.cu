// Instantiations of the register pass kernel: complex64 folded passes (any
// group width) and passes reducing measurement bins (4-qubit groups).
#include "sv_pass_reg.cuh"
#include "sv_pass_whole.cuh"

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


constexpr int WHOLE_THREADS = 128;

// per warp: matrices, stage words, expanded matrices (as k_pass_reg)
size_t pass_whole_smem_bytes(const PassDesc& p) {
    const size_t m = (size_t)((p.mat_elems + 1) & ~1);
    return (WHOLE_THREADS / 32) * (m * 8 + 4 * MAX_STAGES * 4 + m * 16);
}

int pass_whole_blocks_per_sm(int n) { return n >= 10 ? 2 : 4; }

cudaError_t launch_pass_whole(const DevBatch& d, const PassDesc& p, int grid, cudaStream_t s) {
    const size_t smem = pass_whole_smem_bytes(p);
    if (p.n == 9) k_pass_whole<4><<<grid, WHOLE_THREADS, smem, s>>>(d, p);
    else if (p.n == 10) k_pass_whole<5><<<grid, WHOLE_THREADS, smem, s>>>(d, p);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace sv
