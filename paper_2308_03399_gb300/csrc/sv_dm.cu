// Density-matrix method: the exact final distribution of a noisy circuit,
// from which every shot is then sampled (the alternative to multi-shot
// simulation the paper weighs in Sections II and III-C: exact, but its
// memory grows as 4^n).
//
// rho is stored as a state of 2n qubits, vec(rho)[r + c 2^n] = rho[r][c], so
// the pass kernels evolve it (a gate U is U on the row qubits and conj(U) on
// the column qubits; a channel is the superoperator sum_i K_i (x) conj(K_i)
// on both).  The kernels here read the final distribution p_j = rho[j][j]
// and draw every shot's key from it: the first j with u < C_j, C the running
// float64 sum in index order (the selection rule of Table I), u the shot's
// Philox draw for the final op.
#include <cuda_runtime.h>

#include <cstdint>

#include "sv_internal.h"
#include "sv_sample.cuh"

namespace sv {

template <class R>
__global__ void __launch_bounds__(256) k_dm_diag(const typename svs::Cx<R>::T* rho, int n, double* p) {
    const int64_t dim = 1ll << n;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < dim; j += (int64_t)gridDim.x * blockDim.x)
        p[j] = (double)rho[j + (j << n)].x;  // the diagonal is real; its imaginary part is rounding
}

// per chunk of L probabilities: their float64 sum in a fixed order
__global__ void __launch_bounds__(256) k_dm_chunks(const double* p, int64_t L, int chunks, double* sums) {
    __shared__ double sh[32];
    for (int c = blockIdx.x; c < chunks; c += gridDim.x) {
        double s = 0.0;
        for (int64_t j = threadIdx.x; j < L; j += blockDim.x) s += p[(int64_t)c * L + j];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
            sums[c] = t;
        }
    }
}

__global__ void k_dm_cum(const double* sums, double* cum, int chunks) { svs::chunk_cum(sums, cum, chunks, 1); }

// one warp per shot: the chunk by a warp ballot over the running sums, then
// the first index by a warp prefix sum over 32 probabilities at a time
__global__ void __launch_bounds__(256) k_dm_sample(const double* p, const double* cum, int64_t L, int chunks,
                                                   uint64_t n_shots, uint64_t seed, uint32_t op, uint64_t* keys,
                                                   double* thr) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t dim = L * chunks;
    for (int64_t s = gw; s < (int64_t)n_shots; s += nw) {
        const double u = svs::philox_uniform(seed, (uint64_t)s, op);
        int c = chunks;
        for (int c0 = 0; c0 < chunks && c == chunks; c0 += 32) {
            const bool hit = c0 + lane < chunks && u < cum[c0 + lane];
            const unsigned m = __ballot_sync(0xffffffffu, hit);
            if (m) c = c0 + __ffs(m) - 1;
        }
        int64_t key = -1;
        double lo = 0.0, hi = 0.0;
        if (c < chunks) {
            double acc = c ? cum[c - 1] : 0.0;
            for (int64_t b0 = 0; b0 < L && key < 0; b0 += 32) {
                const int64_t j = (int64_t)c * L + b0 + lane;
                const double x = b0 + lane < L ? p[j] : 0.0;
                double incl = x;
                for (int o = 1; o < 32; o <<= 1) {
                    const double y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                const unsigned m = __ballot_sync(0xffffffffu, b0 + lane < L && u < acc + incl);
                if (m) {
                    const int f = __ffs(m) - 1;
                    key = (int64_t)c * L + b0 + f;
                    hi = acc + __shfl_sync(0xffffffffu, incl, f);
                    lo = hi - __shfl_sync(0xffffffffu, x, f);
                }
                acc += __shfl_sync(0xffffffffu, incl, 31);
            }
        }
        if (key < 0) {  // u at or past the rounded total: the last entry with p > 0
            for (int64_t top = dim; top > 0 && key < 0; top -= 32) {
                const int64_t j = top - 32 + lane;
                const double x = j >= 0 ? p[j] : 0.0;
                const unsigned m = __ballot_sync(0xffffffffu, j >= 0 && x > 0.0);
                if (m) {
                    const int f = 31 - __clz(m);
                    key = top - 32 + f;
                    hi = cum[chunks - 1];
                    lo = hi - __shfl_sync(0xffffffffu, x, f);
                }
            }
            if (key < 0) key = dim - 1;
        }
        if (lane == 0) {
            keys[s] = (uint64_t)key;
            if (thr) {
                thr[2 * s] = lo;
                thr[2 * s + 1] = hi;
            }
        }
    }
}

cudaError_t launch_dm_final(const void* rho, int prec, int n, double* p, double* sums, double* cum, int chunks,
                            uint64_t n_shots, uint64_t seed, uint32_t op, uint64_t* keys, double* thr, int n_sm,
                            cudaStream_t s) {
    const int64_t dim = 1ll << n;
    const int grid = 4 * n_sm;
    if (prec) k_dm_diag<double><<<grid, 256, 0, s>>>(static_cast<const double2*>(rho), n, p);
    else k_dm_diag<float><<<grid, 256, 0, s>>>(static_cast<const float2*>(rho), n, p);
    k_dm_chunks<<<grid, 256, 0, s>>>(p, dim / chunks, chunks, sums);
    k_dm_cum<<<1, 32, 0, s>>>(sums, cum, chunks);
    k_dm_sample<<<grid, 256, 0, s>>>(p, cum, dim / chunks, chunks, n_shots, seed, op, keys, thr);
    return cudaGetLastError();
}

}  // namespace sv
