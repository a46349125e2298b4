// Final sampling for callers that cannot allocate device memory.
//
// sv_final_sample_noalloc draws one key per state (the sampling measure of
// sv_counts / sv_run_circuit) from states the caller already holds on the
// device, writing keys to a device buffer the caller also provides.  Its
// only working memory is the file-scope array below: 1 MiB of float64
// partial sums that every device which loads the library keeps until the
// process exits.  Nothing here calls cudaMalloc, cudaFree or an allocating
// library routine.
//
// The kernels use the same building blocks as the batch path's final
// sampling (sv_sample.cuh: same chunking, same per-thread order, same
// fixed-order combination), so a state gives the same key through either
// entry point.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/sv.h"
#include "sv_sample.cuh"

namespace sv {
void set_last_error(const std::string& msg);  // sv_runtime.cu
}

namespace {

constexpr int NA_MAX_DEVICES = 64;
constexpr size_t NA_SCRATCH_DOUBLES = 131072;  // 1 MiB
constexpr int NA_MAX_CHUNKS = 1024;  // chunk count limit (as in the batch path)

static __device__ __align__(256) double na_scratch[NA_SCRATCH_DOUBLES];

double* na_scratch_ptr[NA_MAX_DEVICES] = {};
std::mutex na_mutex;

// per (state, chunk): sum of |psi_j|^2 over the chunk's contiguous range
template <class R>
__global__ void __launch_bounds__(256) na_partials(const typename svs::Cx<R>::T* states, int64_t dim, int chunks,
                                                  int n_states, double* scratch) {
    __shared__ double red_sh[32];
    const int64_t L = dim / chunks;
    const int64_t items = (int64_t)n_states * chunks;
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
        const int st = (int)(it / chunks), c = (int)(it % chunks);
        const double s = svs::chunk_sum<R>(states + (int64_t)st * dim + c * L, L, red_sh);
        if (threadIdx.x == 0) scratch[(int64_t)st * chunks + c] = s;
    }
}

// per state (one warp): running sum of its chunk sums, in place
__global__ void __launch_bounds__(256) na_cum(int chunks, int n_states, double* scratch) {
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int st = gw; st < n_states; st += nw)
        svs::chunk_cum(scratch + (int64_t)st * chunks, scratch + (int64_t)st * chunks, chunks, 1);
}

// per state (one warp): its key
template <class R>
__global__ void __launch_bounds__(256) na_sample(const typename svs::Cx<R>::T* states, int64_t dim, int chunks,
                                                int n_states, const uint64_t* shots, uint64_t seed, uint32_t op,
                                                uint64_t* keys, const double* scratch) {
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int st = gw; st < n_states; st += nw) {
        const double u = svs::philox_uniform(seed, shots[st], op);
        double lo, hi;
        const int64_t key = svs::sample_warp<R>(states + (int64_t)st * dim, dim, chunks,
                                                scratch + (int64_t)st * chunks, 1, u, &lo, &hi);
        if ((threadIdx.x & 31) == 0) keys[st] = (uint64_t)key;
    }
}

}  // namespace

extern "C" sv_status sv_final_sample_noalloc(const void* states, sv_prec prec, int n_qubits, uint32_t n_states,
                                             const uint64_t* shots, uint64_t seed, uint32_t op, uint64_t* keys,
                                             void* cuda_stream) {
    if (!states || !shots || !keys) {
        sv::set_last_error("sv_final_sample_noalloc: states, shots and keys must be device pointers");
        return SV_EINVAL;
    }
    if (prec != SV_C64 && prec != SV_C128) {
        sv::set_last_error("sv_final_sample_noalloc: bad precision");
        return SV_EINVAL;
    }
    if (n_qubits < 1 || n_qubits > 30 || n_states == 0) {
        sv::set_last_error("sv_final_sample_noalloc: n_qubits must be 1..30 and n_states >= 1");
        return SV_EINVAL;
    }
    const int64_t dim = 1ll << n_qubits;
    const int64_t c0 = dim / 2048;
    const int chunks = (int)(c0 < 1 ? 1 : (c0 > NA_MAX_CHUNKS ? NA_MAX_CHUNKS : c0));
    if ((uint64_t)n_states * (uint64_t)chunks > NA_SCRATCH_DOUBLES) {
        sv::set_last_error("sv_final_sample_noalloc: n_states x chunks = " +
                           std::to_string((uint64_t)n_states * chunks) + " partial sums exceed the static scratch of " +
                           std::to_string(NA_SCRATCH_DOUBLES) + " (chunks = min(max(2^n / 2048, 1), 1024))");
        return SV_EINVAL;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
        cudaGetLastError();
        sv::set_last_error("sv_final_sample_noalloc: no usable current device");
        return SV_ECUDA;
    }
    double* scratch = nullptr;
    {
        // once per device, with that device current: the device address of
        // the static scratch (its name in host code is only a stand-in)
        std::lock_guard<std::mutex> lock(na_mutex);
        if (!na_scratch_ptr[dev]) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, na_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                sv::set_last_error(std::string("sv_final_sample_noalloc: cudaGetSymbolAddress: ") +
                                   cudaGetErrorString(e));
                return SV_ECUDA;
            }
            na_scratch_ptr[dev] = static_cast<double*>(p);
        }
        scratch = na_scratch_ptr[dev];
    }
    int n_sm = 0;
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    const int grid = 2 * (n_sm > 0 ? n_sm : 1);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (prec == SV_C128) {
        const double2* st = static_cast<const double2*>(states);
        na_partials<double><<<grid, 256, 0, s>>>(st, dim, chunks, (int)n_states, scratch);
        na_cum<<<grid, 256, 0, s>>>(chunks, (int)n_states, scratch);
        na_sample<double><<<grid, 256, 0, s>>>(st, dim, chunks, (int)n_states, shots, seed, op, keys, scratch);
    } else {
        const float2* st = static_cast<const float2*>(states);
        na_partials<float><<<grid, 256, 0, s>>>(st, dim, chunks, (int)n_states, scratch);
        na_cum<<<grid, 256, 0, s>>>(chunks, (int)n_states, scratch);
        na_sample<float><<<grid, 256, 0, s>>>(st, dim, chunks, (int)n_states, shots, seed, op, keys, scratch);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        sv::set_last_error(std::string("sv_final_sample_noalloc: launch: ") + cudaGetErrorString(e));
        return SV_ECUDA;
    }
    return SV_OK;
}
