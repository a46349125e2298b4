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
// The kernels repeat the arithmetic of k_final_partials / k_final_sample in
// sv_kernels.cu (same chunking, same per-thread order, same fixed-order
// combination), so a state gives the same key through either entry point.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/sv.h"

namespace sv {
void set_last_error(const std::string& msg);  // sv_runtime.cu
}

namespace {

constexpr int NA_MAX_DEVICES = 64;
constexpr size_t NA_SCRATCH_DOUBLES = 131072;  // 1 MiB
constexpr int NA_MAX_CHUNKS = 1024;

static __device__ __align__(256) double na_scratch[NA_SCRATCH_DOUBLES];

double* na_scratch_ptr[NA_MAX_DEVICES] = {};
std::mutex na_mutex;

template <class R> struct NaCplx;
template <> struct NaCplx<float> { using T = float2; };
template <> struct NaCplx<double> { using T = double2; };

template <class R> struct NaAcc;
template <> struct NaAcc<double> {
    double s;
    __device__ __forceinline__ void zero() { s = 0.0; }
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double get() const { return s; }
};
template <> struct NaAcc<float> {  // float-float pair, Knuth TwoSum
    float hi, lo;
    __device__ __forceinline__ void zero() { hi = 0.f; lo = 0.f; }
    __device__ __forceinline__ void add(float x) {
        float s = __fadd_rn(hi, x);
        float bp = __fsub_rn(s, hi);
        float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
        hi = s;
        lo = __fadd_rn(lo, e);
    }
    __device__ __forceinline__ double get() const { return (double)hi + (double)lo; }
};

// Philox4x32-10 (Salmon et al., SC'11), key = seed, counter = (shot, op, 0)
__device__ __forceinline__ double na_uniform(uint64_t seed, uint64_t shot, uint32_t op) {
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    uint32_t c0 = (uint32_t)shot, c1 = (uint32_t)(shot >> 32), c2 = op, c3 = 0u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t h0 = __umulhi(0xD2511F53u, c0), l0 = 0xD2511F53u * c0;
        const uint32_t h1 = __umulhi(0xCD9E8D57u, c2), l1 = 0xCD9E8D57u * c2;
        const uint32_t n0 = h1 ^ c1 ^ k0, n2 = h0 ^ c3 ^ k1;
        c0 = n0;
        c1 = l1;
        c2 = n2;
        c3 = l0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return (double)(((((uint64_t)c0) << 32) | (uint64_t)c1) >> 11) * 0x1.0p-53;
}

__device__ __forceinline__ double na_block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    return s;
}

// per (state, chunk): sum of |psi_j|^2 over the chunk's contiguous range
template <class R>
__global__ void __launch_bounds__(256) na_partials(const typename NaCplx<R>::T* states, int64_t dim, int chunks,
                                                  int n_states, double* scratch) {
    using T = typename NaCplx<R>::T;
    __shared__ double red_sh[32];
    const int64_t L = dim / chunks;
    const int64_t items = (int64_t)n_states * chunks;
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
        const int st = (int)(it / chunks), c = (int)(it % chunks);
        const T* g = states + (int64_t)st * dim + c * L;
        NaAcc<R> a;
        a.zero();
        for (int64_t j = threadIdx.x; j < L; j += blockDim.x) {
            const T v = g[j];
            a.add(v.x * v.x + v.y * v.y);
        }
        const double s = na_block_sum(a.get(), red_sh);
        if (threadIdx.x == 0) scratch[(int64_t)st * chunks + c] = s;
    }
}

// per state: chunk by binary search over chunk totals, then a warp prefix
// sum over 32 amplitudes at a time; the first j with u < C_j is the key
template <class R>
__global__ void __launch_bounds__(256) na_sample(const typename NaCplx<R>::T* states, int64_t dim, int chunks,
                                                int n_states, const uint32_t* shots, uint64_t seed, uint32_t op,
                                                uint64_t* keys, const double* scratch) {
    using T = typename NaCplx<R>::T;
    __shared__ double cum[NA_MAX_CHUNKS];
    const int64_t L = dim / chunks;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int st = blockIdx.x; st < n_states; st += gridDim.x) {
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int c = 0; c < chunks; ++c) {
                s += scratch[(int64_t)st * chunks + c];
                cum[c] = s;
            }
        }
        __syncthreads();
        if (warp != 0) continue;
        const T* g = states + (int64_t)st * dim;
        const double u = na_uniform(seed, shots[st], op);
        int clo = 0, chi = chunks;
        while (clo < chi) {
            const int mid = (clo + chi) >> 1;
            if (u < cum[mid]) chi = mid;
            else clo = mid + 1;
        }
        int64_t key = -1;
        if (clo < chunks) {
            double acc = clo ? cum[clo - 1] : 0.0;
            const int64_t j0 = (int64_t)clo * L;
            for (int64_t blk = 0; blk < L && key < 0; blk += 32) {
                double pj = 0.0;
                if (blk + lane < L) {
                    const T v = g[j0 + blk + lane];
                    pj = (double)v.x * (double)v.x + (double)v.y * (double)v.y;
                }
                double incl = pj;
                for (int o = 1; o < 32; o <<= 1) {
                    const double y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                const unsigned hit = __ballot_sync(0xffffffffu, (blk + lane < L) && u < acc + incl);
                if (hit) key = j0 + blk + (__ffs(hit) - 1);
                acc += __shfl_sync(0xffffffffu, incl, 31);
            }
        }
        if (key < 0 && lane == 0) {  // u at or past the rounded total: last nonzero entry
            for (int64_t j = dim - 1; j >= 0; --j) {
                const T v = g[j];
                if ((double)v.x * (double)v.x + (double)v.y * (double)v.y > 0) {
                    key = j;
                    break;
                }
            }
            if (key < 0) key = dim - 1;
        }
        if (lane == 0) keys[st] = (uint64_t)key;
    }
}

}  // namespace

extern "C" sv_status sv_final_sample_noalloc(const void* states, sv_prec prec, int n_qubits, uint32_t n_states,
                                             const uint32_t* shots, uint64_t seed, uint32_t op, uint64_t* keys,
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
        na_sample<double><<<grid, 256, 0, s>>>(st, dim, chunks, (int)n_states, shots, seed, op, keys, scratch);
    } else {
        const float2* st = static_cast<const float2*>(states);
        na_partials<float><<<grid, 256, 0, s>>>(st, dim, chunks, (int)n_states, scratch);
        na_sample<float><<<grid, 256, 0, s>>>(st, dim, chunks, (int)n_states, shots, seed, op, keys, scratch);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        sv::set_last_error(std::string("sv_final_sample_noalloc: launch: ") + cudaGetErrorString(e));
        return SV_ECUDA;
    }
    return SV_OK;
}
