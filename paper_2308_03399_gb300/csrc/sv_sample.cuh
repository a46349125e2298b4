// Philox draws and the final sampling building blocks (Section IV-B-2's
// sampling measure), used by
// the batch path (sv_kernels.cu) and by sv_final_sample_noalloc
// (sv_noalloc.cu), so both give the same key for the same state and draw.
//
// A state of 2^n amplitudes is cut into `chunks` contiguous chunks of L
// amplitudes.  chunk_sum() gives one chunk's sum of |psi_j|^2 (one CTA,
// float-float or float64 per thread, fixed-order combination); chunk_cum()
// turns a state's chunk sums into a running sum (one warp, fixed order);
// sample_warp() draws one key: the chunk by a two-level warp search over the
// running sums, then the first j with u < C_j by a warp prefix sum over 256
// amplitudes at a time (8 per lane), all in float64.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace svs {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32
// multiplies with the published multipliers and Weyl key increments.
// key = (seed lo, seed hi), counter = (shot lo, shot hi, op, 0); the draw is
// the top 53 bits of words 0 and 1.
__device__ __forceinline__ uint64_t philox_k53(uint64_t seed, uint64_t shot, uint32_t op) {
    uint32_t key0 = (uint32_t)seed, key1 = (uint32_t)(seed >> 32);
    uint32_t w0 = (uint32_t)shot, w1 = (uint32_t)(shot >> 32), w2 = op, w3 = 0u;
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t a_hi = __umulhi(0xD2511F53u, w0), a_lo = 0xD2511F53u * w0;
        const uint32_t b_hi = __umulhi(0xCD9E8D57u, w2), b_lo = 0xCD9E8D57u * w2;
        const uint32_t n0 = b_hi ^ w1 ^ key0;
        const uint32_t n2 = a_hi ^ w3 ^ key1;
        w0 = n0;
        w1 = b_lo;
        w2 = n2;
        w3 = a_lo;
        key0 += 0x9E3779B9u;
        key1 += 0xBB67AE85u;
    }
    return ((((uint64_t)w0) << 32) | (uint64_t)w1) >> 11;
}

// the uniform draw u = k * 2^-53 in [0, 1)
__device__ __forceinline__ double philox_uniform(uint64_t seed, uint64_t shot, uint32_t op) {
    return (double)philox_k53(seed, shot, op) * 0x1.0p-53;
}

template <class R> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };

template <class R> struct Sum;
template <> struct Sum<double> {
    double s = 0.0;
    __device__ __forceinline__ void add_sq(double x, double y) { s += x * x + y * y; }
    __device__ __forceinline__ double get() const { return s; }
};
// float-float pair (Knuth's TwoSum); the squares of float32 values enter
// exactly: x*x rounded plus its error fma(x, x, -x*x) (Dekker's product)
template <> struct Sum<float> {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float x) {
        float s = __fadd_rn(hi, x);
        float bp = __fsub_rn(s, hi);
        float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
        hi = s;
        lo = __fadd_rn(lo, e);
    }
    __device__ __forceinline__ void add_sq(float x, float y) {
        const float px = __fmul_rn(x, x), py = __fmul_rn(y, y);
        const float ex = __fmaf_rn(x, x, -px), ey = __fmaf_rn(y, y, -py);
        add(px);
        add(py);
        lo = __fadd_rn(lo, __fadd_rn(ex, ey));
    }
    __device__ __forceinline__ double get() const { return (double)hi + (double)lo; }
};

// sum of |psi_j|^2 over g[0..L), whole CTA; result valid in thread 0
template <class R>
__device__ __forceinline__ double chunk_sum(const typename Cx<R>::T* g, int64_t L, double* sh32) {
    Sum<R> a;
    // a thread adds j = tid, tid + blockDim, ... in increasing order; the
    // loads of eight consecutive terms are issued before their adds
    const int64_t bd = blockDim.x;
    for (int64_t j0 = threadIdx.x; j0 < L; j0 += 8 * bd) {
        typename Cx<R>::T v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (j0 + k * bd < L) v[k] = g[j0 + k * bd];
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (j0 + k * bd < L) a.add_sq(v[k].x, v[k].y);
    }
    double x = a.get();
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh32[threadIdx.x >> 5] = x;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh32[w];
    return s;
}

// running sum of sums[0..chunks) (stride `stride` doubles) into cum (same
// stride), one warp
__device__ __forceinline__ void chunk_cum(const double* sums, double* cum, int chunks, int stride) {
    const int lane = threadIdx.x & 31;
    const int per = (chunks + 31) / 32;
    const int c0 = lane * per, c1 = min(c0 + per, chunks);
    double t = 0.0;
    for (int c = c0; c < c1; ++c) t += sums[(int64_t)c * stride];
    double incl = t;
    for (int o = 1; o < 32; o <<= 1) {
        const double y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    double run = incl - t;
    for (int c = c0; c < c1; ++c) {
        run += sums[(int64_t)c * stride];
        cum[(int64_t)c * stride] = run;
    }
}

// one key for draw u from the state g (whole warp; result in every lane)
template <class R>
__device__ __forceinline__ int64_t sample_warp(const typename Cx<R>::T* g, int64_t dim, int chunks,
                                               const double* cum, int stride, double u, double* lo_out,
                                               double* hi_out) {
    using T = typename Cx<R>::T;
    const int lane = threadIdx.x & 31;
    const int64_t L = dim / chunks;
    // chunk: first c with u < cum[c], coarse blocks of 32 then within
    int c = chunks;
    {
        const int nb = (chunks + 31) / 32;
        int blk = nb;
        for (int b0 = 0; b0 < nb && blk == nb; b0 += 32) {
            const int bi = b0 + lane;
            const int last = min(bi * 32 + 31, chunks - 1);
            const bool hit = bi < nb && u < cum[(int64_t)last * stride];
            const unsigned m = __ballot_sync(0xffffffffu, hit);
            if (m) blk = b0 + __ffs(m) - 1;
        }
        if (blk < nb) {
            const int ci = blk * 32 + lane;
            const bool hit = ci < chunks && u < cum[(int64_t)ci * stride];
            const unsigned m = __ballot_sync(0xffffffffu, hit);
            if (m) c = blk * 32 + __ffs(m) - 1;
        }
    }
    int64_t key = -1;
    double lo = 0.0, hi = 0.0;
    if (c < chunks) {
        double acc = c ? cum[(int64_t)(c - 1) * stride] : 0.0;
        const int64_t j0 = (int64_t)c * L;
        for (int64_t blk = 0; blk < L && key < 0; blk += 256) {
            double pe[8];
            double tot = 0.0;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int64_t j = blk + lane * 8 + e;
                double p = 0.0;
                if (j < L) {
                    const T v = g[j0 + j];
                    p = (double)v.x * (double)v.x + (double)v.y * (double)v.y;
                }
                pe[e] = p;
                tot += p;
            }
            double incl = tot;
            for (int o = 1; o < 32; o <<= 1) {
                const double y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const double base = acc + (incl - tot);
            const unsigned m = __ballot_sync(0xffffffffu, u < acc + incl);
            if (m) {
                const int f = __ffs(m) - 1;
                int64_t k = -1;
                double h = 0.0, l = 0.0;
                if (lane == f) {
                    double run = base;
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const double before = run;
                        run += pe[e];
                        if (k < 0 && u < run && blk + lane * 8 + e < L) {
                            k = j0 + blk + lane * 8 + e;
                            l = before;
                            h = run;
                        }
                    }
                }
                key = __shfl_sync(0xffffffffu, k, f);
                lo = __shfl_sync(0xffffffffu, l, f);
                hi = __shfl_sync(0xffffffffu, h, f);
            }
            acc += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
    if (key < 0) {  // u at or past the rounded total: the last nonzero entry
        const double total = cum[(int64_t)(chunks - 1) * stride];
        for (int64_t top = dim; top > 0 && key < 0; top -= 32) {
            const int64_t j = top - 32 + lane;
            double p = 0.0;
            if (j >= 0) {
                const T v = g[j];
                p = (double)v.x * (double)v.x + (double)v.y * (double)v.y;
            }
            const unsigned m = __ballot_sync(0xffffffffu, j >= 0 && p > 0);
            if (m) {
                const int f = 31 - __clz(m);
                key = top - 32 + f;
                const double pf = __shfl_sync(0xffffffffu, p, f);
                hi = total;
                lo = total - pf;
            }
        }
        if (key < 0) key = dim - 1;
    }
    *lo_out = lo;
    *hi_out = hi;
    return key;
}

}  // namespace svs
