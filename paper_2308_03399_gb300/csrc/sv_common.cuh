// Device helpers shared by the pass, decide and sampling kernels (complex
// types and arithmetic, float-float accumulators, selection thresholds,
// index helpers, the monomial-matrix test, diagonal-form weights).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "sv_internal.h"
#include "sv_sample.cuh"

namespace sv {

constexpr int PASS_NBUF_H = 4;  // ring buffers of k_pass (PASS_NBUF below)

template <class R> struct Cplx;
template <> struct Cplx<float> { using T = float2; };
template <> struct Cplx<double> { using T = double2; };

template <class T> __device__ __forceinline__ T cmul(T a, T b) {
    T r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
template <class T> __device__ __forceinline__ void cfma(T& acc, T a, T b) {
    acc.x += a.x * b.x - a.y * b.y;
    acc.y += a.x * b.y + a.y * b.x;
}

// Packed float32x2 arithmetic (Blackwell fma.rn.f32x2): a complex
// multiply-accumulate acc += m v is two packed FMAs,
// acc += (m.re, m.re) * (v.re, v.im) and acc += (-m.im, m.im) * (v.im, v.re).
__device__ __forceinline__ unsigned long long pk2(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 upk2(unsigned long long r) {
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
    return make_float2(a, b);
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// Accumulators.  complex128 states sum in float64.  complex64 states sum in
// float-float (an unevaluated pair hi + lo updated with Knuth's TwoSum), which
// carries about 48 bits of precision using only float32 arithmetic; the
// squares of float32 amplitudes are formed in float32 and summed this way.
template <class R> struct Acc;
template <> struct Acc<double> {
    double s;
    __device__ __forceinline__ void zero() { s = 0.0; }
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double get() const { return s; }
};
template <> struct Acc<float> {
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

// Philox4x32-10 draws keyed by (seed; shot, op): svs::philox_k53 /
// svs::philox_uniform (sv_sample.cuh), shared with sv_noalloc.cu
using svs::philox_k53;
using svs::philox_uniform;

// Selection in the integer domain: for u = k * 2^-53, u < c exactly when
// k < ceil(c * 2^53) (the scaling by 2^53 is exact), so a branch turns its
// cumulative table into integer thresholds once and each shot compares
// integers.  Past the last threshold (a table summing to just under 1) the
// choice is the last term with nonzero probability.
__device__ __forceinline__ uint64_t cum_threshold(double c) {
    return c > 0.0 ? __double2ull_ru(c * 0x1.0p53) : 0ull;
}
__device__ __forceinline__ int select_k(uint64_t k, const uint64_t* thr, const double* cum, int R) {
    for (int t = 0; t < R; ++t)
        if (k < thr[t]) return t;
    for (int t = R - 1; t >= 0; --t) {
        const double prev = t ? cum[t - 1] : 0.0;
        if (cum[t] > prev) return t;
    }
    return R - 1;
}

__device__ __forceinline__ void set_err(const DevBatch& d, int code, int info) {
    if (atomicCAS(&d.ctl[CTL_ERR], 0, code) == 0) d.ctl[CTL_ERR_INFO] = info;
}

// insert a zero bit at each of the K ascending positions sp[]
template <int K> __device__ __forceinline__ int insert_zeros(int g, const int* sp) {
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const int p = sp[j];
        g = ((g >> p) << (p + 1)) | (g & ((1 << p) - 1));
    }
    return g;
}

template <int K> __device__ __forceinline__ void sorted_pos(const int32_t* pos, int* sp) {
#pragma unroll
    for (int j = 0; j < K; ++j) sp[j] = pos[j];
#pragma unroll
    for (int i = 0; i < K; ++i)
#pragma unroll
        for (int j = 0; j + 1 < K - i; ++j)
            if (sp[j] > sp[j + 1]) {
                const int t = sp[j];
                sp[j] = sp[j + 1];
                sp[j + 1] = t;
            }
}

// the monomial structure of a 4x4 matrix m (row-major), or 0 when it is not
// monomial; phases go to ph[0..3]
template <class T>
__device__ __forceinline__ int mono_info(const T* m, T* ph) {
    int pi[4];
    for (int q = 0; q < 4; ++q) {
        pi[q] = -1;
        for (int c = 0; c < 4; ++c)
            if (m[q * 4 + c].x != 0 || m[q * 4 + c].y != 0) {
                if (pi[q] >= 0) return 0;
                pi[q] = c;
            }
        if (pi[q] < 0) return 0;
    }
    if ((pi[0] ^ pi[1] ^ pi[2] ^ pi[3]) != 0 || pi[0] == pi[1] || pi[0] == pi[2] || pi[0] == pi[3] ||
        pi[1] == pi[2] || pi[1] == pi[3] || pi[2] == pi[3])
        return 0;
    const int b = pi[0], a1 = pi[1] ^ b, a2 = pi[2] ^ b;
    if ((a1 ^ a2) != (pi[3] ^ b)) return 0;  // not affine (never for 4 points, kept as a guard)
    int word = -1;
    const int tab[6][2] = {{1, 2}, {3, 2}, {1, 3}, {3, 1}, {2, 3}, {2, 1}};
    for (int w = 0; w < 6; ++w)
        if (tab[w][0] == a1 && tab[w][1] == a2) word = w;
    if (word < 0) return 0;
    int unit = 1;
    for (int q = 0; q < 4; ++q) {
        ph[q] = m[q * 4 + pi[q]];
        if (ph[q].x != 1 || ph[q].y != 0) unit = 0;
    }
    return 1 | (unit << 1) | (b << 2) | (word << 4) | (pi[0] << 8) | (pi[1] << 10) | (pi[2] << 12) | (pi[3] << 14);
}

// Per-thread accumulators live in shared memory (acc[r * blockDim + tid]):
// float-float pairs for complex64 states, float64 for complex128.
template <class R> struct AccSlot;
template <> struct AccSlot<float> { using T = float2; };
template <> struct AccSlot<double> { using T = double; };

__device__ __forceinline__ void acc_add(float2* a, float x) {
    Acc<float> t;
    t.hi = a->x;
    t.lo = a->y;
    t.add(x);
    a->x = t.hi;
    a->y = t.lo;
}
__device__ __forceinline__ void acc_add(double* a, double x) { *a += x; }
// a term far below the pair's rounding unit goes straight to the low word
__device__ __forceinline__ void acc_add_lo(float2* a, float x) { a->y = __fadd_rn(a->y, x); }
__device__ __forceinline__ void acc_add_lo(double* a, double x) { *a += x; }
__device__ __forceinline__ double acc_get(float2 a) { return (double)a.x + (double)a.y; }
__device__ __forceinline__ double acc_get(double a) { return a; }

// Fixed-order combination of the 32 lanes' accumulators (result in lane 0).
// Float-float pairs are added as pairs (Knuth's TwoSum of the high parts,
// the low parts folded into the error, then Dekker's Fast2Sum to
// renormalise), so complex64 reductions stay on the FP32 pipe until the
// one conversion of the total.
__device__ __forceinline__ double warp_combine(float2 a) {
    float hi = a.x, lo = a.y;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float bh = __shfl_down_sync(0xffffffffu, hi, o);
        const float bl = __shfl_down_sync(0xffffffffu, lo, o);
        const float s = __fadd_rn(hi, bh);
        const float bp = __fsub_rn(s, hi);
        float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(bh, bp));
        e = __fadd_rn(e, __fadd_rn(lo, bl));
        hi = __fadd_rn(s, e);
        lo = __fsub_rn(e, __fsub_rn(hi, s));
    }
    return (double)hi + (double)lo;
}
__device__ __forceinline__ double warp_combine(double a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    return a;
}

// shared-memory layout of k_pass: ring buffers | matrices | accumulators |
// run offsets | mbarriers
__host__ __device__ inline size_t pass_bytes_before_bars(const PassDesc& p, int threads, size_t amp) {
    const size_t acc = p.red_kind != RED_NONE ? (size_t)p.red_R * threads * 8 : 0;
    return (size_t)PASS_NBUF_H * ((size_t)1 << p.tb) * amp + (size_t)p.mat_elems * amp + acc +
           ((size_t)1 << (p.tb - p.run_bits)) * 4;
}

// Kraus probabilities: quadratic forms v^dagger F_i v over groups of the
// Kraus qubits, F_i = K_i^dagger K_i (Section III-B-2 / IV-A-4).  F holds the
// Rn forms, then their float32 residuals (complex64: each form is hi + lo)

// the weight of diagonal form f on bin r in float64: the pool's value
// (float32 for complex64) plus its float32 residual
template <class T>
__device__ __forceinline__ double diag_weight(const T* W, int R, int k, int f, int r) {
    const double w = (double)W[(f << k) + r].x;
    return sizeof(T) == 8 ? w + (double)W[(R << k) + (f << k) + r].x : w;
}

}  // namespace sv
