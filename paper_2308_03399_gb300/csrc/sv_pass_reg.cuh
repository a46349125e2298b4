// The register-resident pass kernel (k_pass_reg) and its helpers.  The
// kernel's instantiations are compiled in three translation units
// (sv_reg_c64.cu, sv_reg_c64x.cu, sv_reg_c128.cu) so that they build in
// parallel; sv_kernels.cu dispatches to them.
#pragma once

#include "sv_common.cuh"

namespace sv {

// ---------------------------------------------------------------------------
// k_pass_reg: register-resident variant for passes whose qubits (plus qubit
// 0) number WP <= 4.  Each lane holds whole groups of 2^WP amplitudes (the
// amplitudes that differ only in the pass's qubits), loads them straight
// from HBM as 128-bit pairs (qubit 0 is group bit 0), applies every fused
// stage in registers, accumulates the reduction in registers, and stores.
// One warp owns a (branch, chunk) unit; a unit's partial is combined by
// warp shuffles in a fixed order, so no block barrier is needed.
// Stage and reduction positions are group-bit indices (0..WP-1); runtime
// positions are mapped onto compile-time register indices by a switch.
// ---------------------------------------------------------------------------
template <class T, int G, int J>
__device__ __forceinline__ void reg_apply1(T* v, const T* M) {
#pragma unroll
    for (int r = 0; r < G; ++r) {
        if (r & (1 << J)) continue;
        const int r1 = r | (1 << J);
        const T a = v[r], b = v[r1];
        T x, y;
        x.x = M[0].x * a.x - M[0].y * a.y + M[1].x * b.x - M[1].y * b.y;
        x.y = M[0].x * a.y + M[0].y * a.x + M[1].x * b.y + M[1].y * b.x;
        y.x = M[2].x * a.x - M[2].y * a.y + M[3].x * b.x - M[3].y * b.y;
        y.y = M[2].x * a.y + M[2].y * a.x + M[3].x * b.y + M[3].y * b.x;
        v[r] = x;
        v[r1] = y;
    }
}

// 2-qubit matrix, matrix bit 0 on group bit J0, matrix bit 1 on group bit J1
template <class T, int G, int J0, int J1>
__device__ __forceinline__ void reg_apply2(T* v, const T* M) {
    const T* m = M;  // shared memory, read per use (keeps registers for the group)
#pragma unroll
    for (int r = 0; r < G; ++r) {
        if (r & ((1 << J0) | (1 << J1))) continue;
        const int i[4] = {r, r | (1 << J0), r | (1 << J1), r | (1 << J0) | (1 << J1)};
        T a[4], o[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) a[c] = v[i[c]];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            T acc;
            acc.x = 0;
            acc.y = 0;
#pragma unroll
            for (int c = 0; c < 4; ++c) cfma(acc, m[q * 4 + c], a[c]);
            o[q] = acc;
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) v[i[c]] = o[c];
    }
}

// structured one-qubit matrices: shape 1 diagonal, 2 anti-diagonal, +4 when
// the two nonzero entries are real (amplitude damping terms scaled by
// 1/sqrt(p)): a real diagonal costs two multiplies per amplitude
template <class T, int G, int J, int SHAPE>
__device__ __forceinline__ void reg_apply1_shape(T* v, const T* M) {
    const T m0 = (SHAPE & 3) == 1 ? M[0] : M[1], m1 = (SHAPE & 3) == 1 ? M[3] : M[2];
#pragma unroll
    for (int r = 0; r < G; ++r) {
        if (r & (1 << J)) continue;
        const int r1 = r | (1 << J);
        const T a = (SHAPE & 3) == 1 ? v[r] : v[r1], b = (SHAPE & 3) == 1 ? v[r1] : v[r];
        if (SHAPE & 4) {
            v[r].x = m0.x * a.x;
            v[r].y = m0.x * a.y;
            v[r1].x = m1.x * b.x;
            v[r1].y = m1.x * b.y;
        } else {
            v[r] = cmul(m0, a);
            v[r1] = cmul(m1, b);
        }
    }
}

template <class T, int G, int J>
__device__ __forceinline__ void reg_apply1_shaped(T* v, const T* M, int shape) {
    switch (shape) {
    case 1: reg_apply1_shape<T, G, J, 1>(v, M); break;
    case 2: reg_apply1_shape<T, G, J, 2>(v, M); break;
    case 5: reg_apply1_shape<T, G, J, 5>(v, M); break;
    default: reg_apply1_shape<T, G, J, 6>(v, M); break;
    }
}

template <class T, int G>
__device__ __forceinline__ void reg_apply1s_dyn(T* v, int j, const T* M, int shape) {
    switch (j) {
    case 0: reg_apply1_shaped<T, G, 0>(v, M, shape); break;
    case 1: if constexpr (G > 2) reg_apply1_shaped<T, G, 1>(v, M, shape); break;
    case 2: if constexpr (G > 4) reg_apply1_shaped<T, G, 2>(v, M, shape); break;
    default: if constexpr (G > 8) reg_apply1_shaped<T, G, 3>(v, M, shape); break;
    }
}

// complex64 2-qubit matrix with packed FMAs; MX holds every entry expanded as
// ((re, re), (-im, im))
template <int G, int J0, int J1>
__device__ __forceinline__ void reg_apply2_f32x2(float2* v, const ulonglong2* MX) {
#pragma unroll
    for (int r = 0; r < G; ++r) {
        if (r & ((1 << J0) | (1 << J1))) continue;
        const int i[4] = {r, r | (1 << J0), r | (1 << J1), r | (1 << J0) | (1 << J1)};
        unsigned long long ap[4], as[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            ap[c] = pk2(v[i[c]].x, v[i[c]].y);
            as[c] = pk2(v[i[c]].y, v[i[c]].x);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            unsigned long long acc = 0ull;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const ulonglong2 m = MX[q * 4 + c];
                acc = fma2(m.x, ap[c], acc);
                acc = fma2(m.y, as[c], acc);
            }
            v[i[q]] = upk2(acc);
        }
    }
}

template <int G>
__device__ __forceinline__ void reg_apply2x_dyn(float2* v, int j0, int j1, const ulonglong2* MX) {
    const int code = j0 * 4 + j1;
    switch (code) {
    case 1: if constexpr (G > 2) reg_apply2_f32x2<G, 0, 1>(v, MX); break;
    case 4: if constexpr (G > 2) reg_apply2_f32x2<G, 1, 0>(v, MX); break;
    case 2: if constexpr (G > 4) reg_apply2_f32x2<G, 0, 2>(v, MX); break;
    case 8: if constexpr (G > 4) reg_apply2_f32x2<G, 2, 0>(v, MX); break;
    case 6: if constexpr (G > 4) reg_apply2_f32x2<G, 1, 2>(v, MX); break;
    case 9: if constexpr (G > 4) reg_apply2_f32x2<G, 2, 1>(v, MX); break;
    case 3: if constexpr (G > 8) reg_apply2_f32x2<G, 0, 3>(v, MX); break;
    case 12: if constexpr (G > 8) reg_apply2_f32x2<G, 3, 0>(v, MX); break;
    case 7: if constexpr (G > 8) reg_apply2_f32x2<G, 1, 3>(v, MX); break;
    case 13: if constexpr (G > 8) reg_apply2_f32x2<G, 3, 1>(v, MX); break;
    case 11: if constexpr (G > 8) reg_apply2_f32x2<G, 2, 3>(v, MX); break;
    default: if constexpr (G > 8) reg_apply2_f32x2<G, 3, 2>(v, MX); break;
    }
}

// A monomial 2-qubit matrix (one nonzero per row and column: CX, SWAP, CZ,
// controlled phases, ...) is applied as a gather plus phases:
// out[q] = M[q][pi(q)] in[pi(q)].  Every permutation pi of the 4 indices is
// affine over GF(2), pi(q) = A q xor b, and A is a word of at most three
// elementary maps E01: (q0, q1) -> (q0, q1 xor q0) and E10: (q0, q1) ->
// (q0 xor q1, q1), each a swap of register pairs.  Words of A by index:
// I, E01, E10, E01.E10, E10.E01, E01.E10.E01 (the swap of the two bits).
template <class T, int G, int J>
__device__ __forceinline__ void reg_flip_t(T* v) {
#pragma unroll
    for (int r = 0; r < G; ++r) {
        if (r & (1 << J)) continue;
        const T t = v[r];
        v[r] = v[r | (1 << J)];
        v[r | (1 << J)] = t;
    }
}

// v[r] <-> v[r | T] for every r with bit C set and bit T clear: the gather
// of an elementary map with control bit C and target bit T
template <class T, int G, int C, int TB>
__device__ __forceinline__ void reg_cswap(T* v) {
#pragma unroll
    for (int r = 0; r < G; ++r) {
        if (!(r & (1 << C)) || (r & (1 << TB))) continue;
        const T t = v[r];
        v[r] = v[r | (1 << TB)];
        v[r | (1 << TB)] = t;
    }
}

// info: bit 1 unit phases, bits 2-3 b, bits 4-6 the word of A; ph[q] the
// phase of output q (matrix bit 0 on group bit J0, bit 1 on J1)
template <class T, int G, int J0, int J1>
__device__ __forceinline__ void reg_mono(T* v, int info, const T* ph) {
    const int b = (info >> 2) & 3, word = (info >> 4) & 7;
    if (b & 1) reg_flip_t<T, G, J0>(v);
    if (b & 2) reg_flip_t<T, G, J1>(v);
    switch (word) {  // E01 = reg_cswap<J0, J1>, E10 = reg_cswap<J1, J0>, applied left to right
    case 1: reg_cswap<T, G, J0, J1>(v); break;
    case 2: reg_cswap<T, G, J1, J0>(v); break;
    case 3: reg_cswap<T, G, J0, J1>(v); reg_cswap<T, G, J1, J0>(v); break;
    case 4: reg_cswap<T, G, J1, J0>(v); reg_cswap<T, G, J0, J1>(v); break;
    case 5: reg_cswap<T, G, J0, J1>(v); reg_cswap<T, G, J1, J0>(v); reg_cswap<T, G, J0, J1>(v); break;
    default: break;
    }
    if (!(info & 2)) {
#pragma unroll
        for (int e = 0; e < G; ++e) v[e] = cmul(ph[((e >> J0) & 1) | (((e >> J1) & 1) << 1)], v[e]);
    }
}

template <class T, int G>
__device__ __forceinline__ void reg_mono_dyn(T* v, int j0, int j1, int info, const T* ph) {
    switch (j0 * 4 + j1) {
    case 1: if constexpr (G > 2) reg_mono<T, G, 0, 1>(v, info, ph); break;
    case 4: if constexpr (G > 2) reg_mono<T, G, 1, 0>(v, info, ph); break;
    case 2: if constexpr (G > 4) reg_mono<T, G, 0, 2>(v, info, ph); break;
    case 8: if constexpr (G > 4) reg_mono<T, G, 2, 0>(v, info, ph); break;
    case 6: if constexpr (G > 4) reg_mono<T, G, 1, 2>(v, info, ph); break;
    case 9: if constexpr (G > 4) reg_mono<T, G, 2, 1>(v, info, ph); break;
    case 3: if constexpr (G > 8) reg_mono<T, G, 0, 3>(v, info, ph); break;
    case 12: if constexpr (G > 8) reg_mono<T, G, 3, 0>(v, info, ph); break;
    case 7: if constexpr (G > 8) reg_mono<T, G, 1, 3>(v, info, ph); break;
    case 13: if constexpr (G > 8) reg_mono<T, G, 3, 1>(v, info, ph); break;
    case 11: if constexpr (G > 8) reg_mono<T, G, 2, 3>(v, info, ph); break;
    default: if constexpr (G > 8) reg_mono<T, G, 3, 2>(v, info, ph); break;
    }
}

template <class T, int G, int J>
__device__ __forceinline__ void reg_flip(T* v) {
#pragma unroll
    for (int r = 0; r < G; ++r) {
        if (r & (1 << J)) continue;
        const T t = v[r];
        v[r] = v[r | (1 << J)];
        v[r | (1 << J)] = t;
    }
}

template <class T, int G>
__device__ __forceinline__ void reg_flip_dyn(T* v, int j) {
    switch (j) {
    case 0: reg_flip<T, G, 0>(v); break;
    case 1: if constexpr (G > 2) reg_flip<T, G, 1>(v); break;
    case 2: if constexpr (G > 4) reg_flip<T, G, 2>(v); break;
    default: if constexpr (G > 8) reg_flip<T, G, 3>(v); break;
    }
}

// v[e] <- v[e ^ x] for a group-bit mask x
template <class T, int G>
__device__ __forceinline__ void reg_xor_mask(T* v, int x) {
    if (x & 1) reg_flip<T, G, 0>(v);
    if constexpr (G > 2)
        if (x & 2) reg_flip<T, G, 1>(v);
    if constexpr (G > 4)
        if (x & 4) reg_flip<T, G, 2>(v);
    if constexpr (G > 8)
        if (x & 8) reg_flip<T, G, 3>(v);
}

template <class T, int G>
__device__ __forceinline__ void reg_apply1_dyn(T* v, int j, const T* M) {
    switch (j) {
    case 0: reg_apply1<T, G, 0>(v, M); break;
    case 1: if constexpr (G > 2) reg_apply1<T, G, 1>(v, M); break;
    case 2: if constexpr (G > 4) reg_apply1<T, G, 2>(v, M); break;
    default: if constexpr (G > 8) reg_apply1<T, G, 3>(v, M); break;
    }
}

template <class T, int G>
__device__ __forceinline__ void reg_apply2_dyn(T* v, int j0, int j1, const T* M) {
    const int code = j0 * 4 + j1;
    switch (code) {
    case 1: if constexpr (G > 2) reg_apply2<T, G, 0, 1>(v, M); break;
    case 4: if constexpr (G > 2) reg_apply2<T, G, 1, 0>(v, M); break;
    case 2: if constexpr (G > 4) reg_apply2<T, G, 0, 2>(v, M); break;
    case 8: if constexpr (G > 4) reg_apply2<T, G, 2, 0>(v, M); break;
    case 6: if constexpr (G > 4) reg_apply2<T, G, 1, 2>(v, M); break;
    case 9: if constexpr (G > 4) reg_apply2<T, G, 2, 1>(v, M); break;
    case 3: if constexpr (G > 8) reg_apply2<T, G, 0, 3>(v, M); break;
    case 12: if constexpr (G > 8) reg_apply2<T, G, 3, 0>(v, M); break;
    case 7: if constexpr (G > 8) reg_apply2<T, G, 1, 3>(v, M); break;
    case 13: if constexpr (G > 8) reg_apply2<T, G, 3, 1>(v, M); break;
    case 11: if constexpr (G > 8) reg_apply2<T, G, 2, 3>(v, M); break;
    default: if constexpr (G > 8) reg_apply2<T, G, 3, 2>(v, M); break;
    }
}

// quadratic forms of one-qubit Kraus terms over the pairs along group bit J
template <class R, int G, int J>
__device__ __forceinline__ void reg_forms1(const typename Cplx<R>::T* v, const typename Cplx<R>::T* F, int Rn,
                                           Acc<R>* acc) {
#pragma unroll
    for (int r = 0; r < G; ++r) {
        if (r & (1 << J)) continue;
        const auto a = v[r], b = v[r | (1 << J)];
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            if (f >= Rn) break;
            const auto* Ff = F + 4 * f;
            // Re(conj(a)(F00 a + F01 b) + conj(b)(F10 a + F11 b))
            const R fa_x = Ff[0].x * a.x - Ff[0].y * a.y + Ff[1].x * b.x - Ff[1].y * b.y;
            const R fa_y = Ff[0].x * a.y + Ff[0].y * a.x + Ff[1].x * b.y + Ff[1].y * b.x;
            const R fb_x = Ff[2].x * a.x - Ff[2].y * a.y + Ff[3].x * b.x - Ff[3].y * b.y;
            const R fb_y = Ff[2].x * a.y + Ff[2].y * a.x + Ff[3].x * b.y + Ff[3].y * b.x;
            acc[f].add(a.x * fa_x + a.y * fa_y + b.x * fb_x + b.y * fb_y);
            if constexpr (sizeof(R) == 4) {
                // the same form with the residual coefficients: far below an
                // ulp of the term, so it joins the accumulator's low word
                const auto* Fl = F + 4 * (Rn + f);
                const R la_x = Fl[0].x * a.x - Fl[0].y * a.y + Fl[1].x * b.x - Fl[1].y * b.y;
                const R la_y = Fl[0].x * a.y + Fl[0].y * a.x + Fl[1].x * b.y + Fl[1].y * b.x;
                const R lb_x = Fl[2].x * a.x - Fl[2].y * a.y + Fl[3].x * b.x - Fl[3].y * b.y;
                const R lb_y = Fl[2].x * a.y + Fl[2].y * a.x + Fl[3].x * b.y + Fl[3].y * b.x;
                acc[f].lo += a.x * la_x + a.y * la_y + b.x * lb_x + b.y * lb_y;
            }
        }
    }
}

template <class R, int G>
__device__ __forceinline__ void reg_forms1_dyn(const typename Cplx<R>::T* v, int j, const typename Cplx<R>::T* F,
                                               int Rn, Acc<R>* acc) {
    switch (j) {
    case 0: reg_forms1<R, G, 0>(v, F, Rn, acc); break;
    case 1: if constexpr (G > 2) reg_forms1<R, G, 1>(v, F, Rn, acc); break;
    case 2: if constexpr (G > 4) reg_forms1<R, G, 2>(v, F, Rn, acc); break;
    default: if constexpr (G > 8) reg_forms1<R, G, 3>(v, F, Rn, acc); break;
    }
}

constexpr int REG_MAX_RED = 4;
constexpr int REG_MAX_BINS = 16;  // measurement outcomes a register pass reduces (k <= 4)

// Diagonal forms (sum_r w_f[r] |v_r|^2 over the 2^k amplitudes of the
// reduced qubits) are linear in the 2^k bins of |v|^2, so a unit only
// accumulates the bins: every group collects |v|^2 into the bins of the
// reduced qubits (compile-time bin of each amplitude, float32 within the
// group) and adds them to the float-float bin accumulators.  The weights
// are applied once per unit, in float64 (any number of forms, weights at
// full precision).
template <class R, int G, int J0, int J1>
__device__ __forceinline__ void reg_diag_bins(const typename Cplx<R>::T* v, R* q) {
#pragma unroll
    for (int e = 0; e < G; ++e) {
        const int idx = ((e >> J0) & 1) | (J1 >= 0 ? ((e >> (J1 < 0 ? 0 : J1)) & 1) << 1 : 0);
        q[idx] += v[e].x * v[e].x + v[e].y * v[e].y;
    }
}

template <class R, int G>
__device__ __forceinline__ void reg_diag(const typename Cplx<R>::T* v, const PassDesc& p, Acc<R>* acc) {
    R q[4] = {0, 0, 0, 0};
    if (p.red_k == 1) {
        switch (p.red_pos[0]) {
        case 0: reg_diag_bins<R, G, 0, -1>(v, q); break;
        case 1: if constexpr (G > 2) reg_diag_bins<R, G, 1, -1>(v, q); break;
        case 2: if constexpr (G > 4) reg_diag_bins<R, G, 2, -1>(v, q); break;
        default: if constexpr (G > 8) reg_diag_bins<R, G, 3, -1>(v, q); break;
        }
    } else {
        switch (p.red_pos[0] * 4 + p.red_pos[1]) {
        case 1: if constexpr (G > 2) reg_diag_bins<R, G, 0, 1>(v, q); break;
        case 4: if constexpr (G > 2) reg_diag_bins<R, G, 1, 0>(v, q); break;
        case 2: if constexpr (G > 4) reg_diag_bins<R, G, 0, 2>(v, q); break;
        case 8: if constexpr (G > 4) reg_diag_bins<R, G, 2, 0>(v, q); break;
        case 6: if constexpr (G > 4) reg_diag_bins<R, G, 1, 2>(v, q); break;
        case 9: if constexpr (G > 4) reg_diag_bins<R, G, 2, 1>(v, q); break;
        case 3: if constexpr (G > 8) reg_diag_bins<R, G, 0, 3>(v, q); break;
        case 12: if constexpr (G > 8) reg_diag_bins<R, G, 3, 0>(v, q); break;
        case 7: if constexpr (G > 8) reg_diag_bins<R, G, 1, 3>(v, q); break;
        case 13: if constexpr (G > 8) reg_diag_bins<R, G, 3, 1>(v, q); break;
        case 11: if constexpr (G > 8) reg_diag_bins<R, G, 2, 3>(v, q); break;
        default: if constexpr (G > 8) reg_diag_bins<R, G, 3, 2>(v, q); break;
        }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
        if (r < (1 << p.red_k)) acc[r].add(q[r]);
}

// CTA shape of the register path: complex64 at 128 threads and up to 96
// registers (five CTAs, 20 warps per SM; the pass is latency-bound, so
// resident warps matter more than a few spilled words); complex128 at 256
// threads, where the same cap would spill kilobytes
constexpr int REG_PREFETCH = 1;  // groups ahead of a lane's loads that go to L2

template <class R> struct RegCta;
template <> struct RegCta<float> { static constexpr int threads = 128, min_blocks = 5; };
template <> struct RegCta<double> { static constexpr int threads = 256, min_blocks = 1; };


// register-kernel variants: stage by stage, folded (no reduction), and
// stage by stage with measurement bins (complex64)
constexpr int REG_PLAIN = 0, REG_FOLD = 1, REG_BINS = 2;

template <class R, int WP, int PAIRED, int VAR>
__global__ void __launch_bounds__(RegCta<R>::threads, RegCta<R>::min_blocks)
    k_pass_reg(DevBatch d, const __grid_constant__ PassDesc p) {
    constexpr bool FOLD = VAR == REG_FOLD, BINS = VAR == REG_BINS;
    using T = typename Cplx<R>::T;
    constexpr int G = 1 << WP;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    // shared memory, each region one slice per warp: matrices | stage
    // choice, packed form, scale (4 x MAX_STAGES words) | complex64 only:
    // the matrices expanded for packed FMAs | the folded matrix (G x G)
    const int mat_stride = (p.mat_elems + 1) & ~1;
    T* const mats_all = reinterpret_cast<T*>(smem_raw);
    int* const words_all = reinterpret_cast<int*>(mats_all + (size_t)nwarps * mat_stride);
    ulonglong2* const matx_all = reinterpret_cast<ulonglong2*>(words_all + (size_t)nwarps * 4 * MAX_STAGES);
    T* mats = mats_all + (size_t)warp * mat_stride;
    int* w_sel = words_all + (size_t)warp * 4 * MAX_STAGES;
    int* w_packed = w_sel + MAX_STAGES;
    double* w_scale = reinterpret_cast<double*>(w_sel + 2 * MAX_STAGES);
    ulonglong2* matx = matx_all + (size_t)warp * mat_stride;
    float4* fold_m = reinterpret_cast<float4*>(matx_all + (size_t)nwarps * mat_stride) + (size_t)warp * (G / 2) * G;
    // measurement bins (RED_BINS): per warp, bin r of lane l at bins[r * 32 + l]
    // (float-float pairs for complex64), after the folded matrices (none in
    // a pass with a reduction) and, for complex64, the expanded matrices
    using AS = typename AccSlot<R>::T;
    AS* const bins_all = reinterpret_cast<AS*>(reinterpret_cast<unsigned char*>(matx_all) +
                                               (sizeof(T) == 8 ? (size_t)nwarps * mat_stride * 16 : 0));
    AS* bins = bins_all + (size_t)warp * REG_MAX_BINS * 32;
    // bin of each group element: 4 bits per element
    uint64_t binmap = 0;
    if constexpr (BINS)
        for (int e = 0; e < G; ++e) {
            uint64_t bi = 0;
            for (int j = 0; j < p.red_k; ++j) bi |= (uint64_t)((e >> p.red_pos[j]) & 1) << j;
            binmap |= bi << (4 * e);
        }
    uint64_t skipmask = 0;
    // every stage of the pass, in op order, on one group of G amplitudes
    auto apply_stages = [&](T (&v)[G]) {
        for (int s = 0; s < p.n_stages; ++s) {
            if ((skipmask >> s) & 1) continue;
            const Stage& st = p.st[s];
            if (st.kind == ST_DENSE || st.kind == ST_DENSE_BR) {
                if (st.k == 1) {
                    const int shape = w_packed[s];
                    if (shape) reg_apply1s_dyn<T, G>(v, st.pos[0], mats + st.mat, shape);
                    else reg_apply1_dyn<T, G>(v, st.pos[0], mats + st.mat);
                } else if (const int mi = w_packed[s]) {
                    reg_mono_dyn<T, G>(v, st.pos[0], st.pos[1], mi, mats + st.mat);
                } else {
                    if constexpr (sizeof(T) == 8)
                        reg_apply2x_dyn<G>(reinterpret_cast<float2*>(v), st.pos[0], st.pos[1], matx + st.mat);
                    else
                        reg_apply2_dyn<T, G>(v, st.pos[0], st.pos[1], mats + st.mat);
                }
            } else if (st.kind == ST_PAULI_BR) {
                // out[e] = (-i)^ny (-1)^popcount(z & e) in[e ^ x]
                const int info = w_packed[s];
                reg_xor_mask<T, G>(v, info & 15);
                const bool rot = (info >> 4) & 1;
                const int sign = info >> 8;
#pragma unroll
                for (int e = 0; e < G; ++e) {
                    T t = v[e];
                    if (rot) {
                        const R x = t.x;
                        t.x = t.y;
                        t.y = -x;
                    }
                    if ((sign >> e) & 1) {
                        t.x = -t.x;
                        t.y = -t.y;
                    }
                    v[e] = t;
                }
            } else {  // ST_PROJ_BR
                const int info = w_packed[s];
                const R sc = mats[st.mat].x;
#pragma unroll
                for (int e = 0; e < G; ++e) {
                    if ((info >> e) & 1) {
                        v[e].x *= sc;
                        v[e].y *= sc;
                    } else {
                        v[e].x = 0;
                        v[e].y = 0;
                    }
                }
                reg_xor_mask<T, G>(v, (info >> 16) & 15);
            }
        }
    };

    const int n_br = d.ctl[CTL_NBR];
    if (blockIdx.x == 0 && threadIdx.x == 0 && d.pass_log) {
        const int i = atomicAdd(&d.ctl[CTL_NPASS], 1);
        if (i < d.pass_log_cap) d.pass_log[i] = n_br;
    }
    // group offsets: element e of a group sits at base + off[e]
    // element e of a group sits at base + sum of stride[j] over its set bits
    int stride[WP];
#pragma unroll
    for (int j = 0; j < WP; ++j) stride[j] = 1 << p.tile_q[j];
    const int64_t units = (int64_t)n_br * p.chunks;
    const int64_t gw = (int64_t)blockIdx.x * nwarps + warp, tw = (int64_t)gridDim.x * nwarps;
    const int64_t u0 = units * gw / tw, u1 = units * (gw + 1) / tw;
    const int64_t gpu = (d.dim >> WP) / p.chunks;  // groups per unit
    const bool red = p.red_kind != RED_NONE;
    T* const states = reinterpret_cast<T*>(d.states);
    const R* pool = reinterpret_cast<const R*>(d.pool);
    int cur_b = -1;
    for (int64_t u = u0; u < u1; ++u) {
        const int b = (int)(u / p.chunks);
        const int c = (int)(u % p.chunks);
        const int slot = d.br_slot[b];
        if (slot < 0 || slot >= d.n_slots) {
            if (lane == 0) set_err(d, ERR_SLOT, b);
            continue;
        }
        if (b != cur_b) {
            const uint64_t clb = d.br_clbits[b];
            // the shared gates' matrices (and the reduction's coefficients)
            // are loaded for the warp's first branch only; a branch's own
            // stages (choices, parameter sets) on every branch change
            const bool first = cur_b < 0;
            __syncwarp();
            // each lane takes its stages' choices: the loads of different
            // stages overlap instead of forming one chain per stage
            skipmask = 0;
            for (int s0 = 0; s0 < p.n_stages; s0 += 32) {
                const int s = s0 + lane;
                int sk = 0;
                if (s < p.n_stages) {
                    const Stage& st = p.st[s];
                    int sel = 0, packed = 0;
                    double scale = 1.0;
                    if (st.cond_clbit >= 0 && (int)((clb >> st.cond_clbit) & 1ull) != st.cond_val) sk = 1;
                    if (st.kind == ST_DENSE) {
                        // only its condition is per branch
                    } else if (st.pre) {  // batch mode: the branch's one shot, pre-drawn
                        sel = d.pre_sel[(int64_t)st.pend * d.cap_br + d.perm[d.br_start[b]]];
                        packed = d.ipool[st.off + sel];
                        if ((packed & 0xff) == 0) sk = 1;
                    } else if (st.pend == PEND_PSET) {  // the branch's parameter set
                        sel = d.br_pset[b];
                    } else {
                        sel = d.br_sel[(int64_t)st.pend * d.cap_br + b];
                        scale = d.br_scale[(int64_t)st.pend * d.cap_br + b];
                        if (sel < 0) sk = 1;
                        if (st.kind == ST_PAULI_BR && !sk) {
                            packed = d.ipool[st.off + sel];
                            if ((packed & 0xff) == 0) sk = 1;
                        }
                    }
                    // Pauli and projection stages in group form, once per
                    // branch: Pauli: bits 0-3 flip mask, bit 4 the (-i)
                    // factor, bits 8+ the sign of each group element;
                    // projection: bits 0-15 the kept elements, bits 16-19 the
                    // flips of a reset
                    if (!sk && st.kind == ST_PAULI_BR) {
                        const int xm = packed & 15, zm = (packed >> 4) & 15, ny = (packed >> 8) & 3;
                        int xg = 0, zg = 0;
                        for (int j = 0; j < st.k; ++j) {
                            if ((xm >> j) & 1) xg |= 1 << st.pos[j];
                            if ((zm >> j) & 1) zg |= 1 << st.pos[j];
                        }
                        int sign = 0;
                        for (int e = 0; e < G; ++e)
                            if ((((ny >> 1) & 1) ^ (__popc(zg & e) & 1)) != 0) sign |= 1 << e;
                        w_packed[s] = xg | ((ny & 1) << 4) | (sign << 8);
                    } else if (!sk && st.kind == ST_PROJ_BR) {
                        int keep = 0, xr = 0;
                        for (int e = 0; e < G; ++e) {
                            int o = 0;
                            for (int j = 0; j < st.k; ++j) o |= ((e >> st.pos[j]) & 1) << j;
                            if (o == sel) keep |= 1 << e;
                        }
                        if (st.reset)
                            for (int j = 0; j < st.k; ++j)
                                if ((sel >> j) & 1) xr |= 1 << st.pos[j];
                        w_packed[s] = keep | (xr << 16);
                    }
                    w_sel[s] = sel;
                    w_scale[s] = scale;
                }
                skipmask |= (uint64_t)__ballot_sync(0xffffffffu, sk) << s0;
            }
            __syncwarp();
            // matrices: lanes over a stage's entries
            for (int s = 0; s < p.n_stages; ++s) {
                const Stage& st = p.st[s];
                if (st.kind == ST_DENSE ? !first : ((skipmask >> s) & 1)) continue;
                if (st.kind == ST_DENSE || st.kind == ST_DENSE_BR) {
                    const int D2 = 1 << (2 * st.k);
                    const R* src = pool + st.off + (st.kind == ST_DENSE_BR ? (int64_t)w_sel[s] * st.stride : 0);
                    const R sc = (R)w_scale[s];
                    for (int e = lane; e < D2; e += 32) {
                        T m;
                        m.x = src[2 * e] * sc;
                        m.y = src[2 * e + 1] * sc;
                        mats[st.mat + e] = m;
                        if constexpr (sizeof(T) == 8)
                            matx[st.mat + e] = make_ulonglong2(pk2((float)m.x, (float)m.x), pk2(-(float)m.y, (float)m.y));
                    }
                    if (st.k == 2) {
                        // a monomial matrix (permutation times phases) moves
                        // registers instead of multiplying: its structure to
                        // w_packed, its phases over the matrix's first entries
                        __syncwarp();
                        if (lane == 0) {
                            T m[16], ph[4];
                            for (int e = 0; e < 16; ++e) m[e] = mats[st.mat + e];
                            const int mi = mono_info(m, ph);
                            if (mi)
                                for (int q = 0; q < 4; ++q) mats[st.mat + q] = ph[q];
                            w_packed[s] = mi;
                        }
                    }
                    if (st.k == 1 && lane == 0) {
                        // structure of a one-qubit matrix: 1 diagonal, 2 anti-diagonal, +4 real
                        const bool off0 = src[2] == 0 && src[3] == 0 && src[4] == 0 && src[5] == 0;
                        const bool diag0 = src[0] == 0 && src[1] == 0 && src[6] == 0 && src[7] == 0;
                        int shape = off0 ? 1 : (diag0 ? 2 : 0);
                        if (shape == 1 && src[1] == 0 && src[7] == 0) shape |= 4;
                        if (shape == 2 && src[3] == 0 && src[5] == 0) shape |= 4;
                        w_packed[s] = shape;
                    }
                } else if (st.kind == ST_PROJ_BR && lane == 0) {
                    T m;
                    m.x = (R)w_scale[s];
                    m.y = 0;
                    mats[st.mat] = m;
                }
            }
            if (first && (p.red_kind == RED_FORMS || p.red_kind == RED_DIAG)) {  // coefficients, then residuals
                const int E2 = 2 * (p.red_kind == RED_FORMS ? 4 * p.red_R : p.red_R << p.red_k);
                const R* src = pool + p.red_off;
                for (int e = lane; e < E2; e += 32) {
                    T m;
                    m.x = src[2 * e];
                    m.y = src[2 * e + 1];
                    mats[p.mat_elems - E2 + e] = m;
                }
            }
            __syncwarp();
            if constexpr (FOLD && sizeof(T) == 8) {
                // lane c < G runs the stages on the unit vector e_c: its
                // result is column c of the pass's matrix for this branch
                T col[G];
#pragma unroll
                for (int e = 0; e < G; ++e) {
                    col[e].x = e == lane ? (R)1 : (R)0;
                    col[e].y = 0;
                }
                apply_stages(col);
                // rows r and r + 1 of column c side by side: one 128-bit
                // load per column serves two output rows
                if (lane < G)
#pragma unroll
                    for (int r = 0; r < G; r += 2)
                        fold_m[(r / 2) * G + lane] = make_float4(col[r].x, col[r].y, col[r + 1].x, col[r + 1].y);
                __syncwarp();
            }
            cur_b = b;
        }
        Acc<R> acc[REG_MAX_RED];
#pragma unroll
        for (int r = 0; r < REG_MAX_RED; ++r) acc[r].zero();
        if constexpr (BINS)
            for (int r = 0; r < (1 << p.red_k); ++r) bins[r * 32 + lane] = AS{};
        T* gstate = states + (int64_t)slot * d.dim;
        for (int64_t gi = lane; gi < gpu; gi += 32) {
            // base: the group index with zeros inserted at the group qubits
            // (32-bit: a state has at most 2^30 amplitudes)
            auto group_base = [&](int64_t gidx) {
                uint32_t bb = (uint32_t)gidx;
#pragma unroll
                for (int j = 0; j < WP; ++j) {
                    const uint32_t lowm = (uint32_t)stride[j] - 1u;
                    bb = ((bb & ~lowm) << 1) | (bb & lowm);
                }
                return bb;
            };
            const uint32_t base = group_base(c * gpu + gi);
            T* g = gstate + base;
            auto off = [&](int e) {
                int o = 0;
#pragma unroll
                for (int j = 0; j < WP; ++j)
                    if ((e >> j) & 1) o += stride[j];
                return o;
            };
            // the lane's next group goes to L2 ahead of its loads (no
            // registers held): the pass is latency-bound at 20 warps per SM
            if (gi + 32 * REG_PREFETCH < gpu) {
                const T* gn = gstate + group_base(c * gpu + gi + 32 * REG_PREFETCH);
#pragma unroll
                for (int e = 0; e < G; e += (sizeof(T) == 8 && PAIRED) ? 2 : 1)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(gn + off(e)));
            }
            T v[G];
            if constexpr (sizeof(T) == 8 && PAIRED) {
#pragma unroll
                for (int e = 0; e < G; e += 2) {
                    const float4 x = *reinterpret_cast<const float4*>(g + off(e));
                    v[e].x = x.x;
                    v[e].y = x.y;
                    v[e + 1].x = x.z;
                    v[e + 1].y = x.w;
                }
            } else {
#pragma unroll
                for (int e = 0; e < G; ++e) v[e] = g[off(e)];
            }
            if constexpr (FOLD && sizeof(T) == 8) {
                // the pass's stages folded into one G x G matrix (rows r and
                // r + 1 of column c at fold_m[(r / 2) * G + c]); a folded pass
                // has no reduction, so each pair of output rows is stored as
                // soon as it is formed
#pragma unroll 1
                for (int r = 0; r < G; r += 2) {
                    float2 o0 = make_float2(0.f, 0.f), o1 = make_float2(0.f, 0.f);
#pragma unroll
                    for (int c2 = 0; c2 < G; ++c2) {
                        const float4 m = fold_m[(r / 2) * G + c2];
                        const float2 a = v[c2];
                        o0.x = fmaf(m.x, a.x, fmaf(-m.y, a.y, o0.x));
                        o0.y = fmaf(m.x, a.y, fmaf(m.y, a.x, o0.y));
                        o1.x = fmaf(m.z, a.x, fmaf(-m.w, a.y, o1.x));
                        o1.y = fmaf(m.z, a.y, fmaf(m.w, a.x, o1.y));
                    }
                    if constexpr (PAIRED) {
                        *reinterpret_cast<float4*>(g + off(r)) = make_float4(o0.x, o0.y, o1.x, o1.y);
                    } else {
                        g[off(r)] = o0;
                        g[off(r + 1)] = o1;
                    }
                }
            } else {
                apply_stages(v);
                if (p.red_kind == RED_FORMS)
                    reg_forms1_dyn<R, G>(v, p.red_pos[0], mats + p.mat_elems - 8 * p.red_R, p.red_R, acc);
                else if (p.red_kind == RED_DIAG)
                    reg_diag<R, G>(v, p, acc);
                if constexpr (BINS) {
                    // each lane owns its column of the bins: no races
#pragma unroll
                    for (int e = 0; e < G; ++e) {
                        const int bi = (int)((binmap >> (4 * e)) & 15);
                        const R x = v[e].x * v[e].x + v[e].y * v[e].y;
                        if constexpr (sizeof(R) == 4) acc_add(&bins[bi * 32 + lane], x);
                        else bins[bi * 32 + lane] += x;
                    }
                }
                if (p.store) {
                    if constexpr (sizeof(T) == 8 && PAIRED) {
#pragma unroll
                        for (int e = 0; e < G; e += 2)
                            *reinterpret_cast<float4*>(g + off(e)) = make_float4(v[e].x, v[e].y, v[e + 1].x, v[e + 1].y);
                    } else {
#pragma unroll
                        for (int e = 0; e < G; ++e) g[off(e)] = v[e];
                    }
                }
            }
        }
        if (red && p.red_kind == RED_DIAG) {
            // the unit's bins (fixed shuffle tree, float64), then every form
            // from them: lane f writes form f
            const int D = 1 << p.red_k;
            double bin[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                double x = r < D ? acc[r].get() : 0.0;
                if (r < D)
                    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                bin[r] = x;
            }
            if (lane < p.red_R) {
                const T* W = mats + p.mat_elems - 2 * (p.red_R << p.red_k);
                double part = 0.0;
#pragma unroll
                for (int r = 0; r < 4; ++r)
                    if (r < D) part += diag_weight(W, p.red_R, p.red_k, lane, r) * bin[r];
                d.partials[((int64_t)slot * d.max_chunks + c) * MAX_RED + lane] = part;
            }
        } else if (BINS) {
            // every outcome's bin: a fixed float64 shuffle tree over the lanes
            for (int r = 0; r < (1 << p.red_k); ++r) {
                const AS a = bins[r * 32 + lane];
                double x;
                if constexpr (sizeof(R) == 4) x = (double)a.x + (double)a.y;
                else x = a;
                for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
                if (lane == 0) d.partials[((int64_t)slot * d.max_chunks + c) * MAX_RED + r] = x;
            }
        } else if (red) {
#pragma unroll
            for (int r = 0; r < REG_MAX_RED; ++r) {
                if (r >= p.red_R) break;
                // a unit is short: a float64 shuffle tree costs less here
                // than float-float pairs
                double x = acc[r].get();
                for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
                if (lane == 0) d.partials[((int64_t)slot * d.max_chunks + c) * MAX_RED + r] = x;
            }
        }
    }
}

}  // namespace sv
