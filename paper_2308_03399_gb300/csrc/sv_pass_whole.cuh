// Whole-state warp passes (SV_OPT_WHOLE_STATE) for complex64 states of 9 or
// 10 qubits, passes without a reduction.  One warp holds a branch's state:
// lane l holds amplitudes [l G, (l + 1) G), G = 2^(n - 5); physical bits
// 0..NREG-1 index the registers, the rest the lane.  Before each stage its
// qubits are brought into register bits 0..3 by exchanging bits (register
// pairs renamed, or one value per pair crossing lanes by a shuffle), and the
// stage runs on each 16-register group with the register kernel's code; the
// identity layout is restored before the store.  Every stage of the pass
// runs without a block barrier or a trip to memory.
#pragma once
#include "sv_pass_reg.cuh"

namespace sv {

// exchange register bit J with lane bit b: per pair one value crosses lanes
template <int NREG, int J>
__device__ __forceinline__ void ws_swap_reg_lane(float2* v, int b, int lane) {
    const bool hi = (lane >> b) & 1;
#pragma unroll
    for (int r = 0; r < (1 << NREG); ++r) {
        if (r & (1 << J)) continue;
        const int r1 = r | (1 << J);
        const float2 s = hi ? v[r] : v[r1];
        float2 t;
        t.x = __shfl_xor_sync(0xffffffffu, s.x, 1 << b);
        t.y = __shfl_xor_sync(0xffffffffu, s.y, 1 << b);
        if (hi) v[r] = t;
        else v[r1] = t;
    }
}

template <int NREG>
__device__ __forceinline__ void ws_swap_reg_lane_dyn(float2* v, int j, int b, int lane) {
    switch (j) {
    case 0: ws_swap_reg_lane<NREG, 0>(v, b, lane); break;
    case 1: ws_swap_reg_lane<NREG, 1>(v, b, lane); break;
    case 2: ws_swap_reg_lane<NREG, 2>(v, b, lane); break;
    case 3: ws_swap_reg_lane<NREG, 3>(v, b, lane); break;
    default: if constexpr (NREG > 4) ws_swap_reg_lane<NREG, 4>(v, b, lane); break;
    }
}

// exchange register bits J and K (a rename of register pairs)
template <int NREG, int J, int K>
__device__ __forceinline__ void ws_swap_reg_reg(float2* v) {
#pragma unroll
    for (int r = 0; r < (1 << NREG); ++r) {
        if (!((r >> J) & 1) || ((r >> K) & 1)) continue;
        const int r2 = r ^ (1 << J) ^ (1 << K);
        const float2 t = v[r];
        v[r] = v[r2];
        v[r2] = t;
    }
}

template <int NREG>
__device__ __forceinline__ void ws_swap_reg_reg_dyn(float2* v, int j, int k) {
    if (j > k) { const int t = j; j = k; k = t; }
    switch (j * 8 + k) {
    case 1: ws_swap_reg_reg<NREG, 0, 1>(v); break;
    case 2: ws_swap_reg_reg<NREG, 0, 2>(v); break;
    case 3: ws_swap_reg_reg<NREG, 0, 3>(v); break;
    case 10: ws_swap_reg_reg<NREG, 1, 2>(v); break;
    case 11: ws_swap_reg_reg<NREG, 1, 3>(v); break;
    case 19: ws_swap_reg_reg<NREG, 2, 3>(v); break;
    case 4: if constexpr (NREG > 4) ws_swap_reg_reg<NREG, 0, 4>(v); break;
    case 12: if constexpr (NREG > 4) ws_swap_reg_reg<NREG, 1, 4>(v); break;
    case 20: if constexpr (NREG > 4) ws_swap_reg_reg<NREG, 2, 4>(v); break;
    case 28: if constexpr (NREG > 4) ws_swap_reg_reg<NREG, 3, 4>(v); break;
    default: break;
    }
}

// exchange lane bits b and c: lanes whose two bits differ trade everything
template <int NREG>
__device__ __forceinline__ void ws_swap_lane_lane(float2* v, int b, int c, int lane) {
    const unsigned m = (1u << b) | (1u << c);
    const bool differ = ((lane >> b) & 1) != ((lane >> c) & 1);
#pragma unroll
    for (int r = 0; r < (1 << NREG); ++r) {
        float2 t;
        t.x = __shfl_xor_sync(0xffffffffu, v[r].x, m);
        t.y = __shfl_xor_sync(0xffffffffu, v[r].y, m);
        if (differ) v[r] = t;
    }
}

// logical qubit -> physical bit, 4 bits per qubit (n <= 10 -> 40 bits)
struct WsPerm {
    uint64_t f;
    __device__ __forceinline__ int phys(int q) const { return (int)((f >> (4 * q)) & 15); }
    __device__ __forceinline__ void set(int q, int p) { f = (f & ~(15ull << (4 * q))) | ((uint64_t)p << (4 * q)); }
    __device__ __forceinline__ int at(int p, int n) const {
        for (int q = 0; q < n; ++q)
            if (phys(q) == p) return q;
        return -1;
    }
};

// every qubit of qs[0..k-1] into register bits 0..3
template <int NREG>
__device__ __forceinline__ void ws_bring_in(float2* v, WsPerm& P, const int32_t* qs, int k, int n, int lane) {
    for (int i = 0; i < k; ++i) {
        const int p = P.phys(qs[i]);
        if (p < 4) continue;
        int j = 0;
        for (; j < 4; ++j) {
            bool used = false;
            for (int t = 0; t < k; ++t) used = used || P.phys(qs[t]) == j;
            if (!used) break;
        }
        const int victim = P.at(j, n);
        if (p < NREG) ws_swap_reg_reg_dyn<NREG>(v, j, p);
        else ws_swap_reg_lane_dyn<NREG>(v, j, p - NREG, lane);
        P.set(victim, p);
        P.set(qs[i], j);
    }
}

// back to the identity layout (lane qubits home, lanes in order, registers in order)
template <int NREG>
__device__ __forceinline__ void ws_restore(float2* v, WsPerm& P, int n, int lane) {
    for (bool changed = true; changed;) {
        changed = false;
        for (int j = 0; j < NREG; ++j) {
            const int q = P.at(j, n);
            if (q >= NREG) {
                const int other = P.at(q, n);  // the qubit in q's home lane bit
                ws_swap_reg_lane_dyn<NREG>(v, j, q - NREG, lane);
                P.set(q, q);
                P.set(other, j);
                changed = true;
            }
        }
    }
    for (int b = 0; b < n - NREG; ++b) {
        const int q = P.at(NREG + b, n);
        if (q != NREG + b) {
            const int c = P.phys(NREG + b) - NREG;
            ws_swap_lane_lane<NREG>(v, b, c, lane);
            P.set(q, NREG + c);
            P.set(NREG + b, NREG + b);
        }
    }
    for (int j = 0; j < NREG; ++j) {
        const int q = P.at(j, n);
        if (q != j) {
            const int k = P.phys(j);
            ws_swap_reg_reg_dyn<NREG>(v, j, k);
            P.set(q, k);
            P.set(j, j);
        }
    }
}


// one stage on a 16-amplitude register group with explicit positions (< 4);
// Pauli and projection masks are formed here from the raw choice
template <class T>
__device__ __forceinline__ void ws_apply_one(T* v, const Stage& st, const int* pos, int packed, int sel, const T* M,
                                             const ulonglong2* MX) {
    constexpr int G = 16;
    if (st.kind == ST_DENSE || st.kind == ST_DENSE_BR) {
        if (st.k == 1) {
            if (packed) reg_apply1s_dyn<T, G>(v, pos[0], M, packed);
            else reg_apply1_dyn<T, G>(v, pos[0], M);
        } else if (packed) {
            reg_mono_dyn<T, G>(v, pos[0], pos[1], packed, M);
        } else {
            reg_apply2x_dyn<G>(reinterpret_cast<float2*>(v), pos[0], pos[1], MX);
        }
    } else if (st.kind == ST_PAULI_BR) {
        const int xm = packed & 15, zm = (packed >> 4) & 15, ny = (packed >> 8) & 3;
        int xg = 0, zg = 0;
        for (int j = 0; j < st.k; ++j) {
            if ((xm >> j) & 1) xg |= 1 << pos[j];
            if ((zm >> j) & 1) zg |= 1 << pos[j];
        }
        reg_xor_mask<T, G>(v, xg);
#pragma unroll
        for (int e = 0; e < G; ++e) {
            T t = v[e];
            if (ny & 1) {
                const float x = t.x;
                t.x = t.y;
                t.y = -x;
            }
            if ((((ny >> 1) & 1) ^ (__popc(zg & e) & 1)) != 0) {
                t.x = -t.x;
                t.y = -t.y;
            }
            v[e] = t;
        }
    } else {  // ST_PROJ_BR
        int keep = 0, xr = 0;
        for (int e = 0; e < G; ++e) {
            int o = 0;
            for (int j = 0; j < st.k; ++j) o |= ((e >> pos[j]) & 1) << j;
            if (o == sel) keep |= 1 << e;
        }
        if (st.reset)
            for (int j = 0; j < st.k; ++j)
                if ((sel >> j) & 1) xr |= 1 << pos[j];
        const float sc = M[0].x;
#pragma unroll
        for (int e = 0; e < G; ++e) {
            if ((keep >> e) & 1) {
                v[e].x *= sc;
                v[e].y *= sc;
            } else {
                v[e].x = 0;
                v[e].y = 0;
            }
        }
        reg_xor_mask<T, G>(v, xr);
    }
}


// k_pass_whole: a pass over a whole n-qubit state (n = NREG + 5) held by one
// warp; no reduction.  Shared memory as k_pass_reg (matrices, stage words,
// expanded matrices per warp).
template <int NREG>
__global__ void __launch_bounds__(128, NREG > 4 ? 2 : 4) k_pass_whole(DevBatch d, const __grid_constant__ PassDesc p) {
    using T = float2;
    constexpr int G = 1 << NREG, NH = G / 16;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const int mat_stride = (p.mat_elems + 1) & ~1;
    T* const mats_all = reinterpret_cast<T*>(smem_raw);
    int* const words_all = reinterpret_cast<int*>(mats_all + (size_t)nwarps * mat_stride);
    ulonglong2* const matx_all = reinterpret_cast<ulonglong2*>(words_all + (size_t)nwarps * 4 * MAX_STAGES);
    T* mats = mats_all + (size_t)warp * mat_stride;
    int* w_sel = words_all + (size_t)warp * 4 * MAX_STAGES;
    int* w_packed = w_sel + MAX_STAGES;
    double* w_scale = reinterpret_cast<double*>(w_sel + 2 * MAX_STAGES);
    ulonglong2* matx = matx_all + (size_t)warp * mat_stride;
    const int n = p.n;
    const int n_br = d.ctl[CTL_NBR];
    if (blockIdx.x == 0 && threadIdx.x == 0 && d.pass_log) {
        const int i = atomicAdd(&d.ctl[CTL_NPASS], 1);
        if (i < d.pass_log_cap) d.pass_log[i] = n_br;
    }
    T* const states = reinterpret_cast<T*>(d.states);
    const float* pool = reinterpret_cast<const float*>(d.pool);
    bool first = true;
    for (int b = blockIdx.x * nwarps + warp; b < n_br; b += gridDim.x * nwarps) {
        const int slot = d.br_slot[b];
        if (slot < 0 || slot >= d.n_slots) {
            if (lane == 0) set_err(d, ERR_SLOT, b);
            continue;
        }
        const uint64_t clb = d.br_clbits[b];
        __syncwarp();
        uint64_t skipmask = 0;
        for (int s0 = 0; s0 < p.n_stages; s0 += 32) {
            const int s = s0 + lane;
            int sk = 0;
            if (s < p.n_stages) {
                const Stage& st = p.st[s];
                int sel = 0, packed = 0;
                double scale = 1.0;
                if (st.cond_clbit >= 0 && (int)((clb >> st.cond_clbit) & 1ull) != st.cond_val) sk = 1;
                if (st.kind == ST_DENSE) {
                } else if (st.pre) {
                    sel = d.pre_sel[(int64_t)st.pend * d.cap_br + d.perm[d.br_start[b]]];
                    packed = d.ipool[st.off + sel];
                    if ((packed & 0xff) == 0) sk = 1;
                } else if (st.pend == PEND_PSET) {
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
                if (!sk && st.kind == ST_PAULI_BR) w_packed[s] = packed;  // raw: masks at apply time
                w_sel[s] = sel;
                w_scale[s] = scale;
            }
            skipmask |= (uint64_t)__ballot_sync(0xffffffffu, sk) << s0;
        }
        __syncwarp();
        for (int s = 0; s < p.n_stages; ++s) {
            const Stage& st = p.st[s];
            if (st.kind == ST_DENSE ? !first : ((skipmask >> s) & 1)) continue;
            if (st.kind == ST_DENSE || st.kind == ST_DENSE_BR) {
                const int D2 = 1 << (2 * st.k);
                const float* src = pool + st.off + (st.kind == ST_DENSE_BR ? (int64_t)w_sel[s] * st.stride : 0);
                const float sc = (float)w_scale[s];
                for (int e = lane; e < D2; e += 32) {
                    T m;
                    m.x = src[2 * e] * sc;
                    m.y = src[2 * e + 1] * sc;
                    mats[st.mat + e] = m;
                    matx[st.mat + e] = make_ulonglong2(pk2(m.x, m.x), pk2(-m.y, m.y));
                }
                if (st.k == 2) {
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
                    const bool off0 = src[2] == 0 && src[3] == 0 && src[4] == 0 && src[5] == 0;
                    const bool diag0 = src[0] == 0 && src[1] == 0 && src[6] == 0 && src[7] == 0;
                    int shape = off0 ? 1 : (diag0 ? 2 : 0);
                    if (shape == 1 && src[1] == 0 && src[7] == 0) shape |= 4;
                    if (shape == 2 && src[3] == 0 && src[5] == 0) shape |= 4;
                    w_packed[s] = shape;
                }
            } else if (st.kind == ST_PROJ_BR && lane == 0) {
                T m;
                m.x = (float)w_scale[s];
                m.y = 0;
                mats[st.mat] = m;
            }
        }
        __syncwarp();
        first = false;
        // the state: lane l holds amplitudes [l G, (l + 1) G)
        T* g = states + (int64_t)slot * d.dim + (int64_t)lane * G;
        T v[G];
#pragma unroll
        for (int e = 0; e < G; e += 2) {
            const float4 x = *reinterpret_cast<const float4*>(g + e);
            v[e] = make_float2(x.x, x.y);
            v[e + 1] = make_float2(x.z, x.w);
        }
        WsPerm P{0};
        for (int q = 0; q < n; ++q) P.set(q, q);
        for (int s = 0; s < p.n_stages; ++s) {
            if ((skipmask >> s) & 1) continue;
            const Stage& st = p.st[s];
            ws_bring_in<NREG>(v, P, st.pos, st.k, n, lane);
            int pos[4] = {0, 0, 0, 0};
            for (int j = 0; j < st.k && j < 4; ++j) pos[j] = P.phys(st.pos[j]);
#pragma unroll
            for (int h = 0; h < NH; ++h)
                ws_apply_one<T>(v + 16 * h, st, pos, w_packed[s], w_sel[s], mats + st.mat, matx + st.mat);
        }
        ws_restore<NREG>(v, P, n, lane);
#pragma unroll
        for (int e = 0; e < G; e += 2)
            *reinterpret_cast<float4*>(g + e) = make_float4(v[e].x, v[e].y, v[e + 1].x, v[e + 1].y);
    }
}

}  // namespace sv
