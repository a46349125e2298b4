// CUDA kernels of libsv (sm_103a).
//
// Data layout in HBM: states are stored one after another (Section IV-A-2),
// one slot of 2^n amplitudes per live state, complex64 (float2) or
// complex128 (double2).  A live state is a *branch*: the shots that have drawn
// the same outcomes so far share it (Section IV-B); in batch mode every shot
// is its own branch.  Shot ids are kept grouped by branch in `perm`.
//
// Kernels
//   k_pass_reg      a pass over at most 4 qubits: one read and one write of
//                   every live state, each lane holding whole groups of 2^W
//                   amplitudes in registers, applying the fused sequence of
//                   ops (gates; each branch's chosen Pauli string, Kraus
//                   matrix or measurement projection) and reducing the
//                   probabilities the next random op needs.  Persistent over
//                   (branch, unit) items, one warp each.
//   k_pass          the same for wider passes and measurements, on tiles
//                   staged in shared memory by bulk asynchronous copies.
//   k_decide_*      per branch: sum the reduced probabilities in a fixed
//                   order (float64), draw every shot's Philox number for each
//                   op of the decide's chain, choose the outcome tuple,
//                   partition the branch's shots by it, and give every new
//                   group a branch id and a free slot (or park its shots on
//                   the waiting list when none is left).  The small- and
//                   big-branch kernels run side by side.
//   k_predraw       batch mode: every shot's Pauli choices, before the gates.
//   k_copy          copy parent states into the new branches' slots.
//   k_final_*       sampling of all qubits from each branch (sampling measure).
//
// Reductions are deterministic: every (branch, chunk) partial is produced by
// one warp or CTA in a fixed order, so a branch's result does not depend on
// how many other branches run beside it.
#include <cuda_runtime.h>

#include <cstdint>

#include "sv_common.cuh"
#include "sv_pass_reg.cuh"

namespace sv {

// ---------------------------------------------------------------------------
// stage application on a shared-memory tile of 2^tb amplitudes.  Each thread
// takes whole groups (the 2^k amplitudes that differ only in the stage's
// qubits), so threads never touch each other's amplitudes within a stage.
// ---------------------------------------------------------------------------
template <int K> struct GroupIdx {
    int sp[K];
    int off[1 << K];
    __device__ __forceinline__ GroupIdx(const int32_t* pos) {
        sorted_pos<K>(pos, sp);
#pragma unroll
        for (int r = 0; r < (1 << K); ++r) {
            int o = 0;
#pragma unroll
            for (int j = 0; j < K; ++j)
                if ((r >> j) & 1) o |= 1 << pos[j];
            off[r] = o;
        }
    }
};

// a monomial 4x4 matrix (see mono_info) on a tile: out[q] = ph[q] in[pi(q)]
template <class R>
__device__ __noinline__ void stage_mono(typename Cplx<R>::T* tile, int tb, const int32_t* pos, int info,
                                        const typename Cplx<R>::T* ph) {
    using T = typename Cplx<R>::T;
    const GroupIdx<2> gi(pos);
    int offp[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int pq = (info >> (8 + 2 * q)) & 3;
        offp[q] = (pq & 1 ? 1 << pos[0] : 0) | (pq & 2 ? 1 << pos[1] : 0);
    }
    const bool unit = (info >> 1) & 1;
    const int groups = 1 << (tb - 2);
    for (int g = threadIdx.x; g < groups; g += blockDim.x) {
        const int base = insert_zeros<2>(g, gi.sp);
        T a[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) a[q] = tile[base | offp[q]];
#pragma unroll
        for (int q = 0; q < 4; ++q) tile[base | gi.off[q]] = unit ? a[q] : cmul(ph[q], a[q]);
    }
}

// dense 2^K x 2^K matrix (staged in shared memory, already scaled)
template <class R, int K>
__device__ __noinline__ void stage_dense(typename Cplx<R>::T* tile, int tb, const int32_t* pos,
                                         const typename Cplx<R>::T* M) {
    using T = typename Cplx<R>::T;
    constexpr int D = 1 << K;
    const GroupIdx<K> gi(pos);
    const int groups = 1 << (tb - K);
    for (int g = threadIdx.x; g < groups; g += blockDim.x) {
        const int base = insert_zeros<K>(g, gi.sp);
        T v[D];
#pragma unroll
        for (int r = 0; r < D; ++r) v[r] = tile[base | gi.off[r]];
#pragma unroll
        for (int r = 0; r < D; ++r) {
            T acc;
            acc.x = 0;
            acc.y = 0;
#pragma unroll
            for (int c = 0; c < D; ++c) cfma(acc, M[r * D + c], v[c]);
            tile[base | gi.off[r]] = acc;
        }
    }
}

// Pauli string from its parameters (Section IV-A-3): bit flips x, phase
// flips z, number of Y; out[d] = (-i)^ny (-1)^popcount(z & d) in[d ^ x].
template <class R, int K>
__device__ __noinline__ void stage_pauli(typename Cplx<R>::T* tile, int tb, const int32_t* pos, int packed) {
    using T = typename Cplx<R>::T;
    constexpr int D = 1 << K;
    const GroupIdx<K> gi(pos);
    const int xm = packed & 15, zm = (packed >> 4) & 15, ny = (packed >> 8) & 3;
    int offx = 0;
#pragma unroll
    for (int j = 0; j < K; ++j)
        if ((xm >> j) & 1) offx |= 1 << pos[j];
    T ph;
    ph.x = (ny == 0) ? (R)1 : (ny == 2 ? (R)-1 : (R)0);
    ph.y = (ny == 1) ? (R)-1 : (ny == 3 ? (R)1 : (R)0);
    const int groups = 1 << (tb - K);
    for (int g = threadIdx.x; g < groups; g += blockDim.x) {
        const int base = insert_zeros<K>(g, gi.sp);
        T w[D];
#pragma unroll
        for (int r = 0; r < D; ++r) {
            T t = cmul(ph, tile[base | (gi.off[r] ^ offx)]);
            if (__popc(zm & r) & 1) {
                t.x = -t.x;
                t.y = -t.y;
            }
            w[r] = t;
        }
#pragma unroll
        for (int r = 0; r < D; ++r) tile[base | gi.off[r]] = w[r];
    }
}

// projection onto measured outcome sel, scaled by 1/sqrt(P(sel)); with reset
// the kept amplitudes move to the all-zero outcome (Section IV-A-5)
template <class R, int K>
__device__ __noinline__ void stage_proj(typename Cplx<R>::T* tile, int tb, const int32_t* pos, int sel, double scale,
                                        int reset) {
    using T = typename Cplx<R>::T;
    constexpr int D = 1 << K;
    const GroupIdx<K> gi(pos);
    int offsel = 0;
#pragma unroll
    for (int j = 0; j < K; ++j)
        if ((sel >> j) & 1) offsel |= 1 << pos[j];
    const int keep = reset ? 0 : sel;
    const R sc = (R)scale;
    const int groups = 1 << (tb - K);
    for (int g = threadIdx.x; g < groups; g += blockDim.x) {
        const int base = insert_zeros<K>(g, gi.sp);
        T t = tile[base | offsel];
        t.x *= sc;
        t.y *= sc;
        T z;
        z.x = 0;
        z.y = 0;
#pragma unroll
        for (int r = 0; r < D; ++r) tile[base | gi.off[r]] = (r == keep) ? t : z;
    }
}

template <class R>
__device__ __forceinline__ void stage_dispatch(typename Cplx<R>::T* tile, int tb, const Stage& st,
                                               const typename Cplx<R>::T* M, int sel, double scale, int packed,
                                               int mono) {
    if (mono) {
        stage_mono<R>(tile, tb, st.pos, mono, M);
    } else if (st.kind == ST_DENSE || st.kind == ST_DENSE_BR) {
        if (st.k == 1) stage_dense<R, 1>(tile, tb, st.pos, M);
        else if (st.k == 2) stage_dense<R, 2>(tile, tb, st.pos, M);
        else if (st.k == 3) stage_dense<R, 3>(tile, tb, st.pos, M);
        else if (st.k == 4) stage_dense<R, 4>(tile, tb, st.pos, M);
        else stage_dense<R, 5>(tile, tb, st.pos, M);
    } else if (st.kind == ST_PAULI_BR) {
        if (st.k == 1) stage_pauli<R, 1>(tile, tb, st.pos, packed);
        else if (st.k == 2) stage_pauli<R, 2>(tile, tb, st.pos, packed);
        else if (st.k == 3) stage_pauli<R, 3>(tile, tb, st.pos, packed);
        else stage_pauli<R, 4>(tile, tb, st.pos, packed);
    } else {
        if (st.k == 1) stage_proj<R, 1>(tile, tb, st.pos, sel, scale, st.reset);
        else if (st.k == 2) stage_proj<R, 2>(tile, tb, st.pos, sel, scale, st.reset);
        else if (st.k == 3) stage_proj<R, 3>(tile, tb, st.pos, sel, scale, st.reset);
        else stage_proj<R, 4>(tile, tb, st.pos, sel, scale, st.reset);
    }
}

template <class R, int K>
__device__ __noinline__ void reduce_forms(const typename Cplx<R>::T* tile, int tb, const int32_t* pos, int Rn,
                                          const typename Cplx<R>::T* F, typename AccSlot<R>::T* acc) {
    using T = typename Cplx<R>::T;
    constexpr int D = 1 << K;
    const GroupIdx<K> gi(pos);
    const int groups = 1 << (tb - K);
    for (int g = threadIdx.x; g < groups; g += blockDim.x) {
        const int base = insert_zeros<K>(g, gi.sp);
        T v[D];
#pragma unroll
        for (int r = 0; r < D; ++r) v[r] = tile[base | gi.off[r]];
        for (int f = 0; f < Rn; ++f) {
            const T* Ff = F + f * D * D;
            const T* Fl = F + (Rn + f) * D * D;  // float32 residuals of Ff
            R q = 0, ql = 0;
#pragma unroll
            for (int a = 0; a < D; ++a) {
                T fa, fl;
                fa.x = 0;
                fa.y = 0;
                fl.x = 0;
                fl.y = 0;
#pragma unroll
                for (int c = 0; c < D; ++c) {
                    cfma(fa, Ff[a * D + c], v[c]);
                    if constexpr (sizeof(R) == 4) cfma(fl, Fl[a * D + c], v[c]);
                }
                q += v[a].x * fa.x + v[a].y * fa.y;  // Re(conj(v_a) (F v)_a)
                if constexpr (sizeof(R) == 4) ql += v[a].x * fl.x + v[a].y * fl.y;
            }
            acc_add(&acc[f * blockDim.x + threadIdx.x], q);
            // the residual part is far below an ulp of q: it joins the
            // accumulator's low word instead of being rounded away in q + ql
            if constexpr (sizeof(R) == 4) acc_add_lo(&acc[f * blockDim.x + threadIdx.x], ql);
        }
    }
}

// measurement probabilities of the 2^K outcomes of the measured qubits
// (Section IV-A-5): bin r collects |psi_j|^2 of indices whose measured bits
// spell r.  Warp w owns bins w, w + nwarps, ...; lane l adds the bin's
// amplitudes of groups l, l + 32, ... in index order into its accumulator
// acc[r * 32 + l], so a chunk's bin is one fixed-order warp combination.
template <class R, int K>
__device__ __noinline__ void reduce_bins(const typename Cplx<R>::T* tile, int tb, const int32_t* pos,
                                         typename AccSlot<R>::T* acc) {
    using T = typename Cplx<R>::T;
    constexpr int D = 1 << K;
    int sp[K];
    sorted_pos<K>(pos, sp);
    const int groups = 1 << (tb - K);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int r = warp; r < D; r += nw) {
        int off = 0;
#pragma unroll
        for (int j = 0; j < K; ++j)
            if ((r >> j) & 1) off |= 1 << pos[j];
        typename AccSlot<R>::T a = acc[r * 32 + lane];
        for (int g = lane; g < groups; g += 32) {
            const T v = tile[insert_zeros<K>(g, sp) | off];
            acc_add(&a, v.x * v.x + v.y * v.y);
        }
        acc[r * 32 + lane] = a;
    }
}

template <class R>
__device__ __forceinline__ void reduce_dispatch(const typename Cplx<R>::T* tile, int tb, const PassDesc& p,
                                                const typename Cplx<R>::T* F, typename AccSlot<R>::T* acc) {
    if (p.red_kind == RED_BINS || p.red_kind == RED_DIAG) {  // diagonal forms: the bins of |psi|^2
        if (p.red_k == 1) reduce_bins<R, 1>(tile, tb, p.red_pos, acc);
        else if (p.red_k == 2) reduce_bins<R, 2>(tile, tb, p.red_pos, acc);
        else if (p.red_k == 3) reduce_bins<R, 3>(tile, tb, p.red_pos, acc);
        else reduce_bins<R, 4>(tile, tb, p.red_pos, acc);
    } else {
        if (p.red_k == 1) reduce_forms<R, 1>(tile, tb, p.red_pos, p.red_R, F, acc);
        else reduce_forms<R, 2>(tile, tb, p.red_pos, p.red_R, F, acc);
    }
}

// fixed-order block reduction of one float64 per thread; result in thread 0
__device__ __forceinline__ double block_sum(double v, double* sh) {
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

// ---------------------------------------------------------------------------
// bulk asynchronous copies (TMA bulk engine) and mbarriers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void bulk_store(void* dst, const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait: gives up (error word) instead of spinning forever
__device__ __forceinline__ bool mbar_wait(const DevBatch& d, uint64_t* bar, uint32_t parity) {
    for (int it = 0; it < (1 << 24); ++it)
        if (mbar_try_wait(bar, parity)) return true;
    set_err(d, ERR_TIMEOUT, 1);
    return false;
}

// ---------------------------------------------------------------------------
// k_pass: every CTA owns a contiguous range of (branch, chunk) units and
// streams their tiles through a ring of PASS_NBUF shared-memory buffers.
// Warp 0 fetches tile k+2 with bulk copies (one per contiguous run of the
// tile) while all warps apply the stages to tile k; finished tiles go back
// with bulk stores.  Reductions accumulate per thread and are combined per
// chunk in a fixed order.
// ---------------------------------------------------------------------------
constexpr int PASS_NBUF = PASS_NBUF_H;
constexpr int PASS_AHEAD = 2;

template <class R>
__global__ void __launch_bounds__(256, 2) k_pass(DevBatch d, const __grid_constant__ PassDesc p) {
    using T = typename Cplx<R>::T;
    using A = typename AccSlot<R>::T;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int tb = p.tb, run = p.run_bits;
    const int tsize = 1 << tb;
    const int n_runs = 1 << (tb - run);
    const bool red = p.red_kind != RED_NONE;
    T* bufs = reinterpret_cast<T*>(smem_raw);
    T* mats = bufs + PASS_NBUF * tsize;
    A* acc = reinterpret_cast<A*>(mats + p.mat_elems);
    int* hi_tab = reinterpret_cast<int*>(acc + (red ? p.red_R * (int)blockDim.x : 0));
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + ((pass_bytes_before_bars(p, blockDim.x, sizeof(T)) + 7) & ~7ull));
    __shared__ int skip[MAX_STAGES], sel_sh[MAX_STAGES], packed_sh[MAX_STAGES], mono_sh[MAX_STAGES];
    __shared__ double scale_sh[MAX_STAGES];
    __shared__ double wsum[8][MAX_RED];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // complex64 tiles need qubit 0 inside the tile (pairs move as 128 bits)
    if (sizeof(T) == 8 && run < 1) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_err(d, ERR_INDEX, -1);
        return;
    }
    const int n_br = d.ctl[CTL_NBR];
    if (blockIdx.x == 0 && threadIdx.x == 0 && d.pass_log) {
        const int i = atomicAdd(&d.ctl[CTL_NPASS], 1);
        if (i < d.pass_log_cap) d.pass_log[i] = n_br;
    }
    const int64_t units = (int64_t)n_br * p.chunks;
    const int64_t tpc = p.tiles_per_chunk;
    const int64_t u0 = units * blockIdx.x / gridDim.x, u1 = units * (blockIdx.x + 1) / gridDim.x;
    const int64_t t0 = u0 * tpc, nt = (u1 - u0) * tpc;
    if (nt <= 0) return;

    for (int h = threadIdx.x; h < n_runs; h += blockDim.x) {
        int o = 0;
        for (int j = 0; j < tb - run; ++j)
            if ((h >> j) & 1) o |= 1 << p.tile_q[run + j];
        hi_tab[h] = o;
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < PASS_NBUF; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();

    T* const states = reinterpret_cast<T*>(d.states);
    const uint32_t run_bytes = (uint32_t)(sizeof(T) << run);
    // global address of tile i (of this CTA's sequence)
    auto tile_ptr = [&](int64_t i) -> T* {
        const int64_t unit = i / tpc;
        const int b = (int)(unit / p.chunks);
        const int64_t tn = (unit % p.chunks) * tpc + i % tpc;
        int slot = d.br_slot[b];
        if (slot < 0 || slot >= d.n_slots) {
            set_err(d, ERR_SLOT, b);
            slot = 0;
        }
        int64_t base = 0;
        for (int j = 0; j < p.n_nontile; ++j)
            if ((tn >> j) & 1) base |= 1ll << p.nontile_q[j];
        return states + (int64_t)slot * d.dim + base;
    };
    // warp 0: fetch tile k (k-th of this CTA) into its ring buffer
    auto fetch = [&](int64_t k) {
        const int s = (int)(k % PASS_NBUF);
        T* src = tile_ptr(t0 + k);
        if (lane == 0) mbar_expect_tx(&bars[s], (uint32_t)(sizeof(T) << tb));
        __syncwarp();
        for (int j = lane; j < n_runs; j += 32)
            bulk_load(bufs + (size_t)s * tsize + ((size_t)j << run), src + hi_tab[j], run_bytes, &bars[s]);
    };
    if (warp == 0)
        for (int64_t k = 0; k < PASS_AHEAD && k < nt; ++k) fetch(k);

    int cur_b = -1;
    bool ok = true;
    for (int64_t k = 0; k < nt && ok; ++k) {
        const int64_t i = t0 + k;
        const int s = (int)(k % PASS_NBUF);
        if (warp == 0 && k + PASS_AHEAD < nt) {
            bulk_wait_read1();  // the store of tile k-2 has left the buffer
            __syncwarp();
            fence_proxy_async();
            fetch(k + PASS_AHEAD);
        }
        const int64_t unit = i / tpc;
        const int b = (int)(unit / p.chunks);
        const int c = (int)(unit % p.chunks);
        if (b != cur_b) {
            const uint64_t clb = d.br_clbits[b];
            __syncthreads();
            for (int st_i = threadIdx.x; st_i < p.n_stages; st_i += blockDim.x) {
                const Stage& st = p.st[st_i];
                int sk = 0, sel = 0, packed = 0;
                double scale = 1.0;
                if (st.cond_clbit >= 0 && (int)((clb >> st.cond_clbit) & 1ull) != st.cond_val) sk = 1;
                if (st.pre) {  // batch mode: the branch's one shot, pre-drawn
                    sel = d.pre_sel[(int64_t)st.pend * d.cap_br + d.perm[d.br_start[b]]];
                    packed = d.ipool[st.off + sel];
                    if ((packed & 0xff) == 0) sk = 1;
                } else if (st.pend == PEND_PSET) {  // the branch's parameter set
                    sel = d.br_pset[b];
                } else if (st.kind != ST_DENSE) {
                    sel = d.br_sel[(int64_t)st.pend * d.cap_br + b];
                    scale = d.br_scale[(int64_t)st.pend * d.cap_br + b];
                    if (sel < 0) sk = 1;
                    if (st.kind == ST_PAULI_BR && !sk) {
                        packed = d.ipool[st.off + sel];
                        if ((packed & 0xff) == 0) sk = 1;  // identity string: nothing to do
                    }
                }
                skip[st_i] = sk;
                sel_sh[st_i] = sel;
                packed_sh[st_i] = packed;
                scale_sh[st_i] = scale;
            }
            __syncthreads();
            // matrices: the shared gates' (and the reduction's forms) once per
            // CTA, a branch's own choices (Kraus terms, parameter sets) per
            // branch; a matrix that is monomial (CX, CZ, SWAP, phases) moves
            // amplitudes instead of multiplying
            const R* pool = reinterpret_cast<const R*>(d.pool);
            const bool first = cur_b < 0;
            for (int st_i = 0; st_i < p.n_stages; ++st_i) {
                const Stage& st = p.st[st_i];
                if (st.kind != ST_DENSE && st.kind != ST_DENSE_BR) continue;
                if (st.kind == ST_DENSE ? !first : skip[st_i]) continue;
                const int D2 = 1 << (2 * st.k);
                const R* src = pool + st.off + (st.kind == ST_DENSE_BR ? (int64_t)sel_sh[st_i] * st.stride : 0);
                const R sc = (R)scale_sh[st_i];
                for (int e = threadIdx.x; e < D2; e += blockDim.x) {
                    T m;
                    m.x = src[2 * e] * sc;
                    m.y = src[2 * e + 1] * sc;
                    mats[st.mat + e] = m;
                }
            }
            if (first && (p.red_kind == RED_FORMS || p.red_kind == RED_DIAG)) {  // coefficients, then residuals
                const int E2 = 2 * (p.red_R << ((p.red_kind == RED_FORMS ? 2 : 1) * p.red_k));
                const R* src = pool + p.red_off;
                for (int e = threadIdx.x; e < E2; e += blockDim.x) {
                    T m;
                    m.x = src[2 * e];
                    m.y = src[2 * e + 1];
                    mats[p.mat_elems - E2 + e] = m;
                }
            }
            __syncthreads();
            for (int st_i = threadIdx.x; st_i < p.n_stages; st_i += blockDim.x) {
                const Stage& st = p.st[st_i];
                if (st.k != 2 || (st.kind != ST_DENSE && st.kind != ST_DENSE_BR)) continue;
                if (st.kind == ST_DENSE ? !first : skip[st_i]) continue;
                T m[16], ph[4];
                for (int e = 0; e < 16; ++e) m[e] = mats[st.mat + e];
                const int mi = mono_info(m, ph);
                if (mi)
                    for (int q = 0; q < 4; ++q) mats[st.mat + q] = ph[q];  // this stage's own entries
                mono_sh[st_i] = mi;
            }
            if (first)
                for (int st_i = threadIdx.x; st_i < p.n_stages; st_i += blockDim.x)
                    if (p.st[st_i].k != 2 || (p.st[st_i].kind != ST_DENSE && p.st[st_i].kind != ST_DENSE_BR))
                        mono_sh[st_i] = 0;
            __syncthreads();
            cur_b = b;
        }
        const int n_bins = p.red_kind == RED_DIAG ? 1 << p.red_k : p.red_R;  // warp-owned bins
        if (red && i % tpc == 0) {
            if (p.red_kind == RED_BINS || p.red_kind == RED_DIAG)
                for (int r = warp; r < n_bins; r += (int)(blockDim.x >> 5)) acc[r * 32 + lane] = A{};
            else
                for (int r = 0; r < p.red_R; ++r) acc[r * blockDim.x + threadIdx.x] = A{};
        }
        if (!mbar_wait(d, &bars[s], (uint32_t)((k / PASS_NBUF) & 1))) ok = false;
        T* tile = bufs + (size_t)s * tsize;
        for (int st_i = 0; st_i < p.n_stages; ++st_i) {
            if (skip[st_i]) continue;
            const Stage& st = p.st[st_i];
            stage_dispatch<R>(tile, tb, st, mats + st.mat, sel_sh[st_i], scale_sh[st_i], packed_sh[st_i], mono_sh[st_i]);
            __syncthreads();
        }
        if (red) reduce_dispatch<R>(tile, tb, p, mats + p.mat_elems - 2 * (p.red_R << (2 * p.red_k)), acc);
        __syncthreads();
        if (p.store && warp == 0) {
            T* dst = tile_ptr(i);
            fence_proxy_async();
            for (int j = lane; j < n_runs; j += 32)
                bulk_store(dst + hi_tab[j], tile + ((size_t)j << run), run_bytes);
            bulk_commit();
        }
        if (red && i % tpc == tpc - 1) {
            const int slot = d.br_slot[b];
            const bool slot_ok = slot >= 0 && slot < d.n_slots;
            double* part = d.partials + ((int64_t)(slot_ok ? slot : 0) * d.max_chunks + c) * MAX_RED;
            if (p.red_kind == RED_BINS) {
                // each bin lives in one warp: one fixed-order warp combination
                for (int r = warp; r < p.red_R; r += (int)(blockDim.x >> 5)) {
                    const double v = warp_combine(acc[r * 32 + lane]);
                    if (lane == 0 && slot_ok) part[r] = v;
                }
            } else if (p.red_kind == RED_DIAG) {
                // the bins as for a measurement, then every diagonal form
                // from them with float64 weights (thread f: form f)
                for (int r = warp; r < n_bins; r += (int)(blockDim.x >> 5)) {
                    const double v = warp_combine(acc[r * 32 + lane]);
                    if (lane == 0) wsum[0][r] = v;
                }
                __syncthreads();
                if (threadIdx.x < p.red_R && slot_ok) {
                    const T* W = mats + p.mat_elems - 2 * (p.red_R << p.red_k);
                    double v = 0.0;
                    for (int r = 0; r < n_bins; ++r)
                        v += diag_weight(W, p.red_R, p.red_k, (int)threadIdx.x, r) * wsum[0][r];
                    part[threadIdx.x] = v;
                }
            } else {
                // fixed-order combination: lanes by shuffles, warps in order
                for (int r = 0; r < p.red_R; ++r) {
                    const double v = warp_combine(acc[r * blockDim.x + threadIdx.x]);
                    if (lane == 0) wsum[warp][r] = v;
                }
                __syncthreads();
                if (threadIdx.x < p.red_R && slot_ok) {
                    double v = 0.0;
                    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += wsum[w][threadIdx.x];
                    part[threadIdx.x] = v;
                }
            }
        }
    }
    if (warp == 0) bulk_wait_all();
}

// ---------------------------------------------------------------------------
// k_decide: per branch, probabilities (fixed-order float64 sums of the
// partials), one Philox draw per shot and op, the shot's outcome, and a
// partition of the branch's shots by outcome.  A decide may carry a chain
// (DecideDesc::tail): the ops after the head that need no pass in between.
// A shot then draws every op of the chain in program order, each from its
// own counter (shot, op), and its outcome is the tuple.  Branches with more
// than DEC_SMALL shots take a whole CTA (k_decide_big); the others one warp
// (k_decide_small).
// ---------------------------------------------------------------------------
constexpr int DEC_THREADS = 512;
constexpr int DEC_SMALL = 64;

// Sum over the lanes by a fixed xor tree.  Lanes at or past `used` hold
// exact zeros, and adding a zero changes nothing, so the tree can start at
// the level that first mixes the used lanes: the same result in fewer
// float64 adds (each a 16-cycle FP64-pipe instruction on GB300).
__device__ __forceinline__ double warp_sum(double x, int used) {
    int o = 16;
    while (o > 1 && o >= used) o >>= 1;
    for (; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// per-branch tables of one decide (shared memory: one per warp or per CTA)
struct DecTab {
    double p[MAX_TERMS], cum[MAX_TERMS];  // head op: probabilities, running sums
    uint64_t thr[MAX_TERMS];              // head op: integer thresholds
    double sc[MAX_TERMS];                 // head op: 1 / sqrt(p) of every outcome (1 for Pauli)
    double jp[MAX_RED], jcum[MAX_RED];    // chained DEC_KRAUS_J2: p(j | i), row i at i * R2
    uint64_t jthr[MAX_RED];
    double jsc[MAX_RED];                  // chained DEC_KRAUS_J2: 1 / sqrt(p(j | i))
    int bincnt[MAX_TERMS], binbase[MAX_TERMS], binrun[MAX_TERMS];
    int leaf[MAX_TERMS];                  // fork log: branch of each outcome tuple
};

// probabilities of branch b into p_out (and, for Pauli, the table into
// cum_out); one whole warp.  With joint_out (a DEC_KRAUS_J1 head), the
// joint probabilities p_ij are kept there too.
__device__ void warp_probs(const DevBatch& d, const DecideDesc& dd, int b, int slot, double* p_out, double* cum_out,
                           double* joint_out) {
    const int lane = threadIdx.x & 31;
    const int R = dd.R;
    if (dd.kind == DEC_PAULI) {
        for (int r = lane; r < R; r += 32) {
            p_out[r] = dd.cum[r] - (r ? dd.cum[r - 1] : 0.0);
            cum_out[r] = dd.cum[r];
        }
        __syncwarp();
        return;
    }
    // The terms needed are the contiguous entries [base_r, base_r + R*inner)
    // of every chunk's record: p_r = sum over chunks and j < inner of
    // entry base_r + r*inner + j.  Each lane adds its chunks' entries in
    // registers (all loads of a chunk issued together), the lanes' sums are
    // combined by the fixed shuffle tree, and lane 0 adds the inner terms.
    int src = slot, base_r = 0, inner = 1;
    if (dd.kind == DEC_KRAUS_J1) {
        inner = dd.r2;  // p_i = sum over j of the joint p_ij = entry i * r2 + j
    } else if (dd.kind == DEC_KRAUS_J2) {
        // branches forked by the first op still find the joint partials in
        // their parent's slot
        const int cf = d.ctl[CTL_COPY_FIRST], ce = d.ctl[CTL_COPY_END];
        if (b >= cf && b < ce) src = d.br_slot[d.br_parent[b]];
        base_r = d.br_sel[(int64_t)dd.pend_prev * d.cap_br + b] * R;  // p_ij = entry i * R + j
    }
    const int nk = R * inner;
    const double* pp = d.partials + (int64_t)src * d.max_chunks * MAX_RED + base_r;
    double u[MAX_RED];
#pragma unroll
    for (int k = 0; k < MAX_RED; ++k) u[k] = 0.0;
    for (int c = lane; c < dd.chunks; c += 32) {
        const double* q = pp + (int64_t)c * MAX_RED;
#pragma unroll
        for (int k = 0; k < MAX_RED; ++k)
            if (k < nk) u[k] += q[k];
    }
#pragma unroll
    for (int k = 0; k < MAX_RED; ++k)
        if (k < nk) {
            const double t = warp_sum(u[k], dd.chunks);
            if (lane == 0) cum_out[k] = t;  // scratch until the caller forms the table
        }
    __syncwarp();
    // GB300's float64 pipe retires two lanes per clock per SM, shared by every
    // warp there: each term below is computed by its own lane (the same
    // operations in the same order as one lane looping over them)
    for (int k = lane; k < nk; k += 32)
        if (joint_out) joint_out[k] = cum_out[k];
    for (int r = lane; r < R; r += 32) {
        double t = 0.0;
        for (int j = 0; j < inner; ++j) t += cum_out[r * inner + j];
        p_out[r] = t;
    }
    __syncwarp();
    if (dd.kind == DEC_KRAUS_J2) {
        double pi = 0.0;
        for (int r = 0; r < R; ++r) pi += p_out[r];
        double q[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) q[h] = lane + 32 * h < R ? p_out[lane + 32 * h] / pi : 0.0;
        __syncwarp();
#pragma unroll
        for (int h = 0; h < 2; ++h)
            if (lane + 32 * h < R) p_out[lane + 32 * h] = q[h];
    }
    __syncwarp();
}

__device__ __forceinline__ bool chained_j2(const DecideDesc& dd) {
    return dd.n_tail > 0 && dd.tail[0].kind == DEC_KRAUS_J2;
}

// the branch's tables (one warp): head probabilities, running sums and
// thresholds; for a chained DEC_KRAUS_J2, the conditional tables
// p(j | i) = p_ij / sum_j p_ij of every head outcome i (the arithmetic of a
// separate DEC_KRAUS_J2 decide, row by row)
__device__ void branch_tables(const DevBatch& d, const DecideDesc& dd, int b, int slot, DecTab& T) {
    const int lane = threadIdx.x & 31;
    const bool j2 = chained_j2(dd);
    warp_probs(d, dd, b, slot, T.p, T.cum, j2 ? T.jp : nullptr);
    if (lane == 0 && dd.kind != DEC_PAULI) {
        double acc = 0.0;
        for (int r = 0; r < dd.R; ++r) T.cum[r] = (acc += T.p[r]);
    }
    if (j2) {
        // row i of p(j | i) = p_ij / sum_j p_ij and its running sums, entry
        // k = i * R2 + j by lane k (R * R2 <= MAX_RED <= 32)
        const int R2 = dd.tail[0].R, n2 = dd.R * R2;
        double q = 0.0;
        if (lane < n2) {
            const double* row = T.jp + (lane / R2) * R2;
            double pi = 0.0;
            for (int j = 0; j < R2; ++j) pi += row[j];
            q = T.jp[lane] / pi;
        }
        __syncwarp();
        if (lane < n2) T.jp[lane] = q;
        __syncwarp();
        if (lane < n2) {
            const int i = lane / R2, j = lane % R2;
            double acc = 0.0;
            for (int jj = 0; jj <= j; ++jj) acc += T.jp[i * R2 + jj];
            T.jcum[lane] = acc;
            T.jsc[lane] = 1.0 / sqrt(T.jp[lane]);
        }
    }
    __syncwarp();
    for (int r = lane; r < dd.R; r += 32) {
        T.thr[r] = cum_threshold(T.cum[r]);
        T.sc[r] = dd.kind == DEC_PAULI ? 1.0 : 1.0 / sqrt(T.p[r]);
    }
    if (j2)
        for (int k = lane; k < dd.R * dd.tail[0].R; k += 32) T.jthr[k] = cum_threshold(T.jcum[k]);
    __syncwarp();
}

__device__ __forceinline__ void log_choice(int32_t* log_sel, double* log_thr, uint32_t shot, int sel,
                                           const double* cum) {
    if (log_sel) log_sel[shot] = sel;
    if (log_thr) {
        log_thr[2 * (int64_t)shot] = sel ? cum[sel - 1] : 0.0;
        log_thr[2 * (int64_t)shot + 1] = cum[sel];
    }
}

// a shot's outcome tuple over the chain, as a mixed-radix number
__device__ __forceinline__ int chain_draw(const DevBatch& d, const DecideDesc& dd, const DecTab& T, uint32_t shot) {
    const uint64_t gs = d.shot_base + shot;
    int o = select_k(philox_k53(d.seed, gs, dd.op), T.thr, T.cum, dd.R);
    log_choice(dd.log_sel, dd.log_thr, shot, o, T.cum);
    int key = o;
    for (int t = 0; t < dd.n_tail; ++t) {
        const DecideTail& tl = dd.tail[t];
        const double* cum;
        const uint64_t* thr;
        if (tl.kind == DEC_KRAUS_J2) {  // only right after the head: o is the head's outcome
            cum = T.jcum + o * tl.R;
            thr = T.jthr + o * tl.R;
        } else {
            cum = dd.tail_cum + tl.cum_off;
            thr = dd.tail_thr + tl.cum_off;
        }
        o = select_k(philox_k53(d.seed, gs, tl.op), thr, cum, tl.R);
        log_choice(tl.log_sel, tl.log_thr, shot, o, cum);
        key = key * tl.R + o;
    }
    return key;
}

// per-op choices and scales of outcome tuple `key` into branch `leaf`'s
// pending columns; returns the head outcome
__device__ int write_choices(const DevBatch& d, const DecideDesc& dd, const DecTab& T, int leaf, int key) {
    int outc[1 + MAX_TAIL];
    int rest = key;
    for (int t = dd.n_tail - 1; t >= 0; --t) {
        outc[1 + t] = rest % dd.tail[t].R;
        rest /= dd.tail[t].R;
    }
    outc[0] = rest;
    const int oh = outc[0];
    d.br_sel[(int64_t)dd.pend * d.cap_br + leaf] = oh;
    d.br_scale[(int64_t)dd.pend * d.cap_br + leaf] = T.sc[oh];
    for (int t = 0; t < dd.n_tail; ++t) {
        const DecideTail& tl = dd.tail[t];
        const int o = outc[1 + t];
        d.br_sel[(int64_t)tl.pend * d.cap_br + leaf] = o;
        d.br_scale[(int64_t)tl.pend * d.cap_br + leaf] = tl.kind == DEC_KRAUS_J2 ? T.jsc[oh * tl.R + o] : 1.0;
    }
    return oh;
}

// fork events of one branch's decide, per op of the chain (one thread): at
// each op, every node (shots sharing the earlier ops' outcomes) whose shots
// take two or more outcomes logs one event per outcome: (op, node's branch,
// the outcome's branch, outcome, shots, first perm position, and the node's
// first perm position and shots).  A node's
// branch is that of its first outcome tuple, so the events are those of
// deciding the ops one at a time.  The branch's shots are partitioned in
// tuple order, so a node's and an outcome's shots are contiguous perm ranges
// that start at their first tuple's group; later forks only reorder shots inside
// their own branch's range, so the range keeps this set of shot ids until
// the waiting list restarts.
__device__ void log_fork_events(const DevBatch& d, const DecideDesc& dd, const DecTab& T, int start) {
    const int M = 1 + dd.n_tail;
    int stride = dd.nk;
    for (int m = 0; m < M; ++m) {
        const int Rm = m == 0 ? dd.R : dd.tail[m - 1].R;
        const uint32_t op = m == 0 ? dd.op : dd.tail[m - 1].op;
        const int node = stride;  // keys per node at this level
        stride /= Rm;             // keys per outcome of this op within a node
        for (int n0 = 0; n0 < dd.nk; n0 += node) {
            int distinct = 0, first = -1, total = 0;
            for (int o = 0; o < Rm; ++o) {
                int c = 0, f = -1;
                for (int k = n0 + o * stride; k < n0 + (o + 1) * stride; ++k)
                    if (T.bincnt[k] > 0) {
                        c += T.bincnt[k];
                        if (f < 0) f = k;
                    }
                if (c > 0) {
                    ++distinct;
                    total += c;
                    if (first < 0) first = f;
                }
            }
            if (distinct < 2) continue;
            const int parent = T.leaf[first];
            for (int o = 0; o < Rm; ++o) {
                int c = 0, f = -1;
                for (int k = n0 + o * stride; k < n0 + (o + 1) * stride; ++k)
                    if (T.bincnt[k] > 0) {
                        c += T.bincnt[k];
                        if (f < 0) f = k;
                    }
                if (c == 0) continue;
                const int e = atomicAdd(&d.ctl[CTL_NFORK], 1);
                if (e < d.fork_log_cap) {
                    int64_t* ev = d.fork_log + FORK_WORDS * (int64_t)e;
                    ev[0] = op; ev[1] = parent; ev[2] = T.leaf[f]; ev[3] = o; ev[4] = c;
                    ev[5] = start + T.binbase[f];
                    ev[6] = start + T.binbase[first];  // the node's own range
                    ev[7] = total;
                }
            }
        }
    }
}

// Groups of branch b after a decide, built by one whole warp: the outcome
// tuples with shots, in tuple order.  The branch keeps the first; with
// shot-branching every other group becomes a new branch (Section IV-B-2: a
// state forks where its shots' outcomes differ) or, with no free slot left,
// parks its shots on the waiting list.  One atomic on the allocation counter
// reserves the ids of all of the branch's new branches, and each group's
// lane writes its own branch, so a fork costs the same whatever the number
// of groups.  Which branch gets which id depends on timing, but no result
// does: a branch's arithmetic never depends on its id or slot.  k_copy folds
// the counters into the branch count.
__device__ void decide_groups(const DevBatch& d, const DecideDesc& dd, int b, int start, DecTab& T, bool big) {
    if (dd.sample_only) return;  // the choices are drawn and logged; the commit forks
    const int lane = threadIdx.x & 31;
    const int NK = dd.nk;
    // group index of tuples lane and lane + 32 (-1: no shots)
    int gidx[2] = {-1, -1};
    int g = 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int r = lane + 32 * h;
        const bool nz = r < NK && T.bincnt[r] > 0;
        const unsigned m = __ballot_sync(0xffffffffu, nz);
        if (nz) gidx[h] = g + __popc(m & ((1u << lane) - 1u));
        g += __popc(m);
    }
    const unsigned f0 = __ballot_sync(0xffffffffu, gidx[0] == 0), f1 = __ballot_sync(0xffffffffu, gidx[1] == 0);
    const int r0 = f0 ? __ffs(f0) - 1 : 32 + __ffs(f1) - 1;
    const uint64_t cl_parent = d.br_clbits[b];
    const int tail_prod = NK / dd.R;
    auto clbits_of = [&](int key) {
        uint64_t cl = cl_parent;
        if (dd.kind == DEC_MEASURE) {
            const int oh = key / tail_prod;
            for (int j = 0; j < dd.m; ++j) {
                const uint64_t bit = (uint64_t)((oh >> j) & 1);
                cl = (cl & ~(1ull << dd.clbit[j])) | (bit << dd.clbit[j]);
            }
        }
        return cl;
    };
    const bool forks = g > 1 && dd.fork;
    int j0 = 0;
    if (lane == 0) {
        write_choices(d, dd, T, b, r0);
        d.br_clbits[b] = clbits_of(r0);
        if (g > 1 && !dd.fork) set_err(d, ERR_GROUPS, b);
        if (forks) {
            j0 = atomicAdd(&d.ctl[CTL_NALLOC], g - 1);
            if (big) {
                // the small-branch kernel runs at the same time: mark the
                // branch before its count may drop to its range
                *reinterpret_cast<volatile int32_t*>(&d.br_big[b]) = (int32_t)dd.op;
                __threadfence();
            }
            *reinterpret_cast<volatile int32_t*>(&d.br_count[b]) = T.bincnt[r0];
            if (d.fork_log) T.leaf[r0] = b;
        }
    }
    if (!forks) return;
    j0 = __shfl_sync(0xffffffffu, j0, 0);
    const int n_br0 = d.ctl[CTL_NBR], n_free = d.ctl[CTL_NFREE];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int gi = gidx[h];
        if (gi < 1) continue;
        const int r = lane + 32 * h;
        const int j = j0 + gi - 1;
        const int cnt = T.bincnt[r], st = start + T.binbase[r];
        int child = -1;
        if (j < n_free) {
            child = n_br0 + j;
            d.br_slot[child] = d.free_slots[n_free - 1 - j];
            d.br_start[child] = st;
            d.br_count[child] = cnt;
            d.br_clbits[child] = clbits_of(r);
            d.br_parent[child] = b;
            d.br_big[child] = -1;
            d.br_pset[child] = d.br_pset[b];
            for (uint64_t cols = dd.live_cols; cols; cols &= cols - 1) {  // the parent's pending choices
                const int q = __ffsll((long long)cols) - 1;
                d.br_sel[(int64_t)q * d.cap_br + child] = d.br_sel[(int64_t)q * d.cap_br + b];
                d.br_scale[(int64_t)q * d.cap_br + child] = d.br_scale[(int64_t)q * d.cap_br + b];
            }
            write_choices(d, dd, T, child, r);
        } else {
            const int w = atomicAdd(&d.ctl[CTL_NWAIT], cnt);
            for (int i = 0; i < cnt; ++i) d.wait_shots[w + i] = d.perm[st + i];
        }
        if (d.fork_log) T.leaf[r] = child;
    }
    if (d.fork_log) {
        __syncwarp();
        if (lane == 0) log_fork_events(d, dd, T, start);
        __syncwarp();
    }
}

// Branches of up to DEC_THREADS * DEC_SPT shots are staged in shared
// memory: one load of the branch's perm range (all loads of a thread in
// flight together), the draws and bin counts, and the partition written
// straight back into perm (every read of the range has completed before the
// first write).  The loops over the staged shots are not unrolled: they run
// once per launch, on an SM whose instruction cache the pass kernels have
// just filled.  Larger branches stream through perm_tmp.
constexpr int DEC_SPT = 20;
constexpr size_t DEC_BIG_SMEM = (size_t)DEC_SPT * DEC_THREADS * (sizeof(uint32_t) + sizeof(uint8_t));

__global__ void __launch_bounds__(DEC_THREADS, 1) k_decide_big(DevBatch d, const __grid_constant__ DecideDesc dd) {
    __shared__ DecTab T;
    __shared__ int ng_sh, nlist_sh;
    __shared__ int list_sh[DEC_THREADS];
    extern __shared__ __align__(16) unsigned char dec_smem[];
    uint32_t* sm_shot = reinterpret_cast<uint32_t*>(dec_smem);
    uint8_t* sm_key = reinterpret_cast<uint8_t*>(sm_shot + DEC_SPT * DEC_THREADS);
    const int n_br = d.ctl[CTL_NBR];
    const int NK = dd.nk;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31;
    // this CTA's branches are blockIdx.x + j * gridDim.x; its threads look at
    // nth of them at once and list the ones above DEC_SMALL shots
    for (int64_t b0 = blockIdx.x; b0 < n_br; b0 += (int64_t)gridDim.x * nth) {
        __syncthreads();
        if (tid == 0) nlist_sh = 0;
        __syncthreads();
        {
            const int64_t bt = b0 + (int64_t)tid * gridDim.x;
            if (bt < n_br && d.br_count[bt] > DEC_SMALL) list_sh[atomicAdd(&nlist_sh, 1)] = (int)bt;
        }
        __syncthreads();
        const int nlist = nlist_sh;
        for (int li = 0; li < nlist; ++li) {
            const int b = list_sh[li];
            const int cnt = d.br_count[b];
            const int slot = d.br_slot[b], start = d.br_start[b];
            const bool onchip = cnt <= DEC_SPT * nth;
            const int nk = (cnt + nth - 1) / nth;
            if (onchip) {
#pragma unroll
                for (int k = 0; k < DEC_SPT; ++k) {
                    const int i = tid + k * nth;
                    sm_shot[k * nth + tid] = i < cnt ? d.perm[start + i] : 0u;
                }
            }
            __syncthreads();
            if (warp == 0) branch_tables(d, dd, b, slot, T);
            if (tid < NK) {
                T.bincnt[tid] = 0;
                T.binrun[tid] = 0;
            }
            __syncthreads();
            if (onchip) {
#pragma unroll 1
                for (int k = 0; k < nk; ++k) {
                    const int i = tid + k * nth;
                    int key = -1;
                    if (i < cnt) {
                        key = chain_draw(d, dd, T, sm_shot[k * nth + tid]);
                        sm_key[k * nth + tid] = (uint8_t)key;
                    }
                    const unsigned peers = __match_any_sync(0xffffffffu, key);
                    if (key >= 0 && (peers & ((1u << lane) - 1u)) == 0) atomicAdd(&T.bincnt[key], __popc(peers));
                }
            } else {
#pragma unroll 1
                for (int base = 0; base < cnt; base += nth) {  // warp-aggregated bin counts
                    const int i = base + tid;
                    int key = -1;
                    if (i < cnt) {
                        key = chain_draw(d, dd, T, d.perm[start + i]);
                        d.shot_sel[start + i] = key;
                    }
                    const unsigned peers = __match_any_sync(0xffffffffu, key);
                    if (key >= 0 && (peers & ((1u << lane) - 1u)) == 0) atomicAdd(&T.bincnt[key], __popc(peers));
                }
            }
            __syncthreads();
            if (tid == 0) {
                int ng = 0, acc = 0;
                for (int r = 0; r < NK; ++r)
                    if (T.bincnt[r] > 0) {
                        T.binbase[r] = acc;
                        acc += T.bincnt[r];
                        ++ng;
                    }
                ng_sh = ng;
            }
            __syncthreads();
            if (ng_sh > 1 && dd.fork) {
                // partition by outcome in one sweep: positions within a group come
                // from warp-aggregated shared-memory counters, so the order of shots
                // inside a group is not fixed (no result depends on it)
                if (onchip) {
#pragma unroll 1
                    for (int k = 0; k < nk; ++k) {
                        const int i = tid + k * nth;
                        const int key = i < cnt ? (int)sm_key[k * nth + tid] : -1;
                        const unsigned peers = __match_any_sync(0xffffffffu, key);
                        const int rank = __popc(peers & ((1u << lane) - 1u));
                        const int leader = __ffs(peers) - 1;
                        int pos = 0;
                        if (key >= 0 && rank == 0) pos = atomicAdd(&T.binrun[key], __popc(peers));
                        pos = __shfl_sync(0xffffffffu, pos, leader);
                        if (key >= 0) d.perm[start + T.binbase[key] + pos + rank] = sm_shot[k * nth + tid];
                    }
                } else {
#pragma unroll 1
                    for (int base = 0; base < cnt; base += nth) {
                        const int i = base + tid;
                        const int key = (i < cnt) ? d.shot_sel[start + i] : -1;
                        const unsigned peers = __match_any_sync(0xffffffffu, key);
                        const int rank = __popc(peers & ((1u << lane) - 1u));
                        const int leader = __ffs(peers) - 1;
                        int pos = 0;
                        if (key >= 0 && rank == 0) pos = atomicAdd(&T.binrun[key], __popc(peers));
                        pos = __shfl_sync(0xffffffffu, pos, leader);
                        if (key >= 0) d.perm_tmp[start + T.binbase[key] + pos + rank] = d.perm[start + i];
                    }
                    __syncthreads();
                    for (int i = tid; i < cnt; i += nth) d.perm[start + i] = d.perm_tmp[start + i];
                }
                __syncthreads();
            }
            if (warp == 0) decide_groups(d, dd, b, start, T, true);
        }
    }
}

constexpr int DECS_WARPS = 8;

// one warp per branch of at most DEC_SMALL (= 64) shots: two shots per lane,
// held in registers from the first load to the in-place partition
__global__ void __launch_bounds__(DECS_WARPS * 32) k_decide_small(DevBatch d, const __grid_constant__ DecideDesc dd) {
    __shared__ DecTab tabs[DECS_WARPS];
    static_assert(DEC_SMALL == 64, "two shots per lane");
    const int n_br = d.ctl[CTL_NBR];
    const int NK = dd.nk;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    DecTab& T = tabs[warp];
    const int gw = blockIdx.x * DECS_WARPS + warp, nw = gridDim.x * DECS_WARPS;
    for (int b = gw; b < n_br; b += nw) {
        const int cnt = *reinterpret_cast<const volatile int32_t*>(&d.br_count[b]);
        if (cnt > DEC_SMALL) continue;
        // a count the big kernel has just lowered comes after its mark
        __threadfence();
        if (*reinterpret_cast<const volatile int32_t*>(&d.br_big[b]) == (int32_t)dd.op) continue;
        const int slot = d.br_slot[b], start = d.br_start[b];
        uint32_t sh[2];
        sh[0] = lane < cnt ? d.perm[start + lane] : 0u;
        sh[1] = lane + 32 < cnt ? d.perm[start + lane + 32] : 0u;
        branch_tables(d, dd, b, slot, T);
        for (int r = lane; r < NK; r += 32) {
            T.bincnt[r] = 0;
            T.binrun[r] = 0;
        }
        __syncwarp();
        int key[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            key[k] = lane + 32 * k < cnt ? chain_draw(d, dd, T, sh[k]) : -1;
            if (key[k] >= 0) atomicAdd(&T.bincnt[key[k]], 1);
        }
        __syncwarp();
        int ng = 0;
        if (lane == 0) {
            int acc = 0;
            for (int r = 0; r < NK; ++r)
                if (T.bincnt[r] > 0) {
                    T.binbase[r] = acc;
                    acc += T.bincnt[r];
                    ++ng;
                }
        }
        ng = __shfl_sync(0xffffffffu, ng, 0);
        __syncwarp();
        if (ng > 1 && dd.fork) {
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int kk = key[k];
                const unsigned peers = __match_any_sync(0xffffffffu, kk);
                const int rank = __popc(peers & ((1u << lane) - 1u));
                if (kk >= 0) d.perm[start + T.binbase[kk] + T.binrun[kk] + rank] = sh[k];
                __syncwarp();
                if (kk >= 0 && rank == 0) T.binrun[kk] += __popc(peers);
                __syncwarp();
            }
        }
        decide_groups(d, dd, b, start, T, false);
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// k_predraw: Pauli choices of every shot for the Pauli ops of a batch-mode
// circuit, drawn before the first gate (Section IV-A-3 samples Pauli noise
// ahead of applying it).  With one shot per branch a Pauli choice never
// forks anything, so no decide is needed: row q of pre_sel holds op q's
// choice per shot id, and the pass reads its branch's shot's entry.  The
// rows' descriptors sit in the integer pool at `table`, PRE_WORDS each: op,
// R, pool offsets of the R thresholds ceil(C * 2^53) and of the R running
// sums (both 64-bit words as int32 pairs), then the two log pointers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t ipool_u64(const int32_t* ip, int64_t off) {
    return (uint64_t)(uint32_t)ip[off] | ((uint64_t)(uint32_t)ip[off + 1] << 32);
}

__global__ void __launch_bounds__(256) k_predraw(DevBatch d, int n_rows, int table, int n_shots) {
    const int64_t total = (int64_t)n_rows * n_shots;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        const int q = (int)(i / n_shots);
        const uint32_t s = (uint32_t)(i % n_shots);
        const int32_t* e = d.ipool + table + (int64_t)PRE_WORDS * q;
        const uint32_t op = (uint32_t)e[0];
        const int R = e[1];
        const uint64_t* thr = reinterpret_cast<const uint64_t*>(d.ipool + e[2]);
        const double* cum = reinterpret_cast<const double*>(d.ipool + e[3]);
        const int sel = select_k(philox_k53(d.seed, d.shot_base + s, op), thr, cum, R);
        d.pre_sel[(int64_t)q * d.cap_br + s] = (uint8_t)sel;
        int32_t* log_sel = reinterpret_cast<int32_t*>(ipool_u64(d.ipool, table + (int64_t)PRE_WORDS * q + 4));
        double* log_thr = reinterpret_cast<double*>(ipool_u64(d.ipool, table + (int64_t)PRE_WORDS * q + 6));
        log_choice(log_sel, log_thr, s, sel, cum);
    }
}

cudaError_t launch_predraw(const DevBatch& d, int n_rows, int table, int n_shots, int grid, cudaStream_t s) {
    k_predraw<<<grid, 256, 0, s>>>(d, n_rows, table, n_shots);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// k_copy: parent state -> new branch slot (128-bit accesses)
// ---------------------------------------------------------------------------
// The forks of the last decide took ids [n_br, n_br + admitted) and their
// slots; copy each parent state into its children's slots, then (last CTA
// to finish) fold the new branches into the counts.
constexpr int COPY_VPT = 4;

__global__ void __launch_bounds__(256) k_copy(DevBatch d, int64_t state_vec16) {
    __shared__ int last;
    const int first = d.ctl[CTL_NBR];
    const int nalloc = d.ctl[CTL_NALLOC], n_free = d.ctl[CTL_NFREE];
    const int nb = nalloc < n_free ? nalloc : n_free;
    // work item = COPY_VPT * 256 16-byte words (16 KB); a thread issues all
    // its loads before its stores
    const int64_t per_item = COPY_VPT * 256;
    const int64_t items_per_state = (state_vec16 + per_item - 1) / per_item;
    const int64_t items = (int64_t)nb * items_per_state;
    const uint4* src_all = reinterpret_cast<const uint4*>(d.states);
    uint4* dst_all = reinterpret_cast<uint4*>(d.states);
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
        const int id = first + (int)(it / items_per_state);
        const int64_t c = it % items_per_state;
        const int src_slot = d.br_slot[d.br_parent[id]], dst_slot = d.br_slot[id];
        const uint4* src = src_all + (int64_t)src_slot * state_vec16;
        uint4* dst = dst_all + (int64_t)dst_slot * state_vec16;
        const int64_t lo = c * per_item + threadIdx.x;
        uint4 v[COPY_VPT];
#pragma unroll
        for (int k = 0; k < COPY_VPT; ++k)
            if (lo + 256 * k < state_vec16) v[k] = src[lo + 256 * k];
#pragma unroll
        for (int k = 0; k < COPY_VPT; ++k)
            if (lo + 256 * k < state_vec16) dst[lo + 256 * k] = v[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&d.ctl[CTL_DONE], 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        d.ctl[CTL_COPY_FIRST] = first;
        d.ctl[CTL_COPY_END] = first + nb;
        d.ctl[CTL_NBR] = first + nb;
        d.ctl[CTL_NFREE] = n_free - nb;
        d.ctl[CTL_NCOPIED] += nb;
        d.ctl[CTL_NALLOC] = 0;
        d.ctl[CTL_DONE] = 0;
        __threadfence();
    }
}

// ---------------------------------------------------------------------------
// final sampling (Section IV-B-2): per branch, prefix of |psi_j|^2 in index
// order, one draw per shot, first j with u < C_j
// ---------------------------------------------------------------------------
template <class R>
__global__ void __launch_bounds__(256) k_final_partials(DevBatch d, FinalDesc f) {
    using T = typename Cplx<R>::T;
    __shared__ double red_sh[32];
    const int n_br = d.ctl[CTL_NBR];
    const int64_t L = d.dim / f.chunks;
    const int64_t items = (int64_t)n_br * f.chunks;
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
        const int b = (int)(it / f.chunks), c = (int)(it % f.chunks);
        const int slot = d.br_slot[b];
        const T* g = reinterpret_cast<const T*>(d.states) + (int64_t)slot * d.dim + c * L;
        const double s = svs::chunk_sum<R>(g, L, red_sh);
        if (threadIdx.x == 0) d.partials[((int64_t)slot * d.max_chunks + c) * MAX_RED] = s;
    }
}

// per branch (one warp): running sum of the chunk sums (into partials[..][1])
// and the branch of every perm position it owns
__global__ void __launch_bounds__(256) k_final_cum(DevBatch d, FinalDesc f) {
    const int n_br = d.ctl[CTL_NBR];
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int b = gw; b < n_br; b += nw) {
        const int slot = d.br_slot[b], start = d.br_start[b], cnt = d.br_count[b];
        double* base = d.partials + (int64_t)slot * d.max_chunks * MAX_RED;
        svs::chunk_cum(base, base + 1, f.chunks, MAX_RED);
        for (int i = lane; i < cnt; i += 32) d.pos_branch[start + i] = b;
    }
}

// one warp per shot, over all live shots whatever their branch
template <class R>
__global__ void __launch_bounds__(256) k_final_sample(DevBatch d, FinalDesc f) {
    using T = typename Cplx<R>::T;
    const int n_br = d.ctl[CTL_NBR];
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int pos = gw; pos < d.cap_br; pos += nw) {
        const int b = d.pos_branch[pos];
        if (b < 0 || b >= n_br) continue;
        const int start = d.br_start[b], cnt = d.br_count[b];
        if (pos < start || pos >= start + cnt) continue;  // stale entry (waiting shot)
        const int slot = d.br_slot[b];
        const uint32_t s = d.perm[pos];
        const double u = philox_uniform(d.seed, d.shot_base + s, f.op);
        const T* g = reinterpret_cast<const T*>(d.states) + (int64_t)slot * d.dim;
        double lo, hi;
        const int64_t key = svs::sample_warp<R>(g, d.dim, f.chunks,
                                                d.partials + (int64_t)slot * d.max_chunks * MAX_RED + 1, MAX_RED, u,
                                                &lo, &hi);
        if (lane == 0) {
            d.keys[s] = (uint64_t)key;
            if (f.log_sel) f.log_sel[s] = (int32_t)key;
            if (f.log_thr) {
                f.log_thr[2 * (int64_t)s] = lo;
                f.log_thr[2 * (int64_t)s + 1] = hi;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// initialisation
// ---------------------------------------------------------------------------
template <class R>
__global__ void __launch_bounds__(256) k_init(DevBatch d, int n_init) {
    using T = typename Cplx<R>::T;
    // the root slots the reset created (none when a restart finds no
    // waiting shots)
    const int roots = d.ctl[CTL_NBR];
    const int64_t total = (int64_t)(n_init < roots ? n_init : roots) * d.dim;
    T* s = reinterpret_cast<T*>(d.states);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        T v;
        v.x = (i % d.dim == 0) ? (R)1 : (R)0;
        v.y = 0;
        s[i] = v;
    }
}

// a restart whose shot count is read on the device (inside a captured
// graph): the waiting count as the previous round left it
__global__ void k_wait_snapshot(DevBatch d) { d.ctl[CTL_NRUN] = d.ctl[CTL_NWAIT]; }

// from_wait: 0 shots 0 .. n_run-1; 1 the first n_run waiting shots; 2 every
// waiting shot (count from the device)
__global__ void __launch_bounds__(256) k_reset(DevBatch d, int branch_mode, int n_run, int from_wait) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (from_wait == 2) n_run = d.ctl[CTL_NRUN];
    for (int64_t i = t0; i < n_run; i += stride) d.perm[i] = from_wait ? d.wait_shots[i] : (uint32_t)i;
    const int nb = branch_mode ? (n_run > 0 ? 1 : 0) : n_run;
    for (int64_t b = t0; b < nb; b += stride) {
        d.br_slot[b] = (int)b;
        d.br_start[b] = branch_mode ? 0 : (int)b;
        d.br_count[b] = branch_mode ? n_run : 1;
        d.br_clbits[b] = 0;
        d.br_parent[b] = -1;
        d.br_big[b] = -1;
        // batch mode: the shot's own parameter set (shot-branching with a
        // sweep resets through k_reset_psets instead)
        d.br_pset[b] = d.pset_of_shot ? (int32_t)d.pset_of_shot[from_wait ? d.wait_shots[b] : (uint32_t)b] : 0;
        for (int q = 0; q < MAX_PEND; ++q) {
            d.br_sel[(int64_t)q * d.cap_br + b] = 0;
            d.br_scale[(int64_t)q * d.cap_br + b] = 1.0;
        }
    }
    const int n_free = d.n_slots - nb;
    for (int64_t j = t0; j < n_free; j += stride) d.free_slots[j] = d.n_slots - 1 - (int)j;
    if (t0 == 0) {
        d.ctl[CTL_NBR] = nb;
        d.ctl[CTL_NFREE] = n_free;
        d.ctl[CTL_NWAIT] = 0;
        d.ctl[CTL_COPY_FIRST] = 0;
        d.ctl[CTL_COPY_END] = 0;
        d.ctl[CTL_NALLOC] = 0;
        d.ctl[CTL_DONE] = 0;
    }
}

// Shot-branching with a parameter sweep: shots with different parameters
// never share a state, so a run starts with one root branch per parameter
// set that has shots (each a copy of |0...0>).  One CTA counts the shots of
// every set, lays the sets out one after another in perm (a counting sort;
// the order of shots inside a set is not fixed, and no result depends on
// it) and writes the root branches.
constexpr int RESET_PSET_THREADS = 1024;

__global__ void __launch_bounds__(RESET_PSET_THREADS) k_reset_psets(DevBatch d, int n_run, int from_wait) {
    __shared__ int cnt[MAX_PSETS], base[MAX_PSETS], run[MAX_PSETS];
    __shared__ int nb_sh;
    const int tid = threadIdx.x, nth = blockDim.x;
    if (from_wait == 2) n_run = d.ctl[CTL_NRUN];
    const int P = d.n_psets;
    for (int q = tid; q < P; q += nth) {
        cnt[q] = 0;
        run[q] = 0;
    }
    __syncthreads();
    for (int i = tid; i < n_run; i += nth) {
        const uint32_t s = from_wait ? d.wait_shots[i] : (uint32_t)i;
        atomicAdd(&cnt[d.pset_of_shot[s]], 1);
    }
    __syncthreads();
    if (tid == 0) {
        int acc = 0, nb = 0;
        for (int q = 0; q < P; ++q) {
            base[q] = acc;
            if (cnt[q] == 0) continue;
            d.br_slot[nb] = nb;
            d.br_start[nb] = acc;
            d.br_count[nb] = cnt[q];
            d.br_pset[nb] = q;
            acc += cnt[q];
            ++nb;
        }
        if (nb > d.n_slots) {  // the host checks this; a later slot limit could break it
            set_err(d, ERR_SLOT, nb);
            nb = 0;
        }
        nb_sh = nb;
    }
    __syncthreads();
    for (int i = tid; i < n_run; i += nth) {
        const uint32_t s = from_wait ? d.wait_shots[i] : (uint32_t)i;
        const int q = d.pset_of_shot[s];
        d.perm[base[q] + atomicAdd(&run[q], 1)] = s;
    }
    const int nb = nb_sh;
    for (int b = tid; b < nb; b += nth) {
        d.br_clbits[b] = 0;
        d.br_parent[b] = -1;
        d.br_big[b] = -1;
        for (int q = 0; q < MAX_PEND; ++q) {
            d.br_sel[(int64_t)q * d.cap_br + b] = 0;
            d.br_scale[(int64_t)q * d.cap_br + b] = 1.0;
        }
    }
    const int n_free = d.n_slots - nb;
    for (int j = tid; j < n_free; j += nth) d.free_slots[j] = d.n_slots - 1 - j;
    if (tid == 0) {
        d.ctl[CTL_NBR] = nb;
        d.ctl[CTL_NFREE] = n_free;
        d.ctl[CTL_NWAIT] = 0;
        d.ctl[CTL_COPY_FIRST] = 0;
        d.ctl[CTL_COPY_END] = 0;
        d.ctl[CTL_NALLOC] = 0;
        d.ctl[CTL_DONE] = 0;
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
size_t pass_smem_bytes(int prec, const PassDesc& p, int threads) {
    return ((pass_bytes_before_bars(p, threads, prec ? 16 : 8) + 7) & ~(size_t)7) + PASS_NBUF * 8;
}

cudaError_t init_kernels() {
    cudaError_t e = cudaFuncSetAttribute(k_pass<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_pass<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_decide_big, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DEC_BIG_SMEM);
    return e;
}

int pass_reg_threads(int prec) { return prec ? RegCta<double>::threads : RegCta<float>::threads; }

int pass_reg_variant(int prec, const PassDesc& p) {
    if (prec) return REG_PLAIN;
    return p.fold ? REG_FOLD : (p.red_kind == RED_BINS ? REG_BINS : REG_PLAIN);
}

// the instantiations live in sv_reg_c64.cu, sv_reg_c64x.cu and sv_reg_c128.cu;
// folded and measurement-bin passes exist for complex64 only
const void* pass_reg_fn(int prec, int wp, int paired, int var) {
    if (prec) return reg_kernel_c128(wp);
    if (var == REG_FOLD) return reg_kernel_fold_c64(wp, paired);
    if (var == REG_BINS) return reg_kernel_bins_c64(paired);
    return reg_kernel_plain_c64(wp, paired);
}

int pass_reg_blocks_per_sm(int prec, int wp, int paired, int var, size_t smem) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pass_reg_fn(prec, wp, paired, var), pass_reg_threads(prec),
                                                      smem) != cudaSuccess) {
        cudaGetLastError();
        n = 1;
    }
    return n > 0 ? n : 1;
}

size_t pass_reg_smem_bytes(int prec, const PassDesc& p, int threads) {
    const size_t c = prec ? 16 : 8;
    const size_t nw = threads / 32;
    const size_t m = (size_t)((p.mat_elems + 1) & ~1);
    const size_t g = (size_t)1 << p.reg_wp;
    return nw * (m * c + 4 * MAX_STAGES * 4) + (prec ? 0 : nw * m * 16) + (p.fold && !prec ? nw * g * g * 8 : 0) +
           (p.red_kind == RED_BINS ? nw * REG_MAX_BINS * 32 * 8 : 0);
}

cudaError_t launch_pass(const DevBatch& d, int prec, const PassDesc& p, int threads, int grid, cudaStream_t s) {
    if (p.reg_wp > 0) {
        const int threads = pass_reg_threads(prec);
        const size_t smem = pass_reg_smem_bytes(prec, p, threads);
        const void* f = pass_reg_fn(prec, p.reg_wp, p.reg_paired && !prec, pass_reg_variant(prec, p));
        void* args[] = {(void*)&d, (void*)&p};
        return cudaLaunchKernel(f, dim3(grid), dim3(threads), args, smem, s);
    }
    const size_t smem = pass_smem_bytes(prec, p, threads);
    if (prec) k_pass<double><<<grid, threads, smem, s>>>(d, p);
    else k_pass<float><<<grid, threads, smem, s>>>(d, p);
    return cudaGetLastError();
}

static int resident_blocks(const void* fn, int threads, size_t smem = 0) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        n = 1;
    }
    return n > 0 ? n : 1;
}

cudaError_t launch_decide(const DevBatch& d, const DecideDesc& dd, int n_sm, cudaStream_t s, cudaStream_t side,
                          cudaEvent_t ev_fork, cudaEvent_t ev_join) {
    // The two kernels run side by side: the big one on the side stream,
    // forked from and joined back to the batch's stream (a fork / join that
    // graph capture records as two parallel nodes).  A big branch whose
    // count drops to DEC_SMALL or fewer is marked before its count changes,
    // so the small kernel never decides it again (br_big).  Both kernels are
    // latency-bound and grid-stride over the branches, so each launches
    // exactly one resident wave.
    static const int small_per_sm = resident_blocks((const void*)k_decide_small, DECS_WARPS * 32);
    static const int big_per_sm = resident_blocks((const void*)k_decide_big, DEC_THREADS, DEC_BIG_SMEM);
    cudaError_t e = cudaEventRecord(ev_fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(side, ev_fork, 0);
    if (e != cudaSuccess) return e;
    k_decide_big<<<big_per_sm * n_sm, DEC_THREADS, DEC_BIG_SMEM, side>>>(d, dd);
    k_decide_small<<<small_per_sm * n_sm, DECS_WARPS * 32, 0, s>>>(d, dd);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(ev_join, side);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev_join, 0);
    return e;
}



cudaError_t launch_copy(const DevBatch& d, int prec, int grid, cudaStream_t s) {
    const int64_t vec16 = d.dim * (prec ? 16 : 8) / 16;
    k_copy<<<grid, 256, 0, s>>>(d, vec16);
    return cudaGetLastError();
}

cudaError_t launch_final(const DevBatch& d, int prec, const FinalDesc& f, int grid, cudaStream_t s) {
    if (prec) {
        k_final_partials<double><<<4 * grid, 256, 0, s>>>(d, f);  // HBM-bound: 8 CTAs per SM
        k_final_cum<<<grid, 256, 0, s>>>(d, f);
        k_final_sample<double><<<grid, 256, 0, s>>>(d, f);
    } else {
        k_final_partials<float><<<4 * grid, 256, 0, s>>>(d, f);  // HBM-bound: 8 CTAs per SM
        k_final_cum<<<grid, 256, 0, s>>>(d, f);
        k_final_sample<float><<<grid, 256, 0, s>>>(d, f);
    }
    return cudaGetLastError();
}

cudaError_t launch_init(const DevBatch& d, int prec, int n_init_slots, int grid, cudaStream_t s) {
    if (prec) k_init<double><<<grid, 256, 0, s>>>(d, n_init_slots);
    else k_init<float><<<grid, 256, 0, s>>>(d, n_init_slots);
    return cudaGetLastError();
}

cudaError_t launch_reset(const DevBatch& d, int mode_branch, int n_shots_run, int from_wait, int grid,
                         cudaStream_t s) {
    if (from_wait == 2) k_wait_snapshot<<<1, 1, 0, s>>>(d);
    if (mode_branch && d.pset_of_shot) k_reset_psets<<<1, RESET_PSET_THREADS, 0, s>>>(d, n_shots_run, from_wait);
    else k_reset<<<grid, 256, 0, s>>>(d, mode_branch, n_shots_run, from_wait);
    return cudaGetLastError();
}

}  // namespace sv
