// Host runtime of libsv: batch memory, the pass scheduler, CUDA-graph
// capture, and the C ABI declared in include/sv.h.
//
// Scheduler.  Ops are not launched one by one.  Gates and the per-branch
// application of already-sampled noise/measurement choices are queued as
// *stages*; a queue is flushed as one pass launch (one read and one write of
// every live state) when a random op needs probabilities from the current
// state (Kraus, measurement), when the pass would exceed its fusion width,
// or when the state is read.  Pauli choices do not depend on the state
// (Section IV-A-3) and are sampled without touching it: in batch mode all
// of them up front (k_predraw), otherwise by a decide.  A decide that
// follows another with no pass between joins it as a chain, and in
// shot-branching mode each decide is followed by k_copy, so no host
// synchronisation happens inside a circuit (Section IV-A-4).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/sv.h"
#include "sv_internal.h"

using namespace sv;

namespace {

thread_local std::string g_err;

sv_status fail(sv_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

#define CU(call)                                                                                     \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess) return fail(SV_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

struct PendStage {
    int kind, k;
    int q[MAX_STAGE_Q];
    int cond_clbit, cond_val, pend, reset, off, stride;
    int pre;  // ST_PAULI_BR: row of the pre-drawn table (batch mode), not a pending column
};

// a Pauli op of a batch-mode circuit whose choices are drawn up front
struct PreRow {
    uint32_t op;
    int R;
    int thr_off, cum_off;  // integer-pool offsets of the thresholds and running sums
    int32_t* log_sel;
    double* log_thr;
};

enum LType { L_INIT, L_RESET, L_PASS, L_DECIDE, L_ALLOC, L_COPY, L_FINAL, L_PREDRAW };
enum PClass { P_PASS = 0, P_DECIDE, P_ALLOC, P_COPY, P_FINAL, P_INIT, P_OTHER, P_N };

struct Launch {
    LType type;
    int a0 = 0, a1 = 0, a2 = 0;
    uint32_t op = 0;
    PassDesc pass;
    DecideDesc dec;
    FinalDesc fin;
};

// Philox4x32-10 on the host (plain per-shot mode draws on the host, as the
// conventional implementation does); published constants of Salmon et al.
double host_uniform(uint64_t seed, uint64_t shot, uint32_t op) {
    uint32_t k[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t x[4] = {(uint32_t)shot, (uint32_t)(shot >> 32), op, 0u};
    for (int r = 0; r < 10; ++r) {
        const uint64_t m0 = (uint64_t)0xD2511F53u * x[0];
        const uint64_t m1 = (uint64_t)0xCD9E8D57u * x[2];
        const uint32_t y0 = (uint32_t)(m1 >> 32) ^ x[1] ^ k[0];
        const uint32_t y2 = (uint32_t)(m0 >> 32) ^ x[3] ^ k[1];
        x[1] = (uint32_t)m1;
        x[3] = (uint32_t)m0;
        x[0] = y0;
        x[2] = y2;
        k[0] += 0x9E3779B9u;
        k[1] += 0xBB67AE85u;
    }
    const uint64_t top = ((((uint64_t)x[0]) << 32) | x[1]) >> 11;
    return (double)top * (1.0 / 9007199254740992.0);
}

int host_select(double u, const double* cum, int n) {
    for (int t = 0; t < n; ++t)
        if (u < cum[t]) return t;
    for (int t = n - 1; t >= 0; --t)
        if (cum[t] > (t ? cum[t - 1] : 0.0)) return t;
    return n - 1;
}

}  // namespace

namespace sv {
// message for sv_last_error() from other translation units of the library
void set_last_error(const std::string& msg) { g_err = msg; }
}  // namespace sv

struct sv_batch_s {
    int n = 0;
    uint64_t n_shots = 0;
    int n_clbits = 0;
    sv_prec prec = SV_C64;
    sv_mode mode = SV_BATCH;
    uint64_t seed = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // side stream and fork / join events: the two decide kernels run side
    // by side (also inside captured graphs)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int64_t dim = 0;
    size_t amp_bytes = 8, state_bytes = 0;
    int n_slots = 0;
    int tb = 11, chunks = 1, chunks_final = 1;
    int red_chunks = 1;  // chunk records written by the last pass with a reduction
    int threads = 256, grid_pass = 0, grid_small = 0, n_sm = 0;
    int max_active = 8, max_stages = MAX_STAGES;  // max_active is set in sv_alloc_batch
    bool max_active_set = false;  // SV_OPT_MAX_ACTIVE given explicitly (a new tile size keeps it)
    bool threads_set = false;     // SV_OPT_THREADS given explicitly
    bool branch = false;
    // device memory
    std::vector<void*> allocs;
    DevBatch dev{};
    void* d_pool = nullptr;
    int32_t* d_ipool = nullptr;
    size_t pool_cap = 0, ipool_cap = 0;
    // host pool (append-only between resets; pinned staging for async upload)
    std::vector<double> pool;
    std::vector<int32_t> ipool;
    size_t pool_up = 0, ipool_up = 0;
    void* h_pool = nullptr;
    int32_t* h_ipool = nullptr;
    // scheduler
    std::vector<PendStage> pend;
    uint64_t active = 0;
    uint64_t col_used = 0;  // per-branch choice columns held by pending stages
    int mat_used = 0;
    // recorded circuits: a pass takes a dependency-closed subset of the
    // pending stages, so stages on other qubits can wait for a later pass
    bool commute = true;
    bool fold = true;  // SV_OPT_FOLD
    bool whole = false;  // SV_OPT_WHOLE_STATE
    std::vector<Launch>* rec = nullptr;
    bool started = false;
    uint32_t last_random = 0xffffffffu;
    // per-op calls in shot-branching mode: the decide of the last random op
    // has drawn its choices; sv_branch (or the next call) commits its forks
    bool uncommitted = false;
    Launch commit;
    // logging
    bool log = false;
    std::map<uint32_t, std::pair<int32_t*, double*>> logs;
    // statistics
    uint64_t n_launch = 0, n_passes = 0, restarts = 0;
    // profiling
    bool profile = false;
    double prof_ms[P_N] = {};
    int64_t prof_cnt[P_N] = {};
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof_ev;
    // graph cache
    uint64_t graph_hash = 0;
    cudaGraphExec_t graph_exec = nullptr;
    int64_t graph_launches = 0;
    std::vector<uint8_t> graph_pass_store;
    std::vector<uint8_t> pass_store;  // per executed pass: writes the state back
    bool upload_each = false;
    double h2d_bytes = 0;
    int pass_path = 0;  // 0 auto, 1 shared-memory tiles only
    // sv_run_circuits: one graph over several batches (kept by the first)
    uint64_t multi_hash = 0;
    cudaGraphExec_t multi_exec = nullptr;
    cudaGraphExec_t multi_restart_exec = nullptr;  // waiting-list restarts of the same batches
    std::vector<std::vector<Launch>> multi_lists;
    std::vector<uint64_t> multi_gens;
    // the constant pool holds one recorded circuit at a time; every recording
    // (and every growth of the pool) starts a new generation, and a cached
    // graph replays only while the generations it captured are current
    uint64_t pool_gen = 0, graph_gen = 0;
    bool joint = true;  // decide back-to-back one-qubit Kraus pairs from one pass
    bool chain = true;  // decide ops that need no pass between in one launch
    bool predraw = true;  // batch mode: Pauli choices drawn up front, no decides
    std::vector<PreRow> pre_rows;  // of the circuit being recorded
    int pre_cap = 0;               // rows the device table holds
    std::map<int, int> reg_occ;
    int slot_limit = 0;
    // parameter sweep (sv_set_param_sets): every shot's parameter set
    int n_psets = 0;
    std::vector<uint32_t> h_pset;
    // branch tree of the last run (with SV_OPT_LOG in shot-branching modes):
    // per round (the first pass, then each waiting-list restart) the fork
    // events logged by its end and the shot permutation as it stood then
    struct TreeRound {
        int64_t fork_end;
        int n_run;
        std::vector<uint32_t> perm;
    };
    std::vector<TreeRound> tree;
};

namespace {

template <class T> sv_status dalloc(sv_batch b, T** p, size_t count) {
    void* q = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc(&q, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(SV_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    b->allocs.push_back(q);
    *p = reinterpret_cast<T*>(q);
    return SV_OK;
}

int pclass(LType t) {
    switch (t) {
    case L_PASS: return P_PASS;
    case L_DECIDE: return P_DECIDE;
    case L_PREDRAW: return P_DECIDE;
    case L_ALLOC: return P_ALLOC;
    case L_COPY: return P_COPY;
    case L_FINAL: return P_FINAL;
    case L_INIT: return P_INIT;
    default: return P_OTHER;
    }
}

// threads of a tile-path CTA: the batch's setting (default 128: a CTA's
// stages wait on each other's barriers, and more, smaller CTAs keep more
// tiles in flight; measured faster than 256 on whole-state and on 20-qubit
// tiles), at least one per form of the pass's reduction (each thread
// writes one form's partial)
int tile_threads(sv_batch b, const PassDesc& p) {
    int t = b->threads_set ? b->threads : 128;
    while (t < 256 && t < p.red_R) t *= 2;
    return t;
}

int pass_grid(sv_batch b, const PassDesc& p) {
    if (b->grid_pass > 0) return b->grid_pass;
    if (p.whole) return b->n_sm * pass_whole_blocks_per_sm(b->n);
    if (p.reg_wp > 0) {
        const int prec = b->prec == SV_C128;
        const size_t smem = pass_reg_smem_bytes(prec, p, pass_reg_threads(prec));
        const int var = pass_reg_variant(prec, p);
        const int key = ((p.reg_wp * 2 + prec) * 2 + p.reg_paired) * 3 + var;
        auto it = b->reg_occ.find(key * 4096 + (int)(smem / 64));
        int per_sm;
        if (it == b->reg_occ.end()) {
            per_sm = pass_reg_blocks_per_sm(prec, p.reg_wp, p.reg_paired, var, smem);
            b->reg_occ[key * 4096 + (int)(smem / 64)] = per_sm;
        } else {
            per_sm = it->second;
        }
        return b->n_sm * per_sm;
    }
    // k_pass is register-bound at 512 threads per SM (two CTAs of 256);
    // shared memory (tile ring + matrices + accumulators) may allow fewer
    const int threads = tile_threads(b, p);
    const size_t smem = pass_smem_bytes(b->prec == SV_C128, p, threads) + 2048;
    const int per_sm = (int)std::max<size_t>(1, std::min<size_t>(512 / threads, (227 * 1024) / smem));
    return b->n_sm * per_sm;
}

cudaError_t exec_one(sv_batch b, const Launch& L) {
    const int prec = b->prec == SV_C128;
    switch (L.type) {
    case L_INIT: return launch_init(b->dev, prec, L.a0, b->n_sm * 4, b->stream);
    case L_RESET: return launch_reset(b->dev, L.a0, L.a1, L.a2, b->n_sm * 2, b->stream);
    case L_PASS:
        if (L.pass.whole) return launch_pass_whole(b->dev, L.pass, pass_grid(b, L.pass), b->stream);
        return launch_pass(b->dev, prec, L.pass, tile_threads(b, L.pass), pass_grid(b, L.pass), b->stream);
    case L_DECIDE: return launch_decide(b->dev, L.dec, b->n_sm, b->stream, b->side, b->ev_fork, b->ev_join);
    case L_ALLOC: return cudaSuccess;
    case L_COPY: return launch_copy(b->dev, prec, b->n_sm * 4, b->stream);
    case L_FINAL: return launch_final(b->dev, prec, L.fin, b->grid_small, b->stream);
    case L_PREDRAW: return launch_predraw(b->dev, L.a0, L.a1, L.a2, b->n_sm * 4, b->stream);
    }
    return cudaErrorInvalidValue;
}

sv_status exec(sv_batch b, const Launch& L) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (b->profile && !b->rec) {
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, b->stream);
    }
    cudaError_t e = exec_one(b, L);
    if (e != cudaSuccess) return fail(SV_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    if (e0) {
        cudaEventRecord(e1, b->stream);
        b->prof_ev.push_back({pclass(L.type), {e0, e1}});
    }
    b->n_launch += L.type == L_FINAL ? 3 : (L.type == L_DECIDE ? 2 : 1);
    if (L.type == L_PASS) {
        b->n_passes += 1;
        b->pass_store.push_back(L.pass.store ? 1 : 0);
    }
    return SV_OK;
}

sv_status emit(sv_batch b, Launch&& L) {
    if (b->rec) {
        b->rec->push_back(std::move(L));
        return SV_OK;
    }
    return exec(b, L);
}

// ---- pool ------------------------------------------------------------------
// grow the device pool and its pinned staging copy (everything is uploaded
// again afterwards)
sv_status grow_pool(sv_batch b) {
    CU(cudaStreamSynchronize(b->stream));
    size_t pc = b->pool_cap, ic = b->ipool_cap;
    while (pc < b->pool.size()) pc *= 2;
    while (ic < b->ipool.size()) ic *= 2;
    void *dp = nullptr, *hp = nullptr, *di = nullptr, *hi = nullptr;
    if (cudaMalloc(&dp, pc * 8) != cudaSuccess || cudaMallocHost(&hp, pc * 8) != cudaSuccess ||
        cudaMalloc(&di, ic * 4) != cudaSuccess || cudaMallocHost(&hi, ic * 4) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(dp);
        cudaFreeHost(hp);
        cudaFree(di);
        return fail(SV_ENOMEM, "cannot grow the constant pool");
    }
    cudaFree(b->d_pool);
    cudaFreeHost(b->h_pool);
    cudaFree(b->d_ipool);
    cudaFreeHost(b->h_ipool);
    b->d_pool = dp;
    b->h_pool = hp;
    b->d_ipool = (int32_t*)di;
    b->h_ipool = (int32_t*)hi;
    b->pool_cap = pc;
    b->ipool_cap = ic;
    b->pool_gen += 1;
    b->dev.pool = dp;
    b->dev.ipool = (const int32_t*)di;
    b->pool_up = b->ipool_up = 0;
    return SV_OK;
}

sv_status upload_pool(sv_batch b) {
    const size_t rsz = b->prec == SV_C128 ? 8 : 4;
    if (b->pool.size() > b->pool_cap || b->ipool.size() > b->ipool_cap) {
        sv_status st = grow_pool(b);
        if (st) return st;
    }
    if (b->pool.size() > b->pool_up) {
        for (size_t i = b->pool_up; i < b->pool.size(); ++i) {
            if (rsz == 8) reinterpret_cast<double*>(b->h_pool)[i] = b->pool[i];
            else reinterpret_cast<float*>(b->h_pool)[i] = (float)b->pool[i];
        }
        CU(cudaMemcpyAsync((char*)b->d_pool + b->pool_up * rsz, (char*)b->h_pool + b->pool_up * rsz,
                           (b->pool.size() - b->pool_up) * rsz, cudaMemcpyHostToDevice, b->stream));
        b->h2d_bytes += (double)(b->pool.size() - b->pool_up) * rsz;
        b->pool_up = b->pool.size();
    }
    if (b->ipool.size() > b->ipool_up) {
        for (size_t i = b->ipool_up; i < b->ipool.size(); ++i) b->h_ipool[i] = b->ipool[i];
        CU(cudaMemcpyAsync(b->d_ipool + b->ipool_up, b->h_ipool + b->ipool_up,
                           (b->ipool.size() - b->ipool_up) * 4, cudaMemcpyHostToDevice, b->stream));
        b->h2d_bytes += (double)(b->ipool.size() - b->ipool_up) * 4;
        b->ipool_up = b->ipool.size();
    }
    return SV_OK;
}

sv_status reset_pool(sv_batch b) {
    CU(cudaStreamSynchronize(b->stream));  // staging buffers are about to be rewritten
    b->pool.clear();
    b->ipool.clear();
    b->pool_up = b->ipool_up = 0;
    return SV_OK;
}

int pool_matrix(sv_batch b, const double* m, int k, double scale = 1.0) {
    const int off = (int)b->pool.size();
    const int e = 1 << (2 * k);
    for (int i = 0; i < 2 * e; ++i) b->pool.push_back(m[i] * scale);
    return off;
}

// ---- scheduler ---------------------------------------------------------------
// Default fusion width: passes on at most 4 qubits run in registers
// (k_pass_reg), many-stage ones folded; wider fusion goes to shared-memory
// tiles.  Measured on GB300 over 28 circuits of 6-11 qubits, width 4 took
// 30.2 ms in batch mode against 34.7 ms for whole-state tiles.
constexpr int DEFAULT_MAX_ACTIVE = 4;

bool whole_active(sv_batch b);
int local_pos(const int* tile_q, int tb, int q) {
    for (int i = 0; i < tb; ++i)
        if (tile_q[i] == q) return i;
    return -1;
}

// Flush queued stages as one pass; optionally end it with a reduction.
struct RedSpec {
    int kind = RED_NONE, k = 0, R = 0, off = 0;
    int diag_off = -1;  // RED_FORMS whose forms are all diagonal: weights here
    int q[MAX_STAGE_Q] = {};
};

// Rough per-group instruction counts of the register kernel (a group is
// G = 2^wp amplitudes of one lane): every stage costs a dispatch plus its
// arithmetic; a folded pass costs G x G complex products (four FMAs each,
// one shared-memory load per two) and one composition per branch.  The
// folded product is bound by delivering its matrix from shared memory, so
// it has to save half the estimated work to pay.
int stage_group_cost(sv_batch b, const PendStage& ps, int G) {
    int c = 40;  // stage dispatch: descriptor loads, skip test, switch
    if (ps.kind == ST_DENSE || ps.kind == ST_DENSE_BR) {
        const double* m = ps.kind == ST_DENSE ? &b->pool[ps.off] : nullptr;
        auto z = [&](int e) { return m[2 * e] == 0 && m[2 * e + 1] == 0; };
        if (ps.k == 1) {
            const bool shaped = m && ((z(1) && z(2)) || (z(0) && z(3)));
            c += shaped ? 2 * G : (m ? 8 * G : 4 * G);
        } else {
            int nz = 0;
            if (m)
                for (int e = 0; e < 16; ++e) nz += !z(e);
            c += nz == 4 ? 2 * G : 12 * G;
        }
    } else if (ps.kind == ST_PAULI_BR) {
        c += 3 * G;
    } else {
        c += 2 * G;
    }
    return c;
}

bool fold_pays(sv_batch b, const std::vector<const PendStage*>& ss, int wp) {
    const int G = 1 << wp;
    int64_t c = 0;
    for (const PendStage* ps : ss) c += stage_group_cost(b, *ps, G);
    return c * 2 > 3 * (int64_t)(3 * G * G + 60);
}

// can a pass run in registers (k_pass_reg)?  at most 4 qubits, dense stages
// of at most 2 qubits, and no reduction, diagonal forms, <= 4 one-qubit
// forms, or the outcome bins of a measurement of at most 4 qubits
int reg_width(sv_batch b, const RedSpec& red, uint64_t act, const std::vector<const PendStage*>& ss) {
    if (b->pass_path == 1) return 0;
    const int wp = __builtin_popcountll(act);
    if (wp > 4 || wp < 1) return 0;
    for (const PendStage* ps : ss)
        if ((ps->kind == ST_DENSE || ps->kind == ST_DENSE_BR) && ps->k > 2) return 0;
    // measurement bins: complex64 groups of exactly 4 qubits (the kernel
    // variant exists for that shape only)
    if (red.kind == RED_BINS && (wp != 4 || b->prec == SV_C128)) return 0;
    // diagonal forms reduce to 2^k bins (any number of forms); general
    // forms take one accumulator each (at most 4, one qubit)
    if (red.kind == RED_FORMS && red.diag_off < 0 && (red.R > 4 || red.k != 1)) return 0;
    // the per-warp matrix copies must fit the default 48 KB of dynamic
    // shared memory of the register kernels; longer stage lists take tiles
    PassDesc probe;
    memset(&probe, 0, sizeof(probe));
    probe.reg_wp = wp;
    probe.red_kind = red.kind;
    for (const PendStage* ps : ss)
        probe.mat_elems += (ps->kind == ST_DENSE || ps->kind == ST_DENSE_BR) ? 1 << (2 * ps->k)
                                                                            : (ps->kind == ST_PROJ_BR ? 1 : 0);
    if (red.kind == RED_FORMS) probe.mat_elems += 2 * (red.diag_off >= 0 ? red.R << red.k : red.R << (2 * red.k));
    const int prec = b->prec == SV_C128;
    if (pass_reg_smem_bytes(prec, probe, pass_reg_threads(prec)) > 48 * 1024) return 0;
    return wp;
}

uint64_t stage_mask(const PendStage& s) {
    uint64_t m = 0;
    for (int j = 0; j < s.k; ++j) m |= 1ull << s.q[j];
    return m;
}

int stage_mats(const PendStage& s) {
    return (s.kind == ST_DENSE || s.kind == ST_DENSE_BR) ? 1 << (2 * s.k) : (s.kind == ST_PROJ_BR ? 1 : 0);
}

// the stage holds a per-branch choice column (a sampled op's choice)
bool stage_has_col(const PendStage& s) { return s.kind != ST_DENSE && !s.pre && s.pend >= 0; }

// Stages that may wait past a reduction on other qubits: unconditional
// unitaries (gates, Pauli strings, a parameter set's matrix).  The
// probabilities of a Kraus op or a measurement on qubits R do not change
// under a unitary on qubits outside R (it commutes with the forms / the
// projectors and keeps norms); a chosen Kraus matrix or a projection does
// not keep norms, and a conditional gate reads classical bits a later
// measurement may rewrite.
bool stage_deferrable(const PendStage& s) {
    if (s.cond_clbit >= 0) return false;
    return s.kind == ST_DENSE || s.kind == ST_PAULI_BR || (s.kind == ST_DENSE_BR && s.pend == PEND_PSET);
}

// one pass: the pending stages idx (ascending, a dependency-closed subset in
// op order) and an optional reduction; the stages leave the queue and their
// choice columns are free again
sv_status emit_stages(sv_batch b, const std::vector<int>& idx, const RedSpec& red) {
    if (idx.empty() && red.kind == RED_NONE) return SV_OK;
    std::vector<const PendStage*> ss;
    for (int i : idx) ss.push_back(&b->pend[i]);
    Launch L;
    L.type = L_PASS;
    PassDesc& p = L.pass;
    memset(&p, 0, sizeof(p));
    p.n = b->n;
    p.tb = b->tb;
    uint64_t act = 0;
    for (const PendStage* ps : ss) act |= stage_mask(*ps);
    for (int j = 0; j < red.k; ++j) act |= 1ull << red.q[j];
    // a whole-state warp pass: no reduction, stages of at most 4 qubits
    // (dense ones of at most 2), its matrices within 48 KB per CTA
    bool whole = whole_active(b) && red.kind == RED_NONE && !ss.empty();
    if (whole) {
        int m = 0;
        for (const PendStage* ps : ss) {
            if (ps->k > 4 || ((ps->kind == ST_DENSE || ps->kind == ST_DENSE_BR) && ps->k > 2)) whole = false;
            m += (ps->kind == ST_DENSE || ps->kind == ST_DENSE_BR) ? 1 << (2 * ps->k) : (ps->kind == ST_PROJ_BR ? 1 : 0);
        }
        PassDesc probe;
        memset(&probe, 0, sizeof(probe));
        probe.mat_elems = m;
        if (pass_whole_smem_bytes(probe) > 48 * 1024) whole = false;
    }
    const int wp = whole ? 0 : reg_width(b, red, act, ss);
    if (whole) {
        // every qubit, in order: stage positions are the logical qubits
        act = b->n >= 64 ? ~0ull : (1ull << b->n) - 1;
        p.tb = b->n;
        p.whole = 1;
    } else if (wp > 0) {
        // register group: exactly the pass's qubits; with qubit 0 among them
        // complex64 amplitudes move as 128-bit pairs
        p.tb = wp;
        p.reg_paired = (int)(act & 1ull);
    } else {
        // tile: qubit 0 (complex64 moves amplitude pairs 2j, 2j+1 with one
        // 128-bit access), every active qubit, then the lowest others
        act |= 1ull;
    }
    std::vector<int> tq;
    for (int q = 0; q < b->n; ++q)
        if ((act >> q) & 1) tq.push_back(q);
    if ((int)tq.size() > p.tb) return fail(SV_EINTERNAL, "pass holds more qubits than a tile");
    for (int q = 0; q < b->n && (int)tq.size() < p.tb; ++q)
        if (!((act >> q) & 1)) tq.push_back(q);
    std::sort(tq.begin(), tq.end());
    for (int i = 0; i < p.tb; ++i) p.tile_q[i] = tq[i];
    int run = 0;
    while (run < p.tb && p.tile_q[run] == run) ++run;
    p.run_bits = run;
    p.n_nontile = 0;
    for (int q = 0; q < b->n; ++q)
        if (std::find(tq.begin(), tq.end(), q) == tq.end()) p.nontile_q[p.n_nontile++] = q;
    p.reg_wp = wp;
    if (wp > 0) {
        // register path: a warp's unit holds at least REG_UNIT_MIN_AMPS
        // amplitudes, so the fixed-order combination of its reduction is
        // paid once per several hundred groups
        const int64_t unit = std::max<int64_t>(b->dim / b->chunks, REG_UNIT_MIN_AMPS);
        p.chunks = (int)std::max<int64_t>(1, b->dim / unit);
        p.tiles_per_chunk = 1;
    } else {
        // tile path: a chunk spans at least eight tiles (or the whole
        // state), so the fixed-order combination of its reduction is paid
        // once per several tiles
        const int64_t tiles = 1ll << (b->n - p.tb);
        const int64_t tpc = std::max<int64_t>(tiles / b->chunks, std::min<int64_t>(tiles, 8));
        p.chunks = (int)(tiles / tpc);
        p.tiles_per_chunk = (int)tpc;
    }
    if (red.kind != RED_NONE) b->red_chunks = p.chunks;
    int mat = 0;
    if ((int)ss.size() > MAX_STAGES) return fail(SV_EINTERNAL, "pass holds more stages than a pass descriptor");
    p.n_stages = (int)ss.size();
    for (int s = 0; s < p.n_stages; ++s) {
        const PendStage& ps = *ss[s];
        Stage& st = p.st[s];
        st.kind = ps.kind;
        st.k = ps.k;
        for (int j = 0; j < ps.k; ++j) st.pos[j] = local_pos(p.tile_q, p.tb, ps.q[j]);
        st.cond_clbit = ps.cond_clbit;
        st.cond_val = ps.cond_val;
        st.pend = ps.pend;
        st.reset = ps.reset;
        st.off = ps.off;
        st.stride = ps.stride;
        st.pre = ps.pre;
        st.mat = 0;
        if (ps.kind == ST_DENSE || ps.kind == ST_DENSE_BR) {
            st.mat = mat;
            mat += 1 << (2 * ps.k);
        } else if (ps.kind == ST_PROJ_BR && (wp > 0 || p.whole)) {
            st.mat = mat;  // the register and whole-state paths keep the scale here
            mat += 1;
        }
    }
    p.store = p.n_stages > 0;
    p.red_kind = red.kind;
    p.red_k = red.k;
    p.red_R = red.R;
    p.red_off = red.off;
    if (red.kind == RED_FORMS && red.diag_off >= 0) {  // diagonal forms: bins, weights per chunk
        p.red_kind = RED_DIAG;
        p.red_off = red.diag_off;
    }
    for (int j = 0; j < red.k; ++j) p.red_pos[j] = local_pos(p.tile_q, p.tb, red.q[j]);
    // forms (or diagonal weights) and their float32 residuals
    if (p.red_kind == RED_FORMS) mat += 2 * (red.R << (2 * red.k));
    else if (p.red_kind == RED_DIAG) mat += 2 * (red.R << red.k);
    p.mat_elems = mat;
    if (wp > 0 && b->fold && b->prec == SV_C64 && red.kind == RED_NONE && p.store && fold_pays(b, ss, wp)) {
        p.fold = 1;
        if (pass_reg_smem_bytes(0, p, pass_reg_threads(0)) > 48 * 1024) p.fold = 0;
    }
    // the rest of the queue stays pending
    std::vector<PendStage> rest;
    std::vector<char> taken(b->pend.size(), 0);
    for (int i : idx) taken[i] = 1;
    for (size_t i = 0; i < b->pend.size(); ++i) {
        if (taken[i]) {
            if (stage_has_col(b->pend[i])) b->col_used &= ~(1ull << b->pend[i].pend);
        } else {
            rest.push_back(b->pend[i]);
        }
    }
    b->pend.swap(rest);
    b->active = 0;
    b->mat_used = 0;
    for (const PendStage& ps : b->pend) {
        b->active |= stage_mask(ps);
        b->mat_used += stage_mats(ps);
    }
    return emit(b, std::move(L));
}

// every pending stage in one pass
sv_status emit_pass(sv_batch b, const RedSpec& red) {
    std::vector<int> all(b->pend.size());
    for (size_t i = 0; i < all.size(); ++i) all[i] = (int)i;
    return emit_stages(b, all, red);
}

bool fits(sv_batch b, uint64_t act);

bool commute_on(sv_batch b) { return b->commute && b->rec; }

constexpr int POOL_MAX = 2 * MAX_STAGES;  // pending stages that may wait for a later pass

// The stages of the next pass, chosen from the pending queue.  A stage can
// join when every earlier pending stage on one of its qubits has joined
// (stages on disjoint qubits commute), so the pass is a dependency-closed
// subset and runs its stages in op order.  Without a reduction the pass
// grows from the oldest stage; with one (qubits red_q) it starts from the
// stages the reduction must see: those on red_q, every non-deferrable stage,
// and everything earlier on their qubits.  It then takes every stage that
// adds no qubit, and, while the width allows, the stage adding the fewest
// new qubits (ties: the one touching the most of the pass's qubits, then the
// earliest).  Returns false when the required stages do not fit one pass.
bool select_pass(sv_batch b, uint64_t red_q, bool for_red, int red_mats, std::vector<int>& out) {
    const int n = (int)b->pend.size();
    const int budget = MAT_SMEM - 256;
    std::vector<char> in(n, 0);
    uint64_t pq = red_q;
    int cnt = 0, mats = red_mats;
    if (for_red) {
        uint64_t later = 0;
        for (int t = n - 1; t >= 0; --t) {
            const PendStage& s = b->pend[t];
            const uint64_t m = stage_mask(s);
            if ((m & red_q) || !stage_deferrable(s) || (m & later)) {
                in[t] = 1;
                later |= m;
                pq |= m;
                ++cnt;
                mats += stage_mats(s);
            }
        }
        if (!fits(b, pq) || cnt > b->max_stages || (cnt > 0 && mats > budget)) return false;
    } else if (n > 0) {
        in[0] = 1;
        pq |= stage_mask(b->pend[0]);
        cnt = 1;
        mats += stage_mats(b->pend[0]);
    }
    for (;;) {
        bool changed = true;
        while (changed) {  // stages adding no qubit
            changed = false;
            uint64_t blocked = 0;
            for (int t = 0; t < n; ++t) {
                if (in[t]) continue;
                const PendStage& s = b->pend[t];
                const uint64_t m = stage_mask(s);
                if (!(m & blocked) && !(m & ~pq) && cnt < b->max_stages && mats + stage_mats(s) <= budget) {
                    in[t] = 1;
                    ++cnt;
                    mats += stage_mats(s);
                    changed = true;
                } else {
                    blocked |= m;
                }
            }
        }
        int best = -1, best_new = 99, best_touch = -1;
        uint64_t blocked = 0;
        for (int t = 0; t < n; ++t) {
            if (in[t]) continue;
            const PendStage& s = b->pend[t];
            const uint64_t m = stage_mask(s);
            if (!(m & blocked) && fits(b, pq | m) && cnt < b->max_stages && mats + stage_mats(s) <= budget) {
                const int nw = __builtin_popcountll(m & ~pq), touch = __builtin_popcountll(m & pq);
                if (nw < best_new || (nw == best_new && touch > best_touch)) {
                    best = t;
                    best_new = nw;
                    best_touch = touch;
                }
            }
            blocked |= m;
        }
        if (best < 0) break;
        in[best] = 1;
        pq |= stage_mask(b->pend[best]);
        ++cnt;
        mats += stage_mats(b->pend[best]);
    }
    out.clear();
    for (int t = 0; t < n; ++t)
        if (in[t]) out.push_back(t);
    return true;
}

// one pass grown from the oldest pending stage
sv_status emit_oldest(sv_batch b) {
    std::vector<int> idx;
    select_pass(b, 0, false, 0, idx);
    return emit_stages(b, idx, RedSpec());
}

sv_status flush(sv_batch b) {
    if (!commute_on(b)) return emit_pass(b, RedSpec());
    while (!b->pend.empty()) {
        sv_status st = emit_oldest(b);
        if (st) return st;
    }
    return SV_OK;
}

// the pass of a reduction on red.q (forms or bins holding red_mats matrix
// entries), after whatever passes the pending stages need first
sv_status emit_reduction(sv_batch b, const RedSpec& red, int red_mats) {
    uint64_t rq = 0;
    for (int j = 0; j < red.k; ++j) rq |= 1ull << red.q[j];
    if (!commute_on(b)) {
        if (!fits(b, b->active | rq) || b->mat_used + red_mats > MAT_SMEM - 256) {
            sv_status st = flush(b);
            if (st) return st;
        }
        return emit_pass(b, red);
    }
    for (;;) {
        std::vector<int> idx;
        if (select_pass(b, rq, true, red_mats, idx)) return emit_stages(b, idx, red);
        if (b->pend.empty()) return fail(SV_EINTERNAL, "a reduction does not fit one pass");
        sv_status st = emit_oldest(b);
        if (st) return st;
    }
}

int alloc_col(sv_batch b);

// a free per-branch choice column, emitting passes until one is free
sv_status get_col(sv_batch b, int* col) {
    while ((*col = alloc_col(b)) < 0) {
        if (b->pend.empty()) return fail(SV_EINTERNAL, "no free choice column");
        sv_status st = commute_on(b) ? emit_oldest(b) : flush(b);
        if (st) return st;
    }
    return SV_OK;
}

// a free per-branch choice column (-1: none)
int alloc_col(sv_batch b) {
    for (int c = 0; c < MAX_PEND; ++c)
        if (!((b->col_used >> c) & 1)) {
            b->col_used |= 1ull << c;
            return c;
        }
    return -1;
}

// whole-state warp passes apply (complex64 states of 9 or 10 qubits)
bool whole_active(sv_batch b) { return b->whole && b->prec == SV_C64 && (b->n == 9 || b->n == 10); }

// qubits of a pass fit one tile (which always holds qubit 0); with
// whole-state passes a pass may take every qubit
bool fits(sv_batch b, uint64_t act) {
    if (whole_active(b)) return true;
    return __builtin_popcountll(act | 1ull) <= b->tb && __builtin_popcountll(act) <= b->max_active;
}

// make room for a stage on qubits q[0..k-1] with `mats` matrix entries
sv_status make_room(sv_batch b, const int* q, int k, int mats, bool needs_pend) {
    if (commute_on(b)) {
        // the queue may span more qubits than a pass; passes leave it when
        // it is long or holds every choice column
        sv_status st = SV_OK;
        while (!st && ((int)b->pend.size() >= POOL_MAX || (needs_pend && b->col_used == ~0ull)))
            st = emit_oldest(b);
        return st;
    }
    uint64_t act = b->active;
    for (int j = 0; j < k; ++j) act |= 1ull << q[j];
    if (!fits(b, act) || (int)b->pend.size() >= b->max_stages ||
        b->mat_used + mats > MAT_SMEM - 256 || (needs_pend && b->col_used == ~0ull))
        return flush(b);
    return SV_OK;
}

void add_stage(sv_batch b, const PendStage& s) {
    b->pend.push_back(s);
    for (int j = 0; j < s.k; ++j) b->active |= 1ull << s.q[j];
    if (s.kind == ST_DENSE || s.kind == ST_DENSE_BR) b->mat_used += 1 << (2 * s.k);
}

sv_status tree_begin(sv_batch b);

// slots that hold |0...0> when a run (or a waiting-list restart) begins:
// every shot's own in batch mode; in shot-branching mode one root, or one
// per parameter set of a sweep
int root_slots(sv_batch b, int n_run) {
    if (!b->branch) return n_run;
    return b->n_psets > 0 ? std::min(b->n_psets, b->dev.n_slots) : 1;
}

sv_status ensure_started(sv_batch b) {
    if (b->started) return SV_OK;
    if (!b->rec) {  // per-op calls: a new run, a new fork log
        sv_status st = tree_begin(b);
        if (st) return st;
    }
    const int branch = b->branch;
    Launch r;
    r.type = L_RESET;
    r.a0 = branch;
    r.a1 = (int)b->n_shots;
    r.a2 = 0;
    sv_status st = emit(b, std::move(r));
    if (st) return st;
    Launch i;
    i.type = L_INIT;
    i.a0 = root_slots(b, (int)b->n_shots);
    st = emit(b, std::move(i));
    if (st) return st;
    b->started = true;
    return SV_OK;
}

sv_status check_qubits(sv_batch b, int k, const int* q) {
    if (!q && k > 0) return fail(SV_EINVAL, "qubits is NULL");
    for (int j = 0; j < k; ++j) {
        if (q[j] < 0 || q[j] >= b->n) return fail(SV_EINVAL, "qubit out of range");
        for (int i = 0; i < j; ++i)
            if (q[i] == q[j]) return fail(SV_EINVAL, "repeated qubit");
    }
    return SV_OK;
}

sv_status get_log(sv_batch b, uint32_t op, int32_t** sel, double** thr) {
    *sel = nullptr;
    *thr = nullptr;
    if (!b->log) return SV_OK;
    auto it = b->logs.find(op);
    if (it == b->logs.end()) {
        int32_t* s = nullptr;
        double* t = nullptr;
        sv_status st = dalloc(b, &s, b->n_shots);
        if (st) return st;
        st = dalloc(b, &t, 2 * b->n_shots);
        if (st) return st;
        cudaMemsetAsync(s, 0xff, b->n_shots * 4, b->stream);
        it = b->logs.emplace(op, std::make_pair(s, t)).first;
    }
    *sel = it->second.first;
    *thr = it->second.second;
    return SV_OK;
}

// decide (+ fork) for random op `op`; the chosen term is then queued as a stage
// A decide that directly follows another in the recorded launch list (no
// pass between) joins it as a tail op when it needs no new reduction: the
// second op of a joint Kraus pair right after the first, or any Pauli op.
// One launch and one copy then serve the whole chain.
bool chain_decide(sv_batch b, uint32_t op, int kind, int R, const double* cum, int pend) {
    if (!b->rec || b->rec->empty()) return false;
    std::vector<Launch>& rec = *b->rec;
    size_t i = rec.size() - 1;
    if (b->branch) {
        if (rec[i].type != L_COPY || i == 0) return false;
        --i;
    }
    if (rec[i].type != L_DECIDE) return false;
    DecideDesc& h = rec[i].dec;
    if (h.n_tail >= MAX_TAIL || (int64_t)h.nk * R > MAX_TERMS) return false;
    if (kind == DEC_KRAUS_J2) {
        if (h.kind != DEC_KRAUS_J1 || h.n_tail != 0 || R != h.r2) return false;
    } else if (kind != DEC_PAULI) {
        return false;
    }
    int used = 0;
    for (int t = 0; t < h.n_tail; ++t)
        if (h.tail[t].kind == DEC_PAULI) used = std::max(used, h.tail[t].cum_off + h.tail[t].R);
    if (kind == DEC_PAULI && used + R > MAX_TAIL_TERMS) return false;
    DecideTail& tl = h.tail[h.n_tail];
    memset(&tl, 0, sizeof(tl));
    tl.op = op;
    tl.kind = kind;
    tl.R = R;
    tl.pend = pend;
    if (get_log(b, op, &tl.log_sel, &tl.log_thr)) return false;
    if (kind == DEC_PAULI) {
        tl.cum_off = used;
        for (int t = 0; t < R; ++t) {
            h.tail_cum[used + t] = cum[t];
            // ceil(c * 2^53): the scaling is exact, as on the device
            h.tail_thr[used + t] = cum[t] > 0.0 ? (uint64_t)std::ceil(cum[t] * 9007199254740992.0) : 0ull;
        }
    }
    h.n_tail += 1;
    h.nk *= R;
    return true;
}

sv_status emit_decide(sv_batch b, uint32_t op, int kind, int R, const double* cum, int pend, int m,
                      const int* clbits, int r2 = 0, int pend_prev = -1) {
    if (b->chain && chain_decide(b, op, kind, R, cum, pend)) {
        b->last_random = op;
        return SV_OK;
    }
    Launch L;
    L.type = L_DECIDE;
    DecideDesc& d = L.dec;
    memset(&d, 0, sizeof(d));
    d.op = op;
    d.kind = kind;
    d.R = R;
    d.pend = pend;
    d.chunks = b->red_chunks;  // the pass just emitted wrote these
    d.fork = b->branch;
    d.m = m;
    d.r2 = r2;
    d.pend_prev = pend_prev;
    d.nk = R;
    d.live_cols = b->col_used;
    for (int j = 0; j < m; ++j) d.clbit[j] = clbits[j];
    if (cum)
        for (int t = 0; t < R; ++t) d.cum[t] = cum[t];
    sv_status st = get_log(b, op, &d.log_sel, &d.log_thr);
    if (st) return st;
    if (b->branch && !b->rec) {
        // per-op call in shot-branching mode (Section IV-B-2's sample, then
        // branch): this launch draws and logs every shot's choice; the same
        // keyed draws fork the branches when sv_branch commits
        b->commit = L;
        d.sample_only = 1;
        d.fork = 0;
        st = emit(b, std::move(L));
        if (st) return st;
        b->uncommitted = true;
        b->last_random = op;
        return SV_OK;
    }
    st = emit(b, std::move(L));
    if (st) return st;
    if (b->branch) {
        Launch c;
        c.type = L_COPY;
        st = emit(b, std::move(c));
        if (st) return st;
    }
    b->last_random = op;
    return SV_OK;
}

// fork the branches of the last sampled op (per-op calls, shot-branching)
sv_status commit_forks(sv_batch b) {
    if (!b->uncommitted) return SV_OK;
    b->uncommitted = false;
    sv_status st = exec(b, b->commit);
    if (st) return st;
    Launch c;
    c.type = L_COPY;
    return exec(b, c);
}

bool is_unitary(const double* m, int k, double tol) {
    const int D = 1 << k;
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
            std::complex<double> s = 0;
            for (int r = 0; r < D; ++r)
                s += std::conj(std::complex<double>(m[2 * (r * D + i)], m[2 * (r * D + i) + 1])) *
                     std::complex<double>(m[2 * (r * D + j)], m[2 * (r * D + j) + 1]);
            if (std::abs(s - (i == j ? 1.0 : 0.0)) > tol) return false;
        }
    return true;
}

// ---- op implementations (batched modes) --------------------------------------
sv_status op_gate(sv_batch b, int k, const int* q, const double* mat, int cond_clbit, int cond_val) {
    sv_status st = check_qubits(b, k, q);
    if (st) return st;
    if (k < 1 || k > MAX_GATE_Q) return fail(SV_EUNSUPPORTED, "gates act on 1 to 5 qubits");
    if (!mat) return fail(SV_EINVAL, "matrix is NULL");
    {
        uint64_t gq = 1ull;  // a tile always holds qubit 0
        for (int j = 0; j < k; ++j) gq |= 1ull << q[j];
        if (__builtin_popcountll(gq) > b->tb) return fail(SV_EUNSUPPORTED, "the gate's qubits do not fit one tile");
    }
    if (cond_clbit >= b->n_clbits || cond_clbit < -1) return fail(SV_EINVAL, "condition bit out of range");
    if (!is_unitary(mat, k, 1e-10)) return fail(SV_EINVAL, "gate matrix is not unitary");
    if ((st = ensure_started(b))) return st;
    if ((st = make_room(b, q, k, 1 << (2 * k), false))) return st;
    PendStage s{};
    s.kind = ST_DENSE;
    s.k = k;
    for (int j = 0; j < k; ++j) s.q[j] = q[j];
    s.cond_clbit = cond_clbit;
    s.cond_val = cond_val;
    s.off = pool_matrix(b, mat, k);
    add_stage(b, s);
    return SV_OK;
}

// A dense matrix on k <= MAX_GATE_Q qubits that need not be unitary: the
// density-matrix method's superoperators (vec(rho) is a state of 2n qubits)
sv_status op_superop(sv_batch b, int k, const int* q, const double* mat) {
    sv_status st = check_qubits(b, k, q);
    if (st) return st;
    if (k < 1 || k > MAX_GATE_Q) return fail(SV_EUNSUPPORTED, "superoperators act on 1 to 5 qubits");
    if ((st = ensure_started(b))) return st;
    if ((st = make_room(b, q, k, 1 << (2 * k), false))) return st;
    PendStage s{};
    s.kind = ST_DENSE;
    s.k = k;
    for (int j = 0; j < k; ++j) s.q[j] = q[j];
    s.cond_clbit = -1;
    s.off = pool_matrix(b, mat, k);
    add_stage(b, s);
    // a later make_room may flush this stage: its matrix must be on the device
    return upload_pool(b);
}

// Section VI: a gate whose parameters vary between shots.  The matrix of
// every parameter set goes to the pool; the stage takes, per branch, the
// matrix of the branch's parameter set (all shots of a branch share it).
sv_status op_pgate(sv_batch b, int k, const int* q, const double* mats, int n_sets) {
    sv_status st = check_qubits(b, k, q);
    if (st) return st;
    if (k < 1 || k > 2) return fail(SV_EUNSUPPORTED, "parameterized gates act on 1 or 2 qubits");
    if (!mats) return fail(SV_EINVAL, "matrices are NULL");
    if (b->n_psets == 0) return fail(SV_EINVAL, "no parameter sets (sv_set_param_sets) on this batch");
    if (n_sets != b->n_psets) return fail(SV_EINVAL, "one matrix per parameter set of the batch is needed");
    const int E = 1 << (2 * k);
    for (int j = 0; j < n_sets; ++j)
        if (!is_unitary(mats + 2 * (size_t)E * j, k, 1e-10)) return fail(SV_EINVAL, "a parameter set's matrix is not unitary");
    if ((st = ensure_started(b))) return st;
    if ((st = make_room(b, q, k, E, false))) return st;
    PendStage s{};
    s.kind = ST_DENSE_BR;
    s.k = k;
    for (int j = 0; j < k; ++j) s.q[j] = q[j];
    s.cond_clbit = -1;
    s.pend = PEND_PSET;
    s.off = (int)b->pool.size();
    s.stride = 2 * E;
    for (size_t i = 0; i < 2 * (size_t)E * n_sets; ++i) b->pool.push_back(mats[i]);
    add_stage(b, s);
    return SV_OK;
}

int pauli_packed(const char* str, int k) {
    int xm = 0, zm = 0, ny = 0;
    for (int j = 0; j < k; ++j) {
        const char c = str[j];
        if (c == 'X' || c == 'Y') xm |= 1 << j;
        if (c == 'Z' || c == 'Y') zm |= 1 << j;
        if (c == 'Y') ++ny;
    }
    return xm | (zm << 4) | ((ny & 3) << 8);
}

sv_status op_pauli(sv_batch b, uint32_t op, int k, const int* q, int n_terms, const double* cum,
                   const char* paulis) {
    sv_status st = check_qubits(b, k, q);
    if (st) return st;
    if (k < 1 || k > 4) return fail(SV_EUNSUPPORTED, "Pauli noise acts on 1 to 4 qubits");
    if (n_terms < 1 || n_terms > MAX_TERMS) return fail(SV_EUNSUPPORTED, "Pauli noise has 1 to 64 terms");
    if (!cum || !paulis) return fail(SV_EINVAL, "Pauli table is NULL");
    for (int t = 0; t < n_terms; ++t) {
        if (t && cum[t] < cum[t - 1]) return fail(SV_EINVAL, "cumulative probabilities decrease");
        for (int j = 0; j < k; ++j)
            if (!strchr("IXYZ", paulis[t * k + j]) || !paulis[t * k + j]) return fail(SV_EINVAL, "bad Pauli character");
    }
    if ((st = ensure_started(b))) return st;
    // batch mode, whole circuits: the choice of every shot is drawn up front
    // (k_predraw), so the op needs no decide and no pending column
    const bool pre = b->rec && !b->branch && b->predraw &&
                     (uint64_t)(b->pre_rows.size() + 1) * b->n_shots <= PRE_TABLE_BYTES;
    if ((st = make_room(b, q, k, 0, !pre))) return st;
    const int off = (int)b->ipool.size();
    for (int t = 0; t < n_terms; ++t) b->ipool.push_back(pauli_packed(paulis + t * k, k));
    int pend;
    if (pre) {
        PreRow r{};
        r.op = op;
        r.R = n_terms;
        if (b->ipool.size() & 1) b->ipool.push_back(0);  // 64-bit words start 8-byte aligned
        r.thr_off = (int)b->ipool.size();
        for (int t = 0; t < n_terms; ++t) {
            // ceil(C * 2^53): the scaling is exact, as on the device
            const uint64_t thr = cum[t] > 0.0 ? (uint64_t)std::ceil(cum[t] * 9007199254740992.0) : 0ull;
            b->ipool.push_back((int32_t)(uint32_t)thr);
            b->ipool.push_back((int32_t)(uint32_t)(thr >> 32));
        }
        r.cum_off = (int)b->ipool.size();
        for (int t = 0; t < n_terms; ++t) {
            uint64_t bits;
            memcpy(&bits, &cum[t], 8);
            b->ipool.push_back((int32_t)(uint32_t)bits);
            b->ipool.push_back((int32_t)(uint32_t)(bits >> 32));
        }
        if ((st = get_log(b, op, &r.log_sel, &r.log_thr))) return st;
        pend = (int)b->pre_rows.size();
        b->pre_rows.push_back(r);
        b->last_random = op;
    } else {
        if ((st = get_col(b, &pend))) return st;
        if ((st = upload_pool(b))) return st;
        if ((st = emit_decide(b, op, DEC_PAULI, n_terms, cum, pend, 0, nullptr))) return st;
    }
    PendStage s{};
    s.pre = pre ? 1 : 0;
    s.kind = ST_PAULI_BR;
    s.k = k;
    for (int j = 0; j < k; ++j) s.q[j] = q[j];
    s.cond_clbit = -1;
    s.pend = pend;
    s.off = off;
    add_stage(b, s);
    return SV_OK;
}

// F_i = K_i^dagger K_i of every term (row-major complex)
std::vector<std::complex<double>> kraus_forms(const double* kraus, int k, int n_terms) {
    const int D = 1 << k, E = D * D;
    std::vector<std::complex<double>> F((size_t)E * n_terms);
    for (int t = 0; t < n_terms; ++t) {
        const double* K = kraus + 2 * E * t;
        for (int i = 0; i < D; ++i)
            for (int j = 0; j < D; ++j) {
                std::complex<double> s = 0;
                for (int r = 0; r < D; ++r)
                    s += std::conj(std::complex<double>(K[2 * (r * D + i)], K[2 * (r * D + i) + 1])) *
                         std::complex<double>(K[2 * (r * D + j)], K[2 * (r * D + j) + 1]);
                F[(size_t)E * t + i * D + j] = s;
            }
    }
    return F;
}

bool kraus_complete(const std::vector<std::complex<double>>& F, int k, int n_terms) {
    const int D = 1 << k, E = D * D;
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
            std::complex<double> s = 0;
            for (int t = 0; t < n_terms; ++t) s += F[(size_t)E * t + i * D + j];
            if (std::abs(s - (i == j ? 1.0 : 0.0)) > 1e-10) return false;
        }
    return true;
}

// Quadratic-form coefficients carry a second copy holding their float32
// residuals v - (float)v: a complex64 reduction evaluates each form as
// hi + lo, so the coefficients enter at float64-grade accuracy (a float32
// coefficient alone would shift every probability by the same relative
// ~3e-8, which no summation order averages out).  Zero for complex128.
void push_residuals(sv_batch b, int off, int n) {
    for (int i = 0; i < n; ++i) {
        const double v = b->pool[off + i];
        b->pool.push_back(b->prec == SV_C64 ? v - (double)(float)v : 0.0);
    }
}

// push forms (and, when all are diagonal, their diagonals) into the pool,
// each followed by its residuals
void push_forms(sv_batch b, const std::vector<std::complex<double>>& F, int k, int R, RedSpec& red) {
    const int D = 1 << k, E = D * D;
    red.off = (int)b->pool.size();
    bool diag = true;
    for (int f = 0; f < R; ++f)
        for (int i = 0; i < D; ++i)
            for (int j = 0; j < D; ++j) {
                const std::complex<double> v = F[(size_t)E * f + i * D + j];
                b->pool.push_back(v.real());
                b->pool.push_back(v.imag());
                if (i != j && v != 0.0) diag = false;
            }
    push_residuals(b, red.off, 2 * R * E);
    red.diag_off = -1;
    if (diag) {
        red.diag_off = (int)b->pool.size();
        for (int f = 0; f < R; ++f)
            for (int i = 0; i < D; ++i) {
                b->pool.push_back(F[(size_t)E * f + i * D + i].real());
                b->pool.push_back(0.0);
            }
        push_residuals(b, red.diag_off, 2 * R * D);
    }
}

sv_status op_kraus(sv_batch b, uint32_t op, int k, const int* q, int n_terms, const double* kraus) {
    sv_status st = check_qubits(b, k, q);
    if (st) return st;
    if (k < 1 || k > 2) return fail(SV_EUNSUPPORTED, "Kraus noise acts on 1 or 2 qubits");
    if (n_terms < 1 || n_terms > MAX_RED) return fail(SV_EUNSUPPORTED, "Kraus noise has 1 to 16 matrices");
    if (!kraus) return fail(SV_EINVAL, "Kraus matrices are NULL");
    const int D = 1 << k, E = D * D;
    const std::vector<std::complex<double>> F = kraus_forms(kraus, k, n_terms);
    if (!kraus_complete(F, k, n_terms)) return fail(SV_EINVAL, "Kraus matrices are not complete (sum K^dagger K != I)");
    if ((st = ensure_started(b))) return st;
    // the reduction must see every earlier op that does not commute with it
    RedSpec red;
    red.kind = RED_FORMS;
    red.k = k;
    red.R = n_terms;
    for (int j = 0; j < k; ++j) red.q[j] = q[j];
    push_forms(b, F, k, n_terms, red);
    const int mat_off = (int)b->pool.size();
    for (int i = 0; i < 2 * E * n_terms; ++i) b->pool.push_back(kraus[i]);
    if ((st = upload_pool(b))) return st;
    if ((st = emit_reduction(b, red, 2 * n_terms * E))) return st;
    int pend;
    if ((st = get_col(b, &pend))) return st;
    if ((st = emit_decide(b, op, DEC_KRAUS, n_terms, nullptr, pend, 0, nullptr))) return st;
    PendStage s{};
    s.kind = ST_DENSE_BR;
    s.k = k;
    for (int j = 0; j < k; ++j) s.q[j] = q[j];
    s.cond_clbit = -1;
    s.pend = pend;
    s.off = mat_off;
    s.stride = 2 * E;
    if ((st = make_room(b, q, k, E, true))) return st;
    add_stage(b, s);
    return SV_OK;
}

// Two one-qubit Kraus ops on different qubits, back to back: one pass
// reduces the joint probabilities p_ij = ||K2_j K1_i psi||^2 (forms
// F1_i (x) F2_j); op 1 is decided from p_i = sum_j p_ij = ||K1_i psi||^2 and
// op 2, per branch, from p_ij / p_i = ||K2_j (K1_i psi / sqrt(p_i))||^2,
// which is the sequential rule of Section III-B-2 computed in one pass.
sv_status op_kraus_pair(sv_batch b, uint32_t op1, int qa, int n1, const double* k1, uint32_t op2, int qb, int n2,
                        const double* k2) {
    sv_status st;
    int qs[2] = {qa, qb};
    if ((st = check_qubits(b, 2, qs))) return st;
    if (!k1 || !k2) return fail(SV_EINVAL, "Kraus matrices are NULL");
    const std::vector<std::complex<double>> F1 = kraus_forms(k1, 1, n1), F2 = kraus_forms(k2, 1, n2);
    if (!kraus_complete(F1, 1, n1) || !kraus_complete(F2, 1, n2))
        return fail(SV_EINVAL, "Kraus matrices are not complete (sum K^dagger K != I)");
    if ((st = ensure_started(b))) return st;
    // joint forms on [qa, qb]: matrix index bit 0 <-> qa, bit 1 <-> qb
    std::vector<std::complex<double>> F((size_t)16 * n1 * n2);
    for (int i = 0; i < n1; ++i)
        for (int j = 0; j < n2; ++j)
            for (int r = 0; r < 4; ++r)
                for (int c = 0; c < 4; ++c)
                    F[(size_t)16 * (i * n2 + j) + r * 4 + c] = F1[4 * i + (r & 1) * 2 + (c & 1)] *
                                                              F2[4 * j + (r >> 1) * 2 + (c >> 1)];
    RedSpec red;
    red.kind = RED_FORMS;
    red.k = 2;
    red.R = n1 * n2;
    red.q[0] = qa;
    red.q[1] = qb;
    push_forms(b, F, 2, n1 * n2, red);
    const int m1 = (int)b->pool.size();
    for (int i = 0; i < 8 * n1; ++i) b->pool.push_back(k1[i]);
    const int m2 = (int)b->pool.size();
    for (int i = 0; i < 8 * n2; ++i) b->pool.push_back(k2[i]);
    if ((st = upload_pool(b))) return st;
    if ((st = emit_reduction(b, red, 2 * n1 * n2 * 16))) return st;
    int pend1, pend2;
    if ((st = get_col(b, &pend1))) return st;
    if ((st = emit_decide(b, op1, DEC_KRAUS_J1, n1, nullptr, pend1, 0, nullptr, n2, -1))) return st;
    if ((st = get_col(b, &pend2))) return st;
    if ((st = emit_decide(b, op2, DEC_KRAUS_J2, n2, nullptr, pend2, 0, nullptr, n2, pend1))) return st;
    PendStage s{};
    s.kind = ST_DENSE_BR;
    s.k = 1;
    s.cond_clbit = -1;
    s.q[0] = qa;
    s.pend = pend1;
    s.off = m1;
    s.stride = 8;
    add_stage(b, s);
    s.q[0] = qb;
    s.pend = pend2;
    s.off = m2;
    add_stage(b, s);
    return SV_OK;
}

sv_status op_measure(sv_batch b, uint32_t op, int m, const int* q, const int* clbits, int reset) {
    sv_status st = check_qubits(b, m, q);
    if (st) return st;
    if (m < 1 || m > 4) return fail(SV_EUNSUPPORTED, "measurements take 1 to 4 qubits");
    if (!clbits) return fail(SV_EINVAL, "clbits is NULL");
    for (int j = 0; j < m; ++j)
        if (clbits[j] < 0 || clbits[j] >= b->n_clbits) return fail(SV_EINVAL, "classical bit out of range");
    if ((st = ensure_started(b))) return st;
    RedSpec red;
    red.kind = RED_BINS;
    red.k = m;
    red.R = 1 << m;
    for (int j = 0; j < m; ++j) red.q[j] = q[j];
    if ((st = upload_pool(b))) return st;
    if ((st = emit_reduction(b, red, 0))) return st;
    int pend;
    if ((st = get_col(b, &pend))) return st;
    if ((st = emit_decide(b, op, DEC_MEASURE, 1 << m, nullptr, pend, m, clbits))) return st;
    PendStage s{};
    s.kind = ST_PROJ_BR;
    s.k = m;
    for (int j = 0; j < m; ++j) s.q[j] = q[j];
    s.cond_clbit = -1;
    s.pend = pend;
    s.reset = reset ? 1 : 0;
    add_stage(b, s);
    return SV_OK;
}

sv_status op_final(sv_batch b, uint32_t op) {
    sv_status st = ensure_started(b);
    if (st) return st;
    if ((st = upload_pool(b))) return st;
    if ((st = flush(b))) return st;
    Launch L;
    L.type = L_FINAL;
    memset(&L.fin, 0, sizeof(L.fin));
    L.fin.op = op;
    L.fin.chunks = b->chunks_final;
    if ((st = get_log(b, op, &L.fin.log_sel, &L.fin.log_thr))) return st;
    return emit(b, std::move(L));
}

sv_status check_device_error(sv_batch b) {
    int32_t ctl[CTL_WORDS];
    CU(cudaMemcpyAsync(ctl, b->dev.ctl, sizeof(ctl), cudaMemcpyDeviceToHost, b->stream));
    CU(cudaStreamSynchronize(b->stream));
    if (ctl[CTL_ERR] == ERR_TIMEOUT) return fail(SV_ETIMEOUT, "device wait timed out");
    if (ctl[CTL_ERR] != 0) {
        char buf[128];
        snprintf(buf, sizeof(buf), "device error %d (info %d)", ctl[CTL_ERR], ctl[CTL_ERR_INFO]);
        return fail(SV_EINTERNAL, buf);
    }
    return SV_OK;
}

sv_status read_ctl(sv_batch b, int32_t* ctl) {
    CU(cudaMemcpyAsync(ctl, b->dev.ctl, sizeof(int32_t) * CTL_WORDS, cudaMemcpyDeviceToHost, b->stream));
    CU(cudaStreamSynchronize(b->stream));
    return SV_OK;
}

// the end of a round of a logged shot-branching run: keep the shot
// permutation (a fork event's shot set is a range of it, valid until the
// waiting list restarts)
sv_status tree_snapshot(sv_batch b, const int32_t* ctl, int n_run) {
    if (!b->log || !b->branch || !b->dev.fork_log) return SV_OK;
    sv_batch_s::TreeRound r;
    r.fork_end = ctl[CTL_NFORK];
    r.n_run = n_run;
    r.perm.resize(b->n_shots);
    CU(cudaMemcpyAsync(r.perm.data(), b->dev.perm, b->n_shots * 4, cudaMemcpyDeviceToHost, b->stream));
    CU(cudaStreamSynchronize(b->stream));
    b->tree.push_back(std::move(r));
    return SV_OK;
}

// a logged run starts a new fork log and branch tree
sv_status tree_begin(sv_batch b) {
    b->tree.clear();
    if (!b->log || !b->dev.fork_log) return SV_OK;
    CU(cudaMemsetAsync(b->dev.ctl + CTL_NFORK, 0, 4, b->stream));
    return SV_OK;
}

// one op of a flattened circuit, batched modes
sv_status circuit_op(sv_batch b, const sv_circuit* c, int i) {
    const int kind = c->kind[i], k = c->nq[i];
    const int* q = c->qubits + c->q_off[i];
    const double* d = c->data + c->d_off[i];
    switch (kind) {
    case SV_OP_GATE: return op_gate(b, k, q, d, c->cond_clbit[i], c->cond_val[i]);
    case SV_OP_PAULI:
        return op_pauli(b, (uint32_t)i, k, q, c->n_terms[i], d, (const char*)c->paulis + c->s_off[i]);
    case SV_OP_KRAUS: return op_kraus(b, (uint32_t)i, k, q, c->n_terms[i], d);
    case SV_OP_MEASURE: return op_measure(b, (uint32_t)i, k, q, c->clbits + c->cl_off[i], c->reset[i]);
    case SV_OP_FINAL: return op_final(b, (uint32_t)i);
    case SV_OP_PGATE: return op_pgate(b, k, q, d, c->n_terms[i]);
    }
    return fail(SV_EINVAL, "unknown op kind");
}

uint64_t fnv(uint64_t h, const void* p, size_t n) {
    const unsigned char* c = (const unsigned char*)p;
    for (size_t i = 0; i < n; ++i) h = (h ^ c[i]) * 1099511628211ull;
    return h;
}

uint64_t circuit_hash(sv_batch b, const sv_circuit* c) {
    uint64_t h = 1469598103934665603ull;
    h = fnv(h, &c->n_qubits, 12);
    const size_t n = c->n_ops;
    h = fnv(h, c->kind, 4 * n);
    h = fnv(h, c->nq, 4 * n);
    h = fnv(h, c->q_off, 4 * n);
    h = fnv(h, c->n_terms, 4 * n);
    h = fnv(h, c->d_off, 8 * n);
    h = fnv(h, c->cond_clbit, 4 * n);
    h = fnv(h, c->cond_val, 4 * n);
    int64_t dmax = 0, qmax = 0;
    for (size_t i = 0; i < n; ++i) qmax = std::max<int64_t>(qmax, c->q_off[i] + c->nq[i]);
    h = fnv(h, c->qubits, 4 * qmax);
    for (size_t i = 0; i < n; ++i) {
        const int k = c->nq[i];
        int64_t len = 0;
        if (c->kind[i] == SV_OP_GATE) len = 2ll << (2 * k);
        else if (c->kind[i] == SV_OP_PAULI) len = c->n_terms[i];
        else if (c->kind[i] == SV_OP_KRAUS || c->kind[i] == SV_OP_PGATE) len = (int64_t)c->n_terms[i] * (2ll << (2 * k));
        dmax = std::max<int64_t>(dmax, c->d_off[i] + len);
    }
    h = fnv(h, c->data, 8 * dmax);
    for (size_t i = 0; i < n; ++i)
        if (c->kind[i] == SV_OP_PAULI) h = fnv(h, c->paulis + c->s_off[i], (size_t)c->n_terms[i] * c->nq[i]);
    h = fnv(h, &b->mode, sizeof(b->mode));
    return h;
}

// plain per-shot form: one state, one launch per op, host-side choices
sv_status run_plain(sv_batch b, const sv_circuit* c) {
    sv_status st;
    std::vector<uint64_t> keys(b->n_shots);
    for (uint64_t shot = 0; shot < b->n_shots; ++shot) {
        Launch r;
        r.type = L_RESET;
        r.a0 = 0;
        r.a1 = 1;
        r.a2 = 0;
        if ((st = exec(b, r))) return st;
        // perm[0] = shot
        uint32_t s32 = (uint32_t)shot;
        CU(cudaMemcpyAsync(b->dev.perm, &s32, 4, cudaMemcpyHostToDevice, b->stream));
        Launch in;
        in.type = L_INIT;
        in.a0 = 1;
        if ((st = exec(b, in))) return st;
        uint64_t clreg = 0;
        for (int i = 0; i < c->n_ops; ++i) {
            const int kind = c->kind[i], k = c->nq[i];
            const int* q = c->qubits + c->q_off[i];
            const double* d = c->data + c->d_off[i];
            if (kind == SV_OP_GATE) {
                if (c->cond_clbit[i] >= 0 && (int)((clreg >> c->cond_clbit[i]) & 1) != c->cond_val[i]) continue;
                if ((st = op_gate(b, k, q, d, -1, 0))) return st;
                if ((st = upload_pool(b))) return st;
                if ((st = flush(b))) return st;
            } else if (kind == SV_OP_PGATE) {
                // the shot's own parameter set, chosen on the host
                if (b->n_psets == 0 || c->n_terms[i] != b->n_psets)
                    return fail(SV_EINVAL, "parameterized gate without matching parameter sets");
                const uint32_t ps = b->h_pset[shot];
                if ((st = op_gate(b, k, q, d + (size_t)ps * (2ull << (2 * k)), -1, 0))) return st;
                if ((st = upload_pool(b))) return st;
                if ((st = flush(b))) return st;
            } else if (kind == SV_OP_PAULI) {
                const double u = host_uniform(b->seed, b->dev.shot_base + shot, (uint32_t)i);
                const int t = host_select(u, d, c->n_terms[i]);
                const char* str = (const char*)c->paulis + c->s_off[i] + t * k;
                if (pauli_packed(str, k) & 0xff) {
                    // a single-entry table makes the device choice the host's
                    double one[1] = {2.0};
                    if ((st = op_pauli(b, (uint32_t)i, k, q, 1, one, str))) return st;
                    if ((st = flush(b))) return st;
                }
            } else if (kind == SV_OP_KRAUS || kind == SV_OP_MEASURE) {
                // conventional form: one reduction per candidate, read back, compare on the host
                const int R = kind == SV_OP_KRAUS ? c->n_terms[i] : (1 << k);
                const int D = 1 << k, E = D * D;
                std::vector<double> p(R);
                for (int t = 0; t < R; ++t) {
                    RedSpec red;
                    red.k = k;
                    for (int j = 0; j < k; ++j) red.q[j] = q[j];
                    if (kind == SV_OP_KRAUS) {
                        red.kind = RED_FORMS;
                        red.R = 1;
                        red.off = (int)b->pool.size();
                        const double* K = d + 2 * E * t;
                        for (int a = 0; a < D; ++a)
                            for (int bb = 0; bb < D; ++bb) {
                                std::complex<double> s = 0;
                                for (int r = 0; r < D; ++r)
                                    s += std::conj(std::complex<double>(K[2 * (r * D + a)], K[2 * (r * D + a) + 1])) *
                                         std::complex<double>(K[2 * (r * D + bb)], K[2 * (r * D + bb) + 1]);
                                b->pool.push_back(s.real());
                                b->pool.push_back(s.imag());
                            }
                        push_residuals(b, red.off, 2 * E);
                    } else {
                        red.kind = RED_BINS;
                        red.R = 1 << k;
                    }
                    if ((st = upload_pool(b))) return st;
                    if ((st = emit_pass(b, red))) return st;
                    std::vector<double> part(MAX_RED * b->red_chunks);
                    CU(cudaMemcpyAsync(part.data(), b->dev.partials, sizeof(double) * MAX_RED * b->red_chunks,
                                       cudaMemcpyDeviceToHost, b->stream));
                    CU(cudaStreamSynchronize(b->stream));
                    if (kind == SV_OP_KRAUS) {
                        double s = 0;
                        for (int ch = 0; ch < b->red_chunks; ++ch) s += part[ch * MAX_RED];
                        p[t] = s;
                    } else {
                        for (int o = 0; o < R; ++o) {
                            double s = 0;
                            for (int ch = 0; ch < b->red_chunks; ++ch) s += part[ch * MAX_RED + o];
                            p[o] = s;
                        }
                        break;
                    }
                }
                std::vector<double> cum(R);
                double acc = 0;
                for (int t = 0; t < R; ++t) cum[t] = (acc += p[t]);
                const double u = host_uniform(b->seed, b->dev.shot_base + shot, (uint32_t)i);
                const int t = host_select(u, cum.data(), R);
                const double scale = 1.0 / std::sqrt(p[t]);
                if (kind == SV_OP_KRAUS) {
                    const double* K = d + 2 * E * t;
                    PendStage s{};
                    s.kind = ST_DENSE;
                    s.k = k;
                    for (int j = 0; j < k; ++j) s.q[j] = q[j];
                    s.cond_clbit = -1;
                    s.off = pool_matrix(b, K, k, scale);
                    add_stage(b, s);
                } else {
                    // projection (and reset) as a dense matrix on the measured qubits
                    std::vector<double> P(2 * E, 0.0);
                    const int reset = c->reset[i];
                    P[2 * ((reset ? 0 : t) * D + t)] = scale;
                    PendStage s{};
                    s.kind = ST_DENSE;
                    s.k = k;
                    for (int j = 0; j < k; ++j) s.q[j] = q[j];
                    s.cond_clbit = -1;
                    s.off = pool_matrix(b, P.data(), k);
                    add_stage(b, s);
                    const int* cl = c->clbits + c->cl_off[i];
                    for (int j = 0; j < k; ++j)
                        clreg = (clreg & ~(1ull << cl[j])) | ((uint64_t)((t >> j) & 1) << cl[j]);
                }
                if ((st = upload_pool(b))) return st;
                if ((st = flush(b))) return st;
            } else if (kind == SV_OP_FINAL) {
                if ((st = op_final(b, (uint32_t)i))) return st;
            }
        }
        if ((st = reset_pool(b))) return st;
    }
    return SV_OK;
}

// the launch sequence of a whole circuit (without the reset / init of the
// root), with its constants uploaded
// the pre-drawn rows of a recorded circuit: their descriptors go to the
// integer pool, the device table grows to hold them, and the draw is the
// circuit's first launch
sv_status finish_predraw(sv_batch b, std::vector<Launch>& launches) {
    const int n = (int)b->pre_rows.size();
    const int table = (int)b->ipool.size();
    for (const PreRow& r : b->pre_rows) {
        const uint64_t ls = (uint64_t)(uintptr_t)r.log_sel, lt = (uint64_t)(uintptr_t)r.log_thr;
        const int32_t w[PRE_WORDS] = {(int32_t)r.op, r.R, r.thr_off, r.cum_off, (int32_t)(uint32_t)ls,
                                      (int32_t)(uint32_t)(ls >> 32), (int32_t)(uint32_t)lt, (int32_t)(uint32_t)(lt >> 32)};
        b->ipool.insert(b->ipool.end(), w, w + PRE_WORDS);
    }
    if (n > b->pre_cap) {
        sv_status st = dalloc(b, &b->dev.pre_sel, (size_t)n * b->n_shots);
        if (st) return st;
        b->pre_cap = n;
        b->pool_gen += 1;  // kernels take the batch by value
    }
    Launch L;
    L.type = L_PREDRAW;
    L.a0 = n;
    L.a1 = table;
    L.a2 = (int)b->n_shots;
    launches.insert(launches.begin(), L);
    return SV_OK;
}

sv_status record_circuit(sv_batch b, const sv_circuit* c, std::vector<Launch>& launches) {
    sv_status st = reset_pool(b);
    if (st) return st;
    b->pool_gen += 1;
    b->started = true;  // reset / init are issued by the caller, per run
    b->rec = &launches;
    b->col_used = 0;
    b->pre_rows.clear();
    for (int i = 0; i < c->n_ops && !st; ++i) {
        if (b->joint && i + 1 < c->n_ops && c->kind[i] == SV_OP_KRAUS && c->kind[i + 1] == SV_OP_KRAUS &&
            c->nq[i] == 1 && c->nq[i + 1] == 1 && c->qubits[c->q_off[i]] != c->qubits[c->q_off[i + 1]] &&
            c->n_terms[i] * c->n_terms[i + 1] <= MAX_RED) {
            st = op_kraus_pair(b, (uint32_t)i, c->qubits[c->q_off[i]], c->n_terms[i], c->data + c->d_off[i],
                               (uint32_t)(i + 1), c->qubits[c->q_off[i + 1]], c->n_terms[i + 1],
                               c->data + c->d_off[i + 1]);
            ++i;
            continue;
        }
        st = circuit_op(b, c, i);
    }
    if (!st) st = flush(b);
    b->rec = nullptr;
    if (!st && !b->pre_rows.empty()) st = finish_predraw(b, launches);
    if (st) return st;
    return upload_pool(b);
}

// restart the waiting list of a shot-branching batch until it is empty
// (Section IV-B-2), launching one by one
sv_status drain_waiting(sv_batch b, const std::vector<Launch>& launches) {
    int n_run = (int)b->n_shots;
    for (;;) {
        int32_t ctl[CTL_WORDS];
        sv_status st = read_ctl(b, ctl);
        if (st) return st;
        if ((st = tree_snapshot(b, ctl, n_run))) return st;
        if (ctl[CTL_ERR] || ctl[CTL_NWAIT] == 0) return SV_OK;
        n_run = ctl[CTL_NWAIT];
        Launch r;
        r.type = L_RESET;
        r.a0 = 1;
        r.a1 = ctl[CTL_NWAIT];
        r.a2 = 1;
        if ((st = exec(b, r))) return st;
        Launch in;
        in.type = L_INIT;
        in.a0 = root_slots(b, n_run);
        if ((st = exec(b, in))) return st;
        for (const Launch& L : launches)
            if ((st = exec(b, L))) return st;
        b->restarts += 1;
    }
}

}  // namespace

// =============================================================================
// C ABI
// =============================================================================
extern "C" {

const char* sv_last_error(void) { return g_err.c_str(); }

sv_status sv_alloc_batch(int n_qubits, uint64_t n_shots, int n_clbits, sv_prec prec, sv_mode mode, uint64_t seed,
                         uint64_t mem_budget, void* cuda_stream, sv_batch* out) {
    if (!out) return fail(SV_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_qubits < 1 || n_qubits > 30) return fail(SV_EINVAL, "n_qubits must be 1..30");
    if (n_shots == 0 || n_shots > (1ull << 31)) return fail(SV_EINVAL, "n_shots must be 1..2^31");
    if (n_clbits < 0 || n_clbits > 64) return fail(SV_EINVAL, "n_clbits must be 0..64");
    if (prec != SV_C64 && prec != SV_C128) return fail(SV_EINVAL, "bad precision");
    if (mode < SV_PLAIN || mode > SV_BATCH_BRANCH) return fail(SV_EINVAL, "bad mode");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(SV_ECUDA, "no CUDA device");
    }
    sv_batch b = new sv_batch_s();
    b->n = n_qubits;
    b->n_shots = n_shots;
    b->n_clbits = n_clbits;
    b->prec = prec;
    b->mode = mode;
    b->seed = seed;
    b->branch = mode == SV_BRANCH || mode == SV_BATCH_BRANCH;
    b->dim = 1ll << n_qubits;
    b->amp_bytes = prec == SV_C128 ? 16 : 8;
    b->state_bytes = b->dim * b->amp_bytes;
    cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, dev);
    b->grid_small = 2 * b->n_sm;
    b->tb = std::min(n_qubits, prec == SV_C128 ? 10 : 11);
    // Fusion width: when the whole state is one tile, a pass may touch every
    // qubit (the state sits in shared memory); otherwise at most 4, so
    // passes run on the register path (wider passes over a bigger state
    // leave the tile few contiguous low qubits and its bulk copies turn
    // short)
    b->max_active = DEFAULT_MAX_ACTIVE;
    const int64_t tiles = 1ll << (n_qubits - b->tb);
    b->chunks = (int)std::min<int64_t>(tiles, MAX_CHUNKS);
    b->chunks_final = (int)std::min<int64_t>(std::max<int64_t>(b->dim / 2048, 1), MAX_CHUNKS);
    if (cuda_stream) {
        b->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete b;
            return fail(SV_ECUDA, "cudaStreamCreate failed");
        }
        b->own_stream = true;
    }
    if (cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        sv_free_batch(b);
        return fail(SV_ECUDA, "cannot create the decide side stream");
    }
    // slots
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    const int max_chunks = std::max(b->chunks, b->chunks_final);
    const size_t per_slot = b->state_bytes + (size_t)max_chunks * MAX_RED * 8;
    const size_t per_shot = 4 * 8 + MAX_PEND * 12 + 64;
    const size_t fixed = per_shot * n_shots + (64ull << 20);
    size_t budget = mem_budget;
    if (budget == 0) {
        const size_t reserve = std::max<size_t>(1ull << 30, total_b / 50);
        budget = free_b > fixed + reserve ? free_b - fixed - reserve : 0;
    }
    uint64_t slots = budget / per_slot;
    if (mode == SV_PLAIN) slots = std::min<uint64_t>(slots, 1);
    else slots = std::min<uint64_t>(slots, n_shots);
    if (slots == 0) {
        sv_free_batch(b);
        return fail(SV_ENOMEM, "not even one state fits the memory budget");
    }
    if (mode == SV_BATCH && slots < n_shots) {
        sv_free_batch(b);
        return fail(SV_ENOMEM, "batch mode needs one state per shot; use shot-branching or fewer shots");
    }
    b->n_slots = (int)slots;
    DevBatch& d = b->dev;
    d.dim = b->dim;
    d.n = n_qubits;
    d.n_slots = b->n_slots;
    d.cap_br = (int)n_shots;
    d.seed = seed;
    d.max_chunks = max_chunks;
    sv_status st = SV_OK;
    void* states = nullptr;
    if (cudaMalloc(&states, (size_t)b->n_slots * b->state_bytes) != cudaSuccess) {
        cudaGetLastError();
        sv_free_batch(b);
        return fail(SV_ENOMEM, "cannot allocate the state slots");
    }
    b->allocs.push_back(states);
    d.states = states;
    const uint64_t S = n_shots;
    if ((st = dalloc(b, &d.ctl, CTL_WORDS)) || (st = dalloc(b, &d.br_slot, S)) || (st = dalloc(b, &d.br_start, S)) ||
        (st = dalloc(b, &d.br_count, S)) || (st = dalloc(b, &d.br_clbits, S)) || (st = dalloc(b, &d.br_parent, S)) || (st = dalloc(b, &d.br_big, S)) || (st = dalloc(b, &d.br_pset, S)) ||
        (st = dalloc(b, &d.br_sel, S * MAX_PEND)) || (st = dalloc(b, &d.br_scale, S * MAX_PEND)) ||
        (st = dalloc(b, &d.perm, S)) || (st = dalloc(b, &d.perm_tmp, S)) || (st = dalloc(b, &d.shot_sel, S)) ||
        (st = dalloc(b, &d.free_slots, b->n_slots)) || (st = dalloc(b, &d.wait_shots, S)) ||

        (st = dalloc(b, &d.partials, (size_t)b->n_slots * max_chunks * MAX_RED)) || (st = dalloc(b, &d.keys, S)) ||
        (st = dalloc(b, &d.pass_log, 1 << 20)) || (st = dalloc(b, &d.pos_branch, S))) {
        sv_free_batch(b);
        return st;
    }
    b->pool_cap = 1 << 16;
    b->ipool_cap = 1 << 14;
    if (cudaMalloc(&b->d_pool, b->pool_cap * 8) != cudaSuccess ||
        cudaMalloc((void**)&b->d_ipool, b->ipool_cap * 4) != cudaSuccess ||
        cudaMallocHost(&b->h_pool, b->pool_cap * 8) != cudaSuccess ||
        cudaMallocHost((void**)&b->h_ipool, b->ipool_cap * 4) != cudaSuccess) {
        cudaGetLastError();
        sv_free_batch(b);
        return fail(SV_ENOMEM, "cannot allocate the constant pool");
    }
    d.pool = b->d_pool;
    d.ipool = b->d_ipool;
    d.pass_log_cap = 1 << 20;
    if (init_kernels() != cudaSuccess) {
        sv_free_batch(b);
        return fail(SV_ECUDA, "cannot configure the kernels");
    }
    cudaMemsetAsync(d.ctl, 0, CTL_WORDS * 4, b->stream);
    cudaMemsetAsync(d.pos_branch, 0xff, S * 4, b->stream);
    *out = b;
    return SV_OK;
}

sv_status sv_free_batch(sv_batch b) {
    if (!b) return SV_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
    if (b->multi_exec) cudaGraphExecDestroy(b->multi_exec);
    if (b->multi_restart_exec) cudaGraphExecDestroy(b->multi_restart_exec);
    for (auto& e : b->prof_ev) {
        cudaEventDestroy(e.second.first);
        cudaEventDestroy(e.second.second);
    }
    for (void* p : b->allocs) cudaFree(p);
    if (b->d_pool) cudaFree(b->d_pool);
    if (b->d_ipool) cudaFree(b->d_ipool);
    if (b->h_pool) cudaFreeHost(b->h_pool);
    if (b->h_ipool) cudaFreeHost(b->h_ipool);
    if (b->side) {
        cudaStreamSynchronize(b->side);
        cudaStreamDestroy(b->side);
    }
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev_join) cudaEventDestroy(b->ev_join);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return SV_OK;
}

static sv_status set_option(sv_batch b, sv_option opt, int64_t v);

sv_status sv_set_option(sv_batch b, sv_option opt, int64_t v) {
    if (!b) return fail(SV_EINVAL, "batch is NULL");
    const sv_status st = set_option(b, opt, v);
    // options shape the recorded launches (and the device struct the
    // kernels take by value): a cached graph is recorded again
    if (st == SV_OK && opt != SV_OPT_UPLOAD && opt != SV_OPT_PROFILE) b->pool_gen += 1;
    return st;
}

static sv_status set_option(sv_batch b, sv_option opt, int64_t v) {
    switch (opt) {
    case SV_OPT_LOG:
        if (v && !b->dev.fork_log) {
            // waiting-list restarts fork the same shots again: room for many rounds
            b->dev.fork_log_cap = (int)std::min<uint64_t>(64 * b->n_shots + 65536, 1 << 22);
            sv_status st = dalloc(b, &b->dev.fork_log, FORK_WORDS * (size_t)b->dev.fork_log_cap);
            if (st) return st;
        }
        b->log = v != 0;
        if (!v) b->dev.fork_log = nullptr;
        return SV_OK;
    case SV_OPT_TILE_BITS:
        if (v && (v < 2 || v > MAX_TILE_BITS)) return fail(SV_EINVAL, "tile bits must be 2..12");
        if (b->started) return fail(SV_EINVAL, "set the tile size before the first op");
        b->tb = std::min<int>(b->n, v ? (int)v : (b->prec == SV_C128 ? 10 : 11));
        b->chunks = (int)std::min<int64_t>(1ll << (b->n - b->tb), b->dev.max_chunks);
        if (!b->max_active_set) b->max_active = DEFAULT_MAX_ACTIVE;
        return SV_OK;
    case SV_OPT_MAX_ACTIVE:
        b->max_active = v ? (int)std::max<int64_t>(2, v) : DEFAULT_MAX_ACTIVE;
        b->max_active_set = v != 0;
        return SV_OK;
    case SV_OPT_MAX_STAGES: b->max_stages = v ? (int)std::min<int64_t>(std::max<int64_t>(v, 1), MAX_STAGES) : MAX_STAGES; return SV_OK;
    case SV_OPT_THREADS:
        if (v && v != 32 && v != 64 && v != 128 && v != 256) return fail(SV_EINVAL, "threads must be 32, 64, 128 or 256");
        b->threads = v ? (int)v : 256;
        b->threads_set = v != 0;
        return SV_OK;
    case SV_OPT_GRID: b->grid_pass = (int)std::max<int64_t>(0, v); return SV_OK;
    case SV_OPT_PROFILE: b->profile = v != 0; return SV_OK;
    case SV_OPT_UPLOAD: b->upload_each = v != 0; return SV_OK;
    case SV_OPT_JOINT_KRAUS: b->joint = v != 0; return SV_OK;
    case SV_OPT_PASS_PATH:
        if (v < 0 || v > 1) return fail(SV_EINVAL, "pass path must be 0 (auto) or 1 (shared-memory tiles)");
        b->pass_path = (int)v;
        return SV_OK;
    case SV_OPT_SHOT_BASE:
        if (v < 0) return fail(SV_EINVAL, "shot base must be >= 0");
        if (!b->pend.empty()) return fail(SV_EINVAL, "per-op calls are in progress on this batch");
        b->dev.shot_base = (uint64_t)v;
        return SV_OK;
    case SV_OPT_CHAIN_DECIDES: b->chain = v != 0; return SV_OK;
    case SV_OPT_PREDRAW_PAULI: b->predraw = v != 0; return SV_OK;
    case SV_OPT_COMMUTE: b->commute = v != 0; return SV_OK;
    case SV_OPT_FOLD: b->fold = v != 0; return SV_OK;
    case SV_OPT_WHOLE_STATE: b->whole = v != 0; return SV_OK;
    case SV_OPT_SLOT_LIMIT:
        if (v < 0) return fail(SV_EINVAL, "slot limit must be >= 0");
        if (v && b->branch && v < b->n_psets) return fail(SV_EINVAL, "fewer slots than parameter sets");
        b->slot_limit = (int)v;
        if (v && b->branch) b->dev.n_slots = std::min<int>(b->n_slots, (int)v);
        else b->dev.n_slots = b->n_slots;
        return SV_OK;
    }
    return fail(SV_EINVAL, "unknown option");
}

sv_status sv_apply_gate_batch(sv_batch b, int k, const int* qubits, const double* mat, int cond_clbit, int cond_value) {
    if (!b) return fail(SV_EINVAL, "batch is NULL");
    if (sv_status cs = commit_forks(b)) return cs;
    if (b->mode == SV_PLAIN) return fail(SV_EUNSUPPORTED, "plain mode runs whole circuits (sv_run_circuit)");
    sv_status st = op_gate(b, k, qubits, mat, cond_clbit, cond_value);
    if (st) return st;
    return upload_pool(b);
}

sv_status sv_set_param_sets(sv_batch b, const uint32_t* set_of_shot, uint32_t n_sets) {
    if (!b) return fail(SV_EINVAL, "batch is NULL");
    if (!b->pend.empty() || b->uncommitted || b->started)
        return fail(SV_EINVAL, "set the parameter sets before the first op of a run");
    if (n_sets == 0) {
        b->n_psets = 0;
        b->h_pset.clear();
        b->dev.pset_of_shot = nullptr;
        b->dev.n_psets = 0;
        b->pool_gen += 1;
        return SV_OK;
    }
    if (!set_of_shot) return fail(SV_EINVAL, "set_of_shot is NULL");
    if (n_sets > (uint32_t)MAX_PSETS) return fail(SV_EUNSUPPORTED, "at most 1024 parameter sets per batch");
    if (b->branch && n_sets > (uint32_t)b->dev.n_slots)
        return fail(SV_ENOMEM, "shot-branching needs a state slot for every parameter set");
    for (uint64_t s = 0; s < b->n_shots; ++s)
        if (set_of_shot[s] >= n_sets) return fail(SV_EINVAL, "a shot's parameter set is out of range");
    uint32_t* d = nullptr;
    sv_status st = dalloc(b, &d, b->n_shots);
    if (st) return st;
    CU(cudaMemcpyAsync(d, set_of_shot, b->n_shots * 4, cudaMemcpyHostToDevice, b->stream));
    CU(cudaStreamSynchronize(b->stream));
    b->h_pset.assign(set_of_shot, set_of_shot + b->n_shots);
    b->n_psets = (int)n_sets;
    b->dev.pset_of_shot = d;
    b->dev.n_psets = (int)n_sets;
    b->pool_gen += 1;  // cached graphs hold the batch's device struct
    return SV_OK;
}

sv_status sv_apply_param_gate_batch(sv_batch b, int k, const int* qubits, const double* mats, int n_sets) {
    if (!b) return fail(SV_EINVAL, "batch is NULL");
    if (sv_status cs = commit_forks(b)) return cs;
    if (b->mode == SV_PLAIN) return fail(SV_EUNSUPPORTED, "plain mode runs whole circuits (sv_run_circuit)");
    sv_status st = op_pgate(b, k, qubits, mats, n_sets);
    if (st) return st;
    return upload_pool(b);
}

sv_status sv_sample_noise(sv_batch b, uint32_t op, sv_noise_kind kind, int k, const int* qubits, int n_terms,
                          const double* cum_probs, const char* paulis, const double* kraus) {
    if (!b) return fail(SV_EINVAL, "batch is NULL");
    if (sv_status cs = commit_forks(b)) return cs;
    if (b->mode == SV_PLAIN) return fail(SV_EUNSUPPORTED, "plain mode runs whole circuits (sv_run_circuit)");
    if (kind == SV_NOISE_PAULI) return op_pauli(b, op, k, qubits, n_terms, cum_probs, paulis);
    if (kind == SV_NOISE_KRAUS) return op_kraus(b, op, k, qubits, n_terms, kraus);
    return fail(SV_EINVAL, "unknown noise kind");
}

sv_status sv_measure_batch(sv_batch b, uint32_t op, int m, const int* qubits, const int* clbits, int reset) {
    if (!b) return fail(SV_EINVAL, "batch is NULL");
    if (sv_status cs = commit_forks(b)) return cs;
    if (b->mode == SV_PLAIN) return fail(SV_EUNSUPPORTED, "plain mode runs whole circuits (sv_run_circuit)");
    return op_measure(b, op, m, qubits, clbits, reset);
}

sv_status sv_branch(sv_batch b, uint32_t op) {
    if (!b) return fail(SV_EINVAL, "batch is NULL");
    if (b->last_random != op) return fail(SV_EINVAL, "op is not the last random op sampled");
    return commit_forks(b);
}

sv_status sv_get_keys(sv_batch b, uint64_t* keys) {
    if (!b || !keys) return fail(SV_EINVAL, "NULL argument");
    CU(cudaMemcpyAsync(keys, b->dev.keys, b->n_shots * 8, cudaMemcpyDeviceToHost, b->stream));
    CU(cudaStreamSynchronize(b->stream));
    return check_device_error(b);
}

static sv_status histogram(sv_batch b, uint64_t* keys, uint64_t* counts, uint64_t cap, uint64_t* n_out) {
    int32_t ctl[CTL_WORDS];
    sv_status st = read_ctl(b, ctl);
    if (st) return st;
    std::vector<uint64_t> k(b->n_shots);
    CU(cudaMemcpyAsync(k.data(), b->dev.keys, b->n_shots * 8, cudaMemcpyDeviceToHost, b->stream));
    std::vector<uint32_t> perm(b->n_shots);
    std::vector<int32_t> start(ctl[CTL_NBR]), cnt(ctl[CTL_NBR]);
    CU(cudaMemcpyAsync(perm.data(), b->dev.perm, b->n_shots * 4, cudaMemcpyDeviceToHost, b->stream));
    if (ctl[CTL_NBR] > 0) {
        CU(cudaMemcpyAsync(start.data(), b->dev.br_start, 4 * ctl[CTL_NBR], cudaMemcpyDeviceToHost, b->stream));
        CU(cudaMemcpyAsync(cnt.data(), b->dev.br_count, 4 * ctl[CTL_NBR], cudaMemcpyDeviceToHost, b->stream));
    }
    CU(cudaStreamSynchronize(b->stream));
    std::vector<uint64_t> live;
    for (int br = 0; br < ctl[CTL_NBR]; ++br)
        for (int i = 0; i < cnt[br]; ++i) live.push_back(k[perm[start[br] + i]]);
    std::sort(live.begin(), live.end());
    uint64_t n = 0;
    for (size_t i = 0; i < live.size();) {
        size_t j = i;
        while (j < live.size() && live[j] == live[i]) ++j;
        if (n >= cap) return fail(SV_EINVAL, "cap too small for the histogram");
        keys[n] = live[i];
        counts[n] = j - i;
        ++n;
        i = j;
    }
    *n_out = n;
    return SV_OK;
}

sv_status sv_counts(sv_batch b, uint32_t final_op, uint64_t* keys, uint64_t* counts, uint64_t cap, uint64_t* n_out) {
    if (!b || !keys || !counts || !n_out) return fail(SV_EINVAL, "NULL argument");
    if (b->mode == SV_PLAIN) return fail(SV_EUNSUPPORTED, "plain mode runs whole circuits (sv_run_circuit)");
    if (sv_status cs = commit_forks(b)) return cs;
    sv_status st = op_final(b, final_op);
    if (st) return st;
    if ((st = check_device_error(b))) return st;
    return histogram(b, keys, counts, cap, n_out);
}

sv_status sv_waiting(sv_batch b, uint64_t* n_waiting) {
    if (!b || !n_waiting) return fail(SV_EINVAL, "NULL argument");
    if (sv_status cs = commit_forks(b)) return cs;
    int32_t ctl[CTL_WORDS];
    sv_status st = read_ctl(b, ctl);
    if (st) return st;
    *n_waiting = (uint64_t)ctl[CTL_NWAIT];
    return SV_OK;
}

sv_status sv_run_circuit(sv_batch b, const sv_circuit* c, int use_graph) {
    if (!b || !c) return fail(SV_EINVAL, "NULL argument");
    if (c->n_qubits != b->n) return fail(SV_EINVAL, "circuit qubit count differs from the batch");
    if (c->n_clbits > b->n_clbits) return fail(SV_EINVAL, "circuit needs more classical bits than the batch");
    sv_status st;
    if (!b->pend.empty() || b->uncommitted) return fail(SV_EINVAL, "per-op calls are in progress on this batch");
    if (b->mode == SV_PLAIN) {
        b->started = true;
        if ((st = reset_pool(b))) return st;
        if ((st = run_plain(b, c))) return st;
        return check_device_error(b);
    }
    // launch list of the op sequence (after the reset / init of the root)
    const uint64_t h = circuit_hash(b, c);
    const bool cached = use_graph && b->graph_exec && b->graph_hash == h && b->graph_gen == b->pool_gen;
    std::vector<Launch> launches;
    if (!cached && (st = record_circuit(b, c, launches))) return st;
    if (cached && b->upload_each) {
        // the circuit's constants cross the bus again (end-to-end timing)
        b->pool_up = 0;
        b->ipool_up = 0;
        if ((st = upload_pool(b))) return st;
    }
    const int branch = b->branch;
    int from_wait = 0;
    int n_run = (int)b->n_shots;
    if ((st = tree_begin(b))) return st;
    for (int round = 0;; ++round) {
        Launch r;
        r.type = L_RESET;
        r.a0 = branch;
        r.a1 = n_run;
        r.a2 = from_wait;
        if ((st = exec(b, r))) return st;
        Launch in;
        in.type = L_INIT;
        in.a0 = root_slots(b, n_run);
        if ((st = exec(b, in))) return st;
        if (use_graph) {
            if (!cached && round == 0) {
                if (b->graph_exec) {
                    cudaGraphExecDestroy(b->graph_exec);
                    b->graph_exec = nullptr;
                }
                cudaGraph_t g;
                CU(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
                for (const Launch& L : launches) {
                    cudaError_t e = exec_one(b, L);
                    if (e != cudaSuccess) {
                        cudaStreamEndCapture(b->stream, &g);
                        return fail(SV_ECUDA, std::string("capture: ") + cudaGetErrorString(e));
                    }
                }
                CU(cudaStreamEndCapture(b->stream, &g));
                CU(cudaGraphInstantiate(&b->graph_exec, g, 0));
                cudaGraphDestroy(g);
                b->graph_hash = h;
                b->graph_gen = b->pool_gen;
                int64_t nl = 0;
                for (const Launch& L : launches) nl += L.type == L_FINAL ? 3 : (L.type == L_DECIDE ? 2 : 1);
                b->graph_launches = nl;
                b->graph_pass_store.clear();
                for (const Launch& L : launches)
                    if (L.type == L_PASS) b->graph_pass_store.push_back(L.pass.store ? 1 : 0);
            }
            CU(cudaGraphLaunch(b->graph_exec, b->stream));
            b->n_launch += b->graph_launches;
            b->n_passes += b->graph_pass_store.size();
            b->pass_store.insert(b->pass_store.end(), b->graph_pass_store.begin(), b->graph_pass_store.end());
        } else {
            for (const Launch& L : launches)
                if ((st = exec(b, L))) return st;
        }
        if (!branch) break;
        int32_t ctl[CTL_WORDS];
        if ((st = read_ctl(b, ctl))) return st;
        if ((st = tree_snapshot(b, ctl, n_run))) return st;
        if (ctl[CTL_ERR]) break;
        if (ctl[CTL_NWAIT] == 0) break;
        // waiting list (Section IV-B-2): restart its shots from |0...0>
        n_run = ctl[CTL_NWAIT];
        from_wait = 1;
        b->restarts += 1;
        if (!use_graph && launches.empty()) break;
    }
    b->started = false;
    return check_device_error(b);
}

// One CUDA graph in which batch bs[i] runs lists[i] on a branch of its own
// (forked from and joined back to the batches' shared stream), so the
// batches' kernels run side by side.
static sv_status capture_branches(sv_batch* bs, const std::vector<std::vector<Launch>>& lists, cudaGraphExec_t* out) {
    const int n = (int)lists.size();
    sv_batch b0 = bs[0];
    std::vector<cudaStream_t> cs(n, nullptr);
    std::vector<cudaEvent_t> done(n, nullptr);
    cudaEvent_t root = nullptr;
    cudaError_t e = cudaEventCreateWithFlags(&root, cudaEventDisableTiming);
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&cs[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&done[i], cudaEventDisableTiming);
    }
    cudaGraph_t g = nullptr;
    bool capturing = false;
    if (e == cudaSuccess) e = cudaStreamBeginCapture(b0->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        capturing = true;
        e = cudaEventRecord(root, b0->stream);
    }
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        e = cudaStreamWaitEvent(cs[i], root, 0);
        cudaStream_t own = bs[i]->stream;
        bs[i]->stream = cs[i];
        for (size_t j = 0; j < lists[i].size() && e == cudaSuccess; ++j) e = exec_one(bs[i], lists[i][j]);
        bs[i]->stream = own;
        if (e == cudaSuccess) e = cudaEventRecord(done[i], cs[i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b0->stream, done[i], 0);
    }
    if (capturing) {
        const cudaError_t e2 = cudaStreamEndCapture(b0->stream, &g);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
    if (g) cudaGraphDestroy(g);
    for (int i = 0; i < n; ++i) {
        if (cs[i]) cudaStreamDestroy(cs[i]);
        if (done[i]) cudaEventDestroy(done[i]);
    }
    if (root) cudaEventDestroy(root);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *out = nullptr;
        return fail(SV_ECUDA, std::string("capture: ") + cudaGetErrorString(e));
    }
    return SV_OK;
}

static void count_launches(sv_batch b, const std::vector<Launch>& list) {
    for (const Launch& L : list) {
        b->n_launch += L.type == L_FINAL ? 3 : (L.type == L_DECIDE ? 2 : 1);
        if (L.type == L_PASS) {
            b->n_passes += 1;
            b->pass_store.push_back(L.pass.store ? 1 : 0);
        }
    }
}

sv_status sv_run_circuits(sv_batch* bs, const sv_circuit* const* cs, int n, int use_graph) {
    if (!bs || !cs || n < 1) return fail(SV_EINVAL, "sv_run_circuits: NULL or empty arguments");
    sv_status st;
    for (int i = 0; i < n; ++i) {
        if (!bs[i] || !cs[i]) return fail(SV_EINVAL, "sv_run_circuits: NULL batch or circuit");
        if (bs[i]->mode == SV_PLAIN) return fail(SV_EUNSUPPORTED, "sv_run_circuits: plain mode runs one circuit");
        if (bs[i]->stream != bs[0]->stream) return fail(SV_EINVAL, "sv_run_circuits: batches must share one stream");
        if (cs[i]->n_qubits != bs[i]->n) return fail(SV_EINVAL, "sv_run_circuits: circuit / batch qubit counts differ");
        if (!bs[i]->pend.empty()) return fail(SV_EINVAL, "sv_run_circuits: per-op calls are in progress");
        for (int j = 0; j < i; ++j)
            if (bs[j] == bs[i]) return fail(SV_EINVAL, "sv_run_circuits: a batch appears twice");
    }
    sv_batch b0 = bs[0];
    uint64_t h = 1469598103934665603ull;
    for (int i = 0; i < n; ++i) {
        const uint64_t hi = circuit_hash(bs[i], cs[i]);
        h = fnv(h, &hi, 8);
        h = fnv(h, &bs[i], sizeof(void*));
    }
    bool cached = use_graph && b0->multi_exec && b0->multi_hash == h && (int)b0->multi_gens.size() == n;
    for (int i = 0; cached && i < n; ++i) cached = b0->multi_gens[i] == bs[i]->pool_gen;
    if (!cached) {
        b0->multi_lists.assign(n, {});
        for (int i = 0; i < n; ++i) {
            std::vector<Launch>& L = b0->multi_lists[i];
            Launch r;
            r.type = L_RESET;
            r.a0 = bs[i]->branch;
            r.a1 = (int)bs[i]->n_shots;
            r.a2 = 0;
            L.push_back(r);
            Launch in;
            in.type = L_INIT;
            in.a0 = root_slots(bs[i], (int)bs[i]->n_shots);
            L.push_back(in);
            std::vector<Launch> ops;
            if ((st = record_circuit(bs[i], cs[i], ops))) return st;
            L.insert(L.end(), ops.begin(), ops.end());
        }
    }
    for (int i = 0; i < n; ++i)
        if ((st = tree_begin(bs[i]))) return st;
    if (!use_graph) {
        for (int i = 0; i < n; ++i)
            for (const Launch& L : b0->multi_lists[i])
                if ((st = exec(bs[i], L))) return st;
        // shot-branching batches whose forks found no slot: restart their
        // waiting lists one by one
        for (int i = 0; i < n; ++i) {
            if (!bs[i]->branch) continue;
            std::vector<Launch> ops(b0->multi_lists[i].begin() + 2, b0->multi_lists[i].end());
            if ((st = drain_waiting(bs[i], ops))) return st;
        }
    } else {
        if (!cached) {
            if (b0->multi_exec) cudaGraphExecDestroy(b0->multi_exec);
            if (b0->multi_restart_exec) cudaGraphExecDestroy(b0->multi_restart_exec);
            b0->multi_exec = b0->multi_restart_exec = nullptr;
            if ((st = capture_branches(bs, b0->multi_lists, &b0->multi_exec))) return st;
            b0->multi_hash = h;
            b0->multi_gens.resize(n);
            for (int i = 0; i < n; ++i) b0->multi_gens[i] = bs[i]->pool_gen;
        }
        CU(cudaGraphLaunch(b0->multi_exec, b0->stream));
        for (int i = 0; i < n; ++i) count_launches(bs[i], b0->multi_lists[i]);
        // Waiting lists (Section IV-B-2): every shot-branching batch restarts
        // the shots that found no slot, as a new root, in a second cached
        // graph with one branch per batch whose reset reads the waiting
        // count on the device; a batch with none left does no work there.
        // It is replayed until no batch has shots waiting.
        std::vector<int> wait(n, 0);
        bool any = false;
        for (int i = 0; i < n; ++i) {
            if (!bs[i]->branch) continue;
            int32_t ctl[CTL_WORDS];
            if ((st = read_ctl(bs[i], ctl))) return st;
            if ((st = tree_snapshot(bs[i], ctl, (int)bs[i]->n_shots))) return st;
            wait[i] = ctl[CTL_ERR] ? 0 : ctl[CTL_NWAIT];
            any = any || wait[i] > 0;
        }
        std::vector<std::vector<Launch>> rl;
        while (any) {
            if (rl.empty())
                for (int i = 0; i < n; ++i) {
                    std::vector<Launch> L;
                    if (bs[i]->branch) {
                        Launch r;
                        r.type = L_RESET;
                        r.a0 = 1;
                        r.a1 = 0;
                        r.a2 = 2;
                        L.push_back(r);
                        Launch in;
                        in.type = L_INIT;
                        in.a0 = root_slots(bs[i], (int)bs[i]->n_shots);
                        L.push_back(in);
                        L.insert(L.end(), b0->multi_lists[i].begin() + 2, b0->multi_lists[i].end());
                    }
                    rl.push_back(std::move(L));
                }
            if (!b0->multi_restart_exec && (st = capture_branches(bs, rl, &b0->multi_restart_exec))) return st;
            CU(cudaGraphLaunch(b0->multi_restart_exec, b0->stream));
            any = false;
            for (int i = 0; i < n; ++i) {
                if (!bs[i]->branch) continue;
                count_launches(bs[i], rl[i]);
                if (wait[i] == 0) continue;
                bs[i]->restarts += 1;
                int32_t ctl[CTL_WORDS];
                if ((st = read_ctl(bs[i], ctl))) return st;
                if ((st = tree_snapshot(bs[i], ctl, wait[i]))) return st;
                wait[i] = ctl[CTL_ERR] ? 0 : ctl[CTL_NWAIT];
                any = any || wait[i] > 0;
            }
        }
    }
    for (int i = 0; i < n; ++i) {
        bs[i]->started = false;
        if ((st = check_device_error(bs[i]))) return st;
    }
    return SV_OK;
}

// ---- density-matrix method -------------------------------------------------
// the superoperator sum_t K_t (x) conj(K_t) of a k-qubit channel as a
// 2k-qubit matrix: index bits 0..k-1 are the row qubits, k..2k-1 the column
// qubits (row-major complex, re/im interleaved)
static std::vector<double> superop(const std::vector<std::vector<std::complex<double>>>& K, int k) {
    const int D = 1 << k, D2 = D * D;
    std::vector<double> S(2 * (size_t)D2 * D2, 0.0);
    for (const auto& Kt : K)
        for (int r = 0; r < D; ++r)
            for (int c = 0; c < D; ++c)
                for (int r2 = 0; r2 < D; ++r2)
                    for (int c2 = 0; c2 < D; ++c2) {
                        const std::complex<double> v = Kt[r * D + r2] * std::conj(Kt[c * D + c2]);
                        const size_t e = (size_t)(r + D * c) * D2 + (r2 + D * c2);
                        S[2 * e] += v.real();
                        S[2 * e + 1] += v.imag();
                    }
    return S;
}

static std::vector<std::complex<double>> host_matrix(const double* d, int k) {
    const int E = 1 << (2 * k);
    std::vector<std::complex<double>> m(E);
    for (int e = 0; e < E; ++e) m[e] = {d[2 * e], d[2 * e + 1]};
    return m;
}

// the Pauli string of characters s[0..k-1] (s[j] on qubit j of the op) as a
// 2^k x 2^k matrix, scaled by sqrt(p)
static std::vector<std::complex<double>> pauli_matrix_k(const char* s, int k, double p) {
    const int D = 1 << k;
    std::vector<std::complex<double>> m((size_t)D * D, 0.0);
    const std::complex<double> I1(0, 1);
    for (int c = 0; c < D; ++c) {
        int r = c;
        std::complex<double> ph = std::sqrt(p);
        for (int j = 0; j < k; ++j) {
            const int bit = (c >> j) & 1;
            switch (s[j]) {
            case 'X': r ^= 1 << j; break;
            case 'Y': r ^= 1 << j; ph *= bit ? -I1 : I1; break;
            case 'Z': if (bit) ph = -ph; break;
            default: break;
            }
        }
        m[(size_t)r * D + c] = ph;
    }
    return m;
}

extern "C" sv_status sv_dm_run(const sv_circuit* c, sv_prec prec, uint64_t seed, uint64_t n_shots, uint64_t* keys,
                               double* probs, double* thresholds, void* cuda_stream) {
    if (!c) return fail(SV_EINVAL, "circuit is NULL");
    const int n = c->n_qubits;
    if (n < 1 || n > 15) return fail(SV_EUNSUPPORTED, "the density matrix of n qubits is a state of 2n <= 30 qubits");
    if (n_shots && !keys) return fail(SV_EINVAL, "keys is NULL");
    int final_op = -1;
    for (int i = 0; i < c->n_ops; ++i) {
        const int kind = c->kind[i];
        if (kind == SV_OP_MEASURE || kind == SV_OP_PGATE || (kind == SV_OP_GATE && c->cond_clbit[i] >= 0))
            return fail(SV_EUNSUPPORTED, "the density-matrix method takes gates, Pauli and Kraus noise and a final sample");
        if (kind == SV_OP_FINAL) {
            if (i != c->n_ops - 1) return fail(SV_EUNSUPPORTED, "the final sample must be the last op");
            final_op = i;
        }
    }
    if (n_shots && final_op < 0) return fail(SV_EINVAL, "sampling shots needs a final op");
    sv_batch b = nullptr;
    sv_status st = sv_alloc_batch(2 * n, 1, 0, prec, SV_BATCH, seed, 0, cuda_stream, &b);
    if (st) return st;
    // the first call that fails frees the batch through this guard
    struct Guard {
        sv_batch b;
        ~Guard() { sv_free_batch(b); }
    } guard{b};
    for (int i = 0; i < c->n_ops && !st; ++i) {
        const int kind = c->kind[i], k = c->nq[i];
        const int* q = c->qubits + c->q_off[i];
        const double* d = c->data + c->d_off[i];
        std::vector<int> qq(2 * k);
        for (int j = 0; j < k; ++j) {
            qq[j] = q[j];
            qq[k + j] = q[j] + n;
        }
        if (kind == SV_OP_GATE) {
            // U rho U^dagger: U on the row qubits, conj(U) on the column qubits
            if ((st = check_qubits(b, k, q))) break;
            if (!is_unitary(d, k, 1e-10)) {
                st = fail(SV_EINVAL, "gate matrix is not unitary");
                break;
            }
            std::vector<double> conj_u(d, d + (2 << (2 * k)));
            for (size_t e = 1; e < conj_u.size(); e += 2) conj_u[e] = -conj_u[e];
            if ((st = op_superop(b, k, qq.data(), d))) break;
            st = op_superop(b, k, qq.data() + k, conj_u.data());
        } else if (kind == SV_OP_PAULI || kind == SV_OP_KRAUS) {
            if (2 * k > MAX_GATE_Q) {
                st = fail(SV_EUNSUPPORTED, "channels of the density-matrix method act on 1 or 2 qubits");
                break;
            }
            std::vector<std::vector<std::complex<double>>> K;
            if (kind == SV_OP_PAULI) {
                const char* strs = (const char*)c->paulis + c->s_off[i];
                double prev = 0.0;
                for (int t = 0; t < c->n_terms[i]; ++t) {
                    const double pt = d[t] - prev;
                    prev = d[t];
                    if (pt > 0.0) K.push_back(pauli_matrix_k(strs + t * k, k, pt));
                }
            } else {
                for (int t = 0; t < c->n_terms[i]; ++t) K.push_back(host_matrix(d + (size_t)t * (2 << (2 * k)), k));
            }
            const std::vector<double> S = superop(K, k);
            st = op_superop(b, 2 * k, qq.data(), S.data());
        }
    }
    if (st) return st;
    if ((st = upload_pool(b))) return st;
    if ((st = flush(b))) return st;
    // final distribution and the shots' keys
    const int64_t dim = 1ll << n;
    const int chunks = (int)std::min<int64_t>(std::max<int64_t>(dim / 1024, 1), 1024);
    double *p = nullptr, *sums = nullptr, *cum = nullptr, *thr = nullptr;
    uint64_t* dkeys = nullptr;
    if ((st = dalloc(b, &p, dim)) || (st = dalloc(b, &sums, chunks)) || (st = dalloc(b, &cum, chunks)) ||
        (st = dalloc(b, &dkeys, std::max<uint64_t>(n_shots, 1))) ||
        (thresholds && (st = dalloc(b, &thr, 2 * std::max<uint64_t>(n_shots, 1)))))
        return st;
    CU(launch_dm_final(b->dev.states, prec == SV_C128, n, p, sums, cum, chunks, n_shots, seed,
                       (uint32_t)std::max(final_op, 0), dkeys, thr, b->n_sm, b->stream));
    if (probs) CU(cudaMemcpyAsync(probs, p, dim * 8, cudaMemcpyDeviceToHost, b->stream));
    if (n_shots) CU(cudaMemcpyAsync(keys, dkeys, n_shots * 8, cudaMemcpyDeviceToHost, b->stream));
    if (thresholds && n_shots)
        CU(cudaMemcpyAsync(thresholds, thr, n_shots * 16, cudaMemcpyDeviceToHost, b->stream));
    CU(cudaStreamSynchronize(b->stream));
    return check_device_error(b);
}

sv_status sv_get_amplitudes(sv_batch b, uint64_t shot, double* out, uint64_t len) {
    if (!b || !out) return fail(SV_EINVAL, "NULL argument");
    if (len != (uint64_t)b->dim) return fail(SV_EINVAL, "len must be 2^n");
    if (shot >= b->n_shots) return fail(SV_EINVAL, "shot out of range");
    if (sv_status cs = commit_forks(b)) return cs;
    sv_status st = upload_pool(b);
    if (st) return st;
    if ((st = flush(b))) return st;
    int32_t ctl[CTL_WORDS];
    if ((st = read_ctl(b, ctl))) return st;
    const int nb = ctl[CTL_NBR];
    std::vector<uint32_t> perm(b->n_shots);
    std::vector<int32_t> start(nb), cnt(nb), slot(nb);
    CU(cudaMemcpyAsync(perm.data(), b->dev.perm, b->n_shots * 4, cudaMemcpyDeviceToHost, b->stream));
    CU(cudaMemcpyAsync(start.data(), b->dev.br_start, 4 * nb, cudaMemcpyDeviceToHost, b->stream));
    CU(cudaMemcpyAsync(cnt.data(), b->dev.br_count, 4 * nb, cudaMemcpyDeviceToHost, b->stream));
    CU(cudaMemcpyAsync(slot.data(), b->dev.br_slot, 4 * nb, cudaMemcpyDeviceToHost, b->stream));
    CU(cudaStreamSynchronize(b->stream));
    int sl = -1;
    for (int br = 0; br < nb && sl < 0; ++br)
        for (int i = 0; i < cnt[br]; ++i)
            if (perm[start[br] + i] == shot) {
                sl = slot[br];
                break;
            }
    if (sl < 0) return fail(SV_EINVAL, "shot is not in a live branch (waiting list)");
    if (b->prec == SV_C128) {
        CU(cudaMemcpyAsync(out, (char*)b->dev.states + (size_t)sl * b->state_bytes, b->state_bytes,
                           cudaMemcpyDeviceToHost, b->stream));
        CU(cudaStreamSynchronize(b->stream));
    } else {
        std::vector<float> tmp(2 * b->dim);
        CU(cudaMemcpyAsync(tmp.data(), (char*)b->dev.states + (size_t)sl * b->state_bytes, b->state_bytes,
                           cudaMemcpyDeviceToHost, b->stream));
        CU(cudaStreamSynchronize(b->stream));
        for (int64_t i = 0; i < 2 * b->dim; ++i) out[i] = tmp[i];
    }
    return check_device_error(b);
}

sv_status sv_get_outcomes(sv_batch b, uint32_t op, int32_t* sel, double* thr) {
    if (!b || !sel) return fail(SV_EINVAL, "NULL argument");
    auto it = b->logs.find(op);
    if (it == b->logs.end()) return fail(SV_EINVAL, "no log for this op (enable SV_OPT_LOG before sampling)");
    CU(cudaMemcpyAsync(sel, it->second.first, b->n_shots * 4, cudaMemcpyDeviceToHost, b->stream));
    if (thr) CU(cudaMemcpyAsync(thr, it->second.second, b->n_shots * 16, cudaMemcpyDeviceToHost, b->stream));
    CU(cudaStreamSynchronize(b->stream));
    return SV_OK;
}

sv_status sv_get_fork_events(sv_batch b, int64_t* ev, uint64_t cap, uint64_t* n_out) {
    if (!b || !n_out) return fail(SV_EINVAL, "NULL argument");
    if (sv_status cs = commit_forks(b)) return cs;
    if (!b->dev.fork_log) return fail(SV_EINVAL, "enable SV_OPT_LOG first");
    int32_t ctl[CTL_WORDS];
    sv_status st = read_ctl(b, ctl);
    if (st) return st;
    const uint64_t n = std::min<uint64_t>(ctl[CTL_NFORK], b->dev.fork_log_cap);
    *n_out = n;
    if (!ev) return SV_OK;  // size query
    if (n > cap) return fail(SV_EINVAL, "cap too small");
    if (n && ev) {
        std::vector<int64_t> raw(n * FORK_WORDS);
        CU(cudaMemcpyAsync(raw.data(), b->dev.fork_log, n * FORK_WORDS * 8, cudaMemcpyDeviceToHost, b->stream));
        CU(cudaStreamSynchronize(b->stream));
        for (uint64_t e = 0; e < n; ++e)
            for (int w = 0; w < 5; ++w) ev[5 * e + w] = raw[FORK_WORDS * e + w];
    }
    return SV_OK;
}

sv_status sv_get_branch_tree(sv_batch b, int64_t* records, uint64_t cap, uint64_t* n_records, uint32_t* shots,
                             uint64_t shot_cap, uint64_t* n_shot_ids) {
    if (!b || !n_records || !n_shot_ids) return fail(SV_EINVAL, "NULL argument");
    if (!b->dev.fork_log) return fail(SV_EINVAL, "enable SV_OPT_LOG first");
    if (!b->branch) return fail(SV_EINVAL, "the branch tree exists in shot-branching modes only");
    if (sv_status cs = commit_forks(b)) return cs;
    int32_t ctl[CTL_WORDS];
    sv_status st = read_ctl(b, ctl);
    if (st) return st;
    // per-op calls (no sv_run_circuit): one round, the permutation as it is now
    std::vector<sv_batch_s::TreeRound> live;
    const std::vector<sv_batch_s::TreeRound>* rounds = &b->tree;
    if (b->tree.empty()) {
        sv_batch_s::TreeRound r;
        r.fork_end = ctl[CTL_NFORK];
        r.n_run = (int)b->n_shots;
        r.perm.resize(b->n_shots);
        CU(cudaMemcpyAsync(r.perm.data(), b->dev.perm, b->n_shots * 4, cudaMemcpyDeviceToHost, b->stream));
        CU(cudaStreamSynchronize(b->stream));
        live.push_back(std::move(r));
        rounds = &live;
    }
    const int64_t n_ev = rounds->back().fork_end;
    if (n_ev > b->dev.fork_log_cap) return fail(SV_EUNSUPPORTED, "the fork log overflowed; the tree is incomplete");
    std::vector<int64_t> raw((size_t)n_ev * FORK_WORDS);
    if (n_ev) {
        CU(cudaMemcpyAsync(raw.data(), b->dev.fork_log, raw.size() * 8, cudaMemcpyDeviceToHost, b->stream));
        CU(cudaStreamSynchronize(b->stream));
    }
    uint64_t n_ids = 0;
    for (int64_t e = 0; e < n_ev; ++e) n_ids += (uint64_t)(raw[FORK_WORDS * e + 4] + raw[FORK_WORDS * e + 7]);
    *n_records = (uint64_t)n_ev;
    *n_shot_ids = n_ids;
    if (!records && !shots) return SV_OK;  // size query
    if (!records || !shots || (uint64_t)n_ev > cap || n_ids > shot_cap)
        return fail(SV_EINVAL, "records / shots too small for the tree (query the sizes with NULL buffers)");
    uint64_t off = 0;
    size_t r = 0;
    for (int64_t e = 0; e < n_ev; ++e) {
        while (r + 1 < rounds->size() && e >= (*rounds)[r].fork_end) ++r;
        const int64_t* ev = &raw[FORK_WORDS * e];
        const int64_t start = ev[5], cnt = ev[4], pstart = ev[6], pcnt = ev[7];
        if (start < 0 || cnt < 0 || start + cnt > (int64_t)b->n_shots || pstart < 0 || pcnt < cnt ||
            pstart + pcnt > (int64_t)b->n_shots)
            return fail(SV_EINTERNAL, "a fork event's shot range is out of bounds");
        int64_t* rec = records + SV_TREE_WORDS * e;
        rec[0] = (int64_t)r;
        rec[1] = ev[0];
        rec[2] = ev[1];
        rec[3] = ev[2];
        rec[4] = ev[3];
        rec[5] = (int64_t)off;
        rec[6] = cnt;
        rec[7] = (int64_t)(off + cnt);
        rec[8] = pcnt;
        const std::vector<uint32_t>& perm = (*rounds)[r].perm;
        for (int64_t i = 0; i < cnt; ++i) shots[off + i] = perm[start + i];
        for (int64_t i = 0; i < pcnt; ++i) shots[off + cnt + i] = perm[pstart + i];
        off += (uint64_t)(cnt + pcnt);
    }
    return SV_OK;
}

sv_status sv_stats(sv_batch b, double* s) {
    if (!b || !s) return fail(SV_EINVAL, "NULL argument");
    int32_t ctl[CTL_WORDS];
    sv_status st = read_ctl(b, ctl);
    if (st) return st;
    // algorithmic bytes of the passes since the last call: every live state
    // read once, and written once when the pass applies ops
    const int np = std::min<int>(ctl[CTL_NPASS], b->dev.pass_log_cap);
    std::vector<int32_t> nbr(np);
    if (np) CU(cudaMemcpy(nbr.data(), b->dev.pass_log, 4 * np, cudaMemcpyDeviceToHost));
    double bytes = 0;
    for (int i = 0; i < np && i < (int)b->pass_store.size(); ++i)
        bytes += (double)nbr[i] * (double)b->state_bytes * (1.0 + b->pass_store[i]);
    s[0] = ctl[CTL_NBR];
    s[1] = ctl[CTL_NWAIT];
    s[2] = (double)b->n_launch;
    s[3] = (double)b->n_passes;
    s[4] = bytes;
    s[5] = (double)ctl[CTL_NCOPIED] * 2.0 * (double)b->state_bytes;
    s[6] = (double)b->restarts;
    s[7] = b->h2d_bytes;
    b->h2d_bytes = 0;
    b->n_launch = 0;
    b->n_passes = 0;
    b->restarts = 0;
    b->pass_store.clear();
    const int32_t zero[2] = {0, 0};
    CU(cudaMemcpyAsync(b->dev.ctl + CTL_NPASS, zero, 8, cudaMemcpyHostToDevice, b->stream));
    CU(cudaStreamSynchronize(b->stream));
    return SV_OK;
}

sv_status sv_profile(sv_batch b, double* ms, int64_t* cnt) {
    if (!b || !ms || !cnt) return fail(SV_EINVAL, "NULL argument");
    CU(cudaStreamSynchronize(b->stream));
    for (auto& e : b->prof_ev) {
        float t = 0;
        cudaEventElapsedTime(&t, e.second.first, e.second.second);
        b->prof_ms[e.first] += t;
        b->prof_cnt[e.first] += 1;
        cudaEventDestroy(e.second.first);
        cudaEventDestroy(e.second.second);
    }
    b->prof_ev.clear();
    double tot = 0;
    for (int i = 0; i < 7; ++i) {
        ms[i] = b->prof_ms[i];
        cnt[i] = b->prof_cnt[i];
        tot += ms[i];
        b->prof_ms[i] = 0;
        b->prof_cnt[i] = 0;
    }
    ms[7] = tot;
    cnt[7] = 0;
    return SV_OK;
}

sv_status sv_sync(sv_batch b, uint64_t timeout_ns) {
    if (!b) return fail(SV_EINVAL, "batch is NULL");
    if (timeout_ns == 0) {
        CU(cudaStreamSynchronize(b->stream));
        return check_device_error(b);
    }
    const auto t0 = std::chrono::steady_clock::now();
    while (cudaStreamQuery(b->stream) == cudaErrorNotReady) {
        const auto dt = std::chrono::steady_clock::now() - t0;
        if ((uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(dt).count() > timeout_ns)
            return fail(SV_ETIMEOUT, "stream did not finish in time");
    }
    return check_device_error(b);
}

}  // extern "C"
