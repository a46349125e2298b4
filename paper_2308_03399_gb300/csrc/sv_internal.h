// Internal descriptors shared by the host runtime (sv_runtime.cu) and the
// kernels (sv_kernels.cu).  Everything a kernel needs travels by value in
// its parameters, so a launch sequence can be captured into a CUDA graph
// unchanged.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace sv {

constexpr int MAX_TILE_BITS = 12;  // amplitudes of one CTA tile <= 2^12
constexpr int MAX_STAGES = 40;     // ops fused into one pass
constexpr int MAX_PEND = 64;       // per-branch choice columns of random ops whose stages are pending
constexpr int MAX_TERMS = 64;      // terms of one random op (Pauli strings)
constexpr int64_t REG_UNIT_MIN_AMPS = 8192;  // smallest register-path unit
constexpr int PRE_WORDS = 8;                 // integer-pool words per pre-drawn Pauli row
constexpr uint64_t PRE_TABLE_BYTES = 1ull << 30;  // largest pre-drawn Pauli table
constexpr int MAX_RED = 16;        // probabilities reduced by one pass (Kraus terms, 2^m outcomes)
constexpr int MAX_CHUNKS = 1024;   // reduction partials per state
constexpr int MAX_STAGE_Q = 5;     // qubits of one stage (dense gates up to MAX_GATE_Q)
constexpr int MAT_SMEM = 1024;     // complex matrix entries staged in shared memory per pass
// fork log record: op, parent branch, child branch (-1: waiting list), outcome,
// shots, first perm position of the group's shots at the fork, first perm
// position and shots of the forking node
constexpr int FORK_WORDS = 8;
constexpr int MAX_GATE_Q = 5;      // qubits of one dense gate (a 5-qubit matrix fills MAT_SMEM alone)

// Stage kinds: what one fused op does to a group of 2^k amplitudes.
enum : int32_t {
    ST_DENSE = 0,     // shared dense matrix (a gate)
    ST_DENSE_BR = 1,  // per-branch matrix: term table[sel] * scale (a chosen Kraus matrix)
    ST_PAULI_BR = 2,  // per-branch Pauli string from its 4 parameters (Section IV-A-3)
    ST_PROJ_BR = 3    // per-branch projection onto the measured outcome, optional reset
};
// An ST_DENSE_BR stage whose pend is PEND_PSET takes the matrix of the
// branch's parameter set (br_pset) instead of a sampled choice: a gate whose
// parameters differ between shots (a parameter sweep)
constexpr int32_t PEND_PSET = -1;
constexpr int MAX_PSETS = 1024;  // parameter sets of one batch
enum : int32_t { RED_NONE = 0, RED_FORMS = 1, RED_BINS = 2, RED_DIAG = 3 };
// DEC_KRAUS_J1 / _J2: two one-qubit Kraus ops on different qubits decided
// from one joint reduction p_ij = ||K2_j K1_i psi||^2 (partials indexed
// i * r2 + j): op 1 from p_i = sum_j p_ij, op 2 from p_ij / p_i
enum : int32_t { DEC_PAULI = 0, DEC_KRAUS = 1, DEC_MEASURE = 2, DEC_KRAUS_J1 = 3, DEC_KRAUS_J2 = 4 };

// error word codes
enum : int32_t { ERR_NONE = 0, ERR_SLOT = 1, ERR_INDEX = 2, ERR_GROUPS = 3, ERR_TIMEOUT = 4 };

struct Stage {
    int32_t kind;
    int32_t k;
    int32_t pos[MAX_STAGE_Q];  // tile-local bit of stage qubit j (op order)
    int32_t cond_clbit;        // -1: unconditional
    int32_t cond_val;
    int32_t pend;              // pending-choice column (per-branch kinds)
    int32_t reset;             // ST_PROJ_BR
    int32_t off;               // pool offset (real units) / ipool offset (ST_PAULI_BR)
    int32_t stride;            // real units between terms (ST_DENSE_BR)
    int32_t mat;               // offset of this stage's matrix in the shared-memory matrix area
    int32_t pre;               // ST_PAULI_BR: the choice is row `pend` of the pre-drawn table
};

struct PassDesc {
    int32_t n;                 // qubits
    int32_t tb;                // tile bits
    int32_t run_bits;          // tile-local bits [0, run_bits) are global qubits [0, run_bits)
    int32_t tile_q[MAX_TILE_BITS];
    int32_t n_nontile;
    int32_t nontile_q[32];
    int32_t chunks;            // reduction chunks per state
    int32_t tiles_per_chunk;
    int32_t n_stages;
    int32_t store;             // write the tile back
    int32_t mat_elems;         // complex entries of the shared-memory matrix area
    int32_t red_kind, red_k, red_R, red_off;
    int32_t red_pos[MAX_STAGE_Q];
    int32_t reg_wp;            // > 0: register path (k_pass_reg), group of 2^reg_wp amplitudes
    int32_t reg_paired;        // register path: qubit 0 is group bit 0 (128-bit pairs)
    int32_t fold;              // register path, complex64: the stages composed into one
                               // 2^reg_wp x 2^reg_wp matrix per branch, applied once per group
    int32_t whole;             // whole-state warp pass (k_pass_whole): one warp per branch
    Stage st[MAX_STAGES];
};

// An op decided in the same launch as the decide's head op, after it in
// program order, with no pass between: the second op of a joint Kraus pair
// (DEC_KRAUS_J2, probabilities conditional on the head's choice, from the
// same reduction) or a Pauli op (state-independent table).
constexpr int MAX_TAIL = 3;
constexpr int MAX_TAIL_TERMS = 64;
struct DecideTail {
    uint32_t op;
    int32_t kind;              // DEC_KRAUS_J2 (right after a DEC_KRAUS_J1 head) or DEC_PAULI
    int32_t R;
    int32_t pend;
    int32_t cum_off;           // DEC_PAULI: offset of its table in tail_cum / tail_thr
    int32_t* log_sel;
    double* log_thr;
};

struct DecideDesc {
    uint32_t op;
    int32_t kind;              // DEC_*
    int32_t R;                 // terms / outcomes
    int32_t pend;
    int32_t chunks;            // partials to sum
    int32_t fork;              // shot-branching on
    int32_t sample_only;       // draw and log the choices, change no branch (per-op
                               // calls in shot-branching mode: sv_branch commits)
    int32_t m;                 // measured qubits
    int32_t clbit[MAX_STAGE_Q];
    int32_t r2;                // joint Kraus: terms of the second op (partials stride)
    int32_t pend_prev;         // DEC_KRAUS_J2: pending column of the first op's choice
    uint64_t live_cols;        // choice columns whose stages are still pending (forks copy them)
    int32_t* log_sel;          // per shot id, nullable
    double* log_thr;           // 2 per shot id, nullable
    double cum[MAX_TERMS];     // Pauli cumulative table
    // chain: ops decided after the head in the same launch; a shot's outcome
    // is the tuple (head, tail[0], ...), numbered in mixed radix, nk in all
    int32_t n_tail;
    int32_t nk;                // R times the tail's R (<= MAX_TERMS)
    DecideTail tail[MAX_TAIL];
    double tail_cum[MAX_TAIL_TERMS];
    uint64_t tail_thr[MAX_TAIL_TERMS];  // ceil(cum * 2^53), see cum_threshold
};

struct FinalDesc {
    uint32_t op;
    int32_t chunks;
    int32_t* log_sel;
    double* log_thr;
};

// Device state of a batch (pointers into library-owned device memory).
struct DevBatch {
    void* states;              // n_slots * dim amplitudes
    int64_t dim;
    int32_t n;
    int32_t n_slots;
    int32_t cap_br;            // branch ids per run (= shots)
    uint64_t seed;
    uint64_t shot_base;        // global id of shot 0 (Philox counter offset)
    int32_t* ctl;              // control words, see CTL_*
    int32_t* br_slot;
    int32_t* br_start;
    int32_t* br_count;
    uint64_t* br_clbits;
    int32_t* br_parent;
    int32_t* br_big;           // op whose big-branch decide changed the branch's count (-1: none)
    int32_t* br_pset;          // parameter set of the branch's shots (parameter sweeps)
    const uint32_t* pset_of_shot;  // parameter set of every shot id, nullable (no sweep)
    int32_t n_psets;
    int32_t* br_sel;           // [MAX_PEND][cap_br]
    double* br_scale;          // [MAX_PEND][cap_br]
    uint32_t* perm;            // shot ids, grouped by branch
    uint32_t* perm_tmp;
    int32_t* shot_sel;         // per perm position
    int32_t* free_slots;
    uint32_t* wait_shots;
    double* partials;          // [n_slots][max_chunks][MAX_RED]
    int32_t max_chunks;
    const void* pool;          // real-typed constants (matrices, forms)
    const int32_t* ipool;      // integer constants (Pauli parameters)
    uint64_t* keys;            // per shot id
    uint8_t* pre_sel;          // pre-drawn Pauli choices, [row][shot id] (batch mode)
    int32_t* pos_branch;       // branch owning each perm position (final sampling)
    int64_t* fork_log;         // FORK_WORDS per event, nullable
    int32_t fork_log_cap;
    int32_t* pass_log;         // live branches seen by each pass (profiling), nullable
    int32_t pass_log_cap;
};

// control words (ctl[])
enum : int32_t {
    CTL_NBR = 0,        // live branches
    CTL_NFREE = 1,      // free slots
    CTL_NWAIT = 2,      // shots on the waiting list
    CTL_COPY_FIRST = 3, // first branch created by the last alloc
    CTL_COPY_END = 4,
    CTL_ERR = 5,        // error word
    CTL_ERR_INFO = 6,
    CTL_NFORK = 7,      // fork events logged
    CTL_NPASS = 8,      // passes logged
    CTL_NCOPIED = 9,    // branches created by forks (each one state copy)
    CTL_NALLOC = 10,    // new-branch ids handed out by the current decide
    CTL_DONE = 11,      // finished CTAs of k_copy (last one folds the counts)
    CTL_NRUN = 12,      // shots of a restart whose count is read on the device
    CTL_WORDS = 16
};

// launchers (sv_kernels.cu)
cudaError_t launch_init(const DevBatch& d, int prec, int n_init_slots, int grid, cudaStream_t s);
cudaError_t launch_reset(const DevBatch& d, int mode_branch, int n_shots_run, int from_wait, int grid,
                         cudaStream_t s);
cudaError_t launch_pass(const DevBatch& d, int prec, const PassDesc& p, int threads, int grid, cudaStream_t s);
cudaError_t launch_decide(const DevBatch& d, const DecideDesc& dd, int n_sm, cudaStream_t s, cudaStream_t side,
                          cudaEvent_t ev_fork, cudaEvent_t ev_join);
cudaError_t launch_predraw(const DevBatch& d, int n_rows, int table, int n_shots, int grid, cudaStream_t s);
cudaError_t launch_copy(const DevBatch& d, int prec, int grid, cudaStream_t s);
cudaError_t launch_final(const DevBatch& d, int prec, const FinalDesc& f, int grid, cudaStream_t s);
size_t pass_smem_bytes(int prec, const PassDesc& p, int threads);
size_t pass_reg_smem_bytes(int prec, const PassDesc& p, int threads);
int pass_reg_blocks_per_sm(int prec, int wp, int paired, int var, size_t smem);
int pass_reg_variant(int prec, const PassDesc& p);
// register pass kernel instantiations (one translation unit per group)
const void* reg_kernel_plain_c64(int wp, int paired);
const void* reg_kernel_fold_c64(int wp, int paired);
const void* reg_kernel_bins_c64(int paired);
const void* reg_kernel_c128(int wp);
// whole-state warp passes (complex64, 9 or 10 qubits, no reduction)
size_t pass_whole_smem_bytes(const PassDesc& p);
int pass_whole_blocks_per_sm(int n);
cudaError_t launch_pass_whole(const DevBatch& d, const PassDesc& p, int grid, cudaStream_t s);
int pass_reg_threads(int prec);  // CTA size of the register path
cudaError_t init_kernels();
// density-matrix method (sv_dm.cu): diagonal, running sums, one key per shot
cudaError_t launch_dm_final(const void* rho, int prec, int n, double* p, double* sums, double* cum, int chunks,
                            uint64_t n_shots, uint64_t seed, uint32_t op, uint64_t* keys, double* thr, int n_sm,
                            cudaStream_t s);

}  // namespace sv
