/*
 * sv.h -- C ABI of libsv: batched multi-shot state-vector simulation of
 * noisy quantum circuits on one GPU (sm_103a).
 *
 * The method (Doi, Horii, Wood, "Efficient techniques to GPU Accelerations of
 * Multi-Shot Quantum Computing Simulations", arXiv 2308.03399):
 *   - many shots advance through one circuit in the same kernel launches
 *     (Section IV-A-1), each with its own classical register and parameter
 *     buffers (Section IV-A-2);
 *   - every shot samples its own Pauli noise (Section IV-A-3), Kraus noise
 *     (Section IV-A-4) and measurement outcomes (Section IV-A-5) on the GPU,
 *     with no host synchronisation inside a circuit;
 *   - shot-branching (Section IV-B) keeps one state for all shots that have
 *     drawn the same outcomes and forks a copy only where they diverge; a
 *     branch that finds no free memory parks its shots on a waiting list,
 *     which is re-simulated from |0...0> once the live branches finish.
 *
 * Conventions
 *   - Qubit q is bit q of the amplitude index (little-endian).
 *   - A k-qubit matrix on qubits[0..k-1] maps bit j of its row/column index
 *     to qubits[j]; it is row-major complex float64 with re/im interleaved.
 *   - Every op of a circuit has an ordinal `op`; the shot s draws for op
 *     from Philox4x32-10 with key (seed lo, seed hi) and counter
 *     (s lo, s hi, op, 0), u = top 53 bits of the first two words * 2^-53.
 *     A random op chooses the first entry whose cumulative probability
 *     exceeds u (Table I); u at or above the last cumulative value takes the
 *     last entry with nonzero probability.
 *
 * Ownership and ordering
 *   - The library allocates and owns all device memory of a batch (inside
 *     sv_alloc_batch / sv_run_circuit) and frees it in sv_free_batch.
 *   - Host pointers passed in are read (or written) only during the call.
 *   - Work is issued on the batch's CUDA stream in call order; calls that
 *     return host data (sv_counts, sv_get_*) synchronise that stream.
 *   - A batch is used by one host thread at a time.
 *
 * Errors
 *   - Every call returns sv_status; nothing crosses the ABI as an exception.
 *   - sv_last_error() returns a thread-local message for the last failure.
 *   - Device-side problems (an index out of range, a bounded wait that ran
 *     out) are recorded in a device error word and reported as SV_EINTERNAL
 *     or SV_ETIMEOUT by the next synchronising call.
 */
#ifndef SV_H
#define SV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sv_batch_s *sv_batch;

typedef enum {
    SV_OK = 0,
    SV_EINVAL = 1,       /* bad argument (qubit out of range, non-unitary gate, ...) */
    SV_ENOMEM = 2,       /* device memory exhausted or budget too small */
    SV_ECUDA = 3,        /* a CUDA runtime call failed */
    SV_ETIMEOUT = 4,     /* a bounded device-side wait ran out */
    SV_EUNSUPPORTED = 5, /* valid but beyond the library's limits (sizes, qubit counts) */
    SV_EINTERNAL = 6     /* the device error word was set */
} sv_status;

typedef enum { SV_C64 = 0, SV_C128 = 1 } sv_prec;

/* SV_PLAIN:        one state per shot, shots one after another, one launch
 *                  per op, host reads probabilities back for every Kraus and
 *                  measurement choice (the conventional form the paper's
 *                  Section V-B calls "GPU: Base").
 * SV_BATCH:        one state per shot, every shot in every launch (Section IV-A).
 * SV_BRANCH:       shot-branching (Section IV-B); the live branches are the
 *                  batch of every launch (Section VI's combination).
 * SV_BATCH_BRANCH: same as SV_BRANCH (kept as its own name for callers).   */
typedef enum { SV_PLAIN = 0, SV_BATCH = 1, SV_BRANCH = 2, SV_BATCH_BRANCH = 3 } sv_mode;

typedef enum { SV_NOISE_PAULI = 0, SV_NOISE_KRAUS = 1 } sv_noise_kind;

/* Op kinds of a flattened circuit (sv_circuit.kind). */
enum { SV_OP_GATE = 0, SV_OP_PAULI = 1, SV_OP_KRAUS = 2, SV_OP_MEASURE = 3, SV_OP_FINAL = 4, SV_OP_PGATE = 5 };

/* A flattened circuit as struct-of-arrays (all host pointers, n_ops long
 * unless stated).  Op i acts on qubits[q_off[i] .. q_off[i]+nq[i]).
 *   GATE:    data[d_off[i] ..] one 2^k x 2^k matrix; cond_clbit[i] >= 0 makes
 *            it conditional on classical bit cond_clbit[i] == cond_val[i].
 *   PAULI:   n_terms[i] cumulative probabilities at data[d_off[i] ..] and
 *            n_terms[i]*nq[i] characters from "IXYZ" at paulis[s_off[i] ..],
 *            character j acting on qubits[q_off[i]+j] (Table I form).
 *   KRAUS:   n_terms[i] matrices of 2^k x 2^k at data[d_off[i] ..].
 *   MEASURE: nq[i] qubits into classical bits clbits[cl_off[i] ..]; reset[i]
 *            != 0 returns the measured qubits to |0>.
 *   FINAL:   sample every qubit; the sampled index is the count key.
 *   PGATE:   n_terms[i] matrices of 2^k x 2^k at data[d_off[i] ..], one per
 *            parameter set (sv_set_param_sets); a shot applies its own. */
typedef struct {
    int32_t n_qubits, n_clbits, n_ops;
    const int32_t *kind, *nq, *q_off, *cl_off, *n_terms, *s_off, *cond_clbit, *cond_val, *reset;
    const int64_t *d_off;
    const int32_t *qubits, *clbits;
    const double *data;
    const uint8_t *paulis;
} sv_circuit;

/* Batch options (sv_set_option). */
typedef enum {
    SV_OPT_LOG = 0,         /* 1: record per-shot outcomes, thresholds and fork events */
    SV_OPT_TILE_BITS = 1,   /* amplitudes per CTA tile = 2^value (0 = default)          */
    SV_OPT_MAX_ACTIVE = 2,  /* most distinct qubits fused into one pass (0 = default 4:
                               register passes; wider passes use shared-memory
                               tiles)                                               */
    SV_OPT_MAX_STAGES = 3,  /* most ops fused into one pass (0 = default)               */
    SV_OPT_THREADS = 4,     /* threads per CTA of the tile pass kernel: 32, 64, 128 or
                               256 (0 = default 128)                                */
    SV_OPT_GRID = 5,        /* CTAs of the persistent kernels (0 = default)             */
    SV_OPT_PROFILE = 6,     /* 1: time every launch class with CUDA events              */
    SV_OPT_SLOT_LIMIT = 7,  /* cap on state slots (0 = as many as fit); forces waiting  */
    SV_OPT_UPLOAD = 8,      /* 1: sv_run_circuit copies the circuit's constants to the
                               device on every call, even when its graph is cached   */
    SV_OPT_PASS_PATH = 9,   /* 0: passes of <= 4 qubits run in registers, others in
                               shared-memory tiles; 1: shared-memory tiles only      */
    SV_OPT_JOINT_KRAUS = 10, /* 1 (default): sv_run_circuit decides two back-to-back
                               one-qubit Kraus ops on different qubits from one pass
                               (joint probabilities ||K2_j K1_i psi||^2)             */
    SV_OPT_SHOT_BASE = 11,  /* global id of the batch's shot 0 (default 0): shot s
                               draws its random numbers as shot shot_base + s, so
                               disjoint shot ranges of one seed, run by separate
                               processes or devices, merge into the histogram of
                               one run over the union (shots are independent,
                               Section IV-C).  Keys stay indexed by local shot. */
    SV_OPT_CHAIN_DECIDES = 12, /* 1 (default): sv_run_circuit decides, in one launch,
                               an op and the ops after it that need no new pass
                               (the second op of a joint Kraus pair, Pauli ops) */
    SV_OPT_PREDRAW_PAULI = 13, /* 1 (default): in batch mode, sv_run_circuit draws the
                               Pauli choices of every shot in one launch before the
                               first gate (up to 1 GiB of one-byte choices)
                               instead of one decide per Pauli op */
    SV_OPT_COMMUTE = 14,      /* 1 (default): sv_run_circuit lets a pass take a subset
                               of the queued ops: ops on other qubits commute with it
                               and wait for a later pass (a reduction waits only for
                               what it does not commute with), so passes fill up to
                               the fusion width; 0: every pass takes the whole queue */
    SV_OPT_FOLD = 15,         /* 1 (default): a complex64 register pass with no
                               reduction whose stages cost clearly more per group
                               of 2^w amplitudes than one 2^w x 2^w matrix
                               composes them, per branch, into that matrix and
                               applies it once; 0: stage by stage               */
    SV_OPT_WHOLE_STATE = 16   /* 1: complex64 states of 9 or 10 qubits run their
                               passes without a reduction as whole-state warp
                               passes (one warp per branch, every stage in
                               registers, any qubits); 0 (default): passes of at
                               most the fusion width                            */
} sv_option;

/* Allocate a batch of n_shots shots of an n_qubits register.
 *   mode            see sv_mode; SV_BATCH needs one state per shot
 *   seed            Philox key
 *   mem_budget      bytes of device memory for states (0 = all free memory
 *                   less a reserve); SV_BRANCH admits forks against it
 *   cuda_stream     cudaStream_t to run on, or NULL for a private stream
 * Returns SV_EINVAL for n_qubits outside 1..30, n_shots == 0 or
 * n_clbits > 64, SV_ENOMEM when not even one state fits.                  */
sv_status sv_alloc_batch(int n_qubits, uint64_t n_shots, int n_clbits, sv_prec prec, sv_mode mode,
                         uint64_t seed, uint64_t mem_budget, void *cuda_stream, sv_batch *out);

sv_status sv_free_batch(sv_batch b);

sv_status sv_set_option(sv_batch b, sv_option opt, int64_t value);

/* Section IV-A-1: apply one k-qubit gate (1 <= k <= 5: a fused block of
 * gates given as one dense 2^k x 2^k unitary) to every live state.
 * mat is host, 2^k x 2^k complex float64.  cond_clbit = -1 for an
 * unconditional gate; otherwise shots whose classical bit cond_clbit differs
 * from cond_value are left alone (Section IV-A-5).  SV_EINVAL for repeated or
 * out-of-range qubits or a matrix that is not unitary within 1e-10;
 * SV_EUNSUPPORTED for k > 5 or when the gate's qubits plus qubit 0 exceed
 * the tile (SV_OPT_TILE_BITS).                                              */
sv_status sv_apply_gate_batch(sv_batch b, int k, const int *qubits, const double *mat, int cond_clbit,
                              int cond_value);

/* Section VI (shots of one circuit with varied gate parameters): give every
 * shot a parameter set.  set_of_shot: host, n_shots entries < n_sets
 * (n_sets <= 1024; 0 removes the sweep).  Parameterized gates
 * (sv_apply_param_gate_batch, SV_OP_PGATE) then apply to each shot the
 * matrix of its set.  In shot-branching modes shots of different sets never
 * share a state: a run starts with one root branch per set that has shots
 * (each needs a slot: SV_ENOMEM if n_sets exceeds the batch's slots).  Call
 * before the first op of a run; the device copy of the map is the
 * library's.                                                                */
sv_status sv_set_param_sets(sv_batch b, const uint32_t *set_of_shot, uint32_t n_sets);

/* Section VI: a k-qubit gate (k = 1 or 2) whose matrix depends on the
 * shot's parameter set: mats is host, n_sets matrices of 2^k x 2^k complex
 * float64 (n_sets must equal the batch's).  SV_EINVAL for a non-unitary
 * matrix or a batch without parameter sets.                                */
sv_status sv_apply_param_gate_batch(sv_batch b, int k, const int *qubits, const double *mats, int n_sets);

/* Sections III-B and IV-A-3/4: every shot samples one term of a noise model
 * with its own draw for ordinal `op`.
 *   PAULI: n_terms cumulative probabilities (cum_probs) and n_terms*k chars
 *          of "IXYZ" (paulis), k <= 4, n_terms <= 64.
 *   KRAUS: n_terms matrices of 2^k x 2^k (kraus), k <= 2, n_terms <= 16;
 *          term i is chosen with probability ||K_i psi||^2 and applied as
 *          K_i psi / ||K_i psi||.  SV_EINVAL if sum K^dagger K != I
 *          within 1e-10.
 * In SV_BRANCH modes shots of one branch that choose different terms fork
 * the branch (Section IV-B-2).                                             */
sv_status sv_sample_noise(sv_batch b, uint32_t op, sv_noise_kind kind, int k, const int *qubits, int n_terms,
                          const double *cum_probs, const char *paulis, const double *kraus);

/* Section IV-A-5: measure m <= 4 qubits of every shot into classical bits
 * clbits[0..m-1] (bit i of the outcome is qubits[i]); reset != 0 returns
 * the measured qubits to |0>.                                              */
sv_status sv_measure_batch(sv_batch b, uint32_t op, int m, const int *qubits, const int *clbits, int reset);

/* Section IV-B-2: commit the forks of random op `op`, the last op sampled.
 * In shot-branching modes sv_sample_noise / sv_measure_batch draw and log
 * every shot's choice (sv_get_outcomes sees them) without changing any
 * branch; sv_branch then groups each branch's shots by their choice, keeps
 * the group with the smallest choice in the branch's state, and gives every
 * other group a copy of the state in a free slot (or parks it on the waiting
 * list).  The fork draws again with the same keys (seed, shot, op), so it
 * takes exactly the logged choices.  Any later call on the batch commits a
 * pending fork first, so calling sv_branch is optional.  In SV_BATCH mode
 * every shot is its own branch and there is nothing to commit.  SV_EINVAL
 * if `op` is not the last random op sampled.                                */
sv_status sv_branch(sv_batch b, uint32_t op);

/* Section IV-B-2 / Section I: sample every qubit of every live shot with
 * draw ordinal op_final (one sample per shot from its branch's state) and
 * return the histogram of sampled indices: keys[0..*n_out) ascending with
 * counts[]. cap bounds both host arrays; SV_EINVAL if too small.  Shots on
 * the waiting list are not counted (see sv_waiting).  Synchronises.          */
sv_status sv_counts(sv_batch b, uint32_t op_final, uint64_t *keys, uint64_t *counts, uint64_t cap,
                    uint64_t *n_out);

/* Per-shot final keys of the last sv_counts / sv_run_circuit (host array of
 * n_shots).  Synchronises.                                                  */
sv_status sv_get_keys(sv_batch b, uint64_t *keys);

/* Shots currently parked on the waiting list (Section IV-B-2). */
sv_status sv_waiting(sv_batch b, uint64_t *n_waiting);

/* Run a whole circuit for all shots (Sections IV-A and IV-B), restarting
 * the waiting list until it is empty, and leave per-shot keys for
 * sv_get_keys.  use_graph != 0 captures the launch sequence into a CUDA
 * graph once per circuit and replays it.                                    */
sv_status sv_run_circuit(sv_batch b, const sv_circuit *c, int use_graph);

/* Several circuits, one per batch (n of them, batches sharing one stream;
 * batch and branch modes may mix): with use_graph != 0 the launch sequences
 * of all of them, each with its reset, are captured into ONE CUDA graph
 * (cached for the same batches and circuits) in which every circuit is a
 * parallel branch, so independent circuits run side by side on the GPU
 * (the paper's multi-circuit batching, Section VI); without a graph they run
 * one after another.  Shot-branching
 * batches whose forks parked shots on the waiting list then restart them
 * outside the graph until none wait.  Per-shot keys via sv_get_keys.
 * Batches and circuits must stay alive while the graph is cached.           */
sv_status sv_run_circuits(sv_batch *batches, const sv_circuit *const *circuits, int n, int use_graph);

/* Test / introspection ---------------------------------------------------- */

/* State of the branch that holds `shot`, as 2*len float64 (re, im); len
 * must be 2^n.  Synchronises.                                               */
sv_status sv_get_amplitudes(sv_batch b, uint64_t shot, double *out_re_im, uint64_t len);

/* With SV_OPT_LOG: per-shot choice for random op `op` (-1 if the shot did not
 * reach it) and, if thresholds is non-NULL, 2 float64 per shot: the
 * cumulative values just below and at the choice.  Synchronises.            */
sv_status sv_get_outcomes(sv_batch b, uint32_t op, int32_t *per_shot_outcome, double *thresholds);

/* With SV_OPT_LOG: fork events of the last run (sv_run_circuit, or the
 * per-op calls since the batch was last started), 5 int64 each: (op, parent
 * branch, child branch or -1 for the waiting list, outcome, shots).  A
 * parent's own continuing group is reported with child == parent.  With
 * events NULL the call only reports *n_out.  Synchronises.                  */
sv_status sv_get_fork_events(sv_batch b, int64_t *events, uint64_t cap, uint64_t *n_out);

/* Section IV-B-2: with SV_OPT_LOG in shot-branching modes, the branch tree
 * of the last run with the shot set of every fork.  One record per group of
 * a fork (a fork splits a node's shots by their sampled outcome of op),
 * SV_TREE_WORDS int64 each:
 *   (round, op, parent, child, outcome, shot_offset, shot_count,
 *    parent_offset, parent_count)
 *   round    0 for the first pass through the circuit, r for the r-th
 *            restart of the waiting list (each restart is a new root: the
 *            shots that waited)
 *   parent   branch id (within the round) of the forking node; shots
 *            [parent_offset .. +parent_count) are the node's shot set
 *   child    branch id of the group (== parent for the group that keeps the
 *            parent's state, -1 for a group parked on the waiting list)
 *   shots[shot_offset .. shot_offset + shot_count) are the group's shots
 *            (local shot ids)
 * Records come in decide order (the ops of a chained decide together).  A
 * decide that chains several ops assigns slots to its final groups, so a
 * group of an earlier op of the chain may be parked only in part: its
 * record then shows child -1 (or the branch of its first part) and the
 * records of the later op split it.
 * records: host, cap records; shots: host, shot_cap ids.  With both NULL
 * the call only reports *n_records and *n_shot_ids.  SV_EINVAL when a
 * buffer is too small, SV_EUNSUPPORTED when the device log overflowed
 * (min(64 x shots + 65536, 2^22) events).  Synchronises.                   */
#define SV_TREE_WORDS 9
sv_status sv_get_branch_tree(sv_batch b, int64_t *records, uint64_t cap, uint64_t *n_records, uint32_t *shots,
                             uint64_t shot_cap, uint64_t *n_shot_ids);

/* Live branches and run statistics since the previous call.  stats (8
 * doubles): live branches, waiting shots, kernel launches issued, passes,
 * algorithmic bytes of the pass kernels (each live state read once, and
 * written once when the pass applies ops), bytes of fork copies, waiting-
 * list restarts, bytes copied host to device.  Synchronises.               */
sv_status sv_stats(sv_batch b, double *stats);

/* With SV_OPT_PROFILE: milliseconds spent per launch class (8 doubles:
 * pass, decide, alloc, copy, final, init, other, total) and launch counts
 * (8 int64), accumulated since the last call.  Synchronises.                */
sv_status sv_profile(sv_batch b, double *ms, int64_t *launches);

/* Final sampling that allocates nothing.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc, such as
 * a host framework that owns a fixed device-memory budget and forbids its
 * plug-ins to allocate, or a latency-critical loop where cudaMalloc's
 * implicit synchronisation would stall the device.  It draws one key per
 * state exactly as sv_counts / sv_run_circuit do (same Philox draw, same
 * chunked float64 prefix), from states and into keys the caller provides:
 *   states   device, n_states consecutive states of 2^n_qubits amplitudes
 *            (float2 for SV_C64, double2 for SV_C128), read only
 *   shots    device, n_states 64-bit global shot ids: state i draws with
 *            counter (shots[i], op), as the batch path draws for its shot
 *            shot_base + s (SV_OPT_SHOT_BASE)
 *   keys     device, n_states outputs (sampled indices)
 *   cuda_stream  stream to run on (NULL = default stream); asynchronous
 * Draws within rounding distance of a cumulative threshold are not flagged
 * here (the batch path's log reports the thresholds; this call does not).
 * Scratch is a static 1 MiB device array (131072 float64 partial sums) that
 * every GPU loading the library holds until exit; n_states x chunks (chunks
 * = min(max(2^n_qubits / 2048, 1), 1024)) above that limit gives
 * SV_EINVAL.  The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current and keeps it for
 * the life of the process; make that first call before any stream capture,
 * and do not call again after a cudaDeviceReset (the module, and with it the
 * array, may then sit elsewhere).  All calls share the array and it keeps
 * the last call's contents (every value read is written first in the same
 * call); calls whose work overlaps on the GPU race on it.                    */
sv_status sv_final_sample_noalloc(const void *states, sv_prec prec, int n_qubits, uint32_t n_states,
                                  const uint64_t *shots, uint64_t seed, uint32_t op, uint64_t *keys,
                                  void *cuda_stream);

/* Density-matrix method (Sections II and III-C: exact, but 4^n memory): the
 * circuit's density matrix rho evolves on the GPU (gates U rho U^dagger,
 * Pauli and Kraus channels sum_i K_i rho K_i^dagger, held as a state of 2n
 * qubits vec(rho)[r + c 2^n] = rho[r][c]), then every shot is sampled from
 * the exact final distribution p_j = rho[j][j]: shot s takes the first j
 * with u < C_j, u its Philox draw for the final op (counter (s, op)) and C
 * the running float64 sum in index order.
 *   c           gates (unconditional), Pauli and Kraus noise on 1 or 2
 *               qubits, and a last FINAL op; n_qubits <= 15
 *   keys        host, n_shots sampled indices (n_shots may be 0)
 *   probs       host, 2^n float64 (the distribution), nullable
 *   thresholds  host, 2 x n_shots running sums just below and at each key,
 *               nullable
 * Allocates its own device memory for the call (4^n amplitudes) and frees
 * it.  SV_EUNSUPPORTED for measurements, conditional or parameterized gates,
 * or n_qubits > 15.  Synchronises.                                          */
sv_status sv_dm_run(const sv_circuit *c, sv_prec prec, uint64_t seed, uint64_t n_shots, uint64_t *keys,
                    double *probs, double *thresholds, void *cuda_stream);

/* Learned cost model ------------------------------------------------------
 * A small MLP, n_in -> n_hidden -> n_hidden -> 1 with ReLU, that predicts the
 * log run time of a circuit under a candidate configuration (batch or
 * branch mode, fusion width, pass path, ...), trained on the simulator's own
 * timing logs.  Forward, backward (loss = mean over samples of
 * 0.5 (y - t)^2) and Adam run in the library's CUDA kernels; parameters are
 * one float32 array W1[H x n_in] b1[H] W2[H x H] b2[H] w3[H] b3[1].  x is
 * host, row-major n x n_in; t and y are host, n long.  The model owns its
 * device memory and stream; every call synchronises.  (The paper has no
 * learned part; it ends by noting that the technique has to be chosen per
 * application, Section VI.)                                                   */
typedef struct sv_mlp_s *sv_mlp;
sv_status sv_mlp_create(int n_in, int n_hidden, sv_mlp *out);   /* n_in 1..64, n_hidden 1..128 */
sv_status sv_mlp_free(sv_mlp m);
uint64_t sv_mlp_num_params(sv_mlp m);
sv_status sv_mlp_set_params(sv_mlp m, const float *params, uint64_t n);  /* also resets Adam state */
sv_status sv_mlp_get_params(sv_mlp m, float *params, uint64_t n);
sv_status sv_mlp_forward(sv_mlp m, const float *x, int n, float *y);
/* summed gradient of the loss over the n samples (grad: host, num_params) */
sv_status sv_mlp_gradient(sv_mlp m, const float *x, const float *t, int n, float *loss, float *grad);
/* epochs of shuffled minibatch Adam (shuffle keyed by seed); final_loss =
 * the loss over all n samples afterwards                                      */
sv_status sv_mlp_train(sv_mlp m, const float *x, const float *t, int n, int epochs, int batch, float lr,
                       uint64_t seed, float *final_loss);

/* Wait for the batch's stream, at most timeout_ns (0 = no limit). */
sv_status sv_sync(sv_batch b, uint64_t timeout_ns);

const char *sv_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SV_H */
