/*
 * CPU oracle for noisy multi-shot state-vector simulation.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * definition that the CUDA library is checked against.  Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark may load it; the
 * library never does.  It shares no code with the library.
 *
 * What it computes: every shot is simulated on its own, in float64, from
 * |0...0>, walking the flattened op list in order.  This is the definition
 * the paper's batching (Section IV-A) and shot-branching (Section IV-B)
 * must reproduce: both are re-arrangements of this per-shot computation that
 * change the work done, not the per-shot result.
 *
 *   GATE     Section IV-A-1: a dense 2^k x 2^k matrix on the listed qubits,
 *            skipped when its classical condition does not hold
 *            (Section IV-A-5).
 *   PAULI    Section III-B-1 / Table I: draw u, take the first string whose
 *            cumulative probability exceeds u, apply it as a sequence of
 *            one-qubit Pauli matrices.
 *   KRAUS    Section III-B-2 (Kraus listing): for each matrix K_i in order,
 *            p_i = ||K_i psi||^2 is added to a running sum; the first i with
 *            u < sum is applied as K_i psi / sqrt(p_i).
 *   MEASURE  Section IV-A-5 (measure listing): probabilities of the 2^m
 *            outcomes, first outcome whose running sum exceeds u, collapse
 *            and renormalise, write the classical bits, optional reset.
 *   FINAL    Section IV-B-2 / Section I: one sample of all qubits from the
 *            final state; the sampled index is the count key.
 *   PGATE    Section VI (shots of one circuit with varied gate parameters):
 *            n_terms dense matrices, one per parameter set; the shot's own
 *            parameter set picks the matrix it applies.
 *
 * Randomness: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11), key = (seed lo, seed hi), counter =
 * (shot lo, shot hi, op ordinal, 0); u = ((x0 << 32 | x1) >> 11) * 2^-53.
 *
 * Where u is at or above the last cumulative value (possible only through
 * rounding) the last entry with nonzero probability is taken.
 *
 * Compiled with -ffp-contract=off so that x86 and Arm builds round alike.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

enum { O_GATE = 0, O_PAULI = 1, O_KRAUS = 2, O_MEASURE = 3, O_FINAL = 4, O_PGATE = 5 };

typedef struct {
    int32_t n_qubits, n_clbits, n_ops;
    const int32_t *kind, *nq, *q_off, *cl_off, *n_terms, *s_off, *cond_clbit, *cond_val, *reset;
    const int64_t *d_off;
    const int32_t *qubits, *clbits;
    const double *data;
    const uint8_t *paulis;
} orc_circuit;

/* ------------------------------------------------------------------ */
/* Philox4x32-10                                                       */
/* ------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)0xD2511F53u * c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t n0 = (uint32_t)(prod1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)prod1;
        uint32_t n2 = (uint32_t)(prod0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)prod0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

double orc_uniform(uint64_t seed, uint64_t shot, uint32_t op)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {(uint32_t)shot, (uint32_t)(shot >> 32), op, 0u};
    uint32_t x[4];
    orc_philox4x32_10(ctr, key, x);
    uint64_t bits = ((uint64_t)x[0] << 32) | (uint64_t)x[1];
    return (double)(bits >> 11) * (1.0 / 9007199254740992.0);
}

/* ------------------------------------------------------------------ */
/* state operations, written out from their definitions                */
/* ------------------------------------------------------------------ */

/* psi <- M psi on qubits q[0..k-1]; bit r of the matrix index is qubit q[r]. */
static void apply_matrix(cplx *psi, int n, int k, const int32_t *q, const cplx *m)
{
    uint64_t dim = 1ull << n, sub = 1ull << k, tmask = 0;
    cplx v[32], w[32];
    uint64_t idx[32];
    for (int r = 0; r < k; ++r) tmask |= 1ull << q[r];
    for (uint64_t j = 0; j < dim; ++j) {
        if (j & tmask) continue;
        for (uint64_t r = 0; r < sub; ++r) {
            uint64_t i = j;
            for (int b = 0; b < k; ++b)
                if ((r >> b) & 1) i |= 1ull << q[b];
            idx[r] = i;
            v[r] = psi[i];
        }
        for (uint64_t r = 0; r < sub; ++r) {
            cplx acc = 0;
            for (uint64_t c = 0; c < sub; ++c) acc += m[r * sub + c] * v[c];
            w[r] = acc;
        }
        for (uint64_t r = 0; r < sub; ++r) psi[idx[r]] = w[r];
    }
}

static void load_matrix(const double *d, int k, cplx *m)
{
    uint64_t sub = 1ull << k;
    for (uint64_t e = 0; e < sub * sub; ++e) m[e] = d[2 * e] + I * d[2 * e + 1];
}

static double norm2(const cplx *psi, uint64_t dim)
{
    double s = 0.0;
    for (uint64_t j = 0; j < dim; ++j) s += creal(psi[j]) * creal(psi[j]) + cimag(psi[j]) * cimag(psi[j]);
    return s;
}

/* One-qubit Pauli matrices I, X, Y = [[0,-i],[i,0]], Z. */
static void pauli_matrix(char ch, cplx m[4])
{
    m[0] = m[1] = m[2] = m[3] = 0;
    switch (ch) {
    case 'X': m[1] = 1; m[2] = 1; break;
    case 'Y': m[1] = -I; m[2] = I; break;
    case 'Z': m[0] = 1; m[3] = -1; break;
    default: m[0] = 1; m[3] = 1; break;
    }
}

/* first index t with u < cum[t]; past the end, the last t whose
 * probability cum[t] - cum[t-1] is nonzero */
static int select_cumulative(double u, const double *cum, int n)
{
    for (int t = 0; t < n; ++t)
        if (u < cum[t]) return t;
    for (int t = n - 1; t >= 0; --t) {
        double prev = t ? cum[t - 1] : 0.0;
        if (cum[t] > prev) return t;
    }
    return n - 1;
}

static int find_override(uint32_t op, int32_t n_ovr, const uint32_t *ovr_op, const int32_t *ovr_out)
{
    for (int32_t i = 0; i < n_ovr; ++i)
        if (ovr_op[i] == op) return ovr_out[i];
    return -1;
}

/* ------------------------------------------------------------------ */
/* one shot                                                            */
/* ------------------------------------------------------------------ */
/*
 * pset: the shot's parameter set (the matrix PGATE ops apply).
 * Outputs (each nullable, each indexed by op ordinal):
 *   outcome[op]  chosen term / outcome / key for random ops, -1 otherwise
 *   u_log[op]    the draw
 *   c_lo[op], c_hi[op]  cumulative values just below and at the choice
 *   norms[op]    ||psi||^2 after the op
 * key_out: sampled index of the FINAL op; clbits_out: classical register;
 * state_out: 2*2^n doubles, the state when FINAL is reached (or at the end).
 * Returns 0, or -1 on allocation failure / unsupported sizes.
 */
int orc_run_shot(const orc_circuit *c, uint64_t seed, uint64_t shot, int32_t pset,
                 int32_t n_ovr, const uint32_t *ovr_op, const int32_t *ovr_out,
                 int32_t *outcome, double *u_log, double *c_lo, double *c_hi, double *norms,
                 uint64_t *key_out, uint64_t *clbits_out, double *state_out)
{
    const int n = c->n_qubits;
    const uint64_t dim = 1ull << n;
    if (n < 1 || n > 30) return -1;
    cplx *psi = (cplx *)calloc(dim, sizeof(cplx));
    cplx *phi = NULL;
    double *cum = NULL;
    if (!psi) return -1;
    psi[0] = 1.0;
    uint64_t clreg = 0, key = 0;
    int state_saved = 0, rc = 0;

    for (int32_t op = 0; op < c->n_ops; ++op) {
        const int kind = c->kind[op], k = c->nq[op];
        const int32_t *q = c->qubits + c->q_off[op];
        const double *d = c->data + c->d_off[op];
        if (outcome) outcome[op] = -1;
        if (kind == O_GATE) {
            if (c->cond_clbit[op] >= 0 && (int)((clreg >> c->cond_clbit[op]) & 1) != c->cond_val[op]) {
                if (norms) norms[op] = norm2(psi, dim);
                continue;
            }
            cplx m[1024];
            if (k > 5) { rc = -1; break; }
            load_matrix(d, k, m);
            apply_matrix(psi, n, k, q, m);
        } else if (kind == O_PGATE) {
            cplx m[1024];
            if (k > 5 || pset < 0 || pset >= c->n_terms[op]) { rc = -1; break; }
            load_matrix(d + (int64_t)pset * (int64_t)(2ull << (2 * k)), k, m);
            apply_matrix(psi, n, k, q, m);
        } else if (kind == O_PAULI) {
            const int nt = c->n_terms[op];
            double u = orc_uniform(seed, shot, (uint32_t)op);
            int t = select_cumulative(u, d, nt);
            int ov = find_override((uint32_t)op, n_ovr, ovr_op, ovr_out);
            if (ov >= 0) t = ov;
            const uint8_t *s = c->paulis + c->s_off[op] + (int64_t)t * k;
            for (int j = 0; j < k; ++j) {
                cplx m[4];
                pauli_matrix((char)s[j], m);
                apply_matrix(psi, n, 1, q + j, m);
            }
            if (outcome) outcome[op] = t;
            if (u_log) u_log[op] = u;
            if (c_lo) c_lo[op] = t ? d[t - 1] : 0.0;
            if (c_hi) c_hi[op] = d[t];
        } else if (kind == O_KRAUS) {
            const int nt = c->n_terms[op];
            const uint64_t msz = 2ull << (2 * k);
            double u = orc_uniform(seed, shot, (uint32_t)op);
            int ov = find_override((uint32_t)op, n_ovr, ovr_op, ovr_out);
            if (!phi) phi = (cplx *)malloc(dim * sizeof(cplx));
            if (!phi || k > 5) { rc = -1; break; }
            cplx m[1024];
            double sum = 0.0, chosen_p = 0.0, lo = 0.0;
            int chosen = -1, last_nonzero = -1;
            for (int i = 0; i < nt; ++i) {
                memcpy(phi, psi, dim * sizeof(cplx));
                load_matrix(d + i * msz, k, m);
                apply_matrix(phi, n, k, q, m);
                double p = norm2(phi, dim);
                double before = sum;
                sum += p;
                if (p > 0) last_nonzero = i;
                int take = (ov >= 0) ? (i == ov) : (u < sum);
                if (take) { chosen = i; chosen_p = p; lo = before; break; }
            }
            if (chosen < 0) { /* u at or past the rounded total */
                chosen = last_nonzero >= 0 ? last_nonzero : nt - 1;
                memcpy(phi, psi, dim * sizeof(cplx));
                load_matrix(d + chosen * msz, k, m);
                apply_matrix(phi, n, k, q, m);
                chosen_p = norm2(phi, dim);
                lo = sum - chosen_p;
                sum = lo + chosen_p;
            }
            double scale = 1.0 / sqrt(chosen_p);
            for (uint64_t j = 0; j < dim; ++j) psi[j] = phi[j] * scale;
            if (outcome) outcome[op] = chosen;
            if (u_log) u_log[op] = u;
            if (c_lo) c_lo[op] = lo;
            if (c_hi) c_hi[op] = sum;
        } else if (kind == O_MEASURE) {
            const int m = k;
            const uint64_t nout = 1ull << m;
            const int32_t *cl = c->clbits + c->cl_off[op];
            cum = (double *)realloc(cum, nout * sizeof(double));
            if (!cum) { rc = -1; break; }
            double sum = 0.0;
            for (uint64_t o = 0; o < nout; ++o) {
                double p = 0.0;
                for (uint64_t j = 0; j < dim; ++j) {
                    uint64_t bits = 0;
                    for (int b = 0; b < m; ++b) bits |= ((j >> q[b]) & 1ull) << b;
                    if (bits == o) p += creal(psi[j]) * creal(psi[j]) + cimag(psi[j]) * cimag(psi[j]);
                }
                sum += p;
                cum[o] = sum;
            }
            double u = orc_uniform(seed, shot, (uint32_t)op);
            int o = select_cumulative(u, cum, (int)nout);
            int ov = find_override((uint32_t)op, n_ovr, ovr_op, ovr_out);
            if (ov >= 0) o = ov;
            double po = cum[o] - (o ? cum[o - 1] : 0.0);
            double scale = 1.0 / sqrt(po);
            for (uint64_t j = 0; j < dim; ++j) {
                uint64_t bits = 0;
                for (int b = 0; b < m; ++b) bits |= ((j >> q[b]) & 1ull) << b;
                psi[j] = (bits == (uint64_t)o) ? psi[j] * scale : 0.0;
            }
            for (int b = 0; b < m; ++b) {
                uint64_t bit = ((uint64_t)o >> b) & 1ull;
                clreg = (clreg & ~(1ull << cl[b])) | (bit << cl[b]);
            }
            if (c->reset[op]) {
                cplx xm[4];
                pauli_matrix('X', xm);
                for (int b = 0; b < m; ++b)
                    if (((uint64_t)o >> b) & 1ull) apply_matrix(psi, n, 1, q + b, xm);
            }
            if (outcome) outcome[op] = o;
            if (u_log) u_log[op] = u;
            if (c_lo) c_lo[op] = o ? cum[o - 1] : 0.0;
            if (c_hi) c_hi[op] = cum[o];
        } else if (kind == O_FINAL) {
            if (state_out && !state_saved) {
                for (uint64_t j = 0; j < dim; ++j) {
                    state_out[2 * j] = creal(psi[j]);
                    state_out[2 * j + 1] = cimag(psi[j]);
                }
                state_saved = 1;
            }
            double u = orc_uniform(seed, shot, (uint32_t)op);
            double sum = 0.0, before = 0.0;
            int64_t chosen = -1, last_nonzero = -1;
            int ov = find_override((uint32_t)op, n_ovr, ovr_op, ovr_out);
            if (ov < 0) {
                for (uint64_t j = 0; j < dim; ++j) {
                    double p = creal(psi[j]) * creal(psi[j]) + cimag(psi[j]) * cimag(psi[j]);
                    before = sum;
                    sum += p;
                    if (p > 0) last_nonzero = (int64_t)j;
                    if (u < sum) { chosen = (int64_t)j; break; }
                }
                if (chosen < 0) chosen = last_nonzero >= 0 ? last_nonzero : (int64_t)dim - 1;
            } else {
                chosen = ov;
            }
            if (ov >= 0 || u >= sum) {
                /* a forced key, or the fallback: the running sums around the
                 * key that is actually taken */
                before = 0.0;
                for (int64_t j = 0; j < chosen; ++j)
                    before += creal(psi[j]) * creal(psi[j]) + cimag(psi[j]) * cimag(psi[j]);
                double p = creal(psi[chosen]) * creal(psi[chosen]) + cimag(psi[chosen]) * cimag(psi[chosen]);
                sum = before + p;
            }
            key = (uint64_t)chosen;
            if (outcome) outcome[op] = (int32_t)chosen;
            if (u_log) u_log[op] = u;
            if (c_lo) c_lo[op] = before;
            if (c_hi) c_hi[op] = sum;
        } else {
            rc = -1;
            break;
        }
        if (norms) norms[op] = norm2(psi, dim);
    }
    if (state_out && !state_saved && rc == 0)
        for (uint64_t j = 0; j < dim; ++j) {
            state_out[2 * j] = creal(psi[j]);
            state_out[2 * j + 1] = cimag(psi[j]);
        }
    if (key_out) *key_out = key;
    if (clbits_out) *clbits_out = clreg;
    free(psi);
    free(phi);
    free(cum);
    return rc;
}

/*
 * Shots [shot0, shot0 + n_shots), spread over n_threads OpenMP threads (one
 * shot per thread at a time; threads share nothing but the read-only
 * circuit).  psets (nullable: all 0) gives shot shot0+s's parameter set at
 * psets[s].  keys[s] gets shot shot0+s's final key; outcomes (nullable) is
 * n_shots x n_ops; clbits (nullable) is n_shots.  Returns the number of
 * shots that failed (0 on success).
 */
int orc_run_shots(const orc_circuit *c, uint64_t seed, uint64_t shot0, uint64_t n_shots, const uint32_t *psets,
                  int n_threads, uint64_t *keys, int32_t *outcomes, uint64_t *clbits)
{
    int failed = 0;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : failed)
#endif
    for (int64_t s = 0; s < (int64_t)n_shots; ++s) {
        int32_t *oc = outcomes ? outcomes + (uint64_t)s * (uint64_t)c->n_ops : NULL;
        uint64_t key = 0, cl = 0;
        const int32_t ps = psets ? (int32_t)psets[s] : 0;
        if (orc_run_shot(c, seed, shot0 + (uint64_t)s, ps, 0, NULL, NULL, oc, NULL, NULL, NULL, NULL, &key, &cl, NULL))
            failed += 1;
        keys[s] = key;
        if (clbits) clbits[s] = cl;
    }
    (void)n_threads;
    return failed;
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
