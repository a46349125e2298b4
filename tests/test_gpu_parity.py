"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Every case runs on seeded synthetic circuits and compares, shot by shot, the
GPU's choice for every random op with the oracle's (Pauli exactly; state-
dependent choices exactly unless flagged by the threshold rule), the final
keys, and the final amplitudes (1e-12 complex128, 1e-5 complex64)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2308_03399_gb300 import sv
from paper_2308_03399_gb300 import workloads as W
from tests.parity import (canonical_tree_records, check_branch_tree, compare_shots, gpu_tree_records, oracle_refs,
                          run_gpu)

pytestmark = pytest.mark.gpu

MODES = [sv.SV_BATCH, sv.SV_BRANCH]
PRECS = [sv.SV_C64, sv.SV_C128]

SMALL = {
    "brickwork": lambda: W.brickwork(6, 6, 0.05, 0.1, seed=21),
    "su4_kraus": lambda: W.random_su4(5, 4, 0.1, 0.1, seed=22),
    "midmeasure": lambda: W.midcircuit_measure(6, 3, 0.05, [0, 3], seed=23),
    "qft_kraus": lambda: W.qft(5, 0.05, seed=24, kraus=True),
}


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("name", list(SMALL))
def test_small_circuits_match_oracle(name, mode, prec):
    c = SMALL[name]()
    n_shots = 300
    gpu = run_gpu(c, 7, n_shots, mode, prec, want_amps=range(0, n_shots, 37))
    n, flagged = compare_shots(c, 7, gpu, range(n_shots), prec)
    assert flagged <= max(2, n // 1000)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name", ["su4_kraus", "midmeasure", "qft_kraus"])
def test_shared_memory_tile_path_matches_oracle(name, prec):
    # the same circuits with every pass forced onto shared-memory tiles
    c = SMALL[name]()
    gpu = run_gpu(c, 13, 200, sv.SV_BRANCH, prec, opts={sv.SV_OPT_PASS_PATH: 1}, want_amps=[0, 99])
    compare_shots(c, 13, gpu, range(200), prec)


@pytest.mark.parametrize("prec", PRECS)
def test_register_and_tile_paths_agree_on_config2_prefix(prec):
    # first 3 layers of config 2 at 16 qubits: every pass fits the register
    # path; forcing shared-memory tiles must give the same choices
    c = W.random_su4(16, 3, 1e-2, 5e-3, seed=2)
    a = run_gpu(c, 2, 300, sv.SV_BRANCH, prec, want_amps=[0, 7])
    b = run_gpu(c, 2, 300, sv.SV_BRANCH, prec, opts={sv.SV_OPT_PASS_PATH: 1}, want_amps=[0, 7])
    compare_shots(c, 2, a, range(0, 300, 3), prec)
    compare_shots(c, 2, b, range(0, 300, 3), prec)
    for s in (0, 7):
        assert np.abs(a["amps"][s] - b["amps"][s]).max() < (1e-5 if prec == sv.SV_C64 else 1e-12)


@pytest.mark.parametrize("prec", PRECS)
def test_joint_and_separate_kraus_decisions_match_oracle(prec):
    # back-to-back damping on the two qubits of every gate: decided from one
    # joint reduction (default) or from two passes; both follow the oracle
    c = W.random_su4(9, 4, 0.02, 0.2, seed=33)
    a = run_gpu(c, 12, 300, sv.SV_BRANCH, prec, want_amps=[0, 150])
    b = run_gpu(c, 12, 300, sv.SV_BRANCH, prec, opts={sv.SV_OPT_JOINT_KRAUS: 0}, want_amps=[0, 150])
    assert a["stats"]["passes"] < b["stats"]["passes"]
    compare_shots(c, 12, a, range(300), prec)
    compare_shots(c, 12, b, range(300), prec)


@pytest.mark.parametrize("prec", PRECS)
def test_batch_and_branch_logs_identical(prec):
    c = W.random_su4(6, 5, 0.08, 0.1, seed=31)
    a = run_gpu(c, 3, 400, sv.SV_BATCH, prec)
    b = run_gpu(c, 3, 400, sv.SV_BRANCH, prec)
    assert np.array_equal(a["keys"], b["keys"])
    for op in c.random_ops():
        assert np.array_equal(a["sel"][op], b["sel"][op]), op
        assert np.array_equal(a["thr"][op], b["thr"][op]), op


@pytest.mark.parametrize("prec", PRECS)
def test_fork_events_form_the_canonical_tree(prec):
    c = W.midcircuit_measure(5, 3, 0.05, [1, 3], seed=41)
    n_shots = 500
    gpu = run_gpu(c, 5, n_shots, sv.SV_BRANCH, prec)
    rops = [op for op in c.random_ops() if c.ops[op].kind != W.FINAL]
    assert gpu_tree_records(gpu["forks"]) == canonical_tree_records(gpu["sel"], rops, n_shots)
    compare_shots(c, 5, gpu, range(0, n_shots, 7), prec, check_amps=False)


def _oracle_outcomes(c, seed, gpu, n_shots, prec, **kw):
    outs = {}
    compare_shots(c, seed, gpu, range(n_shots), prec, check_amps=False, outcomes_out=outs, **kw)
    return np.stack([outs[s] for s in range(n_shots)])


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name", list(SMALL))
def test_branch_tree_shot_sets_match_oracle(name, prec):
    # every fork's node and group shot sets equal the canonical tree derived
    # from the oracle's outcome logs of all 300 shots (Section IV-B: a state
    # forks exactly where its shots' sampled outcomes diverge)
    c = SMALL[name]()
    n_shots = 300
    gpu = run_gpu(c, 7, n_shots, sv.SV_BRANCH, prec)
    outc = _oracle_outcomes(c, 7, gpu, n_shots, prec)
    rops = [op for op in c.random_ops() if c.ops[op].kind != W.FINAL]
    assert check_branch_tree(gpu["tree"], outc, rops) == 1
    assert len(gpu["tree"][0]) > 0


@pytest.mark.parametrize("chain", [1, 0])
@pytest.mark.parametrize("prec", PRECS)
def test_branch_tree_with_waiting_list_matches_oracle(prec, chain):
    # three slots: groups park on the waiting list and restart as new roots;
    # each round's records are the canonical tree of that round's shots
    c = W.random_su4(6, 4, 0.1, 0.15, seed=71)
    n_shots = 300
    gpu = run_gpu(c, 4, n_shots, sv.SV_BRANCH, prec,
                  opts={sv.SV_OPT_SLOT_LIMIT: 3, sv.SV_OPT_CHAIN_DECIDES: chain})
    assert gpu["stats"]["restarts"] > 0
    outc = _oracle_outcomes(c, 4, gpu, n_shots, prec)
    rops = [op for op in c.random_ops() if c.ops[op].kind != W.FINAL]
    rounds = check_branch_tree(gpu["tree"], outc, rops)
    assert rounds == gpu["stats"]["restarts"] + 1


@pytest.mark.parametrize("prec,n", [(sv.SV_C64, 14), (sv.SV_C128, 13)])
def test_several_tiles_and_chunks(prec, n):
    # 8 tiles per state: stages and reductions span tile and chunk borders
    c = W.random_su4(n, 3, 0.05, 0.05, seed=51)
    gpu = run_gpu(c, 9, 40, sv.SV_BRANCH, prec, want_amps=[0, 17, 39])
    compare_shots(c, 9, gpu, range(40), prec)


@pytest.mark.parametrize("prec", PRECS)
def test_small_tiles_force_many_passes(prec):
    # 4-amplitude tiles: almost every op gets its own pass
    c = W.brickwork(7, 4, 0.05, 0.1, seed=61)
    gpu = run_gpu(c, 2, 120, sv.SV_BATCH, prec, opts={sv.SV_OPT_TILE_BITS: 3, sv.SV_OPT_MAX_ACTIVE: 4},
                  want_amps=[0, 5])
    compare_shots(c, 2, gpu, range(120), prec)


def test_waiting_list_restarts_match_oracle():
    c = W.random_su4(6, 4, 0.1, 0.15, seed=71)
    gpu = run_gpu(c, 4, 200, sv.SV_BRANCH, sv.SV_C128, opts={sv.SV_OPT_SLOT_LIMIT: 3})
    assert gpu["stats"]["restarts"] > 0
    assert (gpu["forks"][:, 2] == -1).any()
    compare_shots(c, 4, gpu, range(200), sv.SV_C128, check_amps=False)


def test_plain_per_shot_form_matches_oracle():
    c = W.midcircuit_measure(5, 2, 0.05, [0, 2], seed=81)
    gpu = run_gpu(c, 6, 40, sv.SV_PLAIN, sv.SV_C128, log=False)
    keys, _, _ = O.run_shots(c, 6, 0, 40, want_outcomes=False)
    assert np.array_equal(gpu["keys"], keys)
    c = W.random_su4(4, 3, 0.1, 0.1, seed=82)
    gpu = run_gpu(c, 6, 40, sv.SV_PLAIN, sv.SV_C128, log=False)
    keys, _, _ = O.run_shots(c, 6, 0, 40, want_outcomes=False)
    assert np.array_equal(gpu["keys"], keys)


def test_graph_and_direct_launches_agree():
    c = W.random_su4(7, 3, 0.05, 0.1, seed=91)
    a = run_gpu(c, 1, 100, sv.SV_BRANCH, sv.SV_C64, use_graph=True)
    b = run_gpu(c, 1, 100, sv.SV_BRANCH, sv.SV_C64, use_graph=False)
    assert np.array_equal(a["keys"], b["keys"])


def test_per_op_calls_match_run_circuit():
    c = W.midcircuit_measure(5, 2, 0.05, [1, 4], seed=92)
    ref = run_gpu(c, 8, 64, sv.SV_BRANCH, sv.SV_C64, log=False)
    with sv.Batch(5, 64, c.n_clbits, sv.SV_C64, sv.SV_BRANCH, 8) as b:
        for i, o in enumerate(c.ops):
            if o.kind == W.GATE:
                b.apply_gate_batch(o.qubits, o.mat, o.cond_clbit, o.cond_val)
            elif o.kind == W.PAULI:
                b.sample_noise_pauli(i, o.qubits, o.cum, o.strings)
                b.branch(i)
            elif o.kind == W.MEASURE:
                b.measure_batch(i, o.qubits, o.clbits, o.reset)  # committed by the next call
            elif o.kind == W.FINAL:
                cnt = b.counts(i)
        keys = b.get_keys()
    assert np.array_equal(keys, ref["keys"])
    assert sum(cnt.values()) == 64


@pytest.mark.parametrize("prec", PRECS)
def test_sample_then_branch_commits_the_logged_choices(prec):
    # per-op calls in shot-branching mode: sampling logs every shot's choice
    # and forks nothing; sv_branch forks on exactly those choices.  The tree
    # and the keys follow the oracle.
    c = W.random_su4(5, 3, 0.1, 0.15, seed=94)
    n_shots = 200
    with sv.Batch(5, n_shots, 1, prec, sv.SV_BRANCH, 9) as b:
        b.set_option(sv.SV_OPT_LOG, 1)
        for i, o in enumerate(c.ops):
            if o.kind == W.GATE:
                b.apply_gate_batch(o.qubits, o.mat)
                continue
            if o.kind == W.FINAL:
                b.counts(i)
                continue
            if o.kind == W.PAULI:
                b.sample_noise_pauli(i, o.qubits, o.cum, o.strings)
            else:
                b.sample_noise_kraus(i, o.qubits, o.kraus)
            before = b.stats()["live_branches"]
            sel = b.get_outcomes(i)
            assert b.stats()["live_branches"] == before  # nothing forked yet
            if i % 2:
                b.branch(i)  # explicit commit; even ops are committed by the next call
                assert b.stats()["live_branches"] >= before
            assert (sel >= 0).all()
        gpu = dict(keys=b.get_keys(), sel={}, thr={}, tree=b.get_branch_tree(), amps={})
        for op in c.random_ops():
            gpu["sel"][op], gpu["thr"][op] = b.get_outcomes(op, thresholds=True)
        with pytest.raises(sv.SvError):
            b.branch(0)  # not the last random op sampled
    outc = _oracle_outcomes(c, 9, gpu, n_shots, prec)
    rops = [op for op in c.random_ops() if c.ops[op].kind != W.FINAL]
    check_branch_tree(gpu["tree"], outc, rops)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("mode", MODES)
def test_wide_dense_gates_match_oracle(mode, prec):
    # fused blocks given as dense 4- and 5-qubit unitaries (shared-memory
    # tile path), mixed with noise, on 9 qubits
    rng = np.random.default_rng(123)
    c = W.Circuit(9)
    for _ in range(3):
        qs = [int(x) for x in rng.choice(9, 5, replace=False)]
        c.gate(qs, W.haar_unitary(32, rng))
        c.depolarizing(qs[:2], 0.05)
        c.kraus([qs[0]], W.amplitude_damping(0.1))
        qs = [int(x) for x in rng.choice(9, 4, replace=False)]
        c.gate(qs, W.haar_unitary(16, rng))
    c.final()
    gpu = run_gpu(c, 31, 150, mode, prec, want_amps=[0, 149])
    compare_shots(c, 31, gpu, range(150), prec)


def test_per_op_five_qubit_gate_matches_oracle():
    rng = np.random.default_rng(5)
    c = W.Circuit(7)
    c.gate([6, 1, 3, 0, 4], W.haar_unitary(32, rng))
    c.gate([2, 5, 1, 6], W.haar_unitary(16, rng))
    c.final()
    ref = O.run_shot(c, 1, 0, want_state=True)["state"]
    with sv.Batch(7, 4, 1, sv.SV_C128, sv.SV_BATCH, 1) as b:
        for o in c.ops[:-1]:
            b.apply_gate_batch(o.qubits, o.mat)
        assert np.abs(b.get_amplitudes(3) - ref).max() < 1e-12
        with pytest.raises(sv.SvError):
            b.apply_gate_batch([0, 1, 2, 3, 4, 5], np.eye(64))


def test_edge_cases_one_qubit_one_shot():
    c = W.Circuit(1)
    c.gate([0], W.H)
    c.kraus([0], W.amplitude_damping(0.3))
    c.depolarizing([0], 0.2)
    c.final()
    for mode in MODES:
        for prec in PRECS:
            gpu = run_gpu(c, 11, 1, mode, prec, want_amps=[0])
            compare_shots(c, 11, gpu, [0], prec)


def test_bad_arguments_are_rejected():
    with sv.Batch(3, 4, 1, sv.SV_C64, sv.SV_BATCH, 1) as b:
        with pytest.raises(sv.SvError):
            b.apply_gate_batch([3], np.eye(2))
        with pytest.raises(sv.SvError):
            b.apply_gate_batch([0, 0], np.eye(4))
        with pytest.raises(sv.SvError):
            b.apply_gate_batch([0], np.array([[1, 1], [0, 1]]))
        with pytest.raises(sv.SvError):
            b.sample_noise_kraus(0, [0], [np.eye(2) * 0.5])
    with pytest.raises(sv.SvError):
        sv.Batch(31, 1)


def test_config1_all_shots_complex128():
    c = W.config1()
    gpu = run_gpu(c, 1, 1000, sv.SV_BATCH, sv.SV_C128, want_amps=[0, 999])
    n, flagged = compare_shots(c, 1, gpu, range(1000), sv.SV_C128)
    assert flagged == 0


def test_config2_sampled_shots_and_tree():
    # the full 10^4-shot run: 200 seeded shots draw by draw against the oracle
    # (run side by side), two of them with their final states
    c = W.config2()
    n_shots = 10_000
    gpu = run_gpu(c, 2, n_shots, sv.SV_BRANCH, sv.SV_C64, want_amps=[0, 4321])
    rng = np.random.default_rng(0)
    shots = sorted(set(rng.choice(n_shots, 198, replace=False).tolist()) | {0, 4321})
    refs = oracle_refs(c, 2, shots, state_shots=(0, 4321))
    compare_shots(c, 2, gpu, shots, sv.SV_C64, refs=refs)
    rops = [op for op in c.random_ops() if c.ops[op].kind != W.FINAL]
    assert gpu_tree_records(gpu["forks"]) == canonical_tree_records(gpu["sel"], rops, n_shots)


def test_config2_circuit_tree_matches_oracle():
    # the same circuit at 1000 shots: every shot against the oracle, and the
    # branch tree with shot sets against the oracle's canonical tree
    c = W.config2()
    n_shots = 1000
    gpu = run_gpu(c, 2, n_shots, sv.SV_BRANCH, sv.SV_C64)
    refs = oracle_refs(c, 2, range(n_shots))
    outs = {}
    compare_shots(c, 2, gpu, range(n_shots), sv.SV_C64, check_amps=False, outcomes_out=outs, refs=refs)
    rops = [op for op in c.random_ops() if c.ops[op].kind != W.FINAL]
    check_branch_tree(gpu["tree"], np.stack([outs[s] for s in range(n_shots)]), rops)


def test_config3_sampled_shots():
    # 20 qubits, 30 rounds of mid-circuit measurements: 16 shots side by side
    c = W.config3()
    n_shots = 256
    gpu = run_gpu(c, 3, n_shots, sv.SV_BRANCH, sv.SV_C64, want_amps=[0])
    shots = list(range(0, 256, 17))
    refs = oracle_refs(c, 3, shots, state_shots=(0,))
    compare_shots(c, 3, gpu, shots, sv.SV_C64, refs=refs)


def test_run_circuits_one_graph_matches_separate_runs():
    # three circuits, mixed modes and precisions' shot counts, one graph
    cs = [W.brickwork(7, 4, 0.02, 0.05, seed=101), W.random_su4(8, 3, 0.05, 0.1, seed=102),
          W.midcircuit_measure(6, 2, 0.03, [1, 4], seed=103)]
    modes = [sv.SV_BATCH, sv.SV_BRANCH, sv.SV_BRANCH]
    shots = [50, 120, 80]
    ref = [run_gpu(c, 20 + i, s, m, sv.SV_C64, log=False)["keys"] for i, (c, m, s) in enumerate(zip(cs, modes, shots))]
    import torch
    stream = torch.cuda.Stream().cuda_stream  # one shared, non-default stream
    structs = [sv.circuit_struct(c.to_arrays()) for c in cs]
    bs = [sv.Batch(c.n_qubits, s, max(1, c.n_clbits), sv.SV_C64, m, 20 + i, mem_budget=1 << 30, stream=stream)
          for i, (c, m, s) in enumerate(zip(cs, modes, shots))]
    bs[2].set_option(sv.SV_OPT_SLOT_LIMIT, 4)  # force a waiting list in one of them
    for b in bs:
        b.set_option(sv.SV_OPT_LOG, 1)
    for _ in range(2):  # the second call replays the cached graph
        sv.run_circuits(bs, structs, use_graph=True)
        for b, r in zip(bs, ref):
            assert np.array_equal(b.get_keys(), r)
    # every shot of every circuit of the graph against the oracle
    for i, (b, c) in enumerate(zip(bs, cs)):
        gpu = dict(keys=b.get_keys(), sel={}, thr={})
        for op in c.random_ops():
            gpu["sel"][op], gpu["thr"][op] = b.get_outcomes(op, thresholds=True)
        compare_shots(c, 20 + i, gpu, range(shots[i]), sv.SV_C64, check_amps=False)
    for b in bs:
        b.close()


def test_run_circuits_uneven_sizes_match_oracle():
    # circuits of 6 to 14 qubits, both modes, side by side in one graph
    cs = [W.brickwork(n, 3, 0.02, 0.05, seed=200 + n) for n in (6, 9, 12, 14)] + \
         [W.random_su4(11, 3, 0.05, 0.1, seed=211)]
    modes = [sv.SV_BATCH, sv.SV_BRANCH, sv.SV_BATCH, sv.SV_BRANCH, sv.SV_BRANCH]
    shots = [64, 40, 32, 24, 48]
    import torch
    stream = torch.cuda.Stream().cuda_stream
    bs = [sv.Batch(c.n_qubits, s, 1, sv.SV_C64, m, 50 + i, mem_budget=1 << 30, stream=stream)
          for i, (c, m, s) in enumerate(zip(cs, modes, shots))]
    for b in bs:
        b.set_option(sv.SV_OPT_LOG, 1)
    sv.run_circuits(bs, [sv.circuit_struct(c.to_arrays()) for c in cs], use_graph=True)
    for i, (b, c) in enumerate(zip(bs, cs)):
        gpu = dict(keys=b.get_keys(), sel={}, thr={})
        for op in c.random_ops():
            gpu["sel"][op], gpu["thr"][op] = b.get_outcomes(op, thresholds=True)
        compare_shots(c, 50 + i, gpu, range(shots[i]), sv.SV_C64, check_amps=False)
        b.close()


def test_alternating_circuits_on_one_batch_replay_correct_graphs():
    # two circuits share one batch: each recording replaces the batch's
    # constants, so a cached graph must not replay the other circuit's data
    a = W.random_su4(6, 3, 0.05, 0.1, seed=111)
    b = W.random_su4(6, 3, 0.05, 0.1, seed=112)
    ka = run_gpu(a, 5, 64, sv.SV_BRANCH, sv.SV_C64, log=False)["keys"]
    kb = run_gpu(b, 5, 64, sv.SV_BRANCH, sv.SV_C64, log=False)["keys"]
    sa, sb = sv.circuit_struct(a.to_arrays()), sv.circuit_struct(b.to_arrays())
    with sv.Batch(6, 64, 1, sv.SV_C64, sv.SV_BRANCH, 5) as bt:
        for c, k in ((sa, ka), (sb, kb), (sa, ka), (sa, ka), (sb, kb)):
            bt.run_circuit(c, use_graph=True)
            assert np.array_equal(bt.get_keys(), k)


@pytest.mark.parametrize("base", [1000, (1 << 33) + 5])
@pytest.mark.parametrize("mode", MODES)
def test_shot_base_draws_global_shots(mode, base):
    c = SMALL["midmeasure"]()
    gpu = run_gpu(c, 9, 120, mode, sv.SV_C128, opts={sv.SV_OPT_SHOT_BASE: base}, want_amps=(0, 77))
    compare_shots(c, 9, gpu, range(120), sv.SV_C128, base=base)


def test_shot_base_plain_form():
    c = W.random_su4(4, 3, 0.1, 0.1, seed=83)
    gpu = run_gpu(c, 6, 30, sv.SV_PLAIN, sv.SV_C128, log=False, opts={sv.SV_OPT_SHOT_BASE: 500})
    keys, _, _ = O.run_shots(c, 6, 500, 30, want_outcomes=False)
    assert np.array_equal(gpu["keys"], keys)


@pytest.mark.parametrize("prec", PRECS)
def test_shot_ranges_concatenate_to_one_run(prec):
    from paper_2308_03399_gb300 import replicas
    c = W.random_su4(7, 4, 0.05, 0.1, seed=93)
    whole = run_gpu(c, 3, 301, sv.SV_BRANCH, prec, log=False)["keys"]
    parts = []
    for r in range(3):
        base, count = replicas.shard(301, 3, r)
        parts.append(replicas.gpu_runner(prec=prec)(c, 3, base, count))
    assert np.array_equal(np.concatenate(parts), whole)
    # a cached graph must not keep the old base
    cs = sv.circuit_struct(c.to_arrays())
    with sv.Batch(7, 100, 1, prec, sv.SV_BRANCH, 3) as b:
        b.run_circuit(cs)
        assert np.array_equal(b.get_keys(), whole[:100])
        b.set_option(sv.SV_OPT_SHOT_BASE, 201)
        b.run_circuit(cs)
        assert np.array_equal(b.get_keys(), whole[201:301])


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("name", ["su4_kraus", "midmeasure", "brickwork"])
def test_chained_and_separate_decides_agree(name, mode, prec):
    # a chain (head op, the second op of a Kraus pair, Pauli ops) decided in
    # one launch takes the same choices as one launch per op
    c = SMALL[name]()
    # batch mode would draw the Pauli ops up front: keep them as decides here
    a = run_gpu(c, 12, 200, mode, prec, opts={sv.SV_OPT_PREDRAW_PAULI: 0})
    b = run_gpu(c, 12, 200, mode, prec, opts={sv.SV_OPT_PREDRAW_PAULI: 0, sv.SV_OPT_CHAIN_DECIDES: 0})
    for op in c.random_ops():
        assert np.array_equal(a["sel"][op], b["sel"][op]), op
    assert np.array_equal(a["keys"], b["keys"])
    assert a["stats"]["launches"] < b["stats"]["launches"]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name", ["brickwork", "midmeasure", "su4_kraus"])
def test_predrawn_pauli_choices_match_decides(name, prec):
    # batch mode draws every shot's Pauli choices in one launch up front;
    # the choices, logs and keys are those of one decide per Pauli op
    c = SMALL[name]()
    a = run_gpu(c, 13, 150, sv.SV_BATCH, prec)
    b = run_gpu(c, 13, 150, sv.SV_BATCH, prec, opts={sv.SV_OPT_PREDRAW_PAULI: 0})
    for op in c.random_ops():
        assert np.array_equal(a["sel"][op], b["sel"][op]), op
        assert np.array_equal(a["thr"][op], b["thr"][op]), op
    assert np.array_equal(a["keys"], b["keys"])
    assert a["stats"]["launches"] < b["stats"]["launches"]
    compare_shots(c, 13, a, range(0, 150, 7), prec)


# ---------------------------------------------------------------------------
# Parameter sweeps (Section VI: shots of one circuit with varied gate
# parameters): each shot applies the matrices of its own parameter set
# ---------------------------------------------------------------------------
def _psets(n_shots, n_sets, seed):
    return np.random.default_rng(seed).integers(0, n_sets, n_shots).astype(np.uint32)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("mode", MODES)
def test_param_sweep_matches_oracle(mode, prec):
    c = W.param_sweep(6, 4, 5, 0.05, seed=300)
    n_shots = 200
    ps = _psets(n_shots, 5, 1)
    gpu = run_gpu(c, 3, n_shots, mode, prec, psets=ps, want_amps=[0, 1, 2, 199])
    compare_shots(c, 3, gpu, range(n_shots), prec, psets=ps)
    if mode == sv.SV_BRANCH:
        # one root per parameter set: no state is shared across sets
        assert gpu["stats"]["live_branches"] >= len(set(ps.tolist()))


def test_param_sweep_waiting_list_and_per_op_calls():
    c = W.param_sweep(5, 3, 4, 0.1, seed=301)
    n_shots = 160
    ps = _psets(n_shots, 4, 2)
    gpu = run_gpu(c, 8, n_shots, sv.SV_BRANCH, sv.SV_C128, psets=ps, opts={sv.SV_OPT_SLOT_LIMIT: 6})
    assert gpu["stats"]["restarts"] > 0
    compare_shots(c, 8, gpu, range(n_shots), sv.SV_C128, check_amps=False, psets=ps)
    # the same circuit through the per-op calls gives the same keys
    with sv.Batch(5, n_shots, 1, sv.SV_C128, sv.SV_BRANCH, 8) as b:
        b.set_param_sets(ps, 4)
        for i, o in enumerate(c.ops):
            if o.kind == W.PGATE:
                b.apply_param_gate_batch(o.qubits, o.kraus)
            elif o.kind == W.GATE:
                b.apply_gate_batch(o.qubits, o.mat)
            elif o.kind == W.PAULI:
                b.sample_noise_pauli(i, o.qubits, o.cum, o.strings)
            else:
                b.counts(i)
        keys = b.get_keys()
    okeys, _, _ = O.run_shots(c, 8, 0, n_shots, want_outcomes=False, psets=ps)
    assert np.array_equal(keys, okeys)
    # plain per-shot form
    gp = run_gpu(c, 8, 40, sv.SV_PLAIN, sv.SV_C128, log=False, psets=ps[:40])
    assert np.array_equal(gp["keys"], okeys[:40])


def test_param_sweep_rejects_bad_sets():
    with sv.Batch(3, 8, 1, sv.SV_C64, sv.SV_BRANCH, 1) as b:
        with pytest.raises(sv.SvError):
            b.set_param_sets(np.full(8, 3, np.uint32), 3)  # set 3 of 3
        with pytest.raises(sv.SvError):
            b.apply_param_gate_batch([0], [np.eye(2)])  # no sets yet
        b.set_param_sets(np.arange(8) % 2, 2)
        with pytest.raises(sv.SvError):
            b.apply_param_gate_batch([0], [np.eye(2)] * 3)  # 3 matrices for 2 sets


# ---------------------------------------------------------------------------
# Passes that take a subset of the queued ops (SV_OPT_COMMUTE): ops on
# other qubits commute with the pass and wait for a later one; a reduction
# waits only for what it does not commute with
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("mode", MODES)
def test_commuting_passes_match_oracle(mode, prec):
    # config 3's round structure (U3 layer, CX ladder, mid-circuit
    # measurement, conditional resets) on 14 qubits: more qubits than a tile
    c = W.midcircuit_measure(14, 3, 0.01, [0, 5, 10], seed=140)
    a = run_gpu(c, 3, 200, mode, prec, want_amps=[0, 199])
    b = run_gpu(c, 3, 200, mode, prec, opts={sv.SV_OPT_COMMUTE: 0})
    assert a["stats"]["passes"] < b["stats"]["passes"]
    compare_shots(c, 3, a, range(200), prec)
    compare_shots(c, 3, b, range(0, 200, 5), prec, check_amps=False)


@pytest.mark.parametrize("kraus", [False, True])
def test_commuting_passes_qft_match_oracle(kraus):
    c = W.qft(13, 0.02, seed=131, kraus=kraus)
    a = run_gpu(c, 4, 120, sv.SV_BRANCH, sv.SV_C64, want_amps=[0, 119])
    b = run_gpu(c, 4, 120, sv.SV_BRANCH, sv.SV_C64, opts={sv.SV_OPT_COMMUTE: 0}, log=False)
    assert a["stats"]["passes"] <= b["stats"]["passes"]
    compare_shots(c, 4, a, range(120), sv.SV_C64)
    rops = [op for op in c.random_ops() if c.ops[op].kind != W.FINAL]
    check_branch_tree(a["tree"], _oracle_outcomes(c, 4, a, 120, sv.SV_C64), rops)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("case", ["qft13", "brick9_w3"])
def test_folded_passes_match_oracle(case, mode):
    # Register passes with many stages and no reduction compose their stages
    # per branch into one 2^w x 2^w matrix (SV_OPT_FOLD): QFT passes on 13
    # qubits hold up to ~30 one- and two-qubit ops on 4 qubits; a 9-qubit
    # brickwork at fusion width 3 folds 8 x 8 matrices.  Folded and
    # stage-by-stage runs give the oracle's shots and the same states.
    if case == "qft13":
        c, opts = W.qft(13, 0.02, seed=133), {}
    else:
        c, opts = W.brickwork(9, 10, 0.02, 0.05, seed=134), {sv.SV_OPT_MAX_ACTIVE: 3}
    amps = [0, 77, 149]
    a = run_gpu(c, 6, 150, mode, sv.SV_C64, opts=opts, want_amps=amps)
    b = run_gpu(c, 6, 150, mode, sv.SV_C64, opts={**opts, sv.SV_OPT_FOLD: 0}, want_amps=amps)
    compare_shots(c, 6, a, range(150), sv.SV_C64)
    compare_shots(c, 6, b, range(0, 150, 10), sv.SV_C64, check_amps=False)
    for s in amps:
        np.testing.assert_allclose(a["amps"][s], b["amps"][s], atol=2e-6)


@pytest.mark.parametrize("threads", [32, 64])
@pytest.mark.parametrize("name", list(SMALL))
def test_small_tile_ctas_match_oracle(name, threads):
    # one- and two-warp CTAs on whole-state tiles: block barriers are warp
    # barriers, reductions with as many forms as threads or more move to a
    # wider CTA
    c = SMALL[name]()
    gpu = run_gpu(c, 12, 200, sv.SV_BATCH, sv.SV_C64, opts={sv.SV_OPT_THREADS: threads}, want_amps=[0, 199])
    compare_shots(c, 12, gpu, range(200), sv.SV_C64)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("case", ["brick9", "brick10", "qft10", "mid10"])
def test_whole_state_passes_match_oracle(case, mode):
    # SV_OPT_WHOLE_STATE: complex64 states of 9 or 10 qubits held by one
    # warp; passes without a reduction take any qubits (bits exchanged
    # between registers and lanes), passes with one keep the other paths
    c = {"brick9": lambda: W.brickwork(9, 8, 0.02, 0.05, seed=141),
         "brick10": lambda: W.brickwork(10, 8, 0.02, 0.05, seed=142),
         "qft10": lambda: W.qft(10, 0.02, seed=143),
         "mid10": lambda: W.midcircuit_measure(10, 3, 0.02, [0, 7], seed=144)}[case]()
    amps = [0, 99, 199]
    a = run_gpu(c, 8, 200, mode, sv.SV_C64, opts={sv.SV_OPT_WHOLE_STATE: 1}, want_amps=amps)
    b = run_gpu(c, 8, 200, mode, sv.SV_C64, want_amps=amps)
    if case.startswith("brick"):
        assert a["stats"]["passes"] < b["stats"]["passes"]
    compare_shots(c, 8, a, range(200), sv.SV_C64)
    for s in amps:
        np.testing.assert_allclose(a["amps"][s], b["amps"][s], atol=2e-6)
