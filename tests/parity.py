"""Comparison of the CUDA path with the oracle, shot by shot (test helper).

Rules (bit-exactness with explained mismatches):
* Pauli choices must match exactly: both sides compare the same float64 draw
  with the same cumulative table.
* Kraus, measurement and final-sample choices compare u against thresholds
  computed from the state.  A mismatch is *flagged* (not failed) only when
  the two sides' values of the boundary threshold between the two outcomes
  differ by at most tol_c and u lies between them (1e-9 padding); the
  oracle then follows the GPU's choice (override) and the comparison goes on.
* Final amplitudes agree within tol_amp along the matched history.
"""
from __future__ import annotations

import numpy as np

from oracle import oracle as O
from paper_2308_03399_gb300 import sv
from paper_2308_03399_gb300 import workloads as W

TOL = {sv.SV_C128: dict(c=1e-10, amp=1e-12), sv.SV_C64: dict(c=1e-5, amp=1e-5)}


def run_gpu(circ, seed, n_shots, mode, prec, use_graph=True, opts=None, want_amps=(), log=True, mem_budget=0,
            psets=None):
    arrays = circ.to_arrays()
    cs = sv.circuit_struct(arrays)
    with sv.Batch(circ.n_qubits, n_shots, max(1, circ.n_clbits), prec, mode, seed, mem_budget=mem_budget) as b:
        if psets is not None:
            b.set_param_sets(psets, int(np.max(psets)) + 1)
        if log:
            b.set_option(sv.SV_OPT_LOG, 1)
        for k, v in (opts or {}).items():
            b.set_option(k, v)
        b.run_circuit(cs, use_graph=use_graph)
        res = dict(keys=b.get_keys(), stats=b.stats())
        if log:
            res["sel"], res["thr"] = {}, {}
            for op in circ.random_ops():
                s, t = b.get_outcomes(op, thresholds=True)
                res["sel"][op], res["thr"][op] = s, t
            if mode in (sv.SV_BRANCH, sv.SV_BATCH_BRANCH):
                res["forks"] = b.get_fork_events()
                res["tree"] = b.get_branch_tree()
        res["amps"] = {s: b.get_amplitudes(s) for s in want_amps}
    return res


def oracle_refs(circ, seed, shots, state_shots=(), base=0, psets=None):
    """First oracle runs of several shots side by side (threads: the C
    oracle releases the interpreter lock), for sizes where one shot takes
    minutes.  Shots in state_shots also return their final state."""
    import os
    from concurrent.futures import ThreadPoolExecutor
    oc = O.OracleCircuit(circ)
    shots = [int(s) for s in shots]
    with ThreadPoolExecutor(max(1, min(len(shots), os.cpu_count() or 1))) as ex:
        futs = {s: ex.submit(O.run_shot, oc, seed, base + s, None, s in state_shots,
                             0 if psets is None else int(psets[s])) for s in shots}
        return {s: f.result() for s, f in futs.items()}


def compare_shots(circ, seed, gpu, shots, prec, check_amps=True, base=0, amp_errs=None, outcomes_out=None,
                  refs=None, psets=None):
    """Compare the GPU's logs of `shots` with the oracle.  Local shot s of the
    GPU batch is the oracle's global shot base + s.  Returns counts of
    checked draws and flagged draws; raises AssertionError on an unexplained
    mismatch.  With amp_errs, each compared shot's (largest absolute, relative
    L2) amplitude error is appended to it.  With outcomes_out (a dict), the
    oracle's outcome log of each shot (after following flagged draws) is
    stored under the shot.  refs: first oracle runs (oracle_refs) to start
    from instead of running each shot here.  psets[s]: local shot s's
    parameter set (parameter sweeps)."""
    tol = TOL[prec]
    oc = O.OracleCircuit(circ)
    kinds = circ.to_arrays()["kind"]
    rops = circ.random_ops()
    n_draws = n_flag = 0
    fin_ops = {op for op in rops if kinds[op] == W.FINAL}
    for s in shots:
        overrides = {}
        ps = 0 if psets is None else int(psets[s])
        ref = refs[int(s)] if refs is not None else O.run_shot(oc, seed, base + int(s), pset=ps)
        for op in rops:
            g = int(gpu["sel"][op][s])
            c = int(ref["outcome"][op])
            n_draws += 1
            if g == c:
                continue
            assert kinds[op] != W.PAULI, f"shot {s} op {op}: Pauli choice {g} != oracle {c}"
            glo, ghi = gpu["thr"][op][s]
            if g < c:
                bg, bc = ghi, ref["c_lo"][op]
            else:
                bg, bc = glo, ref["c_hi"][op]
            u = ref["u"][op]
            ok = abs(bg - bc) <= tol["c"] and min(bg, bc) - 1e-9 <= u <= max(bg, bc) + 1e-9
            assert ok, (f"shot {s} op {op} kind {kinds[op]}: GPU {g} (thr {glo:.17g},{ghi:.17g}) vs oracle {c} "
                        f"(thr {ref['c_lo'][op]:.17g},{ref['c_hi'][op]:.17g}) u={u:.17g}")
            n_flag += 1
            overrides[op] = g
            if op not in fin_ops:  # the final draw changes nothing after it
                ref = O.run_shot(oc, seed, base + int(s), overrides=overrides, pset=ps)
        if outcomes_out is not None:
            outcomes_out[int(s)] = ref["outcome"].copy()
        fin = [op for op in rops if kinds[op] == W.FINAL]
        if fin:
            assert int(gpu["keys"][s]) == int(gpu["sel"][fin[0]][s])
        if check_amps and s in gpu.get("amps", {}):
            if "state" in ref and not set(overrides) - fin_ops:
                st = ref["state"]  # the state before the final draw
            else:
                st = O.run_shot(oc, seed, base + int(s), overrides=overrides, want_state=True, pset=ps)["state"]
            err = np.abs(gpu["amps"][s] - st).max()
            if amp_errs is not None:
                amp_errs.append((float(err), float(np.linalg.norm(gpu["amps"][s] - st) / np.linalg.norm(st))))
            assert err <= tol["amp"], f"shot {s}: amplitude error {err:.3g} > {tol['amp']}"
    return n_draws, n_flag


def gpu_tree_records(forks):
    """Fork events grouped per (op, parent): sorted (outcome, shots) lists."""
    by = {}
    for op, parent, child, outcome, cnt in forks.tolist():
        by.setdefault((op, parent), []).append((outcome, cnt))
    return sorted((op, tuple(sorted(v))) for (op, _), v in by.items())


def canonical_tree_records(sel, rops, n_shots):
    """The canonical tree (oracle.branch_tree) of the same logs in the same
    grouped form."""
    kinds_final = set()
    outc = np.full((n_shots, max(rops) + 1), -1, np.int64)
    for op in rops:
        outc[:, op] = sel[op]
    recs = O.branch_tree(outc, rops)
    by = {}
    for op, parent, child, outcome in recs:
        by.setdefault((op, parent), []).append((outcome, len(child)))
    del kinds_final
    return sorted((op, tuple(sorted(v))) for (op, _), v in by.items())


def check_branch_tree(tree, outcomes, rops):
    """The GPU's branch tree with shot sets (sv_get_branch_tree) against the
    canonical tree of the oracle's per-shot outcome logs (oracle.branch_tree),
    round by round.

    Round 0 starts from all shots.  Its fork records must equal the canonical
    tree of those shots, cut below the groups the GPU parked on the waiting
    list (a parked group is a record with child -1 whose shots do not fork
    again in the same round).  The shots of the parked groups are the root of
    the next round, whose records must equal the canonical tree of just those
    shots, and so on until no group is parked.  outcomes is (shots, ops), -1
    where a shot made no draw; rops the random ops (final sampling
    excluded).  Returns the number of rounds."""
    records, ids = tree
    n_shots = outcomes.shape[0]
    by_round = {}
    for r, op, parent, child, outc, off, cnt, poff, pcnt in records.tolist():
        S = frozenset(ids[off:off + cnt].tolist())
        P = frozenset(ids[poff:poff + pcnt].tolist())
        assert len(S) == cnt and len(P) == pcnt and S <= P, "a group's shots lie inside its node's"
        by_round.setdefault(r, []).append((op, P, S, outc, child))
    root = frozenset(range(n_shots))
    r = 0
    while root:
        evs = by_round.pop(r, [])
        got = {(op, P, S, o) for op, P, S, o, _ in evs}
        assert len(got) == len(evs), f"round {r}: a fork record appears twice"
        for op, P, S, o, _ in evs:
            assert P <= root, f"round {r}: a node holds shots that are not in the round"
        later = {(op, P) for op, P, S, o, _ in evs}
        parked = [S for op, P, S, o, child in evs
                  if child == -1 and not any(P2 == S and op2 > op for op2, P2 in later)]
        idx = sorted(root)
        canon = O.branch_tree(outcomes[idx], rops, shot_ids=idx)
        canon = {rec for rec in canon if not any(rec[1] <= pk for pk in parked)}
        missing, extra = canon - got, got - canon
        assert not missing and not extra, (f"round {r}: {len(missing)} canonical fork records missing, "
                                           f"{len(extra)} unexpected (of {len(canon)})")
        nxt = frozenset().union(*parked) if parked else frozenset()
        assert sum(len(p) for p in parked) == len(nxt), f"round {r}: parked groups overlap"
        root = nxt
        r += 1
    assert not by_round, f"records for rounds {sorted(by_round)} after the waiting list emptied"
    return r
