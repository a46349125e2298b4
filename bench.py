"""Benchmark: noisy shots per second of batched multi-shot simulation with
shot-branching on one GB300, through the libsv C ABI.

Workload (default): 16-qubit random-SU(4) circuit, depth 16, 2-qubit
depolarizing p=1e-2 and amplitude damping gamma=5e-3 (Kraus) after every
gate, final measurement of all qubits, 10^4 shots, batch-shots with
shot-branching, complex64 amplitudes with float64-grade accumulation.

A step is one whole run of the circuit for all shots (reset, every gate,
noise sample, fork, and the final sample of every shot).  Steps are timed
one by one with CUDA events on the stream the library launches on, with an
L2 flush (a 512 MB write) between them, outside the timed events.

Prints ONE JSON line (rank 0).  --impl reference times the CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "noisy shots/sec at 10–28 qubits, batched FP32 vs plain FP64; % HBM roofline"


def workload(name):
    from paper_2308_03399_gb300 import workloads as W
    if name == "cfg2":
        return W.config2(), 10_000, 2
    if name == "cfg1":
        return W.config1(), 1000, 1
    if name == "cfg3":
        return W.config3(), 10_000, 3
    if name == "cfg5":
        return W.config5(), 2000, 5
    # the paper's QFT with 1% depolarizing noise: qft<n> (Pauli), qftk<n> (Kraus)
    for pre, kraus in (("qftk", True), ("qft", False)):
        if name.startswith(pre) and name[len(pre):].isdigit():
            n = int(name[len(pre):])
            return W.qft(n, 0.01, seed=n, kraus=kraus), 4000, n
    raise SystemExit(f"unknown workload {name}")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def pass_traffic(args, alg_bytes_per_launch):
    """DRAM bytes per k_pass launch: the committed ncu record gives the
    ratio of DRAM traffic to algorithmic bytes over every k_pass launch of
    one step of the same circuit at 2000 shots (a case small enough for a
    multi-metric capture); traffic grows in proportion to the live states a
    pass streams, so the full launch's traffic is that ratio times its
    algorithmic bytes.  None when the kernels have changed since the record
    was taken or the workload differs."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "k_pass_traffic_cfg2_su4_16.txt")
    if not os.path.exists(path) or args.shots:
        return None
    rec = dict(ln.split(None, 1) for ln in open(path).read().strip().splitlines())
    # the pass kernels' sources: the kernel file and the headers holding the
    # register kernel and the shared device helpers, hashed in this order
    h = hashlib.sha1()
    for f in ("sv_kernels.cu", "sv_pass_reg.cuh", "sv_common.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2308_03399_gb300", "csrc", f), "rb").read())
    sha = h.hexdigest()
    if rec.get("source_sha1") != sha or rec.get("workload") != f"{args.workload}:{args.mode}:{args.prec}":
        return None
    ratio = float(rec["dram_bytes_per_step"]) / float(rec["algorithmic_bytes_per_step"])
    return {"bytes_per_launch": ratio * alg_bytes_per_launch, "traffic_over_algorithmic": ratio,
            "measured_on": rec.get("measured_on", "")}


def plain_vs_batched(torch, flush_buf):
    """Config 1 (10-qubit brickwork, 1000 shots): the plain per-shot float64
    form (one state, one launch per op, host-side choices -- the paper's
    conventional "GPU: Base") against the batched forms, shots/s each,
    device time with CUDA events."""
    from paper_2308_03399_gb300 import sv
    circ, shots, seed = workload("cfg1")
    cs = sv.circuit_struct(circ.to_arrays())
    stream = torch.cuda.current_stream()
    out = {"workload": circ.name, "shots": shots}
    for key, mode, prec, warm, steps in (("plain_fp64", sv.SV_PLAIN, sv.SV_C128, 1, 1),
                                         ("batched_fp64", sv.SV_BATCH, sv.SV_C128, 3, 3),
                                         ("batched_fp32", sv.SV_BATCH, sv.SV_C64, 3, 3)):
        b = sv.Batch(circ.n_qubits, shots, 1, prec, mode, seed, stream=stream.cuda_stream)
        graph = mode != sv.SV_PLAIN
        for _ in range(warm):
            b.run_circuit(cs, use_graph=graph)
        b.stats()  # counters from here on cover the timed steps
        ms = 0.0
        for _ in range(steps):
            flush_buf.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.run_circuit(cs, use_graph=graph)
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
        st = b.stats()
        b.close()
        out[key + "_shots_per_s"] = shots * steps / (ms / 1e3)
        if mode == sv.SV_PLAIN:
            # the conventional form's cost is launches: one pass per gate and
            # per non-identity Pauli string, and for a Kraus op or a
            # measurement one reduction per term with a host read of it
            launches = st["launches"] / steps
            out["plain_launches_per_shot"] = launches / shots
            out["plain_us_per_launch"] = 1e3 * ms / steps / max(launches, 1)
    out["ratio_fp32_over_plain"] = out["batched_fp32_shots_per_s"] / out["plain_fp64_shots_per_s"]
    out["ratio_fp64_over_plain"] = out["batched_fp64_shots_per_s"] / out["plain_fp64_shots_per_s"]
    return out


def sm_peaks():
    """SM clock from MEASURED_PEAKS.json (else the nominal 2070 MHz) and the
    GB300 per-SM rates that bound a pass held in shared memory: 152 SMs,
    32 banks x 4 B = 128 B of shared memory per clock per SM, and 128 FP32
    FMA lanes (256 flop) per clock per SM."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    mhz, kind = 2070.0, "nominal clock"
    if os.path.exists(p):
        mhz, kind = float(json.load(open(p)).get("sm_max_mhz", 2070.0)), "measured max clock"
    sms = 152
    return {"smem_gbs": sms * 128 * mhz * 1e6 / 1e9, "fp32_tflops": sms * 256 * mhz * 1e6 / 1e12,
            "derivation": f"152 SMs x (128 B smem | 256 FP32 flop) per clock x {mhz:.0f} MHz ({kind})"}


def leg(torch, flush_buf, name, steps, warmup, mode="branch", prec="c64", graph=True):
    """One more workload on the same GPU: shots/s over `steps` timed steps
    (CUDA events, L2 flushed between steps, clocks sampled), then one
    profiled step (CUDA events around every launch) for the pass kernels'
    own time, algorithmic bytes and passes."""
    from paper_2308_03399_gb300 import sv
    circ, n_shots, seed = workload(name)
    m = {"branch": sv.SV_BRANCH, "batch": sv.SV_BATCH}[mode]
    pr = {"c64": sv.SV_C64, "c128": sv.SV_C128}[prec]
    cs = sv.circuit_struct(circ.to_arrays())
    stream = torch.cuda.current_stream()
    b = sv.Batch(circ.n_qubits, n_shots, max(1, circ.n_clbits), pr, m, seed, stream=stream.cuda_stream)
    for _ in range(warmup):
        b.run_circuit(cs, use_graph=graph)
    torch.cuda.synchronize()
    b.stats()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    ms = []
    for _ in range(steps):
        flush_buf.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.run_circuit(cs, use_graph=graph)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    clk = clocks.stop()
    st = b.stats()
    b.set_option(sv.SV_OPT_PROFILE, 1)
    b.profile()
    flush_buf.fill_(1)
    b.run_circuit(cs, use_graph=False)
    prof = b.profile()
    stp = b.stats()
    b.close()
    pass_ms, n_pass = prof["pass"]
    hbm_peak, peak_kind = peaks()
    step_ms = float(np.mean(ms))
    out = {"workload": circ.name, "n_qubits": circ.n_qubits, "shots": n_shots, "mode": mode, "precision": prec,
           "steps": steps, "warmup": warmup, "shots_per_s": n_shots / (step_ms / 1e3), "ms_per_step": step_ms,
           "passes_per_step": st["passes"] / steps, "restarts_per_step": st["restarts"] / steps,
           "algorithmic_pass_bytes_per_step": stp["pass_bytes"],
           "pass_kernel_ms_per_step": pass_ms, "pass_launches_per_step": n_pass,
           "profile_ms_per_step": {k: v[0] for k, v in prof.items()}, "clocks": clk}
    if pass_ms > 0:
        ach = stp["pass_bytes"] / (pass_ms / 1e3) / 1e9
        out["roofline"] = {"bound": "hbm", "kernel": "k_pass (all pass launches)", "achieved": ach,
                           "peak": hbm_peak, "peak_kind": peak_kind, "unit": "GB/s", "frac": ach / hbm_peak}
    return out, circ, n_shots, prof


def cfg1_smem(torch, flush_buf):
    """Config 1 batched in complex64: 1000 states of 8 KB sit in L2 and each
    pass holds its part of a state on chip (registers, or a shared-memory
    tile), so the passes are bound by on-chip bandwidth or the FP32 pipe,
    not HBM.  Algorithmic work per gate and state (every gate acts on
    every shot in batch mode): a k-qubit dense stage reads and writes each
    of the 2^n amplitudes once in shared memory (2 x 8 B) and does 2^k
    complex multiply-adds per amplitude (8 x 2^k flop).  Both are divided by
    the pass kernels' event time of a profiled step."""
    res, circ, n_shots, prof = leg(torch, flush_buf, "cfg1", steps=5, warmup=3, mode="batch", prec="c64")
    from paper_2308_03399_gb300 import workloads as W
    dim = 1 << circ.n_qubits
    smem_b = sum(2 * 8 * dim for o in circ.ops if o.kind == W.GATE) * n_shots
    flop = sum(8 * (1 << len(o.qubits)) * dim for o in circ.ops if o.kind == W.GATE) * n_shots
    pk = sm_peaks()
    t = res["pass_kernel_ms_per_step"] / 1e3
    res.pop("roofline", None)
    if t > 0:
        smem_frac = smem_b / t / 1e9 / pk["smem_gbs"]
        alu_frac = flop / t / 1e12 / pk["fp32_tflops"]
        res["roofline"] = {
            "bound": "smem" if smem_frac >= alu_frac else "alu", "kernel": "pass kernels (library defaults)",
            "smem": {"achieved": smem_b / t / 1e9, "peak": pk["smem_gbs"], "unit": "GB/s", "frac": smem_frac,
                     "algorithmic_bytes_per_step": smem_b},
            "fp32": {"achieved": flop / t / 1e12, "peak": pk["fp32_tflops"], "unit": "TFLOP/s", "frac": alu_frac,
                     "algorithmic_flop_per_step": flop},
            "peak_derivation": pk["derivation"]}
    return res


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.TimeoutExpired):
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_baseline(circ, seed, budget_s=15.0):
    """The oracle as it stands, on the host's cores, on a bounded sample of
    the workload's shots (shots are independent, so shots/s scales); also
    one core on a few shots."""
    from oracle import oracle as O
    oc = O.OracleCircuit(circ)
    threads = O.max_threads()
    t0 = time.perf_counter()
    O.run_shots(oc, seed, 0, 4, 1, want_outcomes=False)
    single = 4 / (time.perf_counter() - t0)
    n = max(threads, 8)
    t0 = time.perf_counter()
    O.run_shots(oc, seed, 0, n, threads, want_outcomes=False)
    dt = time.perf_counter() - t0
    # grow the sample to about budget_s of work
    n2 = int(max(n, min(200 * n, n * budget_s / max(dt, 1e-3))))
    if n2 > n:
        t0 = time.perf_counter()
        O.run_shots(oc, seed, 0, n2, threads, want_outcomes=False)
        dt = time.perf_counter() - t0
        n = n2
    return {"value": n / dt, "unit": "shots/s", "cores": threads, "kind": "oracle", "cpu_model": cpu_model(),
            "single_core_shots_per_s": single,
            "sample": f"{n} shots of the same circuit (oracle float64, OpenMP over shots), {dt:.1f} s; "
                      f"single core: 4 shots"}


def run_reference(args, rank, world):
    circ, n_shots, seed = workload(args.workload)
    if rank != 0:
        return
    from oracle import oracle as O
    oc = O.OracleCircuit(circ)
    threads = O.max_threads()
    per_step = max(threads, args.ref_shots)
    for _ in range(args.warmup):
        O.run_shots(oc, seed, 0, min(per_step, threads), threads, want_outcomes=False)
    t0 = time.perf_counter()
    for i in range(args.steps):
        O.run_shots(oc, seed, i * per_step, per_step, threads, want_outcomes=False)
    dt = time.perf_counter() - t0
    v = per_step * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "shots/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": circ.name, "n_qubits": circ.n_qubits,
                                            "shots_per_step": per_step, "full_shots": n_shots},
            "cpu_baseline": {"value": v, "unit": "shots/s", "cores": threads, "kind": "oracle",
                             "sample": f"{per_step} shots per step (of {n_shots}), float64 oracle"},
            "e2e": {"value": v, "unit": "shots/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_config4(args):
    """Config 4: 64 brickwork circuits of 8-24 qubits, 10^5 shots split
    unevenly, all run from one captured CUDA graph (sv_run_circuits).  Each
    circuit's configuration (batch or branch mode, fusion width, pass path)
    is picked by the learned cost model; with --autotune the same run with
    the exhaustive autotuner's picks (and the time the search itself took)
    is reported beside it."""
    import torch
    from paper_2308_03399_gb300 import sv
    from paper_2308_03399_gb300 import tuner as T
    torch.cuda.set_device(0)
    torch.cuda.set_stream(torch.cuda.Stream())
    circs, shots = __import__("paper_2308_03399_gb300.workloads", fromlist=["config4"]).config4()
    stream = torch.cuda.current_stream()
    flush_buf = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    free = torch.cuda.mem_get_info()[0]
    pool = int(free * 0.8)
    need = [s * (8 << c.n_qubits) for c, s in zip(circs, shots)]
    model = T.CostModel.load()
    cands = T.candidates()

    # the circuits share one memory pool: a circuit may take a state per shot
    # (batch mode) only within its even share of it, so that batch-mode
    # circuits do not push the wide circuits into extra waiting-list rounds
    share = pool // len(circs)

    def picks_by(fn):
        out = []
        for c, s, nd in zip(circs, shots, need):
            ok = [cfg for cfg in cands if cfg["mode"] == "branch" or nd <= share]
            out.append(fn(c, s, ok))
        return out

    def run(picks, label):
        # memory: batch-mode circuits get exactly one state per shot, the
        # branching ones share the rest in proportion to their full need
        batch_need = sum(nd for nd, p in zip(need, picks) if p["mode"] == "batch")
        rest = max(pool - batch_need, 0)
        br_need = sum(nd for nd, p in zip(need, picks) if p["mode"] == "branch") or 1
        bs, structs = [], []
        for c, s, nd, p, i in zip(circs, shots, need, picks, range(len(circs))):
            mode = sv.SV_BATCH if p["mode"] == "batch" else sv.SV_BRANCH
            # per slot: the state plus its reduction partials (<= 1024 chunks x 16 x 8 B)
            st_bytes = (8 << c.n_qubits) + 128 * max(min(max(1 << max(c.n_qubits - 11, 0), 1), 1024), 1)
            budget = s * st_bytes + (1 << 20) if mode == sv.SV_BATCH else \
                max(min(s * st_bytes, rest * nd // br_need), 2 * st_bytes)
            b = sv.Batch(c.n_qubits, s, 1, sv.SV_C64, mode, 4000 + i, mem_budget=budget, stream=stream.cuda_stream)
            b.set_option(sv.SV_OPT_TILE_BITS, p.get("tile", 0))
            b.set_option(sv.SV_OPT_MAX_ACTIVE, p["max_active"])
            b.set_option(sv.SV_OPT_PASS_PATH, p["path"])
            b.set_option(sv.SV_OPT_JOINT_KRAUS, p["joint"])
            bs.append(b)
            structs.append(sv.circuit_struct(c.to_arrays()))
        for _ in range(args.warmup):
            sv.run_circuits(bs, structs, use_graph=True)
        for b in bs:
            b.stats()
        ms = []
        for _ in range(args.steps):
            flush_buf.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sv.run_circuits(bs, structs, use_graph=True)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        sts = [b.stats() for b in bs]
        launches = sum(x["launches"] for x in sts)
        pass_bytes = sum(x["pass_bytes"] for x in sts) / args.steps
        for b in bs:
            b.close()
        ms_step = float(np.mean(ms))
        return {"label": label, "ms_per_step": ms_step, "shots_per_s": sum(shots) / (ms_step / 1e3),
                "gpu_launches_per_step": launches / args.steps,
                "batch_mode_circuits": sum(p["mode"] == "batch" for p in picks),
                "restarts_per_step": sum(x["restarts"] for x in sts) / args.steps,
                "algorithmic_pass_bytes_per_step": pass_bytes,
                # every circuit's passes over the whole step: how busy HBM was
                "step_average_hbm_gbs": pass_bytes / (ms_step / 1e3) / 1e9,
                "per_circuit": [[c.n_qubits, s, p["mode"], x["restarts"] / args.steps, x["pass_bytes"] / args.steps / 1e9]
                                for c, s, p, x in zip(circs, shots, picks, sts)] if args.compare else None}

    t0 = time.perf_counter()
    mlp_picks = picks_by(lambda c, s, ok: model.pick(c, s, ok))
    t_pick = time.perf_counter() - t0
    res = run(mlp_picks, "cost model")
    line = {"metric": METRIC, "value": res["shots_per_s"], "unit": "shots/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": res["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64", "data": "synthetic",
            "config": {"workload": "cfg4_64_brickwork_8_24q", "circuits": len(circs), "shots": sum(shots),
                       "graph": "one CUDA graph for all 64 circuits", "l2": "flushed between steps (512 MB)"},
            "gpu_launches": int(res["gpu_launches_per_step"] * args.steps), "cost_model_pick_s": t_pick,
            "cost_model": res}
    if args.compare or args.autotune:
        # the fixed policies the model has to beat
        line["fixed_branch"] = run([dict(T.DEFAULT) for _ in circs], "fixed: branch, default fusion")
        fits = [dict(T.DEFAULT, mode="batch") if nd <= share else dict(T.DEFAULT) for nd in need]
        line["fixed_batch_where_it_fits"] = run(fits, "fixed: batch where a state per shot fits the circuit's "
                                                      "even share of the pool, else branch")
    if args.autotune:
        t0 = time.perf_counter()
        small = [c for c in cands if c["joint"] == 1 and c["path"] == 0 and c["tile"] == 0 and c["max_active"] in (0, 3, 8)]
        tuned = picks_by(lambda c, s, ok: T.autotune(c, s, cands=[x for x in small if x in ok], reps=1)[0])
        line["autotune_search_s"] = time.perf_counter() - t0
        line["autotuned"] = run(tuned, "autotuner")
    print(json.dumps(line), flush=True)


def run_qft_sweep(args):
    """The paper's own evaluation (Section V-B, V-D) restated on GB300: QFT
    circuits with 1% depolarizing noise after every gate, as a Pauli model
    and as the equivalent Kraus model, 4000 shots, complex64.  For each
    qubit count: shots/s of batched shots (one state per shot, while they
    fit), shot-branching, and the plain per-shot float64 form (timed on a
    sample of shots, shots being independent); the pass kernels' fraction of
    the measured HBM copy bandwidth.  Then the error-ratio sweep at one
    size: Pauli and Kraus noise at p = 1e-3 .. 3e-2, batched and branched."""
    import torch
    from paper_2308_03399_gb300 import sv
    from paper_2308_03399_gb300 import workloads as W
    torch.cuda.set_device(0)
    torch.cuda.set_stream(torch.cuda.Stream())
    stream = torch.cuda.current_stream()
    flush_buf = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    hbm_peak, peak_kind = peaks()
    shots = 4000
    free = torch.cuda.mem_get_info()[0]

    def timed(circ, mode, prec, n_shots, steps):
        cs = sv.circuit_struct(circ.to_arrays())
        b = sv.Batch(circ.n_qubits, n_shots, 1, prec, mode, 5, stream=stream.cuda_stream)
        graph = mode != sv.SV_PLAIN
        b.run_circuit(cs, use_graph=graph)
        b.stats()
        ms = []
        for _ in range(steps):
            flush_buf.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.run_circuit(cs, use_graph=graph)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        st = b.stats()
        out = {"shots_per_s": n_shots / (np.mean(ms) / 1e3), "ms_per_step": float(np.mean(ms)),
               "passes_per_step": st["passes"] / steps, "restarts_per_step": st["restarts"] / steps}
        if mode != sv.SV_PLAIN:
            b.set_option(sv.SV_OPT_PROFILE, 1)
            b.profile()
            b.run_circuit(cs, use_graph=False)
            pr = b.profile()
            stp = b.stats()
            if pr["pass"][0] > 0:
                out["hbm_frac"] = stp["pass_bytes"] / (pr["pass"][0] / 1e3) / 1e9 / hbm_peak
        b.close()
        return out

    rows = []
    sizes = [int(x) for x in args.qft_sizes.split(",")]
    for n in sizes:
        for kind in ("pauli", "kraus"):
            circ = W.qft(n, 0.01, seed=n, kraus=(kind == "kraus"))
            row = {"n": n, "noise": kind, "ops": circ.n_ops}
            if shots * (8 << n) < 0.6 * free:
                row["batch"] = timed(circ, sv.SV_BATCH, sv.SV_C64, shots, 2)
            row["branch"] = timed(circ, sv.SV_BRANCH, sv.SV_C64, shots, 2)
            # the plain form pays a launch per op (per Kraus term and a host
            # round trip for Kraus noise): a sample of the shots
            plain_shots = max(2, min(40, int((4e4 if kind == "pauli" else 1e4) / circ.n_ops)))
            row["plain_fp64"] = timed(circ, sv.SV_PLAIN, sv.SV_C128, plain_shots, 1)
            row["plain_fp64"]["sample_shots"] = plain_shots
            if n <= 14:
                # the density-matrix method (exact distribution, 4^n memory)
                # for the same 4000 shots: the crossover against multi-shot
                cs = sv.circuit_struct(circ.to_arrays())
                sv.dm_run(cs, shots, sv.SV_C64, 5, stream=stream.cuda_stream)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                sv.dm_run(cs, shots, sv.SV_C64, 5, stream=stream.cuda_stream)
                dt = time.perf_counter() - t0
                row["density_matrix"] = {"shots_per_s": shots / dt, "ms_per_run": 1e3 * dt,
                                         "note": "host wall time of sv_dm_run, allocation included"}
            best = max(v["shots_per_s"] for k, v in row.items() if k in ("batch", "branch"))
            row["best_over_plain"] = best / row["plain_fp64"]["shots_per_s"]
            rows.append(row)
            print(json.dumps(row), file=sys.stderr, flush=True)
    ratio = []
    n_r = args.qft_ratio_n
    for p in (1e-3, 3e-3, 1e-2, 3e-2):
        for kind in ("pauli", "kraus"):
            circ = W.qft(n_r, p, seed=n_r, kraus=(kind == "kraus"))
            r = {"n": n_r, "p": p, "noise": kind, "batch": timed(circ, sv.SV_BATCH, sv.SV_C64, shots, 2),
                 "branch": timed(circ, sv.SV_BRANCH, sv.SV_C64, shots, 2)}
            ratio.append(r)
            print(json.dumps(r), file=sys.stderr, flush=True)
    print(json.dumps({"metric": METRIC, "workload": "qft_sweep", "unit": "shots/s", "shots": shots,
                      "precision": "c64 (plain form: c128)", "hbm_peak_gbs": hbm_peak, "peak_kind": peak_kind,
                      "sizes": rows, "error_ratio": ratio}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cfg2")
    ap.add_argument("--mode", default="branch", choices=["branch", "batch", "plain"])
    ap.add_argument("--prec", default="c64", choices=["c64", "c128"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-shots", type=int, default=32)
    ap.add_argument("--shots", type=int, default=0, help="override the workload's shot count (profiling)")
    ap.add_argument("--timed-only", action="store_true", help="skip the end-to-end and roofline phases")
    ap.add_argument("--no-graph", action="store_true", help="launch kernels one by one (profiling)")
    ap.add_argument("--no-plain", action="store_true", help="skip the config-1 plain-vs-batched comparison")
    ap.add_argument("--max-active", type=int, default=0, help="fusion width (qubits per pass), 0 = library default")
    ap.add_argument("--threads", type=int, default=0, help="threads per tile-pass CTA, 0 = library default")
    ap.add_argument("--whole-state", action="store_true", help="whole-state warp passes (9 or 10 qubits, complex64)")
    ap.add_argument("--autotune", action="store_true", help="config 4: also run the autotuner's picks")
    ap.add_argument("--compare", action="store_true", help="config 4: also run the fixed policies")
    ap.add_argument("--no-legs", action="store_true", help="skip the config 1 / 3 / 5 legs of the default run")
    ap.add_argument("--qft-sizes", default="10,12,14,16,18,20", help="qubit counts of the QFT sweep")
    ap.add_argument("--qft-ratio-n", type=int, default=14, help="qubit count of the error-ratio sweep")
    args = ap.parse_args()
    # three warm-up steps for every timed line; config 4's side record and the
    # QFT sweep (minutes per step) may ask for fewer
    args.warmup = max(args.warmup, 1 if args.workload in ("cfg4", "qft") else 3)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "cfg4":
        return run_config4(args)
    if args.workload == "qft":
        return run_qft_sweep(args)

    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a GPU (the library has no CPU path)")
    torch.cuda.set_device(local)
    # one dedicated stream for the library, the L2 flush and the events
    torch.cuda.set_stream(torch.cuda.Stream())
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2308_03399_gb300 import sv

    circ, n_shots, seed = workload(args.workload)
    if args.shots:
        n_shots = args.shots
    mode = {"branch": sv.SV_BRANCH, "batch": sv.SV_BATCH, "plain": sv.SV_PLAIN}[args.mode]
    prec = {"c64": sv.SV_C64, "c128": sv.SV_C128}[args.prec]
    arrays = circ.to_arrays()
    cs = sv.circuit_struct(arrays)
    stream = torch.cuda.current_stream()
    b = sv.Batch(circ.n_qubits, n_shots, max(1, circ.n_clbits), prec, mode, seed, stream=stream.cuda_stream)
    use_graph = mode != sv.SV_PLAIN and not args.no_graph
    # replicas: rank r simulates global shots [r * n_shots, (r + 1) * n_shots) of one seed
    b.set_option(sv.SV_OPT_SHOT_BASE, rank * n_shots)
    if args.max_active:
        b.set_option(sv.SV_OPT_MAX_ACTIVE, args.max_active)
    if args.threads:
        b.set_option(sv.SV_OPT_THREADS, args.threads)
    if args.whole_state:
        b.set_option(sv.SV_OPT_WHOLE_STATE, 1)
    flush_buf = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")

    for _ in range(args.warmup):
        b.run_circuit(cs, use_graph=use_graph)
    torch.cuda.synchronize()
    b.stats()

    # ---- timed region: K steps, device time per step ------------------------
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    step_ms = []
    for _ in range(args.steps):
        flush_buf.fill_(1)  # L2 flush between timed steps (outside the events)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("timed_step")  # lets ncu capture exactly the timed launches
        e0.record(stream)
        b.run_circuit(cs, use_graph=use_graph)
        e1.record(stream)
        torch.cuda.nvtx.range_pop()
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    st = b.stats()
    total_ms = float(sum(step_ms))
    if dist:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = n_shots * world * args.steps / (total_ms / 1e3)
    launches_per_step = st["launches"] / args.steps
    if args.timed_only:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "shots/s", "ms_per_step": total_ms / args.steps,
                              "shots": n_shots, "workload": circ.name, "mode": args.mode, "precision": args.prec,
                              "max_active": args.max_active,
                              "pass_bytes_per_step": st["pass_bytes"] / args.steps,
                              "passes_per_step": st["passes"] / args.steps,
                              "launches_per_step": launches_per_step, "clocks": clk}), flush=True)
        b.close()
        return

    # ---- end to end through the public API with host buffers -----------------
    b.set_option(sv.SV_OPT_UPLOAD, 1)
    b.stats()
    keys = np.zeros(n_shots, np.uint64)
    e2e_ms = []
    for _ in range(max(2, args.steps)):
        flush_buf.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.run_circuit(cs, use_graph=use_graph)
        keys = b.get_keys()  # device -> host read of the step's result
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    st_e2e = b.stats()
    h2d = st_e2e["h2d_bytes"] / len(e2e_ms)
    e2e_value = n_shots * world / (float(np.mean(e2e_ms)) / 1e3)
    b.set_option(sv.SV_OPT_UPLOAD, 0)

    # ---- roofline of the dominant kernel (k_pass), events per launch ---------
    b.set_option(sv.SV_OPT_PROFILE, 1)
    b.stats()
    b.profile()
    prof_steps = 2
    for _ in range(prof_steps):
        flush_buf.fill_(1)
        b.run_circuit(cs, use_graph=False)
    prof = b.profile()
    stp = b.stats()
    b.set_option(sv.SV_OPT_PROFILE, 0)
    pass_ms, n_pass = prof["pass"]
    hbm_peak, peak_kind = peaks()
    achieved = stp["pass_bytes"] / (pass_ms / 1e3) / 1e9 if pass_ms > 0 else 0.0
    traffic = pass_traffic(args, stp["pass_bytes"] / max(n_pass, 1))

    line = {
        "metric": METRIC, "value": value, "unit": "shots/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64" if prec == sv.SV_C64 else "c128",
        "data": "synthetic",
        "config": {"workload": circ.name, "n_qubits": circ.n_qubits, "depth_ops": circ.n_ops, "shots": n_shots,
                   "mode": args.mode, "precision": args.prec, "seed": seed, "l2": "flushed between steps (512 MB)",
                   "parallelism": f"replicas x{world} (disjoint shot ranges)" if world > 1 else "1 GPU"},
        "gpu_launches": int(round(launches_per_step * args.steps)),
        "e2e": {"value": e2e_value, "unit": "shots/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(keys.nbytes)},
        "roofline": {"bound": "hbm", "kernel": "k_pass", "achieved": achieved, "peak": hbm_peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / hbm_peak,
                     "traffic": traffic["bytes_per_launch"] if traffic else None,
                     "traffic_note": (f"ncu DRAM bytes / algorithmic bytes = {traffic['traffic_over_algorithmic']:.3f} "
                                      f"on {traffic['measured_on']}, scaled to this launch") if traffic else None,
                     "algorithmic_bytes_per_launch": stp["pass_bytes"] / max(n_pass, 1),
                     "algorithmic_bytes_per_step": stp["pass_bytes"] / prof_steps,
                     "pass_ms_per_step": pass_ms / prof_steps, "pass_launches_per_step": n_pass / prof_steps,
                     "share_of_step": pass_ms / max(prof["total"][0], 1e-9)},
        "profile_ms_per_step": {k: v[0] / prof_steps for k, v in prof.items()},
        "branches_at_end": st["live_branches"],
        "clocks": clk,
    }
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(circ, seed)
    if rank == 0 and not args.no_plain and world == 1:
        line["plain_vs_batched"] = plain_vs_batched(torch, flush_buf)
    b.close()
    if rank == 0 and world == 1 and not args.no_legs and args.workload == "cfg2":
        # the metric's other sizes: 10 qubits (states in L2, passes on chip),
        # 20 and 28 qubits (the HBM-roofline target), each with its own clocks
        legs = {"cfg1_smem": lambda: cfg1_smem(torch, flush_buf),
                "cfg3": lambda: leg(torch, flush_buf, "cfg3", steps=2, warmup=1)[0],
                "cfg5": lambda: leg(torch, flush_buf, "cfg5", steps=2, warmup=1)[0]}
        line["legs"] = {}
        for k, fn in legs.items():
            torch.cuda.empty_cache()
            line["legs"][k] = fn()
        c3 = line["legs"]["cfg3"]
        c3["passes_per_round"] = c3["passes_per_step"] / 30
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
