"""Shot distribution over processes, one per GPU (Section IV-C, Section V-C).

Shots are independent, so each process simulates a contiguous range of
global shot ids with the same seed: the library draws shot s of a batch as
global shot ``shot_base + s`` (SV_OPT_SHOT_BASE), and every random number is
keyed by (seed, global shot, op).  The histogram of the union is therefore
the sum of the per-range histograms, whatever the partition, and branching
runs locally inside each range.  The one exchange is that sum, done once at
the end over ``torch.distributed`` (gloo on CPU, NCCL on GPUs).
"""
from __future__ import annotations

from typing import Callable

import numpy as np


def shard(n_shots: int, world: int, rank: int) -> tuple[int, int]:
    """(first global shot, shot count) of ``rank``'s contiguous range; the
    first ``n_shots % world`` ranks take one extra shot."""
    if world < 1 or not 0 <= rank < world or n_shots < 0:
        raise ValueError(f"bad partition: n_shots={n_shots} world={world} rank={rank}")
    q, r = divmod(n_shots, world)
    return rank * q + min(rank, r), q + (1 if rank < r else 0)


def histogram(keys) -> dict:
    vals, cnt = np.unique(np.asarray(keys, np.uint64), return_counts=True)
    return {int(v): int(c) for v, c in zip(vals, cnt)}


def merge_counts(local: dict, group=None, device="cpu") -> dict:
    """Sum of every rank's histogram, returned on every rank.  Keys are final
    measurement registers of at most 62 bits, carried as int64."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    keys = np.fromiter(local.keys(), np.int64, len(local))
    cnts = np.fromiter(local.values(), np.int64, len(local))
    n = torch.tensor([len(keys)], dtype=torch.int64, device=device)
    sizes = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(sizes, n, group=group)
    sizes = [int(s.item()) for s in sizes]
    m = max(sizes)
    if m == 0:
        return {}
    buf = torch.zeros((2, m), dtype=torch.int64, device=device)
    buf[0, : len(keys)] = torch.from_numpy(keys)
    buf[1, : len(cnts)] = torch.from_numpy(cnts)
    bufs = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(bufs, buf, group=group)
    out: dict = {}
    for s, b in zip(sizes, bufs):
        b = b.cpu().numpy()
        for k, c in zip(b[0, :s].tolist(), b[1, :s].tolist()):
            out[k] = out.get(k, 0) + c
    return out


def gpu_runner(prec=None, mode=None, use_graph=True, options=None) -> Callable:
    """Runner that simulates a shot range on the current CUDA device through
    the library: (circuit, seed, base, count) -> per-shot keys."""
    from . import sv

    prec = sv.SV_C64 if prec is None else prec
    mode = sv.SV_BRANCH if mode is None else mode

    def run(circ, seed, base, count):
        with sv.Batch(circ.n_qubits, count, max(1, circ.n_clbits), prec, mode, seed) as b:
            b.set_option(sv.SV_OPT_SHOT_BASE, base)
            for opt, v in (options or {}).items():
                b.set_option(opt, v)
            b.run_circuit(sv.circuit_struct(circ.to_arrays()), use_graph=use_graph)
            return b.get_keys()

    return run


def distributed_counts(circ, n_shots: int, seed: int, runner: Callable | None = None, group=None,
                       device=None) -> dict:
    """Histogram of ``n_shots`` shots of ``circ`` spread over the ranks of
    ``group`` (every rank calls this; every rank gets the merged result).
    ``runner(circ, seed, base, count)`` returns the keys of global shots
    [base, base + count); by default it is the library on the current GPU."""
    import torch.distributed as dist

    rank, world = dist.get_rank(group), dist.get_world_size(group)
    base, count = shard(n_shots, world, rank)
    if runner is None:
        runner = gpu_runner()
    local = histogram(runner(circ, seed, base, count)) if count else {}
    if device is None:
        device = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    return merge_counts(local, group, device)
