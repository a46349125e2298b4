"""Shot distribution over ranks (Section IV-C): contiguous shot ranges, one
histogram merge.  The ranks run as gloo processes on the CPU with the oracle
as each rank's simulator, so the host logic (partition, shot offsets, merge)
is checked against one oracle run over all shots."""
import json
import os
import socket
import subprocess
import sys

import pytest

from oracle import oracle as O
from paper_2308_03399_gb300 import replicas

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
import replica_worker  # noqa: E402


@pytest.mark.parametrize("n_shots", [0, 1, 5, 7, 100, 1001])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_shard_is_a_contiguous_partition(n_shots, world):
    ranges = [replicas.shard(n_shots, world, r) for r in range(world)]
    pos = 0
    for base, count in ranges:
        assert base == pos and count >= 0
        pos += count
    assert pos == n_shots
    counts = [c for _, c in ranges]
    assert max(counts) - min(counts) <= 1


def test_shard_rejects_bad_arguments():
    with pytest.raises(ValueError):
        replicas.shard(10, 0, 0)
    with pytest.raises(ValueError):
        replicas.shard(10, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run_ranks(tmp_path, name, n_shots, seed, world=2, mistake="none"):
    out = str(tmp_path / f"merged_{name}_{n_shots}_{mistake}")
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE=str(world), LOCAL_RANK=str(r),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), OMP_NUM_THREADS="1")
        procs.append(subprocess.Popen([sys.executable, os.path.join(HERE, "replica_worker.py"), out, name,
                                       str(n_shots), str(seed), mistake], env=env))
    for p in procs:
        assert p.wait(timeout=120) == 0
    res = []
    for r in range(world):
        with open(f"{out}.{r}") as f:
            res.append({int(k): v for k, v in json.load(f).items()})
    return res


@pytest.mark.parametrize("name,n_shots,world", [("mid", 37, 2), ("su4", 64, 2), ("su4", 1, 2), ("mid", 50, 3)])
def test_gloo_merge_equals_one_run(tmp_path, name, n_shots, world):
    seed = 2024
    merged = _run_ranks(tmp_path, name, n_shots, seed, world=world)
    keys = O.run_shots(replica_worker.circuit(name), seed, 0, n_shots, want_outcomes=False)[0]
    want = O.counts(keys)
    for m in merged:  # every rank holds the merged histogram
        assert m == want
    assert sum(merged[0].values()) == n_shots


def test_gloo_merge_catches_a_missing_shot_offset(tmp_path):
    seed = 2024
    wrong = _run_ranks(tmp_path, "su4", 64, seed, mistake="nobase")
    keys = O.run_shots(replica_worker.circuit("su4"), seed, 0, 64, want_outcomes=False)[0]
    assert sum(wrong[0].values()) == 64
    assert wrong[0] != O.counts(keys)
