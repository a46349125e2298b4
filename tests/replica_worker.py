"""One rank of the shot-distribution test: runs its shot range through the
oracle and writes the merged histogram (launched with RANK / WORLD_SIZE /
MASTER_ADDR / MASTER_PORT set, as torchrun would)."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import torch.distributed as dist  # noqa: E402

from oracle import oracle as O  # noqa: E402
from paper_2308_03399_gb300 import replicas  # noqa: E402
from paper_2308_03399_gb300 import workloads as W  # noqa: E402


def circuit(name):
    if name == "mid":
        return W.midcircuit_measure(5, 2, 0.02, [1, 3], seed=11, name="mid5")
    return W.random_su4(4, 3, 0.01, 0.01, seed=12, name="su4_4")


def main():
    out, name, n_shots, seed, mistake = sys.argv[1], sys.argv[2], int(sys.argv[3]), int(sys.argv[4]), sys.argv[5]
    dist.init_process_group("gloo")
    circ = circuit(name)

    def runner(c, s, base, count):
        # mistake "nobase": every rank starts at global shot 0 (planted on the CPU)
        b = 0 if mistake == "nobase" else base
        return O.run_shots(c, s, b, count, threads=1, want_outcomes=False)[0]

    merged = replicas.distributed_counts(circ, n_shots, seed, runner=runner)
    with open(f"{out}.{dist.get_rank()}", "w") as f:
        json.dump({str(k): v for k, v in merged.items()}, f)
    dist.barrier()
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
