"""One rank of the two-rank sharding test (run as a subprocess by
tests/test_shard_gloo.py): takes its share of a list of independent SPI
problems, computes their variances with the oracle (the CPU stand-in for the
GPU solve of `paper_1305_5683_gb300.shard.solve_share`), and gathers every
rank's results with gloo."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def main():
    rank, world, out = int(sys.argv[1]), int(sys.argv[2]), sys.argv[3]
    import torch.distributed as dist
    import oracle
    from paper_1305_5683_gb300 import shard
    from spigen import generate_uneven
    dist.init_process_group("gloo", rank=rank, world_size=world)
    probs = generate_uneven(5)
    costs = np.array([p.n ** 2 for p in probs], dtype=float)  # any positive estimate
    parts = shard.assign(costs, world)
    mine = parts[rank]
    local = [oracle.OracleFactor.from_problem(probs[i]).inv_diag() for i in mine]
    allv = shard.gather(local, mine, len(probs))
    if rank == 0:
        np.savez(out, *allv)
    dist.barrier()
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
