"""Host logic of the multi-GPU path for the batched configurations:
assignment of independent problems to ranks and the host-side gather, run
as two gloo ranks on the CPU (no GPU and no data-path collective)."""
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

import oracle
from paper_1305_5683_gb300 import shard
from spigen import generate_uneven, random_spd

HERE = os.path.dirname(os.path.abspath(__file__))


def test_assign_partitions_and_balances():
    rng = np.random.default_rng(0)
    costs = rng.lognormal(0.0, 1.5, 257)
    for world in (1, 2, 3, 8):
        parts = shard.assign(costs, world)
        allidx = np.sort(np.concatenate(parts))
        assert np.array_equal(allidx, np.arange(len(costs)))
        loads = np.array([costs[p].sum() for p in parts])
        # longest-processing-time bound: no rank exceeds the mean by more than the largest job
        assert loads.max() <= costs.sum() / world + costs.max() + 1e-9
    assert [list(p) for p in shard.assign([5.0, 1.0, 1.0, 3.0], 2)] == [[0], [1, 2, 3]]
    with pytest.raises(ValueError):
        shard.assign([1.0], 0)


def test_costs_come_from_the_host_analysis():
    small, large = random_spd(40, 0.1, 1), random_spd(400, 0.02, 2)
    c = shard.problem_costs([small, large])
    assert c.shape == (2,) and 0 < c[0] < c[1]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_gather_every_problem(tmp_path):
    out = str(tmp_path / "gathered.npz")
    env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()))
    procs = [subprocess.Popen([sys.executable, os.path.join(HERE, "gloo_shard_worker.py"), str(r), "2", out], env=env)
             for r in range(2)]
    try:
        rcs = [p.wait(timeout=300) for p in procs]
    finally:
        for p in procs:
            if p.poll() is None:
                p.kill()
    assert rcs == [0, 0]
    got = np.load(out)
    probs = generate_uneven(5)
    assert len(got.files) == len(probs)
    for i, p in enumerate(probs):
        ref = oracle.OracleFactor.from_problem(p).inv_diag()
        assert np.array_equal(got[f"arr_{i}"], ref)
