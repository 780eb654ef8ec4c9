"""Several GPUs for the batched configurations: independent problems (or
energy bands) need no exchange, so each rank takes a share, runs it as one
block-diagonal forest on its own GPU, and the per-problem results are
gathered on the host.  There is no collective on the data path; the only
communication is the final host-side gather.

Shares are balanced by the analysis' work estimate (factor flops plus
variance flops, computed on the host without a device), assigned longest
first to the least-loaded rank.
"""
from __future__ import annotations

import numpy as np


def problem_costs(problems) -> np.ndarray:
    """Estimated device work of each problem (host-side analysis only)."""
    from .spi import Solver
    costs = []
    for p in problems:
        s = Solver.for_problem(p)
        info = s.info()
        s.close()
        costs.append(info["factor_flops"] + info["diag_flops_all"])
    return np.asarray(costs, dtype=np.float64)


def assign(costs, world: int) -> list[np.ndarray]:
    """Longest-processing-time-first assignment: problems in decreasing cost,
    each to the rank with the least cost so far (lowest rank on ties).
    Returns one ascending index array per rank; together they partition
    range(len(costs))."""
    if world < 1:
        raise ValueError("world must be >= 1")
    costs = np.asarray(costs, dtype=np.float64)
    order = np.argsort(-costs, kind="stable")
    load = np.zeros(world)
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        r = int(np.argmin(load))
        parts[r].append(int(i))
        load[r] += costs[i]
    return [np.array(sorted(p), dtype=np.int64) for p in parts]


def solve_share(problems, indices, **solver_options):
    """Factor, solve and compute all variances of problems[indices] on this
    rank's current CUDA device as one forest.  Returns (x list, variance list)
    in the order of `indices`, as host arrays."""
    from .spi import Solver
    share = [problems[i] for i in indices]
    if not share:
        return [], []
    s = Solver.for_problems(share, **solver_options)
    s.factor(np.concatenate([p.values for p in share]))
    x = s.solve(np.concatenate([p.b for p in share]))
    v = s.diag_inverse()
    offs = np.cumsum([0] + [p.n for p in share])
    s.close()
    return ([x[offs[k]:offs[k + 1]] for k in range(len(share))],
            [v[offs[k]:offs[k + 1]] for k in range(len(share))])


def gather(local_results, indices, total: int, group=None) -> list:
    """All ranks' per-problem results, in problem order, on every rank
    (torch.distributed object gather; any backend)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    objs = [None] * world
    dist.all_gather_object(objs, ([int(i) for i in indices], [np.asarray(a) for a in local_results]), group=group)
    out: list = [None] * total
    for idx, arrs in objs:
        for i, a in zip(idx, arrs):
            out[i] = a
    if any(a is None for a in out):
        raise RuntimeError("some problems were assigned to no rank")
    return out
