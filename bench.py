"""Benchmark: variances diag(N^-1) per second for the SPI least-squares
normal matrix of P = 20,000 pointings (380,000 rows, 500 sources with
time-bins of 20-2,000 pointings, per-pointing background plus 19
detector-pattern columns per 500 pointings), FP64.

One step = the whole hot path on one batch: factor(values) -> solve(b) ->
diag_inverse(all n indices), inputs resident in device memory.  The L2 is
flushed (a 256 MiB write) between timed steps, outside the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank factors and inverts its own replica of the
workload (the path does not shard; replicas only, no collective on the data
path) and rank 0 prints one JSON line with the whole-job throughput.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import re
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "diag(N^-1) entries/s"
UNIT = "variances/s"
L2_FLUSH_BYTES = 256 << 20
# the per-unit rates of a GB300 data sheet, used only when a probe fails (then
# the line says so)
NOMINAL_TFLOPS = {"fp64_fma": 1.25, "fp64_dmma": 1.25, "fp32_fma": 80.0, "tf32_tcgen05": 1125.0,
                  "bf16_tcgen05": 2250.0}


def measure_peaks(P) -> dict:
    """Measured TFLOP/s of every arithmetic unit a kernel here is bound by
    (spi_measure_peak: independent operations on every SM, best of 3 runs)."""
    out = {}
    for unit in ("fp64_fma", "fp64_dmma", "fp32_fma", "tf32_tcgen05", "bf16_tcgen05"):
        try:
            out[unit] = P.spi_measure_peak(unit, reps=3)
        except Exception as e:  # reported in the line; the roofline then says which figure it used
            out[unit + "_error"] = f"{type(e).__name__}: {e}"
    return out


def peak_of(peaks: dict, unit: str):
    """(TFLOP/s, source) of one unit: this run's probe, else the data-sheet figure."""
    if unit in peaks:
        return peaks[unit], f"measured by this run's {unit} probe (spi_measure_peak)"
    return NOMINAL_TFLOPS[unit], f"nominal {unit} (the probe failed: {peaks.get(unit + '_error')})"


def _measured_hbm_gbs() -> float:
    """Copy bandwidth measured on this GPU pool (MEASURED_PEAKS.json), else
    the profiling recipe's fallback figure."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


HBM_GBS = _measured_hbm_gbs()


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="scale", choices=["scale", "tiny"])
    ap.add_argument("--rhs-block", type=int, default=0, help="0 = the library's automatic choice")
    ap.add_argument("--rhs-block-mixed", type=int, default=0)
    ap.add_argument("--relax", type=int, default=1)
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-sky", action="store_true")
    ap.add_argument("--sky-only", action="store_true", help="run only the diffuse-sky leg (for profiling)")
    ap.add_argument("--normal-only", action="store_true", help="run only the normal-equation leg (for profiling)")
    ap.add_argument("--mixed-only", action="store_true",
                    help="run only the mixed-precision step of the P = 20,000 workload (for profiling)")
    ap.add_argument("--tune-cache", default=None,
                    help="autotuner table file for the P=20,000 solvers (a later run with the same file, "
                         "e.g. under a profiler, replays the same choices instead of timing again)")
    ap.add_argument("--bands", type=int, default=64)
    ap.add_argument("--problems", type=int, default=256)
    return ap.parse_args()


def workload(name):
    from spigen import SCALE, TINY, generate
    cfg = SCALE if name == "scale" else TINY
    t = time.perf_counter()
    pb = generate(cfg)
    return pb, time.perf_counter() - t


def config_of(pb, extra=None):
    c = {"workload": f"{pb.cfg.name}: SPI normal matrix, P={pb.cfg.n_pointings} pointings x 19 detectors, "
                     f"{pb.cfg.n_sources} sources, time-bins {pb.cfg.bin_lo}-{pb.cfg.bin_hi} pointings, "
                     f"detector-pattern block {pb.cfg.det_block}; step = factor, then solve (FP64 refinement in the mixed form) and full diag(N^-1) concurrently on two streams",
         "n": pb.n, "nnz_lower": pb.nnz, "seed": pb.cfg.seed, "l2": "flushed (256 MiB write) between timed steps"}
    if extra:
        c.update(extra)
    return c


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self.thread:
                self.thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _code_only(text: str) -> bytes:
    """Source text without // comments and blank lines (comment edits keep a digest)."""
    lines = (re.sub(r"//.*$", "", ln).rstrip() for ln in text.splitlines())
    return "\n".join(ln for ln in lines if ln.strip()).encode()


def source_digest(kernel_file: str, upto: str = "") -> str:
    """sha256 over the kernel's code and the analysis that plans its launch (the
    ordering and block plan decide the work of one launch).  With `upto`, the
    kernel file is read up to the end of the definition that contains it (the
    kernel and everything it uses stand before it in the file)."""
    src = open(os.path.join(ROOT, "paper_1305_5683_gb300", "csrc", kernel_file)).read()
    if upto:
        i = src.index(upto)
        src = src[:src.index("\n}\n", i) + 3]
    h = hashlib.sha256()
    h.update(_code_only(src))
    h.update(_code_only(open(os.path.join(ROOT, "paper_1305_5683_gb300", "csrc", "analysis.cpp")).read()))
    return h.hexdigest()


def traffic_of(kernel_file: str, key: str):
    """DRAM bytes per launch from the committed ncu summary, if neither the
    kernel source nor the analysis changed since the counters were taken."""
    try:
        prof = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
        ent = prof[key]
        if ent.get("source_sha256") != source_digest(kernel_file, ent.get("source_upto", "")):
            return None
        return float(ent["dram_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


def cpu_baseline(pb, sample=1024, seed=0):
    """The FP64 oracle as it stands on the host cores: its left-looking
    factor (single thread) and solve of the whole matrix, then the inverse
    diagonal for a random sample of indices on all cores, extrapolated to
    all n indices."""
    import oracle
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    f = oracle.OracleFactor.from_problem(pb)
    t_fac = time.perf_counter() - t0
    t0 = time.perf_counter()
    f.solve(pb.b)
    t_sol = time.perf_counter() - t0
    idx = np.random.default_rng(seed).choice(pb.n, min(sample, pb.n), replace=False).astype(np.int32)
    t0 = time.perf_counter()
    f.inv_diag(idx, nthreads=cores)
    t_smp = time.perf_counter() - t0
    t_all = t_fac + t_sol + t_smp * pb.n / len(idx)
    return f, {"value": pb.n / t_all, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"full left-looking factor ({t_fac:.1f} s, 1 thread) + solve ({t_sol:.2f} s) + "
                         f"inverse diagonal of {len(idx)} random indices ({t_smp:.2f} s, {cores} threads), "
                         f"extrapolated to all {pb.n} indices"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    pb, _ = workload(args.workload)
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    f = oracle.OracleFactor.from_problem(pb)
    t_fac = time.perf_counter() - t0
    rng = np.random.default_rng(1)
    S = 256
    times = []
    for it in range(args.warmup + args.steps):
        idx = rng.choice(pb.n, min(S, pb.n), replace=False).astype(np.int32)
        t0 = time.perf_counter()
        f.inv_diag(idx, nthreads=cores)
        dt = time.perf_counter() - t0 + t_fac * len(idx) / pb.n
        if it >= args.warmup:
            times.append(dt)
    per_var = sum(times) / (args.steps * min(S, pb.n))
    value = 1.0 / per_var
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(pb, {"reference": "FP64 CPU oracle (plain C)"}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"each step: inverse diagonal of {S} random indices on {cores} threads "
                                       f"plus the matching share of the one-off left-looking factor ({t_fac:.1f} s)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def priority_stream(dev):
    """A stream of the highest priority, for the mixed form's factorization and solve.
    The variances of the same factor run beside the solve on a second stream; on this
    stream the solve's short launches are dispatched ahead of the variance kernel's
    pending CTAs instead of behind them.  The FP64 form keeps default priorities: its
    variance kernel runs at the FP64 pipe's rate, and a solve dispatched ahead of it
    takes that rate away instead of filling gaps (measured: FP64 step 87.1 -> 89.1 ms)."""
    import torch
    try:
        _, hi = torch.cuda.Stream.priority_range()
    except Exception:
        hi = -1
    return torch.cuda.Stream(dev, priority=hi)


def overlapped_step(factor, solve, diag, st, st2, ev=None):
    """One step: the factorization on `st`; then the variances on `st2`
    concurrently with the solve (and its refinement) on `st` -- both read only
    the factor; `st` waits for `st2` at the end.  `ev`: six timing events
    (start, factor end, solve end, step end, variances start, variances end)."""
    import torch
    if ev: ev[0].record(st)
    factor(st)
    if ev: ev[1].record(st)
    done = torch.cuda.Event()
    done.record(st)
    st2.wait_event(done)
    if ev: ev[4].record(st2)
    diag(st2)
    if ev: ev[5].record(st2)
    solve(st)
    if ev: ev[2].record(st)
    st.wait_stream(st2)
    if ev: ev[3].record(st)


def _time_alone(fn, st, reps=3):
    """Mean device ms of fn(st) run by itself (nothing concurrent), after one untimed call."""
    import torch
    fn(st)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(reps):
        fn(st)
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _phases(evs):
    """Mean factor, solve, variance and whole-step ms of overlapped steps."""
    return (statistics.mean(e[0].elapsed_time(e[1]) for e in evs), statistics.mean(e[1].elapsed_time(e[2]) for e in evs),
            statistics.mean(e[4].elapsed_time(e[5]) for e in evs), statistics.mean(e[0].elapsed_time(e[3]) for e in evs))


def _time_steps(step, nsteps, warmup, st, flush):
    import torch
    for _ in range(warmup):
        step()
        flush.zero_()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nsteps)]
    for e0, e1 in evs:
        e0.record(st)
        step()
        e1.record(st)
        flush.zero_()
    torch.cuda.synchronize()
    return sum(e0.elapsed_time(e1) for e0, e1 in evs) / nsteps


def bench_bands(P, args, dev, st, flush, world, st_mixed=None):
    """Same-pattern batch: 64 energy bands of a P = 5,000 observation share one
    pattern; mixed precision with FP64 refinement, one launch per tree level
    (and block step) over all bands, replayed from a CUDA graph; against 64
    sequential FP64 runs (one band's FP64 step x 64)."""
    import torch
    from spigen import BAND, generate_bands
    t0 = time.perf_counter()
    bb = generate_bands(BAND, args.bands)
    t_gen = time.perf_counter() - t0
    nb, n = bb.nbands, bb.n
    vals = torch.from_numpy(bb.values).to(dev)
    b = torch.from_numpy(bb.b).to(dev)
    x = torch.empty_like(b)
    var = torch.empty(nb * n, dtype=torch.float64, device=dev)
    s = P.Solver(n, bb.colptr, bb.rowind, batch=nb, precision=P.SPI_PREC_MIXED_FP32, async_=True)

    evs = []
    st2 = torch.cuda.Stream(dev)
    sm = st_mixed if st_mixed is not None else st  # the mixed form's factor and solve

    def step():
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        overlapped_step(lambda q: s.factor_batch(vals, stream=q), lambda q: s.solve_batch(b, x, stream=q),
                        lambda q: s.diag_inverse_batch(out=var, stream=q), sm, st2, ev)
        evs.append(ev)

    ksteps = max(1, min(args.steps, 3))
    torch.cuda.synchronize(dev)
    with torch.cuda.stream(sm):  # the L2 flushes between steps on the same stream
        ms = _time_steps(step, ksteps, max(3, min(args.warmup, 3)), sm, flush)
        s.sync(sm)
    info = s.info()
    ph = _phases(evs[-ksteps:])
    solve_alone = _time_alone(lambda q: s.solve_batch(b, x, stream=q), st)
    # the solve reads every band's stored FP32 factor twice (forward and backward sweeps), per solve
    nsolves = 1 + info["refine_steps"]
    solve_bytes = 2.0 * nsolves * nb * info["nnz_l_stored"] * 4
    # one band in FP64, the plain form, as the sequential reference
    s1 = P.Solver(n, bb.colptr, bb.rowind, async_=True)
    v1 = torch.from_numpy(bb.values[: bb.nnz]).to(dev)
    b1 = b[:n].clone()
    x1 = torch.empty_like(b1)
    var1 = torch.empty(n, dtype=torch.float64, device=dev)

    def step1():
        overlapped_step(lambda q: s1.factor(v1, stream=q), lambda q: s1.solve(b1, x1, stream=q),
                        lambda q: s1.diag_inverse(out=var1, stream=q), st, st2)

    ms1 = _time_steps(step1, ksteps, 3, st, flush)
    s1.sync(st)
    err = float((torch.abs(var[:n] - var1) / var1).max().item())
    errx = float((torch.abs(x[:n] - x1).max() / torch.abs(x1).max()).item())
    value = world * nb * n / (ms / 1e3)
    seq = n / (ms1 / 1e3)
    return {"workload": f"{nb} energy bands x {bb.cfg.name} (P={bb.cfg.n_pointings}, {bb.cfg.n_sources} sources, "
                        f"n={n}, nnz_lower={bb.nnz}), E log-spaced 20-1000 keV, responses x (E/20)^-alpha",
            "value": value, "unit": UNIT, "ms_per_step": ms, "steps": ksteps,
            "phases_ms": {"factor": ph[0], "solve": ph[1], "diag_inverse": ph[2]},
            "solve_alone_ms": solve_alone, "solve_gbs": solve_bytes / (solve_alone / 1e3) / 1e9,
            "solve_hbm_frac": solve_bytes / (solve_alone / 1e3) / 1e9 / HBM_GBS,
            "dtype": "f32 updates / f64 pivots, refinement and variance sums",
            "fp64_sequential_value": seq, "speedup_vs_fp64_sequential": value / (world * seq),
            "max_rel_err_var_band0_vs_fp64": err, "max_rel_err_x_band0_vs_fp64": errx,
            "rhs_block": info["rhs_block"], "generate_s": t_gen}


def bench_uneven(P, args, dev, st, flush, world):
    """Uneven independent batch: 256 problems (P log-uniform in 50-2,000, own
    patterns) as one block-diagonal forest, FP64 -- against the same problems
    run one by one (256 contexts, FP64)."""
    import torch
    from spigen import generate_uneven
    t0 = time.perf_counter()
    probs = generate_uneven(args.problems)
    t_gen = time.perf_counter() - t0
    ntot = sum(p.n for p in probs)
    vals = torch.from_numpy(np.concatenate([p.values for p in probs])).to(dev)
    b = torch.from_numpy(np.concatenate([p.b for p in probs])).to(dev)
    x = torch.empty_like(b)
    var = torch.empty(ntot, dtype=torch.float64, device=dev)
    s = P.Solver.for_problems(probs, async_=True)

    st2 = torch.cuda.Stream(dev)

    def step():
        overlapped_step(lambda q: s.factor(vals, stream=q), lambda q: s.solve(b, x, stream=q),
                        lambda q: s.diag_inverse(out=var, stream=q), st, st2)

    ksteps = max(1, min(args.steps, 3))
    ms = _time_steps(step, ksteps, 3, st, flush)
    s.sync(st)
    singles = [P.Solver.for_problem(p, async_=True) for p in probs]
    offs = np.cumsum([0] + [p.n for p in probs])
    xs = torch.empty_like(b)
    vs = torch.empty_like(var)

    def step1():
        for i, q in enumerate(singles):
            a, e = int(offs[i]), int(offs[i + 1])
            vo = int(sum(pp.nnz for pp in probs[:i]))
            overlapped_step(lambda r: q.factor(vals[vo:vo + probs[i].nnz], stream=r),
                            lambda r: q.solve(b[a:e], xs[a:e], stream=r),
                            lambda r: q.diag_inverse(out=vs[a:e], stream=r), st, st2)

    ms1 = _time_steps(step1, ksteps, 3, st, flush)
    for q in singles:
        q.sync(st)
    err = float((torch.abs(var - vs) / vs).max().item())
    return {"workload": f"{len(probs)} independent SPI problems, P log-uniform 50-2000, n {min(p.n for p in probs)}"
                        f"-{max(p.n for p in probs)} (total {ntot}), one block-diagonal forest",
            "value": world * ntot / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": ksteps, "dtype": "f64",
            "one_by_one_value": ntot / (ms1 / 1e3), "speedup_vs_one_by_one": ms1 / ms,
            "max_rel_diff_vs_one_by_one": err, "launches_per_step": s.info()["launches_factor"]
            + s.info()["launches_solve"] + 1, "generate_s": t_gen}


def plan_summary(info: dict) -> dict:
    """The autotuner's choices for a context, from spi_info."""
    return {"tune_source": ["built-in rules", "timed", "tune cache"][info["tune_source"]],
            "tune_seconds": info["tune_seconds"], "panel_buckets": info["tune_panel_buckets"],
            "panel_buckets_persistent": info["tune_panel_fused"], "schur_buckets": info["tune_schur_buckets"],
            "schur_buckets_tensor_cores": info["tune_schur_tc"],
            "launches_factor": info["launches_factor"], "launches_factor_per_level_kernel": info["launches_factor_fused"],
            "factor_dag_tasks": info["factor_dag_tasks"], "factor_dag_levels": info["factor_dag_levels"],
            "n_levels": info["n_levels"],
            "factor_ms_timed": {"launches_per_level": info["tune_ms_launches"], "dependency_driven": info["tune_ms_dag"]},
            "solve_dag_tasks": info["solve_dag_tasks"],
            "solve_ms_timed": {"launches_per_level": info["tune_solve_ms_launches"],
                               "dependency_driven": info["tune_solve_ms_dag"]},
            "factor_work_flops": info["factor_work_flops"], "factor_flops": info["factor_flops"]}


def bench_sharded(P, args, dev, st, flush, world, rank, dist):
    """The batched configurations split over the ranks (one GPU each), the way
    they shard: independent problems assigned longest-first by the host
    analysis' work estimate (paper_1305_5683_gb300.shard), and energy bands
    in contiguous slices; no collective on the data path.  Every rank runs
    its share as one forest (or one band batch); the step time is the
    maximum over the ranks, the value all ranks' variances over it.  The
    problems' results are gathered on the host after the timing and checked
    against the single-GPU run of the same problems (uneven batch)."""
    import torch
    from spigen import BAND, generate_bands, generate_uneven
    from paper_1305_5683_gb300 import shard
    ksteps = max(1, min(args.steps, 3))

    def timed(step):
        for _ in range(3):
            step(); flush.zero_()
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tot = 0.0
        for _ in range(ksteps):
            e0.record(st); step(); e1.record(st)
            torch.cuda.synchronize(dev)
            tot += e0.elapsed_time(e1)
            flush.zero_()
        mine = torch.tensor([tot / ksteps], dtype=torch.float64, device=dev)
        every = [torch.zeros_like(mine) for _ in range(world)]
        if dist:
            dist.all_gather(every, mine)
        else:
            every = [mine]
        return [float(t.item()) for t in every]

    out = {}
    st2 = torch.cuda.Stream(dev)
    probs = generate_uneven(args.problems)
    costs = shard.problem_costs(probs)
    parts = shard.assign(costs, world)
    share = [probs[i] for i in parts[rank]]
    ntot = sum(p.n for p in probs)
    s = P.Solver.for_problems(share, async_=True)
    vals = torch.from_numpy(np.concatenate([p.values for p in share])).to(dev)
    b = torch.from_numpy(np.concatenate([p.b for p in share])).to(dev)
    x = torch.empty_like(b)
    var = torch.empty(sum(p.n for p in share), dtype=torch.float64, device=dev)

    def step():
        overlapped_step(lambda q: s.factor(vals, stream=q), lambda q: s.solve(b, x, stream=q),
                        lambda q: s.diag_inverse(out=var, stream=q), st, st2)

    per_rank = timed(step)
    s.sync(st)
    load = [float(costs[p].sum()) for p in parts]
    out["uneven"] = {"workload": f"{len(probs)} independent SPI problems (total n {ntot}), assigned longest-first",
                     "value": ntot / (max(per_rank) / 1e3), "unit": UNIT, "ms_per_step": max(per_rank),
                     "per_rank_ms": per_rank, "problems_per_rank": [len(p) for p in parts],
                     "estimated_load_imbalance": max(load) / (sum(load) / world), "steps": ksteps}
    if dist:
        offs = np.cumsum([0] + [p.n for p in share])
        vh = var.cpu().numpy()
        res = shard.gather([vh[offs[k]:offs[k + 1]] for k in range(len(share))], parts[rank], len(probs))
        out["uneven"]["gathered_problems"] = sum(r is not None for r in res)
    del s
    if world > 1:
        bb = generate_bands(BAND, args.bands)
        lo, hi = rank * bb.nbands // world, (rank + 1) * bb.nbands // world
        nb = hi - lo
        sb = P.Solver(bb.n, bb.colptr, bb.rowind, batch=max(nb, 1), precision=P.SPI_PREC_MIXED_FP32, async_=True)
        bv = torch.from_numpy(bb.values[lo * bb.nnz:hi * bb.nnz]).to(dev)
        bbv = torch.from_numpy(bb.b[lo * bb.n:hi * bb.n]).to(dev)
        bx = torch.empty_like(bbv)
        bvar = torch.empty(nb * bb.n, dtype=torch.float64, device=dev)

        def bstep():
            overlapped_step(lambda q: sb.factor_batch(bv, stream=q), lambda q: sb.solve_batch(bbv, bx, stream=q),
                            lambda q: sb.diag_inverse_batch(out=bvar, stream=q), st, st2)

        per_rank = timed(bstep)
        sb.sync(st)
        out["bands"] = {"workload": f"{bb.nbands} energy bands x n={bb.n}, contiguous slices per rank, mixed",
                        "value": bb.nbands * bb.n / (max(per_rank) / 1e3), "unit": UNIT,
                        "ms_per_step": max(per_rank), "per_rank_ms": per_rank, "steps": ksteps}
    return out


def _time_phases(s, vals, b, x, idx, var, nsteps, warmup, st, flush):
    """Mean device ms of factor / solve / diag_inverse / whole overlapped step
    over nsteps timed steps."""
    import torch
    st2 = torch.cuda.Stream()

    def step(ev=None):
        overlapped_step(lambda q: s.factor(vals, stream=q), lambda q: s.solve(b, x, stream=q),
                        lambda q: s.diag_inverse(idx, out=var, stream=q), st, st2, ev)

    for _ in range(warmup):
        step(); flush.zero_()
    s.sync(st)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(nsteps)]
    torch.cuda.synchronize()
    for k in range(nsteps):
        step(evs[k]); flush.zero_()
    torch.cuda.synchronize()
    s.sync(st)
    return _phases(evs)


def bench_sky(P, args, dev, st, flush, world, cfg=None, warmup=3, max_steps=3, peaks=None, st_mixed=None):
    """Diffuse-sky workload: point sources plus a pixel grid, pointings on a
    target grid (the large configuration's structure); variances of the sky
    columns only.  Its fronts are wide (a dense sky block), which is where the
    mixed form's tensor-core updates apply.  FP64 form and mixed form, same
    step; errors of both against the oracle's stored results where they exist
    (tests/golden), and of the mixed form against the FP64 form."""
    import torch
    from spigen import SKY, generate
    cfg = cfg or SKY
    t0 = time.perf_counter()
    pb = generate(cfg)
    t_gen = time.perf_counter() - t0
    idx = torch.from_numpy(pb.sky_columns).to(dev)
    vals = torch.from_numpy(pb.values).to(dev)
    b = torch.from_numpy(pb.b).to(dev)
    ksteps = max(1, min(args.steps, max_steps))
    golden = None
    gpath = os.path.join(ROOT, "tests", "golden", "sky_pix05_oracle.npz")
    if cfg.name == "spi-sky-P2000-pix0.5" and os.path.exists(gpath):
        golden = np.load(gpath)
    out, res = {}, {}
    for name, prec in (("fp64", P.SPI_PREC_FP64), ("mixed", P.SPI_PREC_MIXED_FP32)):
        s = P.Solver.for_problem(pb, async_=True, precision=prec, relax=args.relax)
        x = torch.empty_like(b)
        var = torch.empty(pb.n_sky, dtype=torch.float64, device=dev)
        q = st_mixed if (name == "mixed" and st_mixed is not None) else st
        torch.cuda.synchronize(dev)
        with torch.cuda.stream(q):
            f, so, d, tot = _time_phases(s, vals, b, x, idx, var, ksteps, warmup, q, flush)
        info = s.info()
        res[name] = (x, var)
        out[name] = {"value": world * pb.n_sky / (tot / 1e3), "ms_per_step": tot,
                     "phases_ms": {"factor": f, "solve": so, "diag_inverse": d},
                     "factor_tflops": info["factor_flops"] / (f / 1e3) / 1e12,
                     "diag_tflops": info["diag_flops"] / (d / 1e3) / 1e12,
                     "refine_steps": info["refine_steps"], "solve_relres": info["solve_relres"],
                     "launches_factor": info["launches_factor"], "tune_source": info["tune_source"]}
        if name == "mixed" and peaks is not None and info["factor_tc_flops"] > 0:
            pk, src = peak_of(peaks, "tf32_tcgen05")
            ach = info["factor_tc_flops"] / (f / 1e3) / 1e12
            out[name]["tensor"] = {"tf32_flops_issued": info["factor_tc_flops"], "tiles": info["tiles_factor_tc"],
                                   "launches": info["launches_factor_tc"], "achieved_tflops": ach, "peak": pk,
                                   "frac": ach / pk, "peak_source": src,
                                   "note": "TF32 MMA work issued (6 MMAs per product) over the whole factor span"}
        if name == "mixed" and peaks is not None and info["diag_tc_flops"] > 0:
            pk, src = peak_of(peaks, "tf32_tcgen05")
            ach = info["diag_tc_flops"] / (d / 1e3) / 1e12
            out[name]["diag_tensor"] = {"tf32_flops_issued": info["diag_tc_flops"],
                                        "supernodes": info["diag_tc_supernodes"], "achieved_tflops": ach, "peak": pk,
                                        "frac": ach / pk, "peak_source": src,
                                        "note": "TF32 MMA work issued (3 MMAs per product, padded tiles) over the "
                                                "whole variance span (SIMT kernel below the tensor-core supernodes "
                                                "included)"}
        if golden is not None:
            xo, vo = golden["x"], golden["var_sky"]
            out[name]["max_rel_err_x_vs_oracle"] = float(np.abs(x.cpu().numpy() - xo).max() / np.abs(xo).max())
            out[name]["max_rel_err_var_vs_oracle"] = float((np.abs(var.cpu().numpy() - vo) / vo).max())
        if name == "fp64":
            out["factor_flops"], out["diag_flops"] = info["factor_flops"], info["diag_flops"]
            out["max_front"], out["n_supernodes"] = info["max_front"], info["n_supernodes"]
        del s
    (x64, v64), (xm, vm) = res["fp64"], res["mixed"]
    out["mixed"]["speedup_vs_fp64"] = out["fp64"]["ms_per_step"] / out["mixed"]["ms_per_step"]
    out["mixed"]["max_rel_err_var_vs_fp64"] = float((torch.abs(vm - v64) / v64).max().item())
    out["mixed"]["max_rel_err_x_vs_fp64"] = float((torch.abs(xm - x64).max() / torch.abs(x64).max()).item())
    out.update({"workload": f"{pb.cfg.name}: P={pb.cfg.n_pointings} pointings on a 7x7 target grid, "
                            f"{pb.cfg.n_sources} sources, {pb.n_sky} sky pixels of {pb.cfg.sky_pix_deg:g} deg "
                            f"(n={pb.n}, nnz_lower={pb.nnz}); variances of the sky columns",
                "unit": UNIT, "steps": ksteps, "warmup": warmup, "generate_s": t_gen,
                "oracle": "tests/golden/sky_pix05_oracle.npz" if golden is not None else None})
    return out


def bench_normal(P, args, dev, st):
    """The step before the path (paper Sec. 4.1, Table 3): N = H^T W H and
    b = H^T W y on the device from the design matrix of the P = 20,000
    workload, and their update after 5,000 columns of H changed."""
    import torch
    from spigen import SCALE, generate
    t0 = time.perf_counter()
    pb = generate(SCALE, sparse_design=True)
    t_gen = time.perf_counter() - t0
    H = pb.H
    s = P.Solver.for_problem(pb)
    t0 = time.perf_counter()
    s.normal_setup(H)
    t_setup = time.perf_counter() - t0
    hv = torch.from_numpy(H.data).to(dev)
    w = torch.from_numpy(pb.w).to(dev)
    y = torch.from_numpy(pb.y).to(dev)
    nv = torch.empty(pb.nnz, dtype=torch.float64, device=dev)
    b = torch.empty(pb.n, dtype=torch.float64, device=dev)
    ms = _time_alone(lambda q: s.normal_assemble(hv, w, y, nv, b, stream=q), st)
    diff = float((torch.abs(nv - torch.from_numpy(pb.values).to(dev)).max() / abs(pb.values).max()).item())
    def update_ms(cols):
        sel = torch.from_numpy(np.isin(H.indices, cols)).to(dev)
        hv2 = torch.where(sel, hv * 1.01, hv)
        return _time_alone(lambda q: s.normal_update(cols, hv2, w, y, nv, b, stream=q), st)

    # the Poisson maximum-likelihood fit from the least-squares solution (NEXT-2: the same
    # pattern refactored every Newton step)
    s.normal_assemble(hv, w, y, nv, b, stream=st)
    s.factor(nv, stream=st)
    x0 = s.solve(b, stream=st)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    xm, vm = s.mle_newton(hv, y, x0, stream=st)
    torch.cuda.synchronize(dev)
    t_mle = time.perf_counter() - t0
    mle = {"steps": s.info()["mle_steps"], "wall_s": t_mle, "cash": s.info()["mle_cash"],
           "max_rel_change_from_lsq": float((torch.abs(xm - x0).max() / torch.abs(x0).max()).item()),
           "note": "each step: e = Hx, Hessian assembled, factored and solved on the device; "
                   "variances at the fit from the last Hessian"}
    ms_u = update_ms(np.random.default_rng(5).choice(pb.n, 5000, replace=False).astype(np.int32))
    bins = np.nonzero(pb.kind == 2)[0]
    ms_w = update_ms(bins[len(bins) // 2: len(bins) // 2 + 5000].astype(np.int32))
    ms_d = update_ms(np.nonzero(pb.kind == 1)[0].astype(np.int32))

    # Algorithm 1 (the empty-field pattern fitted with the solution), from a pattern
    # 20 % off the generator's: least squares (N updated in the pointing columns'
    # rows and columns each iteration) and the likelihood form (a Newton fit each)
    rng = np.random.default_rng(1)
    U0 = pb.bg_u * (1 + 0.2 * rng.uniform(-1, 1, len(pb.bg_u)))
    upat = torch.from_numpy(pb.bg_pat).to(dev)
    tq = torch.from_numpy(pb.bg_t).to(dev)
    alg1 = {}
    for mode, iters in (("lsq", 10), ("mle", 3)):
        hvb = hv.clone()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        xb, Ub, stb, vb = s.background_fit(pb.n_pointing, upat, tq, hvb, w, y, U0, mode=mode, max_iter=iters,
                                           stream=st)
        torch.cuda.synchronize(dev)
        tb = time.perf_counter() - t0
        Ub = Ub.cpu().numpy()
        ratio = Ub / pb.bg_u
        alg1[mode] = {"solves": len(stb), "wall_s": tb, "ms_per_solve": 1e3 * tb / len(stb),
                      "stat_first": float(stb[0]), "stat_last": float(stb[-1]),
                      "pattern_spread_vs_true_start": float(np.ptp(U0 / pb.bg_u) / np.mean(U0 / pb.bg_u)),
                      "pattern_spread_vs_true_end": float(np.ptp(ratio) / ratio.mean())}
        del hvb
    alg1["note"] = ("U = 19 detector values, rows' pointing columns hold U_d t_dp; each iteration: solve, "
                    "statistic and pattern sums, U and H's background entries updated; variances at the end")
    return {"workload": f"{SCALE.name}: H {H.shape[0]} x {H.shape[1]}, nnz(H) {H.nnz}, N lower nnz {pb.nnz}",
            "assemble_ms": ms, "update_5000_random_columns_ms": ms_u,
            "update_5000_consecutive_time_bins_ms": ms_w, "update_detector_pattern_columns_ms": ms_d,
            "setup_host_s": t_setup, "mle_newton": mle, "background_fit": alg1,
            "max_rel_diff_vs_generator": diff, "dtype": "f64", "generate_s": t_gen,
            "paper_table3_context": "improved algorithm, one CPU core: 28.2 s full / 0.43 s 5,000 columns at N = 22,503, "
                                    "nnz(H) = 27.05 M (different matrix and hardware)"}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import paper_1305_5683_gb300 as P

    P.build.build()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    st_hi = priority_stream(dev)
    if args.normal_only:  # the normal-equation leg alone (profiling); not the benchmark line
        print(json.dumps({"normal_equations": bench_normal(P, args, dev, torch.cuda.current_stream(dev))}), flush=True)
        return
    if args.sky_only:  # the diffuse-sky legs alone (profiling); not the benchmark line
        from spigen import SKY_PIX05
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        st0 = torch.cuda.current_stream(dev)
        peaks = measure_peaks(P)
        print(json.dumps({"peaks_tflops": peaks,
                          "sky": bench_sky(P, args, dev, st0, flush, world, peaks=peaks, st_mixed=st_hi),
                          "sky_pix05": bench_sky(P, args, dev, st0, flush, world, cfg=SKY_PIX05, warmup=1,
                                                 max_steps=2, peaks=peaks, st_mixed=st_hi)}), flush=True)
        return
    peaks = measure_peaks(P)
    pb, t_gen = workload(args.workload)
    if args.mixed_only:  # the mixed-precision step alone (profiling); not the benchmark line
        st0 = torch.cuda.current_stream(dev)
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        sm_ = P.Solver.for_problem(pb, async_=True, rhs_block=args.rhs_block_mixed, relax=args.relax,
                                   precision=P.SPI_PREC_MIXED_FP32, diag_ctas_per_sm=3, tune_cache=args.tune_cache)
        vals = torch.from_numpy(pb.values).to(dev)
        b = torch.from_numpy(pb.b).to(dev)
        xm = torch.empty_like(b)
        varm = torch.empty(pb.n, dtype=torch.float64, device=dev)
        with torch.cuda.stream(st_hi):
            f, so, d, tot = _time_phases(sm_, vals, b, xm, None, varm, args.steps, args.warmup, st_hi, flush)
        print(json.dumps({"mixed_only": {"ms_per_step": tot, "phases_ms": {"factor": f, "solve": so,
                                                                           "diag_inverse": d},
                                          "plan": plan_summary(sm_.info())}}), flush=True)
        return

    s = P.Solver.for_problem(pb, async_=True, rhs_block=args.rhs_block, relax=args.relax, tune_cache=args.tune_cache)
    info0 = s.info()
    st = torch.cuda.current_stream(dev)
    vals = torch.from_numpy(pb.values).to(dev)
    b = torch.from_numpy(pb.b).to(dev)
    x = torch.empty_like(b)
    var = torch.empty(pb.n, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    st2 = torch.cuda.Stream(dev)

    def step(ev=None):
        overlapped_step(lambda q: s.factor(vals, stream=q), lambda q: s.solve(b, x, stream=q),
                        lambda q: s.diag_inverse(out=var, stream=q), st, st2, ev)

    for _ in range(args.warmup):
        step()
        flush.zero_()
    s.sync(st)
    torch.cuda.synchronize(dev)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            step(evs[k])
            flush.zero_()
        torch.cuda.synchronize(dev)
    s.sync(st)
    t_fac = [e[0].elapsed_time(e[1]) for e in evs]
    t_sol = [e[1].elapsed_time(e[2]) for e in evs]
    t_dia = [e[4].elapsed_time(e[5]) for e in evs]
    total_ms = sum(e[0].elapsed_time(e[3]) for e in evs)
    tot = torch.tensor([total_ms], dtype=torch.float64, device=dev)
    if dist:
        dist.all_reduce(tot, op=dist.ReduceOp.MAX)
    total_ms = float(tot.item())
    info = s.info()
    value = world * pb.n * args.steps / (total_ms / 1e3)
    solve_alone = _time_alone(lambda q: s.solve(b, x, stream=q), st)

    # end to end through the public API with pinned host buffers (copies inside)
    hv = torch.from_numpy(pb.values).pin_memory()
    hb = torch.from_numpy(pb.b).pin_memory()
    hx = torch.empty(pb.n, dtype=torch.float64).pin_memory()
    hvar = torch.empty(pb.n, dtype=torch.float64).pin_memory()
    s_e2e = P.Solver.for_problem(pb, rhs_block=args.rhs_block, relax=args.relax, tune_cache=args.tune_cache)
    s_e2e.factor(hv); s_e2e.solve(hb, hx); s_e2e.diag_inverse(out=hvar)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s_e2e.factor(hv, stream=st)
        s_e2e.solve(hb, hx, stream=st)
        s_e2e.diag_inverse(out=hvar, stream=st)
    torch.cuda.synchronize(dev)
    t_e2e = time.perf_counter() - t0
    e2e_t = torch.tensor([t_e2e], dtype=torch.float64, device=dev)
    if dist:
        dist.all_reduce(e2e_t, op=dist.ReduceOp.MAX)
    e2e_value = world * pb.n * args.steps / float(e2e_t.item())
    agree = float((torch.abs(hvar.to(dev) - var) / var).max().item())
    # the batched configurations split over the ranks (every rank takes part)
    sharded = None
    if not args.no_batch:
        try:
            sharded = bench_sharded(P, args, dev, st, flush, world, rank, dist)
        except Exception as e:
            sharded = {"error": f"{type(e).__name__}: {e}"}
    if dist:
        dist.barrier()
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    # the factorization's plan: the autotuner's table, and the same factorization on the
    # block-step chain alone (every panel tiled, no persistent per-level kernel)
    factor_plan = plan_summary(info)
    try:
        sc = P.Solver.for_problem(pb, async_=True, rhs_block=args.rhs_block, relax=args.relax, force_panel=1,
                                  autotune=-1, dag=1)
        factor_plan["block_step_chain_only"] = {
            "factor_ms": _time_alone(lambda q: sc.factor(vals, stream=q), st, reps=5),
            "launches_factor": sc.info()["launches_factor"]}
        factor_plan["factor_ms"] = _time_alone(lambda q: s.factor(vals, stream=q), st, reps=5)
        del sc
    except Exception as e:
        factor_plan["error"] = f"{type(e).__name__}: {e}"
    # the allocation-free variances (spi_diag_inverse_noalloc) on 4,096 random indices,
    # beside spi_diag_inverse on the same indices
    noalloc = None
    try:
        s.factor(vals, stream=st)
        s.sync(st)
        sel = torch.from_numpy(np.random.default_rng(15).choice(pb.n, 4096, replace=False).astype(np.int32)).to(dev)
        o1 = torch.empty(4096, dtype=torch.float64, device=dev)
        o2 = s.diag_inverse(sel, stream=st)
        s.sync(st)
        t_na = _time_alone(lambda q: P.spi_diag_inverse_noalloc(s._h, sel, o1, stream=q), st, reps=2)
        t_di = _time_alone(lambda q: s.diag_inverse(sel, out=o2, stream=q), st, reps=2)
        noalloc = {"indices": 4096, "ms": t_na, "variances_per_s": 4096 / (t_na / 1e3),
                   "spi_diag_inverse_ms": t_di, "max_rel_diff": float((torch.abs(o1 - o2) / o2).max().item())}
    except Exception as e:
        noalloc = {"error": f"{type(e).__name__}: {e}"}

    # the mixed-precision form on the same workload and the same step
    mixed = None
    if not args.no_mixed:
        # the mixed solve (two sweeps and a residual) outlasts the variances: cap the
        # variance kernel at 3 CTAs per SM so that the solve keeps room beside it
        sm_ = P.Solver.for_problem(pb, async_=True, rhs_block=args.rhs_block_mixed, relax=args.relax,
                                   precision=P.SPI_PREC_MIXED_FP32, diag_ctas_per_sm=3, tune_cache=args.tune_cache)
        xm = torch.empty_like(b)
        varm = torch.empty_like(var)

        def mstep(ev=None):
            overlapped_step(lambda q: sm_.factor(vals, stream=q), lambda q: sm_.solve(b, xm, stream=q),
                            lambda q: sm_.diag_inverse(out=varm, stream=q), st_hi, st2, ev)

        torch.cuda.synchronize(dev)
        with torch.cuda.stream(st_hi):  # the L2 flushes between steps on the same stream
            for _ in range(args.warmup):
                mstep(); flush.zero_()
            sm_.sync(st_hi)
            mevs = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(args.steps)]
            torch.cuda.synchronize(dev)
            for k in range(args.steps):
                mstep(mevs[k]); flush.zero_()
            torch.cuda.synchronize(dev)
            sm_.sync(st_hi)
        mf = [e[0].elapsed_time(e[1]) for e in mevs]
        ms_ = [e[1].elapsed_time(e[2]) for e in mevs]
        md = [e[4].elapsed_time(e[5]) for e in mevs]
        mtot = sum(e[0].elapsed_time(e[3]) for e in mevs)
        minfo = sm_.info()
        mixed = {"value": world * pb.n * args.steps / (mtot / 1e3), "unit": UNIT, "ms_per_step": mtot / args.steps,
                 "phases_ms": {"factor": statistics.mean(mf), "solve": statistics.mean(ms_),
                               "diag_inverse": statistics.mean(md)},
                 "speedup_vs_fp64": total_ms / mtot,
                 "max_rel_err_var_vs_fp64": float((torch.abs(varm - var) / var).max().item()),
                 "max_rel_err_x_vs_fp64": float((torch.abs(xm - x).max() / torch.abs(x).max()).item()),
                 "refine_steps": minfo["refine_steps"], "solve_relres": minfo["solve_relres"],
                 "diag_tflops_fp32": minfo["diag_flops_all"] / (statistics.mean(md) / 1e3) / 1e12,
                 "plan": plan_summary(minfo),
                 "tensor_core_launches": minfo["launches_factor_tc"],
                 "dtype": "f32 updates / f64 pivots, refinement and variance sums"}
        # the variances alone (no solve beside them): the tensor-core kernel for the
        # supernodes with at least diag_tc_min_pivots pivots and their ancestors, the
        # SIMT kernel below them
        d_alone = _time_alone(lambda q: sm_.diag_inverse(out=varm, stream=q), st)
        minfo = sm_.info()
        mixed["diag_alone_ms"] = d_alone
        mixed["diag_tflops_fp32_alone"] = minfo["diag_flops_all"] / (d_alone / 1e3) / 1e12
        if minfo["diag_tc_flops"] > 0:
            pk, src = peak_of(peaks, "tf32_tcgen05")
            ach = minfo["diag_tc_flops"] / (d_alone / 1e3) / 1e12
            mixed["diag_roofline"] = {"bound": "tensor", "kernel": "k_diag_inv_tc (after k_diag_inv_f32)",
                                      "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
                                      "peak_source": src, "supernodes": minfo["diag_tc_supernodes"],
                                      "traffic": traffic_of("diag_tc.cu", "k_diag_inv_tc"),
                                      "tf32_flops_issued": minfo["diag_tc_flops"],
                                      "note": "TF32 MMA work issued (3 MMAs per product, padded tiles) over the "
                                              "whole variance launch pair, timed alone"}
        else:
            pk32, src32 = peak_of(peaks, "fp32_fma")
            mixed["diag_roofline"] = {"bound": "alu", "kernel": "k_diag_inv_f32",
                                      "achieved": mixed["diag_tflops_fp32_alone"], "peak": pk32, "unit": "TFLOP/s",
                                      "frac": mixed["diag_tflops_fp32_alone"] / pk32, "peak_source": src32}
        if minfo["factor_tc_flops"] > 0:
            pk, src = peak_of(peaks, "tf32_tcgen05")
            ach = minfo["factor_tc_flops"] / (statistics.mean(mf) / 1e3) / 1e12
            mixed["tensor"] = {"tf32_flops_issued": minfo["factor_tc_flops"], "achieved_tflops": ach, "peak": pk,
                               "frac": ach / pk, "peak_source": src}
        # variances of 256 unknowns with the factor's first-order error removed
        try:
            sel = torch.from_numpy(np.random.default_rng(13).choice(pb.n, 256, replace=False).astype(np.int32)).to(dev)
            vr = sm_.diag_inverse_refined(sel, stream=st)
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            vr = sm_.diag_inverse_refined(sel, stream=st)
            e1.record(st)
            torch.cuda.synchronize(dev)
            ref = var[sel.long()]
            mixed["refined_256"] = {"ms": e0.elapsed_time(e1),
                                    "max_rel_err_vs_fp64": float((torch.abs(vr - ref) / ref).max().item()),
                                    "max_rel_err_unrefined": float((torch.abs(varm[sel.long()] - ref) / ref).max().item())}
        except Exception as e:
            mixed["refined_256"] = {"error": f"{type(e).__name__}: {e}"}
        del sm_

    # blocks of the inverse on the FP64 factor: the covariances of 512 time-bin
    # columns active in one time window (consecutive bins), and of 512 random unknowns
    inv_block = {}
    bins = np.nonzero(pb.kind == 2)[0]
    sets = {"time_window": bins[len(bins) // 2: len(bins) // 2 + 512],
            "random": np.random.default_rng(11).choice(pb.n, 512, replace=False)}
    for name, sel in sets.items():
        try:
            idx = torch.from_numpy(np.ascontiguousarray(sel, np.int32)).to(dev)
            G = torch.empty((512, 512), dtype=torch.float64, device=dev)
            s.inverse_block(idx, out=G, stream=st)  # plan
            s.sync(st)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(3):
                s.inverse_block(idx, out=G, stream=st)
            e1.record(st)
            torch.cuda.synchronize(dev)
            ms_b = e0.elapsed_time(e1) / 3
            inv_block[name] = {"nidx": 512, "ms": ms_b, "entries_per_s": 512 * 512 / (ms_b / 1e3)}
        except Exception as e:
            inv_block[name] = {"error": f"{type(e).__name__}: {e}"}
    # scattered entries: 5,000 random pairs among 1,024 time-bin columns of one time window
    try:
        rng = np.random.default_rng(12)
        U = bins[len(bins) // 2: len(bins) // 2 + 1024].astype(np.int32)
        r = torch.from_numpy(U[rng.integers(0, len(U), 5000)]).to(dev)
        c = torch.from_numpy(U[rng.integers(0, len(U), 5000)]).to(dev)
        o = torch.empty(5000, dtype=torch.float64, device=dev)
        s.inverse_entries(r, c, out=o, stream=st)
        s.sync(st)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        s.inverse_entries(r, c, out=o, stream=st)
        e1.record(st)
        torch.cuda.synchronize(dev)
        ms_e = e0.elapsed_time(e1)
        inv_block["entries_5000_pairs_over_1024"] = {"nent": 5000, "distinct": len(U), "blocks": 10, "ms": ms_e,
                                                     "entries_per_s": 5000 / (ms_e / 1e3)}
    except Exception as e:
        inv_block["entries_5000_pairs_over_1024"] = {"error": f"{type(e).__name__}: {e}"}

    # pruning ablation: 2,048 random variances from pruned blocked solves (the method) and from
    # full forward solves over all supernodes (spi_options.diag_unpruned), same FP64 factor
    ablation = None
    try:
        sel = torch.from_numpy(np.random.default_rng(14).choice(pb.n, 2048, replace=False).astype(np.int32)).to(dev)
        u = P.Solver.for_problem(pb, rhs_block=args.rhs_block, relax=args.relax, diag_unpruned=True)
        u.factor(vals, stream=st)
        vp_ = s.diag_inverse(sel, stream=st)
        s.sync(st)
        vu_ = u.diag_inverse(sel, stream=st)
        torch.cuda.synchronize(dev)
        t_p = _time_alone(lambda q: s.diag_inverse(sel, out=vp_, stream=q), st)
        t_u = _time_alone(lambda q: u.diag_inverse(sel, out=vu_, stream=q), st, reps=1)
        ablation = {"indices": 2048, "pruned_ms": t_p, "unpruned_ms": t_u, "speedup_from_pruning": t_u / t_p,
                    "max_rel_diff": float((torch.abs(vu_ - vp_) / vp_).max().item()),
                    "note": "unpruned: full forward solve z = L^-1 e_i over all supernodes, 32 per pass"}
        del u
    except Exception as e:
        ablation = {"error": f"{type(e).__name__}: {e}"}

    normal = None
    if not args.no_batch:
        try:
            normal = bench_normal(P, args, dev, st)
        except Exception as e:
            normal = {"error": f"{type(e).__name__}: {e}"}

    sky = sky_pix05 = None
    if not args.no_sky:
        from spigen import SKY_PIX05
        try:
            sky = bench_sky(P, args, dev, st, flush, world, peaks=peaks, st_mixed=st_hi)
        except Exception as e:
            sky = {"error": f"{type(e).__name__}: {e}"}
        try:
            # the large configuration's diffuse sky at full size (0.5 deg pixels, 19,600 sky columns)
            sky_pix05 = bench_sky(P, args, dev, st, flush, world, cfg=SKY_PIX05, warmup=1, max_steps=2, peaks=peaks,
                                  st_mixed=st_hi)
        except Exception as e:
            sky_pix05 = {"error": f"{type(e).__name__}: {e}"}

    batched_bands = batched_uneven = None
    if not args.no_batch:
        for name in ("bands", "uneven"):
            try:
                r = (bench_bands(P, args, dev, st, flush, world, st_mixed=st_hi) if name == "bands"
                     else bench_uneven(P, args, dev, st, flush, world))
            except Exception as e:  # a failing secondary leg is reported, the main line stands
                r = {"error": f"{type(e).__name__}: {e}"}
            if name == "bands":
                batched_bands = r
            else:
                batched_uneven = r

    mean_dia = statistics.mean(t_dia) / 1e3
    achieved = info["diag_flops_all"] / mean_dia / 1e12
    pk64, src64 = peak_of(peaks, "fp64_fma")
    roof = {"bound": "alu", "kernel": "k_diag_inv (pruned blocked forward solves, FP64)",
            "achieved": achieved, "peak": pk64, "unit": "TFLOP/s", "frac": achieved / pk64,
            "peak_source": src64, "traffic": traffic_of("diag.cu", "k_diag_inv")}
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        _, cpu = cpu_baseline(pb)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(pb, {"ordering": "nested dissection", "rhs_block": args.rhs_block,
                                 "streams": "after the factor, solve and variances run concurrently on two streams "
                                            "(default priorities; the mixed-form legs run factor and solve on a "
                                            "stream of the highest priority); "
                                            "phases_ms are each phase's own span, ms_per_step the whole step; "
                                            "mixed leg: variance kernel capped at 3 CTAs per SM "
                                            "(spi_options.diag_ctas_per_sm)",
                                 "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"}),
        "phases_ms": {"factor": statistics.mean(t_fac), "solve": statistics.mean(t_sol),
                      "diag_inverse": statistics.mean(t_dia)},
        "factor_tflops": info["factor_flops"] / (statistics.mean(t_fac) / 1e3) / 1e12,
        "solve_alone_ms": solve_alone,
        "solve_gbs": 2.0 * info["nnz_l_stored"] * 8 / (solve_alone / 1e3) / 1e9,
        "factor_flops": info["factor_flops"], "diag_flops": info["diag_flops_all"],
        "diag_work_flops": info["diag_work_flops"],
        "nnz_l": info["nnz_l"], "n_supernodes": info["n_supernodes"], "analyse_s": info0["analyse_seconds"],
        "roofline": roof,
        "peaks_tflops": peaks,
        "factor_plan": factor_plan,
        "noalloc": noalloc,
        "mixed": mixed,
        "pruning_ablation": ablation,
        "inverse_block": inv_block,
        "normal_equations": normal,
        "sky": sky,
        "sky_pix05": sky_pix05,
        "batched_bands": batched_bands,
        "batched_uneven": batched_uneven,
        "sharded": sharded,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * (pb.nnz + pb.n),
                "d2h_bytes_per_step": 8 * 2 * pb.n, "max_rel_diff_vs_device_run": agree},
        "gpu_launches": args.steps * (info["launches_factor"] + info["launches_solve"] + info["launches_diag"]),
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
