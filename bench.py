#!/usr/bin/env python
"""Throughput of the TENO-D gas-kinetic scheme on one GB300 (or N replicas).

Workload: 2-D Riemann problem, configuration 3 (paper Sec. 5.6 (a)) on a
1024 x 1024 grid with the split at (0.8, 0.8), zero-gradient boundaries,
CFL 0.5, Euler collision time.  A step is one full S2O4 step (both stages,
both directions) of the whole grid with the CFL time step computed on the
device.  Metric: cell-updates per second (cells x steps / time).

Primary value: float32 reconstruction + flux with float64 state and S2O4
accumulation; the float64 path is timed on the same GPU and reported under
"fp64".  Timing: W warm-up steps, then K steps, each bracketed by CUDA
events on the library's stream with a 256 MB L2 flush between steps (outside
the events).  The sweep kernels are also timed individually by the
library's event profiler for the roofline.

Further legs on the same GPU, reported as objects of the same JSON line:
"ensemble" (4096 independent 1-D Riemann problems of 200..4000 cells to
t = 0.15 in one persistent launch, cell-updates/s), "weno_ao" (the main
workload with the WENO5-AO reconstruction), "conventional_2d" (the same with
the WENO5-Z and TENO5 GKS of Sec. 3.1, 4.1), "recon_1d" (Sod's tube on 2^22
cells with the TENO-D, WENO5-Z and TENO5 face reconstructions), "viscous" (Navier-Stokes
viscous shock tube on 2048 x 1024, 200 steps from t = 0), "errors_vs_oracle"
(both GPU paths against the FP64 oracle on the CPU baseline's sample) and
"adjoint" (the
hand-written adjoint on a 512 x 512 isentropic vortex, 700 steps to t = 2,
checkpoint every 20 steps: backward ms per step, float32 and float64),
"developed" / "value_developed" (the main workload timed again from
t = 0.4, where the quadrant waves have developed), "charvars" (the main
workload with TENO-D in characteristic variables, Sec. 3.1),
"paper_workloads" (the double Mach reflection at 960 x 240 to t = 0.2, the
Titarev-Toro wave at 1000 cells to t = 5 and the Riemann configuration 6 at
400^2 to t = 0.6, whole runs in both precisions), "flips" (TENO-D
selections the float32 path makes otherwise than the float64 path, per step
of both timed windows), "oracle_by_config" (the oracle's throughput on
bounded samples of the other configurations, one copy per host core) and
"errors_vs_oracle" per configuration.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_GRID = 1024
METRIC = "TENO-D GKS cell-updates/s (2-D Riemann configuration 3, 1024^2)"
UNIT = "cell-updates/s"
# GB300: 152 SMs x 128 FP32 lanes, 2 flops per fused multiply-add
SMS, FP32_LANES = 152, 128


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--fp64-steps", type=int, default=10)
    p.add_argument("--cpu-sample", type=int, default=96, help="grid of the oracle's bounded sample")
    p.add_argument("--skip-cpu", action="store_true", help="omit the CPU-oracle baseline (profiling runs)")
    p.add_argument("--no-ensemble", dest="ensemble", action="store_false",
                   help="omit the batched 1-D ensemble leg")
    p.add_argument("--no-adjoint", dest="adjoint", action="store_false",
                   help="omit the adjoint leg")
    p.add_argument("--adjoint-steps", type=int, default=700,
                   help="steps of the adjoint leg (700 = t = 2; fewer for profiling runs)")
    p.add_argument("--no-adjoint-fp64", dest="adjoint_fp64", action="store_false",
                   help="omit the float64 run of the adjoint leg")
    p.add_argument("--ensemble-max-steps", type=int, default=0,
                   help="cap the ensemble leg at this many steps per problem (profiling runs)")
    p.add_argument("--ensemble-launch", default="",
                   help="THREADS,BLOCKS_PER_SM for the ensemble leg instead of the autotuner")
    p.add_argument("--no-viscous", dest="viscous", action="store_false",
                   help="omit the viscous shock tube leg")
    p.add_argument("--no-weno-ao", dest="weno_ao", action="store_false",
                   help="omit the WENO5-AO and conventional (WENO5-Z, TENO5) 2-D legs")
    p.add_argument("--no-recon-1d", dest="recon_1d", action="store_false",
                   help="omit the 1-D leg that times TENO-D, WENO5-Z and TENO5 face reconstructions")
    p.add_argument("--no-paper", dest="paper", action="store_false",
                   help="omit the paper-size workload legs (double Mach reflection, Titarev-Toro, config 6)")
    p.add_argument("--no-charvars", dest="charvars", action="store_false",
                   help="omit the characteristic-variable TENO-D leg")
    p.add_argument("--no-developed", dest="developed", action="store_false",
                   help="omit the developed-flow timing window (t = 0.4)")
    p.add_argument("--cpu-budget", type=float, default=4.0,
                   help="seconds of oracle time per configuration on all host cores")
    return p.parse_args()


def rank_info():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        self.proc.wait()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for k, name in enumerate(names):
                if f[5 + k].lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "samples": len(sm), "reasons": sorted(reasons)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def sweep_traffic_from_profiles():
    """DRAM bytes per sweep launch from the committed ncu summary, if any."""
    path = os.path.join(ROOT, "profiles", "sweep_fp32_riemann1024.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    return float(m.group(1)) if m else None


def sweep_pipe_from_profiles(name="sweep_fp32_riemann1024.md", pipe="FMA"):
    """Pipe activity of a sweep kernel (ncu sm__pipe_*_cycles_active, launch
    1, fraction) from the committed ncu summary, if any: the FP32 (FMA) or
    FP64 pipe throughput against its peak, beside the flop-based fraction."""
    path = os.path.join(ROOT, "profiles", name)
    try:
        text = open(path).read()
    except OSError:
        return None
    m = re.search(r"^\| %s pipe %% \| ([0-9.]+)" % pipe, text, re.M)
    return float(m.group(1)) / 100.0 if m else None


def host_info():
    """Host cores available to this process and the CPU model."""
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        import platform
        model = platform.processor() or platform.machine()
    return cores, model


def _oracle_on_threads(make, advance, budget_s, threads):
    """The oracle as it stands on `threads` host threads: every thread steps
    its own copy of a sample (make(k) -> state; advance(state) -> (state,
    cell-updates)) until budget_s has passed (the oracle's C calls release
    the interpreter lock, so the threads run in parallel).  Returns
    (cell-updates/s over all threads, cell-updates, seconds)."""
    from concurrent.futures import ThreadPoolExecutor

    def work(k):
        st = make(k)
        cu = 0.0
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < budget_s:
            st, c = advance(st)
            cu += c
        return cu

    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        cus = list(ex.map(work, range(threads)))
    el = time.perf_counter() - t0
    return sum(cus) / el, sum(cus), el


def cpu_baseline(steps_budget_s=10.0, n=96, budget_all=4.0):
    """The oracle as it stands, on the host cores, on a bounded sample: the
    same problem on an n x n grid, CFL steps, single thread for
    ~steps_budget_s (its state is the errors' sample), then one copy per
    host core for ~budget_all.  The headline value is the all-core one."""
    import oracle as O
    from paper_2309_10534_gb300 import workloads as WL

    s = WL.riemann2d(n, split=0.8)
    P = O.make_problem(2, n, n, **s.problem_kwargs())
    W = s.W
    t0 = time.perf_counter()
    steps = 0
    while True:
        W = O.step(P, W, O.dt(P, W))
        steps += 1
        if time.perf_counter() - t0 > steps_budget_s:
            break
    el = time.perf_counter() - t0
    single = n * n * steps / el
    cores, model = host_info()

    def adv(st):
        return O.step(P, st, O.dt(P, st)), n * n

    allv, cu, el_all = _oracle_on_threads(lambda k: s.W.copy(), adv, budget_all, cores)
    return ({"value": allv, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": model,
             "sample": "%dx%d grid of the same problem, CFL steps from t = 0, one copy per host core for %.0f s "
                       "(%.3g cell-updates)" % (n, n, el_all, cu),
             "single_thread": {"value": single, "cores": 1,
                               "sample": "%dx%d grid, %d CFL steps, one thread" % (n, n, steps)}},
            (s, W, steps))


def oracle_by_config(budget_s, cores):
    """The oracle's throughput on bounded samples of the other workloads, one
    copy per host core (cell-updates/s; one cell-update = one cell advanced
    by one S2O4 step)."""
    import numpy as np
    import oracle as O
    from paper_2309_10534_gb300 import workloads as WL
    out = {}

    def restartable(s, P, t_end):
        def make(k):
            return [s.W.copy(), 0.0]

        def adv(st):
            W, t = st
            if t >= t_end:
                W, t = s.W.copy(), 0.0
            dt = min(O.dt(P, W), t_end - t)
            return [O.step(P, W, dt), t + dt], s.nx * s.ny
        return make, adv

    s = WL.sod(400)
    P = O.make_problem(1, 400, **s.problem_kwargs())
    v, cu, el = _oracle_on_threads(*restartable(s, P, 0.2), budget_s, cores)
    out["1_sod400"] = {"value": v, "unit": UNIT, "cores": cores, "sample": "Sod 400 cells, CFL steps to t = 0.2 "
                       "(restarted), one run per core"}
    s = WL.viscous_shock_tube(64, 32)
    P = O.make_problem(2, 64, 32, **s.problem_kwargs())
    v, cu, el = _oracle_on_threads(*restartable(s, P, 1.0), budget_s, cores)
    out["3_viscous"] = {"value": v, "unit": UNIT, "cores": cores,
                        "sample": "viscous shock tube (Re 200, Pr 0.73, walls) on 64 x 32, CFL steps from t = 0"}
    E = WL.ensemble_1d()
    order = np.argsort(E.ncells, kind="stable")

    def make_e(k):
        return [k, None, 0.0, None]

    def adv_e(st):
        k, W, t, P = st
        if W is None or t >= E.t_end:
            k = (k + cores) % E.ncells.size if W is not None else k
            idx = int(order[k % E.ncells.size])
            n = int(E.ncells[idx])
            W = E.W[:, E.offsets[idx]:E.offsets[idx] + n][:, None, :].copy()
            P = O.make_problem(1, n, tau="euler")
            t = 0.0
        dt = min(O.dt(P, W), E.t_end - t)
        n = W.shape[-1]
        try:
            W = O.step(P, W, dt)
        except RuntimeError:  # a member whose state turns non-physical: next problem
            return [k, None, E.t_end, P], n
        return [k, W, t + dt, P], n
    v, cu, el = _oracle_on_threads(make_e, adv_e, budget_s, cores)
    out["4_ensemble"] = {"value": v, "unit": UNIT, "cores": cores,
                         "sample": "members of the seeded 4096-problem ensemble, smallest first, one per core at a "
                                   "time, to t = 0.15"}
    s = WL.isentropic_vortex(n=32, seed=2309, amplitude=1e-3)
    P = O.make_problem(2, 32, 32, lx=10.0, ly=10.0, bc=("periodic",) * 4, tau="zero")
    dtv = 2.0 / 700 * 16

    def adv_v(st):
        return O.step(P, st, dtv), 32 * 32
    v, cu, el = _oracle_on_threads(lambda k: s.W.copy(), adv_v, budget_s, cores)
    out["5_adjoint_forward"] = {"value": v, "unit": UNIT, "cores": cores,
                                "sample": "forward S2O4 steps of the isentropic vortex (tau = 0) on 32 x 32; the "
                                          "oracle has no adjoint (its reference gradient is central differences: "
                                          "two forward runs per direction)"}
    return out


def _errs(got, ref):
    import numpy as np
    e = np.abs(got - ref)
    return {"l1_rel": float(e.sum() / np.abs(ref).sum()), "linf_rel": float(e.max() / np.abs(ref).max())}


def oracle_errors(gks, sample):
    """Stated errors of both GPU paths against the FP64 oracle, per
    configuration, on samples the oracle finishes in seconds: relative L1
    (sum |e| / sum |W|) and relative Linf (max |e| / max |W|) over all
    conserved variables.  For the float32 path the oracle's own spread under
    float32-level perturbations (1e-7 of the state before every step) is
    given beside it (1e-7 of the initial state, or of the state before every
    step, the larger): TENO-D's cut-offs make shock runs depend
    discontinuously on rounding (see "flips")."""
    import numpy as np
    import oracle as O
    from paper_2309_10534_gb300 import workloads as WL
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from oracle_envelope import fp32_envelope, fp64_envelope
    out = {}
    # config 2: the CPU baseline's own sample
    s, W_or, steps = sample
    e = {"sample": "%dx%d riemann2d_config3, %d CFL steps" % (s.nx, s.ny, steps)}
    for precision in ("fp64", "fp32"):
        S = gks.solver_for(s, precision)
        for _ in range(steps):
            S.step(0.0)
        e[precision] = _errs(S.get_state(), W_or)
        S.close()
    out["2_riemann2d"] = e
    # config 1: Sod, 400 cells, the whole run
    s = WL.sod(400)
    P = O.make_problem(1, 400, **s.problem_kwargs())
    Wo, spread = fp32_envelope(P, s.W, 0.2, seeds=(0, 1))
    e = {"sample": "Sod 400 cells to t = 0.2 (the whole run)", "fp32_oracle_spread_l1_rel": spread}
    for precision in ("fp64", "fp32"):
        S = gks.solver_for(s, precision)
        S.advance_to(0.2)
        e[precision] = _errs(S.get_state(), Wo)
        S.close()
    out["1_sod400"] = e
    # config 3: the viscous shock tube on a reduced grid
    s = WL.viscous_shock_tube(64, 32)
    P = O.make_problem(2, 64, 32, **s.problem_kwargs())
    Wo, spread = fp32_envelope(P, s.W, 1.0, seeds=(0, 1), max_steps=10)
    e = {"sample": "viscous shock tube (Re 200, Pr 0.73) on 64 x 32, 10 CFL steps",
         "fp32_oracle_spread_l1_rel": spread}
    for precision in ("fp64", "fp32"):
        S = gks.solver_for(s, precision)
        S.advance_to(1.0, max_steps=10)
        e[precision] = _errs(S.get_state(), Wo)
        S.close()
    out["3_viscous"] = e
    # config 4: the 16 smallest members of the seeded ensemble to t = 0.15
    from concurrent.futures import ThreadPoolExecutor
    E = WL.ensemble_1d()
    pick = [int(k) for k in np.argsort(E.ncells, kind="stable")[:16]]

    def one(k):
        n = int(E.ncells[k])
        P = O.make_problem(1, n, tau="euler")
        W0 = E.W[:, E.offsets[k]:E.offsets[k] + n][:, None, :]
        try:
            ref = O.run(P, W0, E.t_end)[0][:, 0, :]
            s64 = fp64_envelope(P, W0, E.t_end, seeds=(0,))[1]
            s32 = fp32_envelope(P, W0, E.t_end, seeds=(0,))[1]
            return ref, s64, s32
        except RuntimeError:
            return None
    with ThreadPoolExecutor(max_workers=16) as ex:
        res = list(ex.map(one, pick))
    refs = [r[0] if r else None for r in res]
    spreads = {"fp64": [r[1] if r else None for r in res], "fp32": [r[2] if r else None for r in res]}
    sizes = E.ncells[pick]
    Wsub = np.concatenate([E.W[:, E.offsets[k]:E.offsets[k] + E.ncells[k]] for k in pick], axis=1)
    off = np.concatenate([[0], np.cumsum(sizes)])
    e = {"sample": "the 16 smallest members of the seeded ensemble (%d..%d cells) to t = 0.15; errors over the "
                   "members the oracle completes; each member's error is also divided by the oracle's own spread "
                   "at that path's rounding level (relative perturbations of the initial state, or of every "
                   "step's state, the larger spread: 1e-15 for float64, 1e-7 for float32)" % (sizes.min(), sizes.max())}
    for precision in ("fp64", "fp32"):
        B = gks.Batch(sizes, np.ones(len(pick)), precision=precision)
        B.set_state(Wsub)
        B.advance_to(E.t_end, allow_failed=True)
        got = B.get_state()
        _, _, err, _ = B.progress()
        B.close()
        l1, linf, ratio, used = [], [], [], 0
        for j, ref in enumerate(refs):
            if ref is None or err[j]:
                continue
            r = _errs(got[:, off[j]:off[j + 1]], ref)
            l1.append(r["l1_rel"])
            linf.append(r["linf_rel"])
            ratio.append(r["l1_rel"] / max(spreads[precision][j], 1e-300))
            used += 1
        e[precision] = {"l1_rel_max": max(l1), "l1_rel_mean": float(np.mean(l1)), "linf_rel_max": max(linf),
                        "members": used, "max_ratio_to_oracle_spread": max(ratio)}
    out["4_ensemble"] = e
    # config 5: the adjoint's forward map (isentropic vortex, tau = 0) on 32 x 32
    s = WL.isentropic_vortex(n=32, seed=2309, amplitude=1e-3)
    P = O.make_problem(2, 32, 32, lx=10.0, ly=10.0, bc=("periodic",) * 4, tau="zero")
    dtv = 2.0 / 700 * 16
    Wo = s.W.copy()
    for _ in range(20):
        Wo = O.step(P, Wo, dtv)
    e = {"sample": "isentropic vortex (tau = 0, smooth: no selection switches) on 32 x 32, 20 steps"}
    for precision in ("fp64", "fp32"):
        S = gks.Solver(2, 32, 32, lx=10.0, ly=10.0, bc=("periodic",) * 4, precision=precision, tau="zero")
        S.set_state(s.W)
        for _ in range(20):
            S.step(dtv)
        e[precision] = _errs(S.get_state(), Wo)
        S.close()
    out["5_adjoint_forward"] = e
    return out


def run_reference(args):
    rank, _, world = rank_info()
    if rank != 0:
        return
    import oracle as O
    from paper_2309_10534_gb300 import workloads as WL

    n = 64
    s = WL.riemann2d(n, split=0.8)
    P = O.make_problem(2, n, n, **s.problem_kwargs())
    W = s.W
    for _ in range(args.warmup):
        W = O.step(P, W, O.dt(P, W))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        W = O.step(P, W, O.dt(P, W))
    el = time.perf_counter() - t0
    value = n * n * args.steps / el
    sample = "%dx%d grid of the same problem per step (bounded sample), single thread" % (n, n)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "riemann2d_config3", "grid": "%dx%d" % (N_GRID, N_GRID), "cfl": 0.5, "split": 0.8,
                       "precision": "fp64 (the oracle)", "parallelism": "1 host thread",
                       "sample": "each step a %dx%d grid of the same problem (bounded sample; the metric is "
                                 "per cell-update)" % (n, n)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def ensemble_leg(gks, WL, stream, peak32, max_steps=0, launch=None, rank=0, world=1, dist=None):
    """4096 independent 1-D Riemann problems (200..4000 cells, seeded) to
    t = 0.15 in one persistent launch, float32 flux / float64 state, launch
    shape from the autotuner.  One untimed run captures the graph; the timed
    run replays it from the same initial state.  Cell-updates = sum over
    problems of cells x steps taken (a problem flagged non-physical stops
    early and counts only its own steps).  With N ranks the problems are
    split longest-first over the ranks (no collective on the data path);
    value = all ranks' cell-updates / the slowest rank's time."""
    import numpy as np
    import torch
    E = WL.ensemble_1d()
    shard = gks.partition_lpt(E.ncells.astype(np.float64) ** 2, world)[rank]
    ncells = E.ncells[shard]
    W = np.concatenate([E.W[:, E.offsets[k]:E.offsets[k] + E.ncells[k]] for k in shard], axis=1)
    E = WL.Ensemble(ncells, np.concatenate([[0], np.cumsum(ncells)[:-1]]), W, E.left[shard], E.right[shard],
                    E.gamma, E.t_end)
    B = gks.Batch(E.ncells, np.ones(E.ncells.size), precision="fp32")
    B.set_stream(stream.cuda_stream)
    B.set_state(E.W)
    if launch:
        th, bp = launch
        B.set_launch(th, bp)
    else:
        th, bp, _ = B.tune(0.005, use_cache=False)
    B.advance_to(E.t_end, max_steps=max_steps, allow_failed=True)
    B.set_state(E.W)
    L0 = B.launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    nbad = B.advance_to(E.t_end, max_steps=max_steps, allow_failed=True)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    t, steps, err, _ = B.progress()
    cu = float((E.ncells.astype(np.float64) * steps).sum())
    done = (err == 0)
    cu_done = float((E.ncells.astype(np.float64) * steps)[done].sum())
    dev = stream.device if dist is not None and dist.get_backend() == "nccl" else None
    ms = gks.reduce_scalars([ms], "max", dist, dev)[0]
    cu, nbad, cu_done = gks.reduce_scalars([cu, nbad, cu_done], "sum", dist, dev)
    fpc = gks.count_flops(1, "fp32", "euler", 1.0)["flops_per_cell_update"]
    tf = fpc * cu / (ms * 1e-3) / 1e12
    launches = B.launches() - L0   # graph replays, one kernel each
    B.close()
    return {"value": cu / (ms * 1e-3), "unit": UNIT, "workload": "ensemble_1d_riemann",
            "problems_per_rank": int(E.ncells.size), "cells_per_rank": int(E.ncells.sum()), "t_end": E.t_end,
            "scaling": "strong", "n_gpus": world,
            "ms": ms, "cell_updates": cu, "max_steps_per_problem": int(steps.max()),
            "flagged_nonphysical": int(nbad),
            "completed_set": {"value": cu_done / (ms * 1e-3), "unit": UNIT, "cell_updates": cu_done,
                              "problems": int(E.ncells.size - nbad),
                              "note": "cell-updates of the problems that reached t_end only, over the same time"},
            "launch": {"threads": th, "blocks_per_sm": bp},
            "gpu_launches": launches,
            "precision": "fp32 reconstruction+flux, fp64 state and S2O4 accumulation",
            "flops_per_cell_update": fpc,
            "roofline": {"bound": "alu", "kernel": "k_batch<float>", "achieved": tf, "peak": peak32,
                         "unit": "TFLOP/s", "frac": tf / peak32,
                         "basis": "whole launch vs measured FP32 FMA peak"}}


def weno_ao_leg(gks, WL, stream, peak32, steps, warmup, recon="weno_ao"):
    """The same 1024^2 Riemann workload with another reconstruction: WENO5-AO
    (Sec. 3.2, the scheme the paper compares against), or the conventional
    WENO5-Z / TENO5 GKS (Sec. 3.1, 4.1); float32 flux, CUDA events around
    each step, 256 MB L2 flush between steps, sweep kernels timed by the
    library's event profiler for the roofline."""
    import torch
    s = WL.riemann2d(N_GRID, split=0.8, t_end=0.8)
    S = gks.solver_for(s, "fp32", recon=recon)
    S.set_stream(stream.cuda_stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=stream.device)
    for _ in range(warmup):
        S.step(0.0)
    ms, sn, sms = timed_and_profiled(S, stream, flush, steps)
    S.diagnostics()
    S.close()
    cells = N_GRID * N_GRID
    fm = gks.count_flops(2, "fp32", "euler", 1.0, recon=recon)
    launch_ms = sms / max(sn, 1)
    tf = fm["flops_per_cell_sweep"] * cells / (launch_ms * 1e-3) / 1e12
    return {"value": cells * steps / (ms * 1e-3), "unit": UNIT, "workload": "riemann2d_config3_" + recon,
            "grid": "%dx%d" % (N_GRID, N_GRID), "steps": steps, "ms_per_step": ms / steps,
            "flops_per_cell_update": fm["flops_per_cell_update"],
            "roofline": {"bound": "alu", "kernel": "k2d_sweep<float, %s>" % recon, "achieved": tf, "peak": peak32,
                         "unit": "TFLOP/s", "frac": tf / peak32, "launch_ms": launch_ms}}


N_1D = 1 << 22


def recon_1d_leg(gks, WL, stream, peak32, steps, warmup):
    """The 1-D path with each face reconstruction: TENO-D (the paper's
    scheme) and the conventional WENO5-Z and TENO5 GKS (Sec. 3.1, 4.1; face
    values, slopes by Eq. 3.11, equilibrium slope by Eq. 3.12).  Workload:
    Sod's tube on 2^22 cells (Euler tau), float32 flux, CFL steps, CUDA
    events around each step, 256 MB L2 flush between steps; the stage
    kernels timed by the library's event profiler for the roofline."""
    import torch
    s = WL.sod(N_1D)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=stream.device)
    out = {}
    for recon in ("teno_d", "weno_z", "teno5"):
        S = gks.solver_for(s, "fp32", recon=recon)
        S.set_stream(stream.cuda_stream)
        for _ in range(warmup):
            S.step(0.0)
        ms, sn, sms = timed_and_profiled(S, stream, flush, steps)
        S.diagnostics()
        S.close()
        fm = gks.count_flops(1, "fp32", "euler", 1.0, recon=recon)
        launch_ms = sms / max(sn, 1)
        tf = fm["flops_per_cell_sweep"] * N_1D / (launch_ms * 1e-3) / 1e12
        out[recon] = {"value": N_1D * steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps,
                      "flops_per_cell_update": fm["flops_per_cell_update"],
                      "roofline": {"bound": "alu", "kernel": "k1d_stage<float, %s>" % recon, "achieved": tf,
                                   "peak": peak32, "unit": "TFLOP/s", "frac": tf / peak32, "launch_ms": launch_ms}}
    return {"workload": "sod_1d", "cells": N_1D, "steps": steps, "precision": "fp32", "by_recon": out}


def viscous_leg(gks, WL, stream, precision, steps):
    """Navier-Stokes viscous shock tube (Re = 200, Pr = 0.73, no-slip walls,
    symmetric top) on 2048 x 1024: `steps` CFL steps from t = 0 (the full run
    to t = 1 takes ~1e5 viscous-limited steps), CUDA events around each step,
    256 MB L2 flush between steps."""
    import torch
    s = WL.viscous_shock_tube(2048, 1024, Re=200.0, Pr=0.73)
    S = gks.solver_for(s, precision)
    S.set_stream(stream.cuda_stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=stream.device)
    for _ in range(2):
        S.step(0.0)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    for k in range(steps):
        flush.zero_()
        ev[k][0].record(stream)
        S.step(0.0)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    S.diagnostics()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    cells = 2048 * 1024
    S.close()
    return {"value": cells * steps / (ms * 1e-3), "unit": UNIT, "workload": "viscous_shock_tube",
            "grid": "2048x1024", "steps": steps, "ms_per_step": ms / steps, "tau": "ns", "Re": 200.0,
            "Pr": 0.73, "precision": precision}


def adjoint_leg(gks, WL, stream, precision, steps=700):
    """Hand-written adjoint on the isentropic vortex (strength 5, periodic
    [0, 10]^2, 512 x 512, smooth seeded density perturbation of RMS 1e-3):
    J = integral of rho^2 at t = 2 in 700 fixed steps (CFL 0.5), checkpoint
    every 20 steps.  Forward (with checkpoints) and backward (segment
    recomputation + adjoint steps) timed with CUDA events on the solver's
    stream; ms per step of each."""
    import numpy as np
    import torch
    n, k = 512, 20
    dt = 2.0 / 700
    s = WL.isentropic_vortex(n=n, seed=2309, amplitude=1e-3)
    S = gks.Solver(2, n, n, lx=10.0, ly=10.0, bc=("periodic",) * 4, precision=precision, tau="zero")
    S.set_stream(stream.cuda_stream)
    A = gks.Adjoint(S, k)
    dev = stream.device
    W0 = torch.from_numpy(s.W).to(dev)
    # warm-up: every buffer of the timed passes, and one full checkpoint
    # segment forward and backward, so that the backward pass's segment graph
    # is captured and instantiated before the timed region (a one-time host
    # cost of ~800 captured launches)
    # (the objective's seed below is formed with the same torch operations,
    # so that their first-use loading stays outside the timed region)
    A.reserve(steps)
    S.set_state(W0)
    A.forward(k, dt)
    WN = torch.empty_like(W0)

    def seed():
        S.get_state(WN)
        gWN = torch.zeros_like(W0)
        gWN[0] = 2.0 * WN[0] * (s.dx * s.dy)
        return gWN

    A.backward(seed())
    S.set_state(W0)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    L0, A0 = S.kernel_launches(), A.launches()
    torch.cuda.synchronize()
    ev[0].record(stream)
    A.forward(steps, dt)
    ev[1].record(stream)
    gWN = seed()
    ev[2].record(stream)
    gW0 = A.backward(gWN)
    ev[3].record(stream)
    torch.cuda.synchronize()
    fwd, bwd = ev[0].elapsed_time(ev[1]), ev[2].elapsed_time(ev[3])
    launches = (S.kernel_launches() - L0) + (A.launches() - A0)
    drho = torch.from_numpy(s.extra["delta_rho"]).to(dev)
    u, v = W0[1] / W0[0], W0[2] / W0[0]
    g = gW0[0] + u * gW0[1] + v * gW0[2] + 0.5 * (u * u + v * v) * gW0[3]
    dJ = float((g * drho).sum())
    A.close()
    S.close()
    return {"value": bwd / steps, "unit": "ms/step", "workload": "isentropic_vortex_adjoint",
            "grid": "%dx%d" % (n, n), "steps": steps, "dt": dt, "checkpoint_every": k,
            "forward_ms_per_step": fwd / steps, "backward_ms": bwd, "forward_ms": fwd,
            "gpu_launches": launches, "dJ_deps": dJ,
            "precision": ("fp32 reconstruction+flux, fp64 state and cotangents" if precision == "fp32"
                          else "fp64")}


def flips_leg(gks, WL, s, steps, warmup, t_dev=None):
    """TENO-D selection flips between the precisions (gks_selection_flips) on
    the input state of every step of the timed window (steps warmup+1 ..
    warmup+steps from t = 0), and of as many steps from t_dev: per step the
    selections the float32 path would make otherwise than the float64 path
    on the same float64 state (normal and tangential, both directions).  The
    states are those of the float32-flux run (its state is float64)."""
    S = gks.solver_for(s, "fp32")

    def window(k):
        nf = tf = ns = ts = uf = 0
        for _ in range(k):
            f = S.selection_flips()
            nf += f["normal_flips"]
            tf += f["tangential_flips"]
            ns += f["normal_selections"]
            ts += f["tangential_selections"]
            uf += f["unresolved_flips"]
            S.step(0.0)
        return {"normal_per_step": nf / k, "tangential_per_step": tf / k,
                "fraction_of_selections": (nf + tf) / max(ns + ts, 1),
                "selections_per_step": (ns + ts) / k,
                "unresolved_per_step": uf / k}
    for _ in range(warmup):
        S.step(0.0)
    out = {"timed_window": window(steps)}
    if t_dev:
        S.advance_to(t_dev)
        out["developed_window"] = window(steps)
        out["developed_window"]["t_start"] = t_dev
    S.close()
    return out


def timed_steps(S, stream, flush, K):
    """K steps, each bracketed by CUDA events on the solver's stream, with
    an L2 flush before each (outside the events); ms in total."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    torch.cuda.synchronize()
    for k in range(K):
        flush.zero_()
        ev[k][0].record(stream)
        S.step(0.0)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev)


def timed_and_profiled(S, stream, flush, K):
    """(ms of K uninstrumented steps, sweep launches and sweep ms of K more
    steps with the library's per-kernel events on)."""
    ms = timed_steps(S, stream, flush, K)
    S.profile(True)
    S.profile_read(0)
    timed_steps(S, stream, flush, K)
    sn, sms = S.profile_read(0)
    S.profile(False)
    return ms, sn, sms


def charvars_leg(gks, WL, stream, peak32, steps, warmup):
    """The main workload with TENO-D in characteristic variables (Sec. 3.1),
    float32 flux: cell-updates/s and the sweep's flop rate."""
    import torch
    s = WL.riemann2d(N_GRID, split=0.8, t_end=0.8)
    S = gks.solver_for(s, "fp32", charvars=1)
    S.set_stream(stream.cuda_stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=stream.device)
    for _ in range(warmup):
        S.step(0.0)
    ms, sn, sms = timed_and_profiled(S, stream, flush, steps)
    S.diagnostics()
    S.close()
    cells = N_GRID * N_GRID
    fm = gks.count_flops(2, "fp32", "euler", 1.0, charvars=1)
    launch_ms = sms / max(sn, 1)
    tf = fm["flops_per_cell_sweep"] * cells / (launch_ms * 1e-3) / 1e12
    return {"value": cells * steps / (ms * 1e-3), "unit": UNIT, "workload": "riemann2d_config3_charvars",
            "grid": "%dx%d" % (N_GRID, N_GRID), "steps": steps, "ms_per_step": ms / steps,
            "flops_per_cell_update": fm["flops_per_cell_update"],
            "roofline": {"bound": "alu", "kernel": "k2d_sweep<float, charvars>", "achieved": tf, "peak": peak32,
                         "unit": "TFLOP/s", "frac": tf / peak32, "launch_ms": launch_ms}}


def paper_run(gks, s, precision, stream, max_steps=0):
    """A whole run of a paper workload to its end time (CFL steps, CUDA-graph
    replays of the library's advance), timed with CUDA events on the
    library's stream after an untimed warm-up run; cell-updates/s."""
    import torch
    S = gks.solver_for(s, precision)
    S.set_stream(stream.cuda_stream)
    S.advance_to(s.t_end, max_steps=16)  # warm-up: graphs captured
    S.set_state(s.W)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    try:
        steps, t = S.advance_to(s.t_end, max_steps=max_steps)
    except gks.GKSError as e:
        # a run that leaves the scheme's robustness (a cell average turns
        # non-physical) is reported with the time it reached, not timed
        torch.cuda.synchronize()
        d = S.diagnostics(check=False)
        S.close()
        return {"value": None, "unit": UNIT, "failed": str(e)[:160], "t_reached": float(d.t),
                "steps": int(d.steps)}
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    S.diagnostics()
    S.close()
    cells = s.nx * s.ny
    return {"value": cells * steps / (ms * 1e-3), "unit": UNIT, "steps": int(steps), "t": t, "ms": ms}


def paper_legs(gks, WL, stream):
    """The paper's other workloads at the paper's sizes: Sod's tube (Sec. 5.2,
    400 cells to t = 0.2; launch-latency bound), the double Mach
    reflection (Sec. 5.7, 960 x 240 to t = 0.2), the Titarev-Toro
    shock-entropy wave (Sec. 5.3, 1000 cells to t = 5) and the Riemann
    configuration 6 (Sec. 5.6 (b), 400^2 to t = 0.6), both precisions."""
    out = {}
    for name, s in (("sod400", WL.sod(400)), ("dmr", WL.double_mach(960, 240, t_end=0.2)),
                    ("titarev_toro", WL.titarev_toro(1000)),
                    ("riemann_cfg6", WL.riemann2d_config6(400, t_end=0.6))):
        d = {"grid": "%dx%d" % (s.nx, s.ny) if s.dim == 2 else "%d" % s.nx, "t_end": s.t_end}
        d["fp32"] = paper_run(gks, s, "fp32", stream)
        d["fp64"] = paper_run(gks, s, "fp64", stream)
        out[name] = d
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    rank, local_rank, world = rank_info()
    import numpy as np
    import torch

    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(local_rank)
    from paper_2309_10534_gb300 import build

    if rank == 0:
        build.build()
    if dist:
        dist.barrier()
    from paper_2309_10534_gb300 import gks
    from paper_2309_10534_gb300 import workloads as WL

    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    s = WL.riemann2d(N_GRID, split=0.8, t_end=0.8)
    cells = N_GRID * N_GRID
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def solver(precision):
        S = gks.solver_for(s, precision)
        S.set_stream(stream.cuda_stream)
        return S

    def timed(S, K, W):
        """K steps timed with CUDA events and no instrumentation (the value),
        then K more with the library's per-kernel events on (the sweep's own
        launch time for the roofline)."""
        for _ in range(W):
            S.step(0.0)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        L0 = S.kernel_launches()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        for k in range(K):
            flush.zero_()
            ev[k][0].record(stream)
            S.step(0.0)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        launches = S.kernel_launches() - L0
        ms = sum(a.elapsed_time(b) for a, b in ev)
        S.profile(True)
        S.profile_read(0)
        S.profile_read(1)
        S.profile_read(2)
        for k in range(K):
            flush.zero_()
            S.step(0.0)
        torch.cuda.synchronize()
        sweep_n, sweep_ms = S.profile_read(0)
        S.profile(False)
        return ms, launches, sweep_n, sweep_ms

    # measured FMA-chain peaks of this GPU (the roofline denominators)
    peak32 = gks.alu_peak("fp32", 200.0)
    peak64 = gks.alu_peak("fp64", 200.0)
    clocks = ClockSampler(local_rank)
    clocks.start()
    S32 = solver("fp32")
    ms32, launches32, sn32, sms32 = timed(S32, args.steps, args.warmup)
    devw = None
    T_DEV = 0.4
    if args.developed:
        # the same solver advanced (untimed) to t = 0.4, where the quadrant
        # waves have developed, then K more timed steps
        S32.advance_to(T_DEV)
        msd = timed_steps(S32, stream, flush, args.steps)  # the value, no instrumentation
        S32.profile(True)
        S32.profile_read(0)
        timed_steps(S32, stream, flush, args.steps)  # the sweep's own launch time
        dn, dms = S32.profile_read(0)
        S32.profile(False)
        devw = {"value": cells * args.steps * world / (msd * 1e-3), "unit": UNIT, "t_start": T_DEV,
               "steps": args.steps, "ms_per_step": msd / args.steps, "sweep_launch_ms": dms / max(dn, 1)}
    S64 = solver("fp64")
    k64 = max(1, args.fp64_steps)
    ms64, launches64, sn64, sms64 = timed(S64, k64, min(args.warmup, 3))
    ens = None
    if args.ensemble:
        launch = tuple(int(x) for x in args.ensemble_launch.split(",")) if args.ensemble_launch else None
        ens = ensemble_leg(gks, WL, stream, peak32, args.ensemble_max_steps, launch, rank, world, dist)
    ao = weno_ao_leg(gks, WL, stream, peak32, args.steps, args.warmup) if args.weno_ao else None
    conv2d = ({r: weno_ao_leg(gks, WL, stream, peak32, args.steps, args.warmup, recon=r) for r in ("weno_z", "teno5")}
              if args.weno_ao else None)
    r1d = recon_1d_leg(gks, WL, stream, peak32, args.steps, args.warmup) if args.recon_1d else None
    visc = None
    if args.viscous:
        visc = viscous_leg(gks, WL, stream, "fp32", 200)
        visc["fp64"] = viscous_leg(gks, WL, stream, "fp64", 10)
    chv = charvars_leg(gks, WL, stream, peak32, args.steps, args.warmup) if args.charvars else None
    pap = paper_legs(gks, WL, stream) if args.paper else None
    adj = None
    if args.adjoint:
        adj = adjoint_leg(gks, WL, stream, "fp32", args.adjoint_steps)
        if args.adjoint_fp64:
            adj["fp64"] = adjoint_leg(gks, WL, stream, "fp64", args.adjoint_steps)
    clk = clocks.stop()

    # same number of steps on both paths from the same state: relative L1 of fp32 vs fp64
    S32b = solver("fp32")
    for _ in range(min(args.warmup, 3) + 2 * k64):  # the steps timed() gave S64
        S32b.step(0.0)
    W32 = S32b.get_state()
    W64 = S64.get_state()
    rel_l1 = float(np.abs(W32 - W64).sum() / np.abs(W64).sum())
    S32b.close()

    # end to end through the public API with host buffers (pinned)
    host_in = torch.from_numpy(np.ascontiguousarray(s.W)).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    Se = solver("fp32")
    Se.set_state(host_in.numpy())
    Se.step(0.0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        Se.set_state(host_in.numpy())          # H2D of the step's input (synchronising)
        Se.step(0.0)
        Se.get_state_into(host_out.numpy())    # D2H of the step's result (synchronising)
    torch.cuda.synchronize()
    e2e_seq_s = time.perf_counter() - t0
    Se.close()
    # the same calls on two contexts with their own streams, alternating: the
    # copies are enqueued asynchronously from page-locked memory
    # (GKS_HOST_PINNED_ASYNC), so one context's copy-in and copy-out overlap
    # the other's step; every step still moves its input in and its result out
    pipe = []
    for _ in range(2):
        st_k = torch.cuda.Stream(device=dev)
        S_k = gks.solver_for(s, "fp32")
        S_k.set_stream(st_k.cuda_stream)
        pipe.append((S_k, torch.empty_like(host_in).pin_memory()))
    for S_k, o_k in pipe:
        S_k.set_state_async(host_in)
        S_k.step(0.0)
        S_k.get_state_async(o_k)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        S_k, o_k = pipe[k % 2]
        S_k.set_state_async(host_in)
        S_k.step(0.0)
        S_k.get_state_async(o_k)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_same = all(bool(torch.equal(o_k, host_out)) for _, o_k in pipe)
    for S_k, _ in pipe:
        S_k.close()

    times = torch.tensor([ms32, ms64, e2e_s, e2e_seq_s], dtype=torch.float64, device=dev)
    if dist:
        dist.all_reduce(times, op=dist.ReduceOp.MAX)
    ms32, ms64, e2e_s, e2e_seq_s = times.tolist()
    if rank != 0:
        dist.barrier() if dist else None
        return

    fm = gks.count_flops(2, "fp32", "euler", 1.0)
    fm64 = gks.count_flops(2, "fp64", "euler", 1.0)
    sweep_avg_ms = sms32 / max(sn32, 1)
    flops_per_launch = fm["flops_per_cell_sweep"] * cells
    achieved = flops_per_launch / (sweep_avg_ms * 1e-3) / 1e12
    nominal = SMS * FP32_LANES * 2 * 2.070e9 / 1e12
    peak = peak32
    fp64_tflops = fm64["flops_per_cell_update"] * cells * k64 / (ms64 * 1e-3) / 1e12
    value = cells * args.steps * world / (ms32 * 1e-3)
    line = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms32 / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "riemann2d_config3", "grid": "%dx%d" % (N_GRID, N_GRID),
                   "precision": "fp32 reconstruction+flux, fp64 state and S2O4 accumulation",
                   "cfl": 0.5, "split": 0.8, "l2": "256 MB flush between timed steps",
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "fp64": {"value": cells * k64 * world / (ms64 * 1e-3), "unit": UNIT, "steps": k64,
                 "ms_per_step": ms64 / k64, "flops_per_cell_update": fm64["flops_per_cell_update"],
                 "roofline": {"bound": "alu", "achieved": fp64_tflops, "peak": peak64, "unit": "TFLOP/s",
                              "frac": fp64_tflops / peak64, "basis": "whole step vs measured FP64 FMA peak",
                              "fp64_pipe_active_ncu": sweep_pipe_from_profiles("sweep_fp64_riemann1024.md", "FP64")}},
        "fp32_rel_l1_vs_fp64": rel_l1,
        "gpu_launches": launches32,
        "e2e": {"value": cells * args.steps * world / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": int(s.W.nbytes), "d2h_bytes_per_step": int(s.W.nbytes),
                "method": "set_state_async (pinned) + step + get_state_async per step, alternating two "
                          "contexts on two streams so copies overlap the other context's step",
                "results_match_sequential": e2e_same,
                "sequential": {"value": cells * args.steps * world / e2e_seq_s, "unit": UNIT,
                               "method": "one context, synchronous set_state / step / get_state"}},
        "roofline": {"bound": "alu", "kernel": "k2d_sweep<float>", "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak, "traffic": sweep_traffic_from_profiles(),
                     "flops_per_launch": flops_per_launch, "launch_ms": sweep_avg_ms,
                     "peak_basis": "measured FP32 FMA-chain throughput on this GPU (gks_alu_peak)",
                     "peak_nominal": nominal,
                     "sweep_share_of_step": sms32 / ms32 if ms32 else None,
                     "fma_pipe_active_ncu": sweep_pipe_from_profiles()},
        "flops_per_cell_update": fm["flops_per_cell_update"],
        "clocks": clk,
    }
    if ens:
        line["ensemble"] = ens
    if ao:
        line["weno_ao"] = ao
    if conv2d:
        line["conventional_2d"] = conv2d
    if r1d:
        line["recon_1d"] = r1d
    if visc:
        line["viscous"] = visc
    if adj:
        line["adjoint"] = adj
    if devw:
        line["value_developed"] = devw["value"]
        line["developed"] = devw
    if chv:
        line["charvars"] = chv
    if pap:
        line["paper_workloads"] = pap
    line["flips"] = flips_leg(gks, WL, s, args.steps, args.warmup, T_DEV if args.developed else None)
    if world == 1 and not args.skip_cpu:
        line["cpu_baseline"], sample = cpu_baseline(n=args.cpu_sample, budget_all=args.cpu_budget)
        line["oracle_by_config"] = oracle_by_config(args.cpu_budget, line["cpu_baseline"]["cores"])
        line["errors_vs_oracle"] = oracle_errors(gks, sample)
    print(json.dumps(line))
    if dist:
        dist.barrier()


if __name__ == "__main__":
    main()
