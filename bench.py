#!/usr/bin/env python
"""Newton-step BDDC-GMRES solve time on one GB300, FP32-local vs FP64.

Default workload: the idealised left ventricle with quadratic P2 tetrahedra
(3,004,479 free DoFs), 4096 uneven level-1 subdomains (2048 surface patches
x 2 transmural slabs, sizes +-30%) nested in 64 level-2 subdomains,
three-level BDDC with primal space VEF on both levels and an FP64 coarsest
solve, Guccione + active stress, follower endocardial pressure, clamped
base, 8 load steps.

A step is one Newton step of the solve (residual and tangent assembly,
BDDC setup, FGMRES to 1e-8 relative residual, update).  The timed steps
replay, in order and cyclically, the Newton states of the first load steps
of a solve computed untimed beforehand (which load steps is part of the
workload description printed in ``config``).  The primary value uses FP32
local operators (FP64 assembly, GMRES, vectors and coarsest solve); the
FP64 path is timed on a subset of the same states, and the speedup pairs
the two precisions state by state.

Multi-GPU: the path does not shard across GPUs in this build; N ranks run N
independent replicas (weak scaling) and the time is the max over ranks.

--impl reference times the oracle (plain FP64 CPU implementation) on the
host cores instead, on a bounded sample of the same workload.
"""
import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Newton-step BDDC-GMRES solve time, FP32-local vs FP64, at 1e-8 rel residual"
UNIT = "ms/Newton step"
WORKLOAD = "lv_p2"


def _slab(name, **kw):
    return lambda: __import__("workloads").slab_config(name, **kw)


def _lv(name, **kw):
    return lambda: __import__("workloads").lv_config(name, **kw)


def _with_scaling(build, scaling):
    def f():
        prob = build()
        prob["scaling"] = scaling
        return prob
    return f


# name -> workload: description, problem builder, BDDC levels, GMRES restart,
# load steps whose Newton states are replayed (None: all), FP64 states timed
W = {}
W["lv_p2"] = dict(
    desc="left-ventricle shell, P2 tets, 3,004,479 free DoFs, 4096 uneven subdomains (2048 surface "
         "patches x 2 slabs, +-30%) nested in 64 level-2 subdomains, three-level BDDC, primal VEF/VEF, "
         "FP64 coarsest solve, endocardial follower pressure 2 kPa + activation 15 kPa over 8 load "
         "steps; the Newton states of load steps 1-2 (load 1/8 and 2/8) replayed",
    build=_lv("lv_p2"), levels=3, restart=1000, n_load=2, fp64_states=4, n_parts=4096, its_ref=300)
W["lv_p1"] = dict(
    desc="left-ventricle shell, P1 tets, 1,007,235 free DoFs, 512 uneven subdomains (+-30%), primal "
         "VEF, two-level (dense FP64 coarse), endocardial pressure 2 kPa + activation 15 kPa over 8 load "
         "steps; the Newton states of load steps 1-2 replayed",
    build=_lv("lv_p1"), levels=2, restart=1000, n_load=2, fp64_states=4, n_parts=512, its_ref=150)
W["slab48_q1"] = dict(
    desc="48x48x12 Q1 hex slab [0,4]x[0,4]x[0,1], 64 box subdomains (4x4x4), primal VE, n_free=86436, "
         "follower pressure 1 kPa + activation 30 kPa, 4 load steps; every Newton state of the solve",
    build=_slab("slab48_q1"), levels=2, restart=100, n_load=None, fp64_states=None)
W["slab24_q2"] = dict(
    desc="24x24x6 Q2 hex slab [0,4]x[0,4]x[0,1], 64 box subdomains (8x4x2), primal VEF, n_free=86436, "
         "follower pressure 1 kPa + activation 30 kPa, 4 load steps; every Newton state of the solve",
    build=_slab("slab24_q2"), levels=2, restart=100, n_load=None, fp64_states=None)
W["lv_p1_ml"] = dict(
    desc="left-ventricle shell, P1 tets, 1,007,235 free DoFs, 512 uneven subdomains nested in 16 level-2 "
         "subdomains, three-level BDDC, primal VEF/VEF; Newton states of load steps 1-2",
    build=_lv("lv_p1", n_parts2=16), levels=3, restart=1000, n_load=2, fp64_states=4, n_parts=512,
    its_ref=150)
W["slab48_q1_ver"] = dict(
    desc="48x48x12 Q1 hex slab as slab48_q1 with primal VE plus the rotations of every edge",
    build=_slab("slab48_q1", primal="VER"), levels=2, restart=100, n_load=None, fp64_states=3)
W["slab48_q1_dlx"] = dict(
    desc="48x48x12 Q1 hex slab as slab48_q1 (primal VE) with deluxe scaling",
    build=_with_scaling(_slab("slab48_q1"), "deluxe"), levels=2, restart=100, n_load=None, fp64_states=3)
W["lv_p2_dlx"] = dict(
    desc=W["lv_p2"]["desc"] + "; deluxe scaling on level 1",
    build=_with_scaling(_lv("lv_p2"), "deluxe"), levels=3, restart=1000, n_load=2, fp64_states=2,
    n_parts=4096, its_ref=300)
# reduced ventricles (same generator) for profiler captures that must stay a
# few GB on the device
W["lv_p1_small"] = dict(
    desc="left-ventricle shell, P1 tets, 5 x 64 x 32 rings, 64 subdomains",
    build=lambda: __import__("workloads").lv_problem(nt=5, ntheta=64, nu=32, order=1, n_parts=64,
                                                     load_steps=8, gamma=0.25 * 6.0e4),
    levels=2, restart=300, n_load=1, fp64_states=1, n_parts=64, its_ref=90)
W["lv_p2_small"] = dict(
    desc="left-ventricle shell, P2 tets, 5 x 64 x 32 rings, 128 subdomains (64 patches x 2 slabs) in 8 "
         "level-2 subdomains",
    build=lambda: __import__("workloads").lv_problem(nt=5, ntheta=64, nu=32, order=2, n_parts=128,
                                                     n_parts2=8, n_layers=2, load_steps=8,
                                                     gamma=0.25 * 6.0e4),
    levels=3, restart=300, n_load=1, fp64_states=1, n_parts=128, its_ref=90)
WORKLOADS = W


def _parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=16)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-states", type=int, default=None,
                    help="FP64 states timed (default: the workload's setting)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle-budget-s", type=float, default=150.0)
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--max-gmres", type=int, default=3000)
    ap.add_argument("--mode", default="bench", choices=["bench", "kernels", "step"],
                    help="kernels: one BDDC setup and a few applies and SpMVs of the workload; "
                         "step: one FP32 Newton step from d = 0 at the first load level (short "
                         "programs for profiler captures)")
    return ap.parse_args()


def _dist_init():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clock and throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def _cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


# ------------------------------------------------------- the oracle on the CPU
#
# Slabs: one full oracle Newton step of the workload (d = 0, first load
# level) in a fresh process.  Ventricles (far too large for the oracle): a
# sample of 16 level-1 subdomains of the workload that touch the clamped
# base, with their elements, loads and clamped nodes (workloads.
# lv_part_problem), through the oracle's assembly, BDDC setup and three
# GMRES iterations; the Newton step of the whole workload is extrapolated as
# (subdomains / 16) x (assembly + setup + iterations x time per iteration),
# with the GMRES iterations of the GPU's FP32 path.  Linear scaling in the
# number of subdomains favours the CPU (the oracle's setup and apply grow
# faster than that), and so does leaving out its coarse levels.

SAMPLE_PARTS = 16

_ORACLE_STEP = r"""
import json, sys, time
sys.path.insert(0, %(root)r)
import numpy as np
import workloads
from oracle.assembly import FEProblem
from oracle.bddc import BDDC, Classification
from oracle.krylov import gmres
name, first = %(name)r, %(first)d
if name.startswith("slab"):
    prob = workloads.slab_config(name)
    maxit = 3000
else:
    full = workloads.lv_config(name)
    cp = workloads.clamped_parts(full)
    parts = [cp[(first + i) %% len(cp)] for i in range(%(nparts)d)]
    prob = workloads.lv_part_problem(full, parts)
    maxit = 3
if %(sync)d:
    # all-cores run: wait until every process has built its mesh
    print("ready", flush=True)
    sys.stdin.readline()
t0 = time.perf_counter()
fe = FEProblem(prob)
cl = Classification(fe, prob["elem_part"], prob["n_parts"])
d = np.zeros(fe.n_free)
lam = 1.0 / prob["load_steps"]
t1 = time.perf_counter()
r = fe.residual(d, lam)
K, (Ke, Kf) = fe.tangent(d, lam)
t2 = time.perf_counter()
pc = BDDC(fe, Ke, Kf, prob["primal"], cl)
t3 = time.perf_counter()
x, its, _ = gmres(lambda v: K @ v, -r, pc.apply, tol=1e-8, restart=1000, maxiter=maxit)
d = d + x
t4 = time.perf_counter()
print(json.dumps({"prep": t1 - t0, "assemble": t2 - t1, "setup": t3 - t2, "gmres": t4 - t3,
                  "its": its, "n_free": fe.n_free}))
"""


def _oracle_proc(name, first, threads, sync=False):
    code = _ORACLE_STEP % {"root": ROOT, "name": name, "first": first, "nparts": SAMPLE_PARTS,
                           "sync": int(sync)}
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(threads)
    return subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                            stdin=subprocess.PIPE if sync else None, text=True, env=env)


def _collect(proc, timeout):
    out, err = proc.communicate(timeout=timeout)
    if proc.returncode != 0:
        raise RuntimeError(err[-2000:])
    return json.loads(out.strip().splitlines()[-1])


def _extrapolate(name, s, its):
    """ms per Newton step of the whole workload from one sample."""
    if name.startswith("slab"):
        return 1000.0 * (s["assemble"] + s["setup"] + s["gmres"])
    n_parts = int(WORKLOADS[name]["n_parts"])
    per_it = s["gmres"] / max(1, s["its"])
    return 1000.0 * (n_parts / SAMPLE_PARTS) * (s["assemble"] + s["setup"] + its * per_it)


def _sample_text(name, s, its):
    if name.startswith("slab"):
        return ("one full oracle Newton step of %s at d=0, load 1/4 (%d GMRES its), single-threaded, "
                "fresh process" % (name, s["its"]))
    n_parts = int(WORKLOADS[name]["n_parts"])
    return ("oracle assembly, BDDC setup and %d GMRES iterations (d=0, load 1/8) on %d clamped level-1 "
            "subdomains of %s (%d free DoFs), extrapolated x%d to the workload's %d subdomains with %.0f "
            "GMRES iterations per Newton step; linear in the subdomain count and without the oracle's "
            "coarse levels (both favour the CPU)"
            % (s["its"], SAMPLE_PARTS, name, s["n_free"], n_parts // SAMPLE_PARTS, n_parts, its))


def oracle_baseline(name, its, all_cores=True, timeout=900):
    """(single-thread ms/Newton step, all-cores ms/Newton step, cores used,
    sample description) of the oracle on the workload."""
    ncpu = os.cpu_count() or 1
    s = _collect(_oracle_proc(name, 0, 1), timeout)
    single = _extrapolate(name, s, its)
    sample = _sample_text(name, s, its)
    allc, cores = None, 1
    if all_cores and ncpu > 1:
        # all host cores: independent samples (different subdomains) in
        # parallel, one process per core; the per-subdomain loops of the
        # oracle's setup and apply parallelise the same way
        # one process per core; the clock starts once every process has
        # built its sample (mesh generation is not part of a Newton step)
        procs = [_oracle_proc(name, SAMPLE_PARTS * i, 1, sync=True) for i in range(ncpu)]
        for p in procs:
            if p.stdout.readline().strip() != "ready":
                raise RuntimeError(p.communicate(timeout=timeout)[1][-2000:])
        for p in procs:
            p.stdin.write("go\n")
            p.stdin.flush()
        t0 = time.perf_counter()
        res = [_collect(p, timeout) for p in procs]
        wall = time.perf_counter() - t0
        work = sum(r["prep"] + r["assemble"] + r["setup"] + r["gmres"] for r in res)
        eff = work / (ncpu * wall)
        allc = single / (ncpu * eff)
        cores = ncpu
        sample += ("; all cores: %d samples in parallel, one per core, parallel efficiency %.2f"
                   % (ncpu, eff))
    return single, allc, cores, sample


def run_reference(args, world, rank):
    """The oracle on the host cores: each step is one oracle sample of the
    workload (see oracle_baseline), single-threaded, extrapolated with the
    workload's recorded GMRES iteration count; the number of timed steps is
    capped so that the run stays within the time budget."""
    if rank != 0:
        return
    spec = WORKLOADS[args.workload]
    its = spec.get("its_ref", 0)
    times = []
    sample = ""
    t_start = time.perf_counter()
    while len(times) < max(1, args.steps):
        t_one = time.perf_counter()
        s = _collect(_oracle_proc(args.workload, SAMPLE_PARTS * len(times), 1), 900)
        times.append(_extrapolate(args.workload, s, its))
        sample = _sample_text(args.workload, s, its)
        if time.perf_counter() - t_start + (time.perf_counter() - t_one) > args.oracle_budget_s:
            break
    ms = statistics.mean(times)
    sample += "; %d sample(s) timed of %d steps requested, no warm-up" % (len(times), args.steps)
    line = {
        "impl": "reference", "metric": METRIC, "value": ms, "unit": UNIT, "n_gpus": args.gpus,
        "steps": len(times), "warmup": 0, "steps_requested": args.steps,
        "warmup_requested": args.warmup, "ms_per_step": ms, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": spec["desc"], "workload_name": args.workload},
        "cpu_baseline": {"value": ms, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                         "cpu_model": _cpu_model()},
        "e2e": {"value": ms, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ the GPU path
TIMER_CLASSES = ("SWEEP_GEMM", "ELEMENT", "APPLY", "SPMV", "ORTH", "SETUP", "LEVEL2_SETUP", "LEVEL2_APPLY",
                 "COARSE_SETUP", "COARSE_APPLY", "SETUP_GEMM_F64")


# DRAM traffic of one BDDC apply per byte of local_bytes, from one ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum over the kernels of
# an apply, lv_p2_small, the same generator and kernels at 194k DoFs).  The
# apply streams every operator once, so its traffic grows with local_bytes,
# and the ratio scales the capture to the full workload.  None: no capture
# for that workload's current kernels.
APPLY_TRAFFIC_PER_LOCAL_BYTE = {"lv_p2": 1.034}


def _opts(pkg, prob, spec, precision, max_gmres):
    ml = {}
    if spec["levels"] == 3:
        ml = dict(levels=3, part2=prob["part2"], n_parts2=prob["n_parts2"], primal2="VEF")
    # FP32: the setup is autotuned when the first Newton step creates the
    # context (sweep block x tile order, timed on that tangent)
    return pkg.SolveOptions(precision=precision, primal=prob["primal"], max_gmres=max_gmres,
                            restart=spec["restart"], precision2=precision,
                            scaling=prob.get("scaling", "counting"), autotune=precision == pkg.FP32, **ml)


def newton_states(P, prob, opts, n_load, torch, records=None):
    """Untimed FP32 solve over the first n_load load steps (all if None):
    every Newton state (d before the step, load factor) in order."""
    n = P.n_free
    d = torch.zeros(n, dtype=torch.float64, device="cuda")
    r = torch.empty_like(d)
    ctx = None
    states = []
    last = prob["load_steps"] if n_load is None else n_load
    for k in range(1, last + 1):
        lam = k / prob["load_steps"]
        P.residual(d, lam, r)
        r0 = float(torch.linalg.vector_norm(r))
        for _ in range(25):
            P.residual(d, lam, r)
            if float(torch.linalg.vector_norm(r)) <= 1e-8 * r0:
                break
            states.append((d.clone(), lam))
            rec, ctx = P.newton_step(d, lam, opts, ctx)
            if rec["status"] != 0:
                raise RuntimeError("Newton step failed during the untimed solve: %r" % rec)
            if records is not None:
                records.append(rec)
    return states, ctx


def _spread(n, k):
    """k indices spread evenly over range(n) (all of them if k >= n)."""
    if k >= n:
        return list(range(n))
    return sorted({int(round(i * (n - 1) / max(1, k - 1))) for i in range(k)})


def run_ours(args, world, rank, local):
    import torch

    import paper_2208_06191_gb300 as pkg

    if world == 1:
        torch.cuda.set_device(local)
    pkg.build()
    pkg.load_library()
    spec = WORKLOADS[args.workload]
    prob = spec["build"]()
    P = pkg.Problem(prob)
    n = P.n_free
    opts32 = _opts(pkg, prob, spec, pkg.FP32, args.max_gmres)
    opts64 = _opts(pkg, prob, spec, pkg.FP64, args.max_gmres)

    solve_recs = []
    states, ctx32 = newton_states(P, prob, opts32, spec["n_load"], torch, solve_recs)
    ns = len(states)
    inf32 = ctx32.info()
    autotune = {"sweep_block": inf32["sweep_block"], "tile_order": inf32["tile_order"],
                "ms_setup_tuned": inf32["ms_setup_tuned"], "ms_setup_default": inf32["ms_setup_default"],
                "ms_tuning": solve_recs[0]["ms_autotune"],
                "candidates": "sweep block 64/128 x GEMM tile order by subdomain/largest first, one timed "
                              "setup each on the first Newton state's tangent"}
    dw = torch.empty_like(states[0][0])

    def run_steps(seq, opts, ctx, records=None):
        for j in seq:
            ds, lam = states[j]
            dw.copy_(ds)
            rec, ctx = P.newton_step(dw, lam, opts, ctx)
            if rec["status"] != 0:
                raise RuntimeError("Newton step did not converge: %r" % rec)
            if records is not None:
                records.append(dict(rec, state=j))
        return ctx

    stream = torch.cuda.current_stream()
    K, Wm = args.steps, args.warmup
    seq = [j % ns for j in range(K)]
    # ---- FP32 local operators (primary value)
    ctx32 = run_steps([j % ns for j in range(Wm)], opts32, ctx32)
    clocks = ClockSampler(local)
    clocks.start()
    recs32 = []
    launches0 = pkg.kernel_launches()
    _barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ctx32 = run_steps(seq, opts32, ctx32, recs32)
    e1.record(stream)
    torch.cuda.synchronize()
    _barrier(world)
    launches = pkg.kernel_launches() - launches0
    clk = clocks.stop()
    ms32 = _max_over_ranks(e0.elapsed_time(e1) / K, world)

    # ---- kernel classes and the per-level split, over two more FP32 steps
    # (after the timed region, so the timed numbers carry no extra events)
    pkg.timer_start(getattr(pkg, "TIMER_" + TIMER_CLASSES[0]))
    for c in TIMER_CLASSES[1:]:
        pkg.timer_enable(getattr(pkg, "TIMER_" + c))
    kseq = _spread(ns, 2)
    krecs = []
    ctx32 = run_steps(kseq, opts32, ctx32, krecs)
    tt = {c: pkg.timer_result(getattr(pkg, "TIMER_" + c)) for c in TIMER_CLASSES}
    pkg.timer_stop()
    nk = len(kseq)
    kernels = {}
    for c, t in tt.items():
        if t["launches"]:
            ms = t["ms"] / t["launches"]
            kernels[c.lower()] = {"launches": t["launches"], "ms_per_launch": ms,
                                  "ms_per_step": t["ms"] / nk,
                                  "GB_per_launch": t["bytes"] / t["launches"] / 1e9,
                                  "GBps": t["bytes"] / t["launches"] / (ms * 1e-3) / 1e9 if ms > 0 else None,
                                  "GFLOP_per_launch": t["flops"] / t["launches"] / 1e9,
                                  "TFLOPs": t["flops"] / t["launches"] / (ms * 1e-3) / 1e12 if ms > 0 else None}

    def per_step(c):
        return tt[c]["ms"] / nk

    if spec["levels"] == 3:
        per_level = {
            "level1_setup_ms": per_step("SETUP") - per_step("LEVEL2_SETUP"),
            "level2_setup_ms": per_step("LEVEL2_SETUP") - per_step("COARSE_SETUP"),
            "coarsest_setup_ms": per_step("COARSE_SETUP"),
            "level1_apply_ms": per_step("APPLY") - per_step("LEVEL2_APPLY"),
            "level2_apply_ms": per_step("LEVEL2_APPLY") - per_step("COARSE_APPLY"),
            "coarsest_apply_ms": per_step("COARSE_APPLY"),
        }
    else:
        per_level = {
            "level1_setup_ms": per_step("SETUP") - per_step("COARSE_SETUP"),
            "coarsest_setup_ms": per_step("COARSE_SETUP"),
            "level1_apply_ms": per_step("APPLY") - per_step("COARSE_APPLY"),
            "coarsest_apply_ms": per_step("COARSE_APPLY"),
        }
    per_level["gmres_spmv_ms"] = per_step("SPMV")
    per_level["gmres_orth_ms"] = per_step("ORTH")
    per_level["assembly_element_kernel_ms"] = per_step("ELEMENT")
    per_level["steps_averaged"] = nk

    # ---- FP64 local operators on a subset of the same states, paired (the
    # FP32 context is released first: both do not fit at 3M DoFs)
    ctx32.close()
    ctx32 = None
    torch.cuda.synchronize()
    n64 = args.fp64_states if args.fp64_states is not None else spec["fp64_states"]
    sel64 = _spread(ns, ns if n64 is None else n64)
    ctx64 = run_steps(sel64[:1], opts64, None)  # context creation, untimed
    recs64 = []
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    ctx64 = run_steps(sel64, opts64, ctx64, recs64)
    f1.record(stream)
    torch.cuda.synchronize()
    ms64 = _max_over_ranks(f0.elapsed_time(f1) / len(sel64), world)
    by_state32 = {}
    for r in recs32:
        by_state32.setdefault(r["state"], []).append(r)
    paired = []
    for r64 in recs64:
        r32 = by_state32.get(r64["state"])
        if r32:
            paired.append({"state": r64["state"], "load": r64["load"],
                           "its32": r32[0]["gmres_its"], "its64": r64["gmres_its"],
                           "ms32": statistics.mean(x["ms_total"] for x in r32), "ms64": r64["ms_total"],
                           "relres32": max(x["gmres_relres"] for x in r32), "relres64": r64["gmres_relres"]})
    speedup = (statistics.mean(p["ms64"] for p in paired) / statistics.mean(p["ms32"] for p in paired)
               if paired else None)

    ctx64.close()
    ctx64 = None
    # ---- end to end through the C ABI with host buffers (pinned); one
    # untimed host step first recreates the FP32 context
    host = torch.empty(n, dtype=torch.float64, pin_memory=True)
    host_np = host.numpy()
    states_h = [(s.cpu().numpy(), lam) for s, lam in states]
    e2e_seq = seq  # the timed region's states, in its order
    host_np[:] = states_h[0][0]
    rec, ctx32 = P.newton_step(host_np, states_h[0][1], opts32, None, host=True)
    torch.cuda.synchronize()
    _barrier(world)
    t0 = time.perf_counter()
    for j in e2e_seq:
        ds, lam = states_h[j]
        host_np[:] = ds
        rec, ctx32 = P.newton_step(host_np, lam, opts32, ctx32, host=True)
        if rec["status"] != 0:
            raise RuntimeError("Newton step did not converge (host path): %r" % rec)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    _barrier(world)
    e2e_ms = _max_over_ranks(1000.0 * (t1 - t0) / len(e2e_seq), world)

    # ---- roofline of the dominant kernel class of the step
    peaks = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6767.1))
    bf16 = float(peaks.get("bf16_tflops", 1888.9))
    ap, gm = kernels.get("apply"), kernels.get("sweep_gemm")
    apply_step = ap["ms_per_step"] if ap else 0.0
    gemm_step = gm["ms_per_step"] if gm else 0.0
    if apply_step >= gemm_step and ap:
        achieved = ap["GBps"]
        ratio = APPLY_TRAFFIC_PER_LOCAL_BYTE.get(args.workload)
        roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                    "frac": achieved / hbm,
                    "traffic": ratio * ap["GB_per_launch"] * 1e9 if ratio else None,
                    "traffic_source": ("ncu DRAM bytes of one apply on lv_p2_small, %.3f per byte of "
                                       "local_bytes, scaled to this workload's local_bytes" % ratio)
                    if ratio else None,
                    "kernel": "BDDC apply (its batched launches, level 2 and coarsest included)",
                    "bytes_per_launch": ap["GB_per_launch"] * 1e9, "ms_per_launch": ap["ms_per_launch"],
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                    "work": "dense local operators read once per apply (local_bytes)"}
    else:
        tf32 = bf16 / 2.0
        achieved = gm["TFLOPs"]
        roofline = {"bound": "tensor", "achieved": achieved, "peak": tf32 / 3.0, "unit": "TFLOP/s",
                    "frac": achieved / (tf32 / 3.0), "traffic": None,
                    "kernel": "FP32 setup GEMMs on tcgen05 (3xTF32)",
                    "flops_per_launch": gm["GFLOP_per_launch"] * 1e9, "ms_per_launch": gm["ms_per_launch"],
                    "peak_source": "MEASURED_PEAKS.json bf16_tflops / 2 (TF32) / 3 (three TF32 passes "
                                   "per FP32 product) (of measured)"}

    def mean(recs, key):
        return statistics.mean(r[key] for r in recs)

    line = {
        "metric": METRIC, "value": ms32, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": Wm,
        "ms_per_step": ms32, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic",
        "config": {
            "workload": spec["desc"], "workload_name": args.workload, "newton_states": ns,
            "replay": "the %d Newton states in solve order, cyclically, one per step" % ns,
            "n_free": n, "parallelism": "replicas", "gmres_restart": spec["restart"],
            "precision": {"local_operators": "f32 (setup GEMMs: tcgen05 3xTF32)", "assembly": "f64",
                          "gmres": "f64", "coarse": "f64" if spec["levels"] == 2 else "level-2 f32, coarsest f64"},
            "l2": "inputs larger than L2 (dense local operators read per BDDC apply: %.1f GB)"
                  % (ap["GB_per_launch"] if ap else 0.0),
        },
        "fp64": {"ms_per_step": ms64, "states": sel64,
                 "gmres_its_mean": mean(recs64, "gmres_its"),
                 "ms_setup": mean(recs64, "ms_setup"), "ms_gmres": mean(recs64, "ms_gmres")},
        "paired_states": paired,
        "speedup_fp32_vs_fp64": speedup,
        "its_fp32_minus_fp64_max": max((p["its32"] - p["its64"] for p in paired), default=None),
        "breakdown_fp32": {"ms_assemble": mean(recs32, "ms_assemble"), "ms_setup": mean(recs32, "ms_setup"),
                           "ms_gmres": mean(recs32, "ms_gmres"),
                           "gmres_its_mean": mean(recs32, "gmres_its"),
                           "gmres_its_max": max(r["gmres_its"] for r in recs32),
                           "gmres_relres_max": max(r["gmres_relres"] for r in recs32),
                           "gmres_second_pass_frac": sum(r["gmres_reorth"] for r in recs32)
                           / max(1, sum(r["gmres_its"] for r in recs32)),
                           "ms_step_median": statistics.median(r["ms_total"] for r in recs32),
                           "ms_step_max": max(r["ms_total"] for r in recs32)},
        "per_level": per_level,
        "autotune": autotune,
        "e2e": {"value": e2e_ms, "unit": UNIT, "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n,
                "steps": len(e2e_seq)},
        "gpu_launches": int(launches),
        "roofline": roofline,
        "kernels": kernels,
    }
    if clk:
        line["clocks"] = clk
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            single, allc, cores, sample = oracle_baseline(args.workload, mean(recs32, "gmres_its"))
            line["cpu_baseline"] = {"value": single, "unit": UNIT, "cores": 1, "kind": "oracle",
                                    "sample": sample, "cpu_model": _cpu_model(),
                                    "all_cores": {"value": allc, "cores": cores}}
        except Exception as exc:  # the baseline is reported, not required
            line["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                                    "sample": "failed: %s" % str(exc)[-300:]}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_kernels(args):
    """One assembly, one FP32 BDDC setup, then 3 applies and 3 SpMVs."""
    import torch

    import paper_2208_06191_gb300 as pkg

    pkg.build()
    pkg.load_library()
    spec = WORKLOADS[args.workload]
    prob = spec["build"]()
    P = pkg.Problem(prob)
    d = torch.zeros(P.n_free, dtype=torch.float64, device="cuda")
    r = torch.empty_like(d)
    tangent = P.assemble_tangent(d, 1.0 / prob["load_steps"], r)
    ml = {}
    if spec["levels"] == 3:
        ml = dict(levels=3, part2=prob["part2"], n_parts2=prob["n_parts2"], primal2="VEF",
                  precision2=pkg.FP32)
    pc = pkg.BDDC(P, precision=pkg.FP32, primal=prob["primal"], scaling=prob.get("scaling", "counting"),
                  **ml).setup()
    z = torch.empty_like(d)
    y = torch.empty_like(d)
    for _ in range(3):
        pc.apply(r, z)
        P.spmv(z, y)
    torch.cuda.synchronize()
    inf = pc.info()
    print(json.dumps({"mode": "kernels", "n_free": P.n_free, "apply_norm": float(z.norm()),
                      "local_bytes": inf["local_bytes"], "nnzb": tangent["nnzb"]}))


def run_step(args):
    """One FP32 Newton step of the workload from d = 0 at the first load
    level, in the benchmark's launch configuration without autotuning."""
    import torch

    import paper_2208_06191_gb300 as pkg

    pkg.build()
    pkg.load_library()
    spec = WORKLOADS[args.workload]
    prob = spec["build"]()
    P = pkg.Problem(prob)
    opts = _opts(pkg, prob, spec, pkg.FP32, args.max_gmres)
    opts.autotune = 0
    d = torch.zeros(P.n_free, dtype=torch.float64, device="cuda")
    rec, ctx = P.newton_step(d, 1.0 / prob["load_steps"], opts)
    torch.cuda.synchronize()
    print(json.dumps({"mode": "step", "n_free": P.n_free, "gmres_its": rec["gmres_its"],
                      "ms_total": rec["ms_total"], "status": rec["status"]}))


def main():
    args = _parse()
    world, rank, local = _dist_init()
    if args.mode == "kernels":
        run_kernels(args)
        return
    if args.mode == "step":
        run_step(args)
        return
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
