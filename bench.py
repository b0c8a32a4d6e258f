#!/usr/bin/env python
"""Newton-step BDDC-GMRES solve time on one GB300, FP32-local vs FP64.

Workload: the 48x48x12 trilinear (Q1) hexahedral slab [0,4]x[0,4]x[0,1]
(86,436 free DoFs) cut into 4x4x4 = 64 box subdomains, vertex + edge-average
primal space, Guccione + active stress at half the peak activation and a
1 kPa follower pressure on the top face, z = 0 clamped, 4 load steps.

A step is one Newton step of the solve (residual and tangent assembly,
BDDC setup, GMRES to 1e-8 relative residual, update).  The timed steps
replay, in order, the Newton states of a full solve computed untimed
beforehand, so the mean over a full cycle is the mean time per Newton step
of the whole solve.  The primary value uses FP32 local operators (FP64
assembly, GMRES, vectors and coarse solve); the FP64 path is timed beside
it.

Multi-GPU: the path does not shard across GPUs in this build; N ranks run N
independent replicas (weak scaling) and the time is the max over ranks.

--impl reference times the oracle (plain FP64 CPU implementation) on the
host cores instead, on a bounded sample of the same workload.
"""
import argparse
import json
import os
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
WORKLOAD = "slab48_q1"

# name -> (description, problem builder, BDDC levels, level-2 groups, load
# steps whose Newton states are replayed (None: all), FP64 steps timed
# (None: one per replayed state, so both precisions see the same states))
WORKLOADS = {
    "slab48_q1": ("48x48x12 Q1 hex slab [0,4]x[0,4]x[0,1], 64 box subdomains (4x4x4), primal VE, "
                  "n_free=86436, follower pressure 1 kPa + activation 30 kPa, 4 load steps",
                  lambda: __import__("workloads").slab_config("slab48_q1"), 2, None, None, 3),
    "slab24_q2": ("24x24x6 Q2 hex slab [0,4]x[0,4]x[0,1], 64 box subdomains (8x4x2), primal VEF, "
                  "n_free=86436, follower pressure 1 kPa + activation 30 kPa, 4 load steps",
                  lambda: __import__("workloads").slab_config("slab24_q2"), 2, None, None, 3),
    "lv_p1": ("left-ventricle shell, P1 tets, ~1.0M free DoFs, 512 uneven subdomains (+-30%), "
              "primal VEF, two-level (dense FP64 coarse), endocardial pressure 2 kPa + activation "
              "15 kPa over 8 load steps; Newton states of the first load step",
              lambda: __import__("workloads").lv_config("lv_p1"), 2, None, 1, None),
    "lv_p1_ml": ("left-ventricle shell, P1 tets, ~1.0M free DoFs, 512 uneven subdomains (+-30%) "
                 "nested in 16 level-2 subdomains, three-level BDDC, primal VEF/VEF, pressure 2 kPa "
                 "+ activation 15 kPa over 8 load steps; Newton states of the first load step",
                 lambda: __import__("workloads").lv_config("lv_p1", n_parts2=16), 3, 16, 1, None),
    "lv_p2": ("left-ventricle shell, P2 tets, ~3.0M free DoFs, 4096 uneven subdomains (2048 "
              "surface patches x 2 slabs) nested in 64 level-2 subdomains, three-level BDDC, "
              "primal VEF/VEF, FP64 coarsest solve, pressure 2 kPa + activation 15 kPa over 8 "
              "load steps; Newton states of the first load step",
              lambda: __import__("workloads").lv_config("lv_p2"), 3, 64, 1, None),
}
WORKLOADS["slab48_q1_ver"] = ("48x48x12 Q1 hex slab as slab48_q1 with primal VE plus the rotations "
                              "of every edge (rigid-body primal constraints)",
                              lambda: __import__("workloads").slab_config("slab48_q1", primal="VER"),
                              2, None, None, 3)


def _with_scaling(build, scaling):
    def f():
        prob = build()
        prob["scaling"] = scaling
        return prob
    return f


WORKLOADS["slab48_q1_dlx"] = ("48x48x12 Q1 hex slab as slab48_q1 (primal VE) with deluxe scaling",
                              _with_scaling(WORKLOADS["slab48_q1"][1], "deluxe"), 2, None, None, 3)
WORKLOADS["lv_p1_dlx"] = (WORKLOADS["lv_p1"][0] + "; deluxe scaling",
                          _with_scaling(WORKLOADS["lv_p1"][1], "deluxe"), 2, None, 1, None)
# reduced ventricles (same generator, 5 x 64 x 32 rings, 64 subdomains) for
# profiler captures that must stay a few GB on the device
WORKLOADS["lv_p1_small"] = ("left-ventricle shell, P1 tets, 5 x 64 x 32 rings, 64 subdomains",
                            lambda: __import__("workloads").lv_problem(
                                nt=5, ntheta=64, nu=32, order=1, n_parts=64, load_steps=8,
                                gamma=0.25 * 6.0e4), 2, None, 1, 1)
WORKLOADS["lv_p2_small"] = ("left-ventricle shell, P2 tets, 5 x 64 x 32 rings, 128 subdomains "
                            "(64 patches x 2 slabs) in 8 level-2 subdomains",
                            lambda: __import__("workloads").lv_problem(
                                nt=5, ntheta=64, nu=32, order=2, n_parts=128, n_parts2=8,
                                n_layers=2, load_steps=8, gamma=0.25 * 6.0e4), 3, 8, 1, 1)
WORKLOADS["lv_p1_small_dlx"] = (WORKLOADS["lv_p1_small"][0] + "; deluxe scaling",
                                _with_scaling(WORKLOADS["lv_p1_small"][1], "deluxe"), 2, None, 1, 1)
WORKLOAD_DESC = WORKLOADS[WORKLOAD][0]


def _parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=16)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle-budget-s", type=float, default=150.0)
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--max-gmres", type=int, default=1000)
    ap.add_argument("--mode", default="bench", choices=["bench", "kernels"],
                    help="kernels: one BDDC setup and a few applies and SpMVs of the workload "
                         "(a short program for profiler captures)")
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
            if len(parts) < 9:
                continue
            try:
                rows.append(parts)
            except Exception:
                pass
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


def _oracle_step_seconds(timeout):
    """One oracle Newton step (d = 0, lambda = 1/4) of the workload, in a
    fresh single-threaded Python process; returns (seconds, gmres its)."""
    code = r"""
import json, sys, time
sys.path.insert(0, %r)
import numpy as np
from workloads import slab_config
from oracle.assembly import FEProblem
from oracle.bddc import BDDC, Classification
from oracle.krylov import gmres
prob = slab_config(%r)
fe = FEProblem(prob)
cl = Classification(fe, prob["elem_part"], prob["n_parts"])
d = np.zeros(fe.n_free)
lam = 1.0 / prob["load_steps"]
t0 = time.perf_counter()
r = fe.residual(d, lam)
K, (Ke, Kf) = fe.tangent(d, lam)
pc = BDDC(fe, Ke, Kf, prob["primal"], cl)
x, its, _ = gmres(lambda v: K @ v, -r, pc.apply, tol=1e-8)
d = d + x
t1 = time.perf_counter()
print(json.dumps({"seconds": t1 - t0, "its": its}))
""" % (ROOT, WORKLOAD)
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       timeout=timeout)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    out = json.loads(r.stdout.strip().splitlines()[-1])
    return out["seconds"], out["its"]


def run_reference(args, world, rank):
    """The oracle on the host cores: each step is one full oracle Newton step
    of the workload at d = 0, lambda = 1/4; the number of timed steps is
    capped so that the run stays within the time budget."""
    if rank != 0:
        return
    times, its = [], []
    t_start = time.perf_counter()
    while len(times) < max(1, args.steps):
        s, i = _oracle_step_seconds(timeout=args.oracle_budget_s * 4)
        times.append(s)
        its.append(i)
        if time.perf_counter() - t_start + s > args.oracle_budget_s:
            break
    ms = 1000.0 * statistics.mean(times)
    sample = ("full oracle Newton step (assembly, BDDC setup with SciPy LU, GMRES to 1e-8) of %s "
              "at d=0, lambda=1/4, single-threaded, %d step(s) timed of %d requested, no warm-up "
              "(each step runs in a fresh process)" % (WORKLOAD, len(times), args.steps))
    line = {
        "impl": "reference", "metric": METRIC, "value": ms, "unit": UNIT, "n_gpus": args.gpus,
        "steps": len(times), "warmup": 0, "steps_requested": args.steps,
        "warmup_requested": args.warmup, "ms_per_step": ms, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC, "gmres_its": its},
        "cpu_baseline": {"value": ms, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": ms, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, world, rank, local):
    import numpy as np
    import torch

    import paper_2208_06191_gb300 as pkg

    if world == 1:
        torch.cuda.set_device(local)
    pkg.build()
    pkg.load_library()
    desc, build_prob, levels, _groups, n_load_rec, fp64_default = WORKLOADS[args.workload]
    prob = build_prob()
    P = pkg.Problem(prob)
    n = P.n_free
    ml = {}
    if levels == 3:
        ml = dict(levels=3, part2=prob["part2"], n_parts2=prob["n_parts2"], primal2="VEF")
    scaling = prob.get("scaling", "counting")
    opts32 = pkg.SolveOptions(precision=pkg.FP32, primal=prob["primal"], max_gmres=args.max_gmres,
                              precision2=pkg.FP32, scaling=scaling, **ml)
    opts64 = pkg.SolveOptions(precision=pkg.FP64, primal=prob["primal"], max_gmres=args.max_gmres,
                              precision2=pkg.FP64, scaling=scaling, **ml)

    # untimed: Newton states of a full FP32 solve (or of its first load steps)
    states = []
    d = torch.zeros(n, dtype=torch.float64, device="cuda")
    r = torch.empty_like(d)
    ctx32 = None
    last = prob["load_steps"] if n_load_rec is None else n_load_rec
    for k in range(1, last + 1):
        lam = k / prob["load_steps"]
        P.residual(d, lam, r)
        r0 = float(torch.linalg.vector_norm(r))
        for _ in range(25):
            P.residual(d, lam, r)
            if float(torch.linalg.vector_norm(r)) <= 1e-8 * r0:
                break
            states.append((d.clone(), lam))
            rec, ctx32 = P.newton_step(d, lam, opts32, ctx32)
            if rec["status"] != 0:
                raise RuntimeError("Newton step failed during the untimed solve: %r" % rec)
    ns = len(states)
    dw = torch.empty_like(d)

    def run_steps(count, opts, ctx, offset=0, records=None):
        for j in range(count):
            ds, lam = states[(offset + j) % ns]
            dw.copy_(ds)
            rec, ctx = P.newton_step(dw, lam, opts, ctx)
            if rec["status"] != 0:
                raise RuntimeError("Newton step did not converge: %r" % rec)
            if records is not None:
                records.append(rec)
        return ctx

    stream = torch.cuda.current_stream()
    K, W = args.steps, args.warmup
    # ---- FP32 local operators (primary value)
    ctx32 = run_steps(W, opts32, ctx32)
    clocks = ClockSampler(local)
    clocks.start()
    recs32 = []
    launches0 = pkg.kernel_launches()
    pkg.timer_start(pkg.TIMER_SWEEP_GEMM)
    _barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ctx32 = run_steps(K, opts32, ctx32, 0, recs32)
    e1.record(stream)
    torch.cuda.synchronize()
    _barrier(world)
    gemm = pkg.timer_stop()
    launches = pkg.kernel_launches() - launches0
    clk = clocks.stop()
    ms32 = _max_over_ranks(e0.elapsed_time(e1) / K, world)

    # per-class kernel times over two more FP32 steps each (after the timed
    # region, so the timed numbers carry no extra events)
    kernels = {}
    for name, cls in (("bddc_apply", pkg.TIMER_APPLY), ("bsr_spmv", pkg.TIMER_SPMV),
                      ("element_kernel", pkg.TIMER_ELEMENT), ("gmres_orth", pkg.TIMER_ORTH)):
        pkg.timer_start(cls)
        ctx32 = run_steps(2, opts32, ctx32)
        t = pkg.timer_stop()
        if t["launches"]:
            ms = t["ms"] / t["launches"]
            kernels[name] = {"launches": t["launches"], "ms_per_launch": ms,
                             "GB_per_launch": t["bytes"] / t["launches"] / 1e9,
                             "GBps": t["bytes"] / t["launches"] / (ms * 1e-3) / 1e9,
                             "GFLOP_per_launch": t["flops"] / t["launches"] / 1e9}

    # ---- FP64 local operators
    ctx64 = run_steps(1, opts64, None)
    recs64 = []
    if args.workload == WORKLOAD:
        K64 = max(1, min(K, args.fp64_steps))
    else:
        K64 = ns if fp64_default is None else max(1, min(K, fp64_default))
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    ctx64 = run_steps(K64, opts64, ctx64, 0, recs64)
    f1.record(stream)
    torch.cuda.synchronize()
    ms64 = _max_over_ranks(f0.elapsed_time(f1) / K64, world)

    # ---- end to end through the C ABI with host buffers (pinned)
    host = torch.empty(n, dtype=torch.float64, pin_memory=True)
    host_np = host.numpy()
    states_h = [(s.cpu().numpy(), lam) for s, lam in states]
    torch.cuda.synchronize()
    _barrier(world)
    t0 = time.perf_counter()
    for j in range(K):
        ds, lam = states_h[j % ns]
        host_np[:] = ds
        rec, ctx32 = P.newton_step(host_np, lam, opts32, ctx32, host=True)
        if rec["status"] != 0:
            raise RuntimeError("Newton step did not converge (host path): %r" % rec)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    _barrier(world)
    e2e_ms = _max_over_ranks(1000.0 * (t1 - t0) / K, world)

    peaks = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    # FP32 FMA peak from unit counts and the maximum SM clock:
    # 152 SMs x 128 FP32 lanes x 2 flop x f_max
    fp32_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12
    achieved = gemm["flops"] / (gemm["ms"] * 1e-3) / 1e12 if gemm["ms"] > 0 else None
    roofline = {
        "bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
        "frac": achieved / fp32_peak if achieved else None, "traffic": None,
        "kernel": "gemm_grouped_kernel<float> (Gauss-Jordan sweep trailing update)",
        "launches": gemm["launches"], "ms_per_launch": gemm["ms"] / max(1, gemm["launches"]),
        "flops_per_launch": gemm["flops"] / max(1, gemm["launches"]),
        "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x %g MHz (unit counts and max clock)" % sm_max,
    }

    def phase(recs, key):
        return statistics.mean(r[key] for r in recs)

    line = {
        "metric": METRIC, "value": ms32, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms32, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic",
        "config": {
            "workload": desc, "workload_name": args.workload, "newton_states": ns,
            "n_free": n, "parallelism": "replicas",
            "precision": {"local_operators": "f32", "assembly": "f64", "gmres": "f64",
                          "coarse": "f64" if levels == 2 else "level-2 f32, coarsest f64"},
            "l2": "inputs larger than L2 (dense local operators ~1.1 GB read per BDDC apply)",
        },
        "fp64": {"ms_per_step": ms64, "steps": K64,
                 "gmres_its_mean": statistics.mean(r["gmres_its"] for r in recs64),
                 "ms_setup": phase(recs64, "ms_setup"), "ms_gmres": phase(recs64, "ms_gmres")},
        "speedup_fp32_vs_fp64": ms64 / ms32,
        "breakdown_fp32": {"ms_assemble": phase(recs32, "ms_assemble"),
                           "ms_setup": phase(recs32, "ms_setup"),
                           "ms_gmres": phase(recs32, "ms_gmres"),
                           "gmres_its_mean": statistics.mean(r["gmres_its"] for r in recs32),
                           "gmres_its_max": max(r["gmres_its"] for r in recs32),
                           "ms_step_median": statistics.median(r["ms_total"] for r in recs32),
                           "ms_step_max": max(r["ms_total"] for r in recs32)},
        "e2e": {"value": e2e_ms, "unit": UNIT, "h2d_bytes_per_step": 8 * n,
                "d2h_bytes_per_step": 8 * n},
        "gpu_launches": int(launches),
        "roofline": roofline,
        "kernels": kernels,
    }
    if clk:
        line["clocks"] = clk
    if args.workload != WORKLOAD:
        line["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": "not run: reported for the default workload only"}
    elif rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            s, its = _oracle_step_seconds(timeout=900)
            line["cpu_baseline"] = {
                "value": 1000.0 * s, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": "one oracle Newton step of the same workload at d=0, lambda=1/4 "
                          "(%d GMRES its), single-threaded, fresh process" % its}
        except Exception as exc:  # the baseline is reported, not required
            line["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                                    "sample": "failed: %s" % str(exc)[-200:]}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_kernels(args):
    """One assembly, one FP32 BDDC setup, then 3 applies and 3 SpMVs."""
    import torch

    import paper_2208_06191_gb300 as pkg

    pkg.build()
    pkg.load_library()
    _desc, build_prob, levels, _groups, _n, _f = WORKLOADS[args.workload]
    prob = build_prob()
    P = pkg.Problem(prob)
    d = torch.zeros(P.n_free, dtype=torch.float64, device="cuda")
    r = torch.empty_like(d)
    P.assemble_tangent(d, 1.0 / prob["load_steps"], r)
    ml = {}
    if levels == 3:
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
    print(json.dumps({"mode": "kernels", "n_free": P.n_free, "apply_norm": float(z.norm())}))


def main():
    args = _parse()
    world, rank, local = _dist_init()
    if args.mode == "kernels":
        run_kernels(args)
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
