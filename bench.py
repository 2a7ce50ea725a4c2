"""Benchmark: block SA-AMG preconditioned CG on a synthetic Q1 elasticity box.

One step = the whole hot path on one problem: setup (Alg. 1: strength,
aggregation, tentative prolongation, smoothed P, R, Galerkin R A P, SPAI0,
coarse factor) followed by the PCG solve to relative residual 1e-8 (Alg. 2
V-cycle preconditioner, Sec. 4).  `value` is the PCG time-to-1e-8 of the
solve (hierarchy built, right-hand side resident in HBM), averaged over the
timed steps; setup time is reported beside it.

Workload (default): 80^3 Q1 hexahedra, 1.59 M DOFs, E = 1 matrix with E = 1000
spherical inclusions at 20 % volume (SplitMix64 seed 2202), nu = 0.3,
clamped at x = 0, traction (0, 0, -1) on x = 1.  Synthetic inputs stand in
for the paper's two matrices, which are not available.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Multi-GPU: one process per GPU (torchrun); every rank solves its own replica
(the single solve does not shard), so scaling is weak and the reported time
is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PCG time-to-1e-8 (s); BSR SpMV GB/s vs HBM peak; mixed/learned vs FP64"
WORKLOADS = {
    "inclusions80": dict(n=80, desc="q1-hex-80^3-inclusions-20pct-E1000", tol=1e-8),
    "inclusions150": dict(n=150, desc="q1-hex-150^3-inclusions-20pct-E1000", tol=1e-8),
    "inclusions120": dict(n=120, desc="q1-hex-120^3-inclusions-20pct-E1000", tol=1e-8),
    "inclusions64": dict(n=64, desc="q1-hex-64^3-inclusions-20pct-E1000", tol=1e-8),
    "inclusions48": dict(n=48, desc="q1-hex-48^3-inclusions-20pct-E1000", tol=1e-8),
    "inclusions40": dict(n=40, desc="q1-hex-40^3-inclusions-20pct-E1000", tol=1e-8),
    "cube10": dict(n=10, desc="q1-hex-10^3-cube-body-load", tol=1e-8),
    "batch64": dict(n=0, desc="64 q1-hex boxes 20^3-60^3, nu U[0.2,0.45], 1-16 body-load RHS each",
                    tol=1e-8),
}


def _problem(name):
    import q1elasticity as q
    w = WORKLOADS[name]
    return q.cube(w["n"]) if name.startswith("cube") else q.inclusions(w["n"])


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", self.gpu_id], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]
        return False

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _gpu_id(torch):
    try:
        return "GPU-" + str(torch.cuda.get_device_properties(0).uuid)
    except Exception:
        return os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0]


def _spmv_roofline(solver, torch, n, nbr, nnzb, reps=40, which=0):
    """Average duration of the solve's fine-level 3x3 SpMV kernel (the
    dominant kernel of the PCG iteration) on the launch stream: which = 0 the
    FP64 copy, 3 the FP32-pair copy of a PREC_DF64 hierarchy (same bytes)."""
    x = torch.randn(n, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    for _ in range(5):
        solver.level_spmv(0, which, x, y)
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(reps):
        solver.level_spmv(0, which, x, y)  # 1 GB of values per launch: larger than L2
    e1.record(s)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / reps
    algo = nnzb * (72 + 4) + (nbr + 1) * 4 + n * 8 + n * 8
    return t, algo


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# dominant kernel from one ncu capture at 48^3, scaled by blocks to the 80^3
# launch, keyed by kernel version.  A kernel change gets a new tag and
# reports null until it is captured again.
NCU_TRAFFIC = {"sell_spmv_kernel<3,3,double,double,PLAIN,NONE>:G1:v5": 1136945011,
               "sell_spmv_kernel<3,3,df32,double,PLAIN,NONE>:G1:v1": 1139997327}


def fp64_peak(amg):
    """Measured FP64 FMA rate (the library's FMA-chain kernel, best of 3) as a
    TFLOP/s peak with its derivation."""
    runs = [amg.fp64_fma_rate() for _ in range(3)]
    best = max(runs, key=lambda r: r["tflops"])
    return best["tflops"], (f"measured: FP64 FMA chains (4, 8 or 16 per thread, 2, 4 or 8 "
                            f"CTAs of 256 threads per SM on {best['num_sms']} SMs), the fastest "
                            f"configuration of 3 runs ({best['seconds'] * 1e3:.1f} ms), "
                            f"2 flops per FMA")


# ------------------------------------------------------------------ CPU baseline (oracle)
def cpu_leg(workload):
    """The oracle, as it stands, on the whole workload: its setup (Alg. 1 in
    scalar CSR) and one PCG solve to 1e-8 from u = 0, single thread.  Both
    are timed with the host clock."""
    import oracle
    p = _problem(workload)
    A = oracle.from_problem(p)
    t0 = time.perf_counter()
    H = oracle.Hierarchy(A, 3, p.B)
    t1 = time.perf_counter()
    u, it, rel = H.solve(p.f, tol=WORKLOADS[workload]["tol"], maxiter=5000)
    t2 = time.perf_counter()
    return {"setup_s": t1 - t0, "solve_s": t2 - t1, "iterations": int(it), "rel_resid": rel,
            "u_norm": float(np.linalg.norm(u)), "levels": H.nlevels, "dofs": p.ndof,
            "nnzb": p.nnzb}


def start_cpu_leg(workload):
    """Run cpu_leg in a child process (this script with --cpu-leg) while the
    GPU measurements proceed; it uses one host core."""
    return subprocess.Popen([sys.executable, os.path.abspath(__file__), "--cpu-leg",
                             "--workload", workload], stdout=subprocess.PIPE,
                            stderr=subprocess.PIPE, text=True)


def finish_cpu_leg(proc, timeout=1200):
    try:
        out, err = proc.communicate(timeout=timeout)
    except subprocess.TimeoutExpired:
        proc.kill()
        return {"error": f"oracle leg exceeded {timeout} s"}
    for line in reversed(out.splitlines()):
        if line.startswith("{"):
            return json.loads(line)
    return {"error": "oracle leg failed: " + err.strip()[-300:]}


def cpu_baseline_record(leg, gpu_iterations):
    if "error" in leg:
        return {"value": None, "unit": "s", "cores": 1, "kind": "oracle", "sample": leg["error"]}
    return {"value": leg["solve_s"], "unit": "s", "cores": 1, "kind": "oracle",
            "sample": (f"the whole workload ({leg['dofs']} DOFs, {leg['nnzb']} blocks): one "
                       f"oracle PCG solve to 1e-8 from u = 0 on its own {leg['levels']}-level "
                       f"hierarchy, timed with the host clock ({leg['iterations']} iterations; "
                       f"the oracle's setup took {leg['setup_s']:.1f} s), single thread, run in "
                       f"a child process beside the GPU measurements"),
            "setup_s": leg["setup_s"], "total_s": leg["setup_s"] + leg["solve_s"],
            "iterations": leg["iterations"], "gpu_iterations": gpu_iterations,
            "rel_resid": leg["rel_resid"]}


REF_SAMPLE_ITERS = 3


def run_reference(args):
    """The oracle as the reference arm, on the same workload.  Untimed: its
    setup and one whole PCG solve to 1e-8 (the oracle's own iteration count
    and time-to-tolerance).  Each step: a bounded sample, a PCG run of
    REF_SAMPLE_ITERS iterations from u = 0 on the same hierarchy; the step's
    value is that time x (the oracle's iterations / REF_SAMPLE_ITERS), in the
    metric's unit.  ms_per_step is the sample's own duration."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    p = _problem(args.workload)
    A = oracle.from_problem(p)
    t0 = time.perf_counter()
    H = oracle.Hierarchy(A, 3, p.B)
    t1 = time.perf_counter()
    tol = WORKLOADS[args.workload]["tol"]
    _, it_full, rel = H.solve(p.f, tol=tol, maxiter=5000)
    t2 = time.perf_counter()
    m = min(REF_SAMPLE_ITERS, it_full)
    vals, secs = [], []
    for k in range(args.warmup + args.steps):
        s0 = time.perf_counter()
        H.solve(p.f, tol=tol, maxiter=m)
        dt = time.perf_counter() - s0
        if k >= args.warmup:
            secs.append(dt)
            vals.append(dt * it_full / m)
    v = float(np.mean(vals))
    sample = (f"oracle on the workload itself ({p.ndof} DOFs, {p.nnzb} blocks), single thread: "
              f"setup {t1 - t0:.1f} s and one whole PCG solve to 1e-8 ({it_full} iterations, "
              f"{t2 - t1:.1f} s) untimed; each step a {m}-iteration PCG sample on that "
              f"hierarchy, value = its time x {it_full}/{m}")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * float(np.mean(secs)), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload]["desc"], "dofs": p.ndof,
                       "nnzb": p.nnzb, "parallelism": "single"},
            "iterations": it_full, "rel_resid": rel, "full_solve_s": t2 - t1,
            "setup_s": t1 - t0,
            "cpu_baseline": {"kind": "oracle", "cores": 1, "sample": sample, "value": v,
                             "unit": "s"},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


LEARN_TRAIN = ((20, 11), (26, 12), (32, 13), (40, 14))  # (elements per side, inclusion seed)


def train_learned(amg, torch, dev):
    """Train the block-smoother network on the GPU on four smaller meshes of
    the same material model (error samples the SPAI0 V-cycle leaves, and
    white noise): (weights, training record)."""
    import q1elasticity as q
    t0 = time.perf_counter()
    train_solvers = []
    T = amg.Trainer(amg.learned_init(0), lr=3e-3)
    for k, (n, seed) in enumerate(LEARN_TRAIN):
        p = q.inclusions(n, seed=seed)
        S = amg.AMG(*_dev_problem(torch, p, dev))
        T.add_generated(S, 8, seed=100 + k)
        train_solvers.append(S)
    loss0, _ = T.eval()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    T.step(200)
    loss1, _ = T.eval()
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    w = T.params()
    T.close()
    del train_solvers
    return w, {"meshes": [f"{n}^3 seed {sd}" for n, sd in LEARN_TRAIN], "samples_per_mesh": 8,
               "adam_steps": 200, "lr": 3e-3, "loss_before": loss0, "loss_after": loss1,
               "train_s": t_train, "problem_setup_s": t1 - t0}


def learned_form(amg, torch, solver, w, f, tol, u_ref, t_spai0, it_spai0, steps):
    """The trained network's blocks in place of SPAI0 on level 0 of `solver`
    (FP64 V-cycle); SPAI0 stays the fallback and the yardstick."""
    s = torch.cuda.current_stream()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    fb = solver.set_learned_smoother(w)
    torch.cuda.synchronize()
    t_infer = time.perf_counter() - t2
    st = solver.stats()
    out = {"inference_s": t_infer, "fallback": fb, "lambda_max_MA": st["learned_lambda"],
           "lambda_max_MA_spai0": st["spai0_lambda"], "spai0_value": t_spai0,
           "spai0_iterations": it_spai0,
           "vcycle": "FP64; level 0 smoothed with learned symmetric 3x3 blocks"}
    t, it_l, res_l, st_l, u_l = _timed_solves(torch, solver, f, tol, steps, 5000, s)
    solver.clear_learned_smoother()
    out.update(value=t, iterations=it_l, rel_resid=res_l, status=st_l,
               err_vs_fp64_solution=float(torch.linalg.norm(u_l - u_ref) / torch.linalg.norm(u_ref)),
               speedup_vs_fp64=t_spai0 / t, iterations_gain_vs_spai0=it_spai0 - it_l)
    return out


def learned_fp32_form(amg, torch, args_dev, w, f, tol, u_ref, t_fp64, fp32_form, steps):
    """The same trained network in the FP32 V-cycle (blocks applied in FP32),
    against SPAI0 in the FP32 V-cycle and the plain FP64 path."""
    s = torch.cuda.current_stream()
    sol = amg.AMG(*args_dev, precision=amg.PREC_FP32)
    fb = sol.set_learned_smoother(w)
    v, it_l, res_l, st_l, u_l = _timed_solves(torch, sol, f, tol, steps, 5000, s)
    del sol
    return {"value": v, "iterations": it_l, "rel_resid": res_l, "status": st_l, "fallback": fb,
            "err_vs_fp64_solution": float(torch.linalg.norm(u_l - u_ref) / torch.linalg.norm(u_ref)),
            "speedup_vs_fp64": t_fp64 / v, "speedup_vs_spai0_fp32": fp32_form["value"] / v,
            "spai0_fp32_iterations": fp32_form["iterations"],
            "vcycle": "FP32 matrices and vectors; level 0 smoothed with the learned blocks in FP32"}


def _dev_problem(torch, p, dev):
    return (torch.from_numpy(p.row_ptr).to(dev), torch.from_numpy(p.col).to(dev),
            torch.from_numpy(p.val).to(dev), torch.from_numpy(p.B).to(dev))


def _solve_form(amg, torch, dargs, f, tol, steps, stream, u_ref=None, maxiter=5000, **kw):
    """Set up a hierarchy with the given parameters (host-clock setup time)
    and time `steps` solves of it: (record, solver, solution)."""
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sol = amg.AMG(*dargs, **kw)
    torch.cuda.synchronize()
    setup = time.perf_counter() - t0
    t, it, res, st, u = _timed_solves(torch, sol, f, tol, steps, maxiter, stream)
    out = {"value": t, "setup_s": setup, "iterations": it, "rel_resid": res, "status": st,
           "levels": sol.nlevels, "operator_bytes": int(sol.stats()["bytes_solve"])}
    if u_ref is not None:
        out["err_vs_fp64_solution"] = float(torch.linalg.norm(u - u_ref) / torch.linalg.norm(u_ref))
    return out, sol, u


def _timed_solves(torch, sol, f, tol, steps, maxiter, stream):
    """(mean CUDA-event time, iterations, residual, status, u) of `steps`
    solves after one untimed solve (graph capture)."""
    sol.solve(f, tol=tol, maxiter=maxiter)
    times = []
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        u, it, res, st = sol.solve(f, tol=tol, maxiter=maxiter)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    return float(np.mean(times)), it, res, st, u


def ilu0_form(amg, torch, dev_args, f, tol, u_ref, fp64, p, stream, steps, sweeps=3):
    """Block ILU(0) smoothing (the relaxation of Sec. 4's experiments), FP64,
    `sweeps` Jacobi sweeps per triangle: on the workload, and on the same
    cube and load without inclusions against SPAI0 there."""
    import q1elasticity as q
    rp, cl, val, B = dev_args
    out = {"sweeps_per_triangle": sweeps,
           "vcycle": "FP64; block ILU(0) on every smoothing level, Jacobi-swept triangles"}
    t0 = time.perf_counter()
    try:
        sol = amg.AMG(rp, cl, val, B, smoother=amg.SMOOTH_ILU0, ilu_sweeps=sweeps)
        torch.cuda.synchronize()
        out["setup_s"] = time.perf_counter() - t0
        t, it, res, st, u = _timed_solves(torch, sol, f, tol, steps, 5000, stream)
        out.update({"value": t, "iterations": it, "rel_resid": res, "status": st,
                    "err_vs_fp64_solution": float(torch.linalg.norm(u - u_ref) /
                                                  torch.linalg.norm(u_ref))})
        del sol
    except amg.AmgError as e:
        out.update({"value": None, "status": e.status, "error": str(e)})
    # the same cube and traction without inclusions (E = 1 everywhere)
    n = round(len(p.row_ptr) ** (1.0 / 3.0)) - 1
    ph = q.make_problem(n, traction=(0.0, 0.0, -1.0))
    d = val.device
    hargs = (torch.from_numpy(ph.row_ptr).to(d), torch.from_numpy(ph.col).to(d),
             torch.from_numpy(ph.val).to(d), torch.from_numpy(ph.B).to(d))
    fh = torch.from_numpy(ph.f).to(d)
    homog = {"workload": f"q1-hex-{n}^3-homogeneous", "dofs": ph.ndof}
    for name, kw in (("spai0", {}), ("ilu0", {"smoother": amg.SMOOTH_ILU0, "ilu_sweeps": sweeps})):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sol = amg.AMG(*hargs, **kw)
        torch.cuda.synchronize()
        setup = time.perf_counter() - t0
        try:
            t, it, res, st, _ = _timed_solves(torch, sol, fh, tol, steps, 5000, stream)
            homog[name] = {"value": t, "iterations": it, "rel_resid": res, "status": st,
                           "setup_s": setup}
        except amg.AmgError as e:  # the Jacobi-swept ILU(0) can break CG down
            homog[name] = {"value": None, "status": e.status, "error": str(e), "setup_s": setup}
        del sol
    if homog["ilu0"]["value"] and homog["spai0"]["value"]:
        homog["ilu0_speedup"] = homog["spai0"]["value"] / homog["ilu0"]["value"]
    out["homogeneous"] = homog
    return out


def reduce_max(dist, values, device):
    """Element-wise maximum over ranks (the slowest rank sets the time);
    the values themselves when there is one rank."""
    import torch
    if dist is None:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def batch_seed(rank):
    """Each rank solves its own batch of 64 boxes (weak scaling: independent
    problems, no collective on the data path); rank 0's is the 1-GPU batch."""
    return 2202 + 1000 * rank


def run_batch(args, amg, torch, rank=0, world=1, dist=None, local=0):
    """64 independent boxes (seeded sizes 20^3-60^3, nu in [0.2, 0.45], 1-16
    random unit body loads each): one batched solve of every right-hand side
    against a loop of single FP64 solves of the same systems.  Under N ranks
    every rank solves its own seeded batch and the step time is the maximum
    over ranks."""
    import q1elasticity as q
    dev = torch.device("cuda", local)
    specs = q.batch_specs(64, seed=batch_seed(rank))
    mats, Bs, F, nrhs = [], [], [], []
    for sp in specs:
        p = q.make_problem(sp["n"], nu=sp["nu"], body=sp["body"])
        mats.append((torch.from_numpy(p.row_ptr).to(dev), torch.from_numpy(p.col).to(dev),
                     torch.from_numpy(p.val).to(dev)))
        Bs.append(torch.from_numpy(p.B).to(dev))
        F.append(torch.from_numpy(np.atleast_2d(p.f).copy()).to(dev))
        nrhs.append(sp["nrhs"])
    s = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    bat = amg.AMGBatch(mats, Bs, nrhs, loop_mode=args.loop_mode)
    torch.cuda.synchronize()
    setup_t = time.perf_counter() - t0
    for _ in range(args.warmup):
        bat.solve(F)
    times = []
    launches0 = amg.kernel_launches()
    with ClockSampler(_gpu_id(torch)) as clk:
        for _ in range(args.steps):
            if dist is not None:
                dist.barrier()
            torch.cuda.synchronize()
            e0, e1 = ev(), ev()
            e0.record(s)
            U, its, res, st = bat.solve(F)
            e1.record(s)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
    launches = amg.kernel_launches() - launches0
    times = reduce_max(dist, times, dev)
    assert st == amg.AMG_OK, st
    info = bat.info()
    del bat
    # the same batch with the V-cycle's SpMMs on FP32-pair values (emulated
    # FP64) and on FP32 values; the CG's A p and true residual stay FP64
    variants = {}
    for vname, vprec, vsm in (("df64", amg.PREC_DF64, amg.SMOOTH_SPAI0),
                              ("fp32", amg.PREC_FP32, amg.SMOOTH_SPAI0),
                              ("bjacobi", amg.PREC_FP64, amg.SMOOTH_BJACOBI),
                              ("bjacobi_fp32", amg.PREC_FP32, amg.SMOOTH_BJACOBI)):
        t0 = time.perf_counter()
        bv = amg.AMGBatch(mats, Bs, nrhs, loop_mode=args.loop_mode, precision=vprec,
                          smoother=vsm)
        torch.cuda.synchronize()
        v_setup = time.perf_counter() - t0
        bv.solve(F)
        v_times = []
        for _ in range(args.steps):
            if dist is not None:
                dist.barrier()
            torch.cuda.synchronize()
            e0, e1 = ev(), ev()
            e0.record(s)
            Uv, itsv, resv, stv = bv.solve(F)
            e1.record(s)
            torch.cuda.synchronize()
            v_times.append(e0.elapsed_time(e1) / 1e3)
        v_times = reduce_max(dist, v_times, dev)
        v_diff = max(float(torch.linalg.norm(Uv[i][j] - U[i][j]) / torch.linalg.norm(U[i][j]))
                     for i in range(len(U)) for j in range(len(U[i])))
        variants[vname] = (float(np.mean(v_times)), stv, v_setup, itsv, resv, v_diff,
                           bv.info()["rhs_tile"])
        del bv
    # the same systems, one FP64 solve per rhs through amg_solve
    loop_setup, loop_solve, its_single, errs = 0.0, 0.0, [], []
    for i in range(64):
        t0 = time.perf_counter()
        one = amg.AMG(*mats[i], Bs[i])
        torch.cuda.synchronize()
        loop_setup += time.perf_counter() - t0
        for j in range(nrhs[i]):
            one.solve(F[i][j])  # warm graph
            e0, e1 = ev(), ev()
            e0.record(s)
            u1, it1, r1, st1 = one.solve(F[i][j])
            e1.record(s)
            torch.cuda.synchronize()
            loop_solve += e0.elapsed_time(e1) / 1e3
            its_single.append(it1)
            errs.append(float(torch.linalg.norm(U[i][j] - u1) / torch.linalg.norm(u1)))
        del one
    loop_solve, loop_setup, setup_t = reduce_max(dist, [loop_solve, loop_setup, setup_t], dev)
    v = float(np.mean(times))
    return {
        "metric": METRIC, "value": v, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * v, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS["batch64"]["desc"], "instances": 64 * world,
                   "rhs_rank0": int(sum(nrhs)), "dofs_rank0": int(info["dofs_total"]),
                   "l2": "inputs larger than L2",
                   "parallelism": (f"dp{world}: every rank its own seeded batch of 64"
                                   if world > 1 else "single")},
        "batch": {"setup_s": setup_t, "rhs_tile_per_level_A_P_R": info["rhs_tile"],
                  "cta_threads_per_level_A_P_R": info["cta_threads"],
                  "ctas_per_sm_per_level_A_P_R": info["ctas_per_sm"],
                  "iterations_max": int(max(max(x) for x in its)),
                  "iterations_mean": float(np.mean([y for x in its for y in x])),
                  "rel_resid_max": float(max(max(x) for x in res)),
                  "loop_of_single_solves_s": loop_solve, "loop_setup_s": loop_setup,
                  "speedup_vs_loop": loop_solve / v,
                  "max_rel_diff_vs_single_solves": max(errs),
                  "single_iterations_mean": float(np.mean(its_single))},
        **{f"batch_{k}": {"value": t, "status": stv, "setup_s": vs,
                          "speedup_vs_loop": loop_solve / t, "speedup_vs_fp64_batch": v / t,
                          "iterations_mean": float(np.mean([y for x in itsv for y in x])),
                          "iterations_max": int(max(max(x) for x in itsv)),
                          "rel_resid_max": float(max(max(x) for x in resv)),
                          "max_rel_diff_vs_fp64_batch": vd, "rhs_tile_per_level_A_P_R": tiles,
                          "vcycle": {"df64": "SpMMs on FP32-pair values (emulated FP64)",
                                     "fp32": "SpMMs on FP32 values, FP32 FMAs, FP64 vectors",
                                     "bjacobi": "FP64 SpMMs, block damped Jacobi smoother",
                                     "bjacobi_fp32": "SpMMs on FP32 values, FP32 FMAs, FP64 "
                                                     "vectors, block damped Jacobi smoother"}[k]
                                    + "; CG A p, dots and true residual in FP64"}
           for k, (t, stv, vs, itsv, resv, vd, tiles) in variants.items()},
        "clocks": clk.summary(), "gpu_launches": int(launches),
    }


def paper_memory_bytes(sol, scalar):
    """The hierarchy's memory in the paper's accounting (Sec. 4 tables):
    A, P and R of every level in the solve's storage (values FP64, int32
    column indices and row pointers; scalar CSR stores every entry of the
    blocks), the smoother diagonal and the coarsest level's dense factor."""
    st = sol.stats()
    total = 0
    for l in range(st["nlevels"]):
        info = sol.level_info(l)
        b, nb, ns = info["bs"], info["nbrows"], 6
        mats = [(info["nnzb_A"], nb, b, b)]
        if not info["is_coarsest"]:
            mats += [(info["nnzb_P"], nb, b, ns), (info["nnzb_P"], info["nagg"], ns, b)]
            total += nb * b * 8  # SPAI0 diagonal
        for nnzb, rows, br, bc in mats:
            if scalar:
                total += nnzb * br * bc * (8 + 4) + (rows * br + 1) * 4
            else:
                total += nnzb * (br * bc * 8 + 4) + (rows + 1) * 4
    return total + st["coarse_n"] ** 2 * 8


def paper_variants(amg, torch, dargs, f, tol, stream, steps, u_ref):
    """Sec. 4's comparison on GB300: NS Scalar (scalar setup, scalar solve),
    NS Hybrid1 (scalar setup, block solve, Listing 1) and NS Block (block
    setup and solve, Listing 2's route): setup (median of 3, host clock around
    amg_setup), solve, total and memory in the paper's accounting."""
    out = {}
    for name, kw, scalar in (("ns_scalar", dict(setup=amg.SETUP_SCALAR,
                                                 storage=amg.STORAGE_SCALAR), True),
                             ("ns_hybrid1", dict(setup=amg.SETUP_SCALAR), False),
                             ("ns_block", {}, False)):
        setups = []
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sol = amg.AMG(*dargs, **kw)
            torch.cuda.synchronize()
            setups.append(time.perf_counter() - t0)
            phases = sol.stats()["setup_phase_seconds"]
            del sol
        rec, sol, _ = _solve_form(amg, torch, dargs, f, tol, steps, stream, u_ref, **kw)
        rec.update(setup_s=float(np.median(setups)), setup_phases_s=phases,
                   total_s=float(np.median(setups)) + rec["value"],
                   memory_mb=paper_memory_bytes(sol, scalar) / 1e6,
                   storage="scalar CSR" if scalar else "blocks",
                   setup=("scalar arithmetic" if kw.get("setup") else "block arithmetic"))
        del sol
        out[name] = rec
    blk = out["ns_block"]
    for name in ("ns_scalar", "ns_hybrid1"):
        v = out[name]
        v.update(block_total_speedup=v["total_s"] / blk["total_s"],
                 block_setup_speedup=v["setup_s"] / blk["setup_s"],
                 block_solve_speedup=v["value"] / blk["value"],
                 block_memory_ratio=blk["memory_mb"] / v["memory_mb"])
    out["paper_rod_ns_block_over_ns_scalar"] = {"total": 0.803 / 1.444, "memory": 114.19 / 205.16,
                                                "hardware": "i5-3570K CPU, ILU(0) smoother"}
    return out


def forms_80(amg, torch, dargs, p, f, tol, solver, stream, steps):
    """Variants on the benchmark workload (same f): V-cycle precision (FP64,
    FP32, BF16, emulated FP64), block vs scalar storage, the block solver
    without rotations, MIS-2 aggregation, block ILU(0), the Galerkin product
    in block vs scalar arithmetic, and the learned smoother."""
    rp, cl, val, B = dargs
    dev = val.device
    PRECS = {"fp64": amg.PREC_FP64, "fp32": amg.PREC_FP32, "bf16": amg.PREC_BF16}
    u_ref, _, _, _ = solver.solve(f, tol=tol, maxiter=5000)
    forms = {}
    for name in ("fp64", "fp32", "bf16", "scalar_fp64", "scalar_fp32", "scalar_bf16"):
        # scalar_*: the same hierarchy with every solve operator in scalar
        # CSR rows (the scalar solver of Sec. 4) instead of blocks
        scalar = name.startswith("scalar_")
        pname = name.split("_")[-1]
        rec, sol, _ = _solve_form(amg, torch, dargs, f, tol, steps, stream, u_ref,
                                  precision=PRECS[pname],
                                  storage=amg.STORAGE_SCALAR if scalar else amg.STORAGE_BLOCK)
        del sol
        rec["storage"] = "scalar CSR rows" if scalar else "blocks"
        rec["vcycle"] = {"fp64": "FP64 matrices and vectors",
                         "fp32": "FP32 matrices and vectors, FP32 accumulation",
                         "bf16": "BF16-stored matrices, FP32 vectors and accumulation"}[pname]
        forms[name] = rec
    for name in ("fp32", "bf16"):
        forms[name]["speedup_vs_fp64"] = forms["fp64"]["value"] / forms[name]["value"]
    forms["paper_variants"] = paper_variants(amg, torch, dargs, f, tol, stream, steps, u_ref)
    # the block solver without a near-nullspace (Sec. 4): B = the three
    # translations, 3-DOF coarse nodes, FP64
    T = torch.zeros((p.ndof, 3), dtype=torch.float64, device=dev)
    for c in range(3):
        T[c::3, c] = 1.0
    rec, sol, _ = _solve_form(amg, torch, (rp, cl, val, T), f, tol, steps, stream, u_ref,
                              maxiter=20000)
    del sol
    rec["vcycle"] = "FP64; near-nullspace = 3 translations (no rotations), 3x3 blocks on every level"
    forms["no_nullspace_fp64"] = rec
    # aggregation on the device (MIS-2) against the host's greedy passes:
    # setup times side by side (median of 3), then the MIS-2 hierarchy's solve
    setups = {"greedy": [], "mis2": []}
    for _ in range(3):
        for agg_name, code in (("greedy", amg.AGG_GREEDY), ("mis2", amg.AGG_MIS2)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sol = amg.AMG(*dargs, aggregation=code)
            torch.cuda.synchronize()
            setups[agg_name].append(time.perf_counter() - t0)
            del sol
    rec, sol, _ = _solve_form(amg, torch, dargs, f, tol, steps, stream, u_ref,
                              aggregation=amg.AGG_MIS2)
    del sol
    rec.update(setup_s=float(np.median(setups["mis2"])),
               greedy_setup_s=float(np.median(setups["greedy"])),
               vcycle="FP64; aggregates from a distance-2 maximal independent set on the device")
    forms["mis2_fp64"] = rec
    # FP64 emulated on FP32 pairs: the V-cycle's matrices as hi + lo floats,
    # FP64 vectors and CG; its fine SpMV against HBM
    peak, _ = _peaks()
    rec, sol, _ = _solve_form(amg, torch, dargs, f, tol, steps, stream, u_ref,
                              precision=amg.PREC_DF64)
    t_sp, algo_sp = _spmv_roofline(sol, torch, p.ndof, p.nnodes, p.nnzb, which=3)
    del sol
    tag = "sell_spmv_kernel<3,3,df32,double,PLAIN,NONE>:G1:v1"
    rec.update(speedup_vs_fp64=forms["fp64"]["value"] / rec["value"],
               fine_spmv={"kernel": tag, "traffic": NCU_TRAFFIC.get(tag),
                          "algorithmic_bytes": algo_sp, "launch_ms": t_sp * 1e3,
                          "achieved_gbs": algo_sp / t_sp / 1e9,
                          "frac_of_measured_hbm": algo_sp / t_sp / 1e9 / peak,
                          "frac_of_nominal_8tbs": algo_sp / t_sp / 8e12},
               vcycle="V-cycle in FP64 emulated on FP32 pairs (hi + lo floats, ~2^-45 per "
                      "product), FP64 vectors; CG's A p, dots and true residual in FP64")
    forms["df64"] = rec
    # block damped Jacobi (the paper's damped Jacobi relaxation over node
    # blocks) in place of SPAI0, FP64 and FP32 V-cycles
    for name, prec in (("bjacobi_fp64", amg.PREC_FP64), ("bjacobi_fp32", amg.PREC_FP32)):
        rec, sol, _ = _solve_form(amg, torch, dargs, f, tol, steps, stream, u_ref,
                                  precision=prec, smoother=amg.SMOOTH_BJACOBI)
        rec["lambda_per_level"] = [sol.level_info(l)["smoother_lambda"]
                                   for l in range(sol.nlevels - 1)]
        del sol
        rec["speedup_vs_fp64_spai0"] = forms["fp64"]["value"] / rec["value"]
        rec["spai0_iterations"] = forms["fp64"]["iterations"]
        rec["vcycle"] = ("block damped Jacobi M_I = (2 w_s / lambda) A_II^-1 on every level, "
                         + ("FP64" if name.endswith("64") else "FP32 matrices and vectors"))
        forms[name] = rec
    forms["ilu0_fp64"] = ilu0_form(amg, torch, dargs, f, tol, u_ref, forms["fp64"], p, stream,
                                   steps)
    for name in ("fp64", "fp32", "bf16"):
        sc, bl = forms["scalar_" + name], forms[name]
        sc["block_speedup"] = sc["value"] / bl["value"]
        sc["block_memory_ratio"] = bl["operator_bytes"] / sc["operator_bytes"]
    # the setup side of the same comparison: each level's Galerkin product
    # R (A P) recomputed with block SpGEMMs and with scalar (1x1) SpGEMMs on
    # the unblocked operators (best of two, wall time incl. symbolic)
    gal = []
    for l in range(solver.nlevels - 1):
        tb = min(solver.galerkin_timing(l, amg.STORAGE_BLOCK)[0] for _ in range(2))
        ts, ds = min(solver.galerkin_timing(l, amg.STORAGE_SCALAR) for _ in range(2))
        gal.append({"level": l, "block_s": tb, "scalar_s": ts, "scalar_rel_diff": ds})
    tb_all, ts_all = sum(g["block_s"] for g in gal), sum(g["scalar_s"] for g in gal)
    forms["galerkin_block_vs_scalar"] = {"block_s": tb_all, "scalar_s": ts_all,
                                         "block_speedup": ts_all / tb_all, "levels": gal}
    # learned smoother: trained on the GPU on four smaller meshes, applied here
    w, training = train_learned(amg, torch, dev)
    lf = learned_form(amg, torch, solver, w, f, tol, u_ref, forms["fp64"]["value"],
                      forms["fp64"]["iterations"], steps)
    lf["training"] = training
    forms["learned"] = lf
    forms["learned_fp32"] = learned_fp32_form(amg, torch, dargs, w, f, tol, u_ref,
                                              forms["fp64"]["value"], forms["fp32"], steps)
    return forms, w


def config_precision_150(amg, torch, dev, stream, steps):
    """150^3 inclusions (10.3 M DOFs): the V-cycle precision forms against
    the FP64 path (time-to-1e-8, iterations, error against the FP64
    solution), and MIS-2 aggregation on the same mesh."""
    p = _problem("inclusions150")
    dargs = _dev_problem(torch, p, dev)
    f = torch.from_numpy(p.f).to(dev)
    tol = WORKLOADS["inclusions150"]["tol"]
    out = {"workload": WORKLOADS["inclusions150"]["desc"], "dofs": p.ndof, "nnzb": p.nnzb,
           "timed_solves_per_form": steps}
    with ClockSampler(_gpu_id(torch)) as clk:
        rec, sol, u_ref = _solve_form(amg, torch, dargs, f, tol, steps, stream)
        del sol
        out["fp64"] = rec
        for name, prec in (("fp32", amg.PREC_FP32), ("bf16", amg.PREC_BF16),
                           ("df64", amg.PREC_DF64)):
            rec, sol, _ = _solve_form(amg, torch, dargs, f, tol, steps, stream, u_ref,
                                      precision=prec)
            del sol
            rec["speedup_vs_fp64"] = out["fp64"]["value"] / rec["value"]
            out[name] = rec
        rec, sol, _ = _solve_form(amg, torch, dargs, f, tol, steps, stream, u_ref,
                                  aggregation=amg.AGG_MIS2)
        del sol
        rec["speedup_vs_fp64"] = out["fp64"]["value"] / rec["value"]
        out["mis2_fp64"] = rec
        for name, prec in (("bjacobi_fp64", amg.PREC_FP64), ("bjacobi_fp32", amg.PREC_FP32)):
            rec, sol, _ = _solve_form(amg, torch, dargs, f, tol, steps, stream, u_ref,
                                      precision=prec, smoother=amg.SMOOTH_BJACOBI)
            del sol
            rec["speedup_vs_fp64"] = out["fp64"]["value"] / rec["value"]
            out[name] = rec
    out["clocks"] = clk.summary()
    out["oracle"] = ("not run at this size: the oracle's setup and solve take tens of minutes "
                     "on one host core; errors are against the FP64 GPU solution, whose "
                     "iterations and solution match the oracle's at 80^3")
    del dargs, f, u_ref
    torch.cuda.empty_cache()
    return out


def config_learned_120(amg, torch, dev, stream, steps, w):
    """120^3 inclusions (5.3 M DOFs), the learned smoother's test mesh: the
    network trained on 20^3-40^3 meshes against SPAI0, in the FP64 and FP32
    V-cycles."""
    p = _problem("inclusions120")
    dargs = _dev_problem(torch, p, dev)
    f = torch.from_numpy(p.f).to(dev)
    tol = WORKLOADS["inclusions120"]["tol"]
    out = {"workload": WORKLOADS["inclusions120"]["desc"], "dofs": p.ndof, "nnzb": p.nnzb,
           "timed_solves_per_form": steps}
    with ClockSampler(_gpu_id(torch)) as clk:
        spai0, sol, u_ref = _solve_form(amg, torch, dargs, f, tol, steps, stream)
        out["spai0_fp64"] = spai0
        out["learned_fp64"] = learned_form(amg, torch, sol, w, f, tol, u_ref, spai0["value"],
                                           spai0["iterations"], steps)
        del sol
        fp32, sol, _ = _solve_form(amg, torch, dargs, f, tol, steps, stream, u_ref,
                                   precision=amg.PREC_FP32)
        del sol
        out["spai0_fp32"] = fp32
        out["learned_fp32"] = learned_fp32_form(amg, torch, dargs, w, f, tol, u_ref,
                                                spai0["value"], fp32, steps)
    out["clocks"] = clk.summary()
    lf = out["learned_fp64"]
    out["verdict"] = ("learned beats SPAI0 in the FP64 V-cycle"
                      if lf["value"] < spai0["value"] and lf["iterations"] < spai0["iterations"]
                      else "no gain over SPAI0 in the FP64 V-cycle on this mesh")
    del dargs, f, u_ref
    torch.cuda.empty_cache()
    return out


def config_batch64(args, amg, torch, steps):
    """The batched form (64 seeded boxes, one graph-launched solve of every
    right-hand side) against a loop of single FP64 solves."""
    import types
    sub = types.SimpleNamespace(steps=steps, warmup=1, loop_mode=args.loop_mode)
    line = run_batch(sub, amg, torch)
    keep = ("value", "unit", "config", "batch", "batch_df64", "batch_fp32", "batch_bjacobi",
            "batch_bjacobi_fp32", "clocks", "gpu_launches", "steps")
    out = {k: line[k] for k in keep if k in line}
    torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="inclusions80", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-leg", action="store_true",
                    help="(internal) run only the oracle's setup and solve on the workload and "
                         "print them as JSON")
    ap.add_argument("--profile-spmv", action="store_true",
                    help="only build the hierarchy and launch the fine SpMV kernel 8 times "
                         "(a short, fixed command for profilers)")
    ap.add_argument("--profile-op", default="",
                    help="LEVEL:OP (OP in A, P, R): like --profile-spmv for that level operator")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "bf16", "df64"],
                    help="V-cycle precision of the main line (CG stays FP64); with "
                         "--profile-spmv / --profile-op, df64 profiles the FP32-pair copies")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the variants on the benchmark workload")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the 150^3 precision, 64-box batch and 120^3 learned sub-records")
    ap.add_argument("--form-steps", type=int, default=5,
                    help="timed solves per variant and sub-record (at most --steps)")
    ap.add_argument("--loop-mode", type=int, default=0,
                    help="1: host-launched CG steps (for profilers); 0: device while loop")
    args = ap.parse_args()
    if args.cpu_leg:
        print(json.dumps(cpu_leg(args.workload)), flush=True)
        return 0
    if args.impl == "reference":
        return run_reference(args)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    profiling = args.profile_spmv or bool(args.profile_op)
    leg = None
    if (world == 1 and not args.no_cpu_baseline and not profiling
            and args.workload != "batch64"):
        leg = start_cpu_leg(args.workload)  # before CUDA is initialised in this process

    import torch
    import paper_2202_09056_gb300 as amg

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    amg.load()
    if args.workload == "batch64":
        line = run_batch(args, amg, torch, rank, world, dist, local)
        if rank == 0:
            print(json.dumps(line), flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return 0
    p = _problem(args.workload)
    dev = torch.device("cuda", local)
    dargs = _dev_problem(torch, p, dev)
    rp, cl, val, B = dargs
    f = torch.from_numpy(p.f).to(dev)
    tol = WORKLOADS[args.workload]["tol"]
    s = torch.cuda.current_stream()
    PRECS = {"fp64": amg.PREC_FP64, "fp32": amg.PREC_FP32, "bf16": amg.PREC_BF16,
             "df64": amg.PREC_DF64}
    prec = PRECS[args.precision]

    def step(timings=None):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(s)
        solver = amg.AMG(rp, cl, val, B, loop_mode=args.loop_mode, precision=prec)
        ev[1].record(s)
        u, it, res, st = solver.solve(f, tol=tol, maxiter=5000)
        ev[2].record(s)
        torch.cuda.synchronize()
        if st != amg.AMG_OK:
            raise RuntimeError(f"solve did not converge: status {st}, {it} its, res {res}")
        if timings is not None:
            timings.append((ev[0].elapsed_time(ev[1]) / 1e3, ev[1].elapsed_time(ev[2]) / 1e3,
                            it, res))
        return solver

    if profiling:
        # a short, fixed sequence for profilers: 8 launches of one level
        # operator's SpMV (PLAIN mode) on the benchmark hierarchy
        df = args.precision == "df64"
        solver = amg.AMG(rp, cl, val, B, precision=amg.PREC_DF64 if df else amg.PREC_FP64)
        lvl, op = (0, "A") if not args.profile_op else args.profile_op.split(":")
        lvl, which = int(lvl), "APR".index(op)
        info = [solver.level_info(l) for l in range(solver.nlevels)]
        nf = info[lvl]["nbrows"] * info[lvl]["bs"]
        nc = info[lvl + 1]["nbrows"] * info[lvl + 1]["bs"] if which else nf
        nx, ny = ((nf, nf), (nc, nf), (nf, nc))[which]
        x = torch.randn(nx, dtype=torch.float64, device=dev)
        y = torch.empty(ny, dtype=torch.float64, device=dev)
        for _ in range(8):
            solver.level_spmv(lvl, which + (3 if df else 0), x, y)
        torch.cuda.synchronize()
        print(json.dumps({"profile_op": f"{lvl}:{op}", "workload": args.workload,
                          "nnzb": info[lvl]["nnzb_P" if which else "nnzb_A"], "x": nx, "y": ny}))
        return 0
    for _ in range(args.warmup):
        solver = step()
        del solver
    timings = []
    launches0 = amg.kernel_launches()
    barrier()
    with ClockSampler(_gpu_id(torch)) as clk:
        t0 = time.perf_counter()
        for _ in range(args.steps):
            solver = step(timings)
        barrier()
        wall = time.perf_counter() - t0
    launches = amg.kernel_launches() - launches0
    setup_t = float(np.mean([t[0] for t in timings]))
    solve_t = float(np.mean([t[1] for t in timings]))
    its = timings[-1][2]
    res = timings[-1][3]
    step_t = setup_t + solve_t
    solve_t, step_t = reduce_max(dist, [solve_t, step_t], dev)

    # end to end through the public API: pinned host f -> device, solve, u -> host
    fh = torch.from_numpy(p.f).pin_memory()
    uh = torch.empty_like(fh).pin_memory()
    fd = torch.empty_like(f)
    e2e = []
    for k in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        fd.copy_(fh, non_blocking=True)
        u, it2, res2, st2 = solver.solve(fd, tol=tol, maxiter=5000)
        uh.copy_(u, non_blocking=True)
        e1.record(s)
        torch.cuda.synchronize()
        if k >= args.warmup:
            e2e.append(e0.elapsed_time(e1) / 1e3)
    e2e_t = float(np.mean(e2e))

    stats = solver.stats()
    levels = [solver.level_info(l) for l in range(stats["nlevels"])]
    padding = [list(solver.padding(l)) for l in range(stats["nlevels"])]
    t_spmv, algo = _spmv_roofline(solver, torch, p.ndof, p.nnodes, p.nnzb)
    peak, peak_kind = _peaks()
    fp64_tflops, fp64_src = fp64_peak(amg)
    achieved = algo / t_spmv / 1e9
    kernel_tag = "sell_spmv_kernel<3,3,double,double,PLAIN,NONE>:G1:v5"
    traffic = NCU_TRAFFIC.get(kernel_tag)
    flops = 2.0 * 9 * p.nnzb
    tflops = flops / t_spmv / 1e12
    fsteps = max(1, min(args.steps, args.form_steps))
    forms, configs, w = None, None, None
    if not args.no_forms:
        forms, w = forms_80(amg, torch, dargs, p, f, tol, solver, s, fsteps)
    if not args.no_configs and args.workload == "inclusions80" and world == 1:
        del solver
        torch.cuda.empty_cache()
        solver = None
        configs = {"precision_150": config_precision_150(amg, torch, dev, s, min(fsteps, 2)),
                   "batch64": config_batch64(args, amg, torch, min(fsteps, 2))}
        if w is not None:
            configs["learned_120"] = config_learned_120(amg, torch, dev, s, min(fsteps, 3), w)
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0
    line = {
        "metric": METRIC, "value": solve_t, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * step_t, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f64 CG / f32 V-cycle",
                                         "bf16": "f64 CG / bf16-stored V-cycle",
                                         "df64": "f64 CG / f32-pair (emulated f64) V-cycle"}[args.precision],
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload]["desc"], "dofs": p.ndof,
                   "nnzb": p.nnzb, "levels": stats["nlevels"],
                   "level_rows": [l["nbrows"] * l["bs"] for l in levels],
                   "coarse_n": stats["coarse_n"], "smoother": "SPAI0 x0.8, V(1,1)",
                   "l2": "inputs larger than L2 (fine A values 1.0 GB)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "iterations": its, "rel_resid": res, "setup_s": setup_t, "total_s": step_t,
        "setup_phases_s": stats["setup_phase_seconds"],
        "operator_complexity": stats["operator_complexity"],
        "memory_mb": stats["bytes_matrices"] / 1e6,
        "clocks": clk.summary(),
        "e2e": {"value": e2e_t, "unit": "s", "h2d_bytes_per_step": 8 * p.ndof,
                "d2h_bytes_per_step": 8 * p.ndof},
        "gpu_launches": int(launches),
        "roofline": {"bound": "alu", "kernel": kernel_tag, "achieved": tflops,
                     "peak": fp64_tflops, "unit": "TFLOP/s", "frac": tflops / fp64_tflops,
                     "traffic": traffic, "peak_source": fp64_src,
                     "algorithmic_flops": flops, "launch_ms": 1e3 * t_spmv,
                     "hbm": {"achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "peak_source": peak_kind,
                             "frac_of_nominal_8tbs": achieved / 8000.0,
                             "algorithmic_bytes": algo}},
        "wall_s": wall,
        "precision": args.precision,
        "forms": forms,
        "configs": configs,
    }
    line["sell_padding"] = padding
    if leg is not None:
        line["cpu_baseline"] = cpu_baseline_record(finish_cpu_leg(leg), its)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
