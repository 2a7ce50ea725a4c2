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
# iterations: the method's PCG iteration count on the workload (the GPU path
# and the oracle agree on it, +-1, in the parity tests); it scales the
# oracle's sampled time per iteration to the whole workload
WORKLOADS = {
    "inclusions80": dict(n=80, desc="q1-hex-80^3-inclusions-20pct-E1000", tol=1e-8,
                         iterations=92),
    "inclusions150": dict(n=150, desc="q1-hex-150^3-inclusions-20pct-E1000", tol=1e-8,
                          iterations=211),
    "inclusions120": dict(n=120, desc="q1-hex-120^3-inclusions-20pct-E1000", tol=1e-8,
                          iterations=91),
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
# dominant kernel from ncu, keyed by kernel version; the summary and the
# command that produced it are in profiles/sell_spmv_3x3_fp64_inclusions48.md
# (48^3 capture, 245.7 MB, scaled by blocks to the 80^3 launch).  A kernel
# change gets a new tag and reports null until it is captured again.
NCU_TRAFFIC = {"sell_spmv_kernel<3,3,double,double,PLAIN,NONE>:G1:v5": 1136945011,
               # profiles/sell_spmv_3x3_df64_inclusions48.md (246.3 MB at 48^3, scaled)
               "sell_spmv_kernel<3,3,df32,double,PLAIN,NONE>:G1:v1": 1139997327}

# FP64 FMA peak of GB300: 152 SMs x 2 DFMA per clock x 2 flop x 2.07 GHz
# (the nominal 1.25 TFLOP/s FP64 rate at the maximum SM clock).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def cpu_baseline(sample_n=40, workload="inclusions80", nnz_full=None):
    """The oracle, as it stands, on a bounded sample of the workload: the same
    material model on a sample_n^3 mesh, setup + PCG to 1e-8, single thread.
    value = the sample's PCG time per iteration per fine-matrix nonzero, times
    the workload's nonzeros and iterations (the oracle's estimated time on the
    whole workload, in the metric's unit); the raw sample time beside it."""
    import oracle
    import q1elasticity as q
    p = q.inclusions(sample_n)
    A = oracle.from_problem(p)
    t0 = time.perf_counter()
    H = oracle.Hierarchy(A, 3, p.B)
    t1 = time.perf_counter()
    _, it, rel = H.solve(p.f, tol=1e-8, maxiter=3000)
    t2 = time.perf_counter()
    w = WORKLOADS.get(workload, {})
    if nnz_full is None:  # fine-level blocks of the whole workload
        nnz_full = _problem(workload).nnzb if workload in WORKLOADS and w.get("n") else p.nnzb
    it_full = w.get("iterations", it)
    scale = (nnz_full / p.nnzb) * (it_full / it)
    return {"value": (t2 - t1) * scale, "unit": "s", "cores": 1, "kind": "oracle",
            "sample": f"oracle setup+PCG on the same material model at {sample_n}^3 elements "
                      f"({p.ndof} DOFs, {p.nnzb} blocks, {it} iterations, PCG {t2 - t1:.2f} s, "
                      f"setup {t1 - t0:.2f} s); value = that PCG time x {nnz_full / p.nnzb:.2f} "
                      f"(blocks) x {it_full}/{it} (iterations) for the whole workload",
            "sample_value": t2 - t1, "setup_s": t1 - t0, "iterations": it}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    steps = []
    base = None
    for _ in range(args.warmup + args.steps):
        base = cpu_baseline(args.ref_sample, args.workload)
        steps.append(base["value"])
    vals = steps[args.warmup:]
    v = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * v,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload]["desc"], "parallelism": "replicas"},
            "cpu_baseline": {"kind": "oracle", "cores": 1, "sample": base["sample"], "value": v,
                             "unit": "s"},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


LEARN_TRAIN = ((20, 11), (26, 12), (32, 13), (40, 14))  # (elements per side, inclusion seed)


def learned_form(amg, torch, solver, f, tol, u_ref, t_spai0, it_spai0, steps):
    """Learned smoother: train the block-smoother network on the GPU on four
    smaller meshes of the same material model (error samples the SPAI0
    V-cycle leaves, and white noise), then solve the benchmark system with it
    in place of SPAI0 on level 0; SPAI0 stays the fallback and the yardstick."""
    import q1elasticity as q
    dev = f.device
    s = torch.cuda.current_stream()
    t0 = time.perf_counter()
    train_solvers = []
    T = amg.Trainer(amg.learned_init(0), lr=3e-3)
    for k, (n, seed) in enumerate(LEARN_TRAIN):
        p = q.inclusions(n, seed=seed)
        S = amg.AMG(torch.from_numpy(p.row_ptr).to(dev), torch.from_numpy(p.col).to(dev),
                    torch.from_numpy(p.val).to(dev), torch.from_numpy(p.B).to(dev))
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
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    fb = solver.set_learned_smoother(w)
    torch.cuda.synchronize()
    t_infer = time.perf_counter() - t2
    st = solver.stats()
    out = {"training": {"meshes": [f"{n}^3 seed {sd}" for n, sd in LEARN_TRAIN],
                        "samples_per_mesh": 8, "adam_steps": 200, "lr": 3e-3,
                        "loss_before": loss0, "loss_after": loss1, "train_s": t_train,
                        "problem_setup_s": t1 - t0},
           "inference_s": t_infer, "fallback": fb, "lambda_max_MA": st["learned_lambda"],
           "lambda_max_MA_spai0": st["spai0_lambda"], "spai0_value": t_spai0,
           "spai0_iterations": it_spai0,
           "vcycle": "FP64; level 0 smoothed with learned symmetric 3x3 blocks"}
    solver.solve(f, tol=tol, maxiter=5000)  # warm-up (graph capture)
    times = []
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        u_l, it_l, res_l, st_l = solver.solve(f, tol=tol, maxiter=5000)
        e1.record(s)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    solver.clear_learned_smoother()
    out.update(value=float(np.mean(times)), iterations=it_l, rel_resid=res_l, status=st_l,
               err_vs_fp64_solution=float(torch.linalg.norm(u_l - u_ref) / torch.linalg.norm(u_ref)),
               speedup_vs_fp64=t_spai0 / float(np.mean(times)))
    out["weights"] = w
    return out


def learned_fp32_form(amg, torch, args_dev, w, f, tol, u_ref, t_fp64, fp32_form, steps):
    """The same trained network in the FP32 V-cycle (blocks applied in FP32),
    against SPAI0 in the FP32 V-cycle and the plain FP64 path."""
    s = torch.cuda.current_stream()
    sol = amg.AMG(*args_dev, precision=amg.PREC_FP32)
    fb = sol.set_learned_smoother(w)
    sol.solve(f, tol=tol, maxiter=5000)  # warm-up (graph capture)
    times = []
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        u_l, it_l, res_l, st_l = sol.solve(f, tol=tol, maxiter=5000)
        e1.record(s)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    v = float(np.mean(times))
    return {"value": v, "iterations": it_l, "rel_resid": res_l, "status": st_l, "fallback": fb,
            "err_vs_fp64_solution": float(torch.linalg.norm(u_l - u_ref) / torch.linalg.norm(u_ref)),
            "speedup_vs_fp64": t_fp64 / v, "speedup_vs_spai0_fp32": fp32_form["value"] / v,
            "spai0_fp32_iterations": fp32_form["iterations"],
            "vcycle": "FP32 matrices and vectors; level 0 smoothed with the learned blocks in FP32"}


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
    for vname, vprec in (("df64", amg.PREC_DF64), ("fp32", amg.PREC_FP32)):
        t0 = time.perf_counter()
        bv = amg.AMGBatch(mats, Bs, nrhs, loop_mode=args.loop_mode, precision=vprec)
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
                                     "fp32": "SpMMs on FP32 values, FP32 FMAs, FP64 vectors"}[k]
                                    + "; CG A p, dots and true residual in FP64"}
           for k, (t, stv, vs, itsv, resv, vd, tiles) in variants.items()},
        "clocks": clk.summary(), "gpu_launches": int(launches),
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="inclusions80", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-sample", type=int, default=40)
    ap.add_argument("--profile-spmv", action="store_true",
                    help="only build the hierarchy and launch the fine SpMV kernel 8 times "
                         "(a short, fixed command for profilers)")
    ap.add_argument("--profile-op", default="",
                    help="LEVEL:OP (OP in A, P, R): like --profile-spmv for that level operator")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "bf16", "df64"],
                    help="V-cycle precision of the main line (CG stays FP64); with "
                         "--profile-spmv / --profile-op, df64 profiles the FP32-pair copies")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the FP32/BF16 V-cycle and learned-smoother comparisons "
                         "on the same workload")
    ap.add_argument("--loop-mode", type=int, default=0,
                    help="1: host-launched CG steps (for profilers); 0: device while loop")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_2202_09056_gb300 as amg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
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
    rp = torch.from_numpy(p.row_ptr).to(dev)
    cl = torch.from_numpy(p.col).to(dev)
    val = torch.from_numpy(p.val).to(dev)
    B = torch.from_numpy(p.B).to(dev)
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

    if args.profile_spmv or args.profile_op:
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
    info0 = solver.level_info(0)
    levels = [solver.level_info(l) for l in range(stats["nlevels"])]
    t_spmv, algo = _spmv_roofline(solver, torch, p.ndof, p.nnodes, p.nnzb)
    peak, peak_kind = _peaks()
    achieved = algo / t_spmv / 1e9
    kernel_tag = "sell_spmv_kernel<3,3,double,double,PLAIN,NONE>:G1:v5"
    traffic = NCU_TRAFFIC.get(kernel_tag)
    flops = 2.0 * 9 * p.nnzb
    tflops = flops / t_spmv / 1e12
    forms = None
    if not args.no_forms and not args.profile_spmv:
        # precision form: the same solve with the V-cycle in FP32 / BF16
        # storage (FP32 accumulation), CG recurrences and dots in FP64
        u_ref, it_ref, _, _ = solver.solve(f, tol=tol, maxiter=5000)
        forms = {}
        for name in ("fp64", "fp32", "bf16", "scalar_fp64", "scalar_fp32", "scalar_bf16"):
            # scalar_*: the same hierarchy with every solve operator in scalar
            # CSR rows (the scalar solver of Sec. 4) instead of blocks
            scalar = name.startswith("scalar_")
            pname = name.split("_")[-1]
            sol = amg.AMG(rp, cl, val, B, precision=PRECS[pname],
                          storage=amg.STORAGE_SCALAR if scalar else amg.STORAGE_BLOCK)
            sol.solve(f, tol=tol, maxiter=5000)  # warm-up (graph capture)
            times = []
            for _ in range(args.steps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(s)
                u_p, it_p, res_p, st_p = sol.solve(f, tol=tol, maxiter=5000)
                e1.record(s)
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1) / 1e3)
            err = float(torch.linalg.norm(u_p - u_ref) / torch.linalg.norm(u_ref))
            forms[name] = {"value": float(np.mean(times)), "iterations": it_p, "rel_resid": res_p,
                           "status": st_p, "err_vs_fp64_solution": err,
                           "operator_bytes": int(sol.stats()["bytes_solve"]),
                           "storage": "scalar CSR rows" if scalar else "blocks",
                           "vcycle": {"fp64": "FP64 matrices and vectors",
                                      "fp32": "FP32 matrices and vectors, FP32 accumulation",
                                      "bf16": "BF16-stored matrices, FP32 vectors and accumulation"}[pname]}
            del sol
        for name in ("fp32", "bf16"):
            forms[name]["speedup_vs_fp64"] = forms["fp64"]["value"] / forms[name]["value"]
        # the block solver without a near-nullspace (Sec. 4): B = the three
        # translations, 3-DOF coarse nodes, FP64
        T = torch.zeros((p.ndof, 3), dtype=torch.float64, device=dev)
        for c in range(3):
            T[c::3, c] = 1.0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sol = amg.AMG(rp, cl, val, T)
        torch.cuda.synchronize()
        t_setup = time.perf_counter() - t0
        sol.solve(f, tol=tol, maxiter=20000)
        times = []
        for _ in range(args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            u_p, it_p, res_p, st_p = sol.solve(f, tol=tol, maxiter=20000)
            e1.record(s)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        forms["no_nullspace_fp64"] = {
            "value": float(np.mean(times)), "iterations": it_p, "rel_resid": res_p, "status": st_p,
            "setup_s": t_setup, "levels": sol.nlevels,
            "err_vs_fp64_solution": float(torch.linalg.norm(u_p - u_ref) / torch.linalg.norm(u_ref)),
            "operator_bytes": int(sol.stats()["bytes_solve"]),
            "vcycle": "FP64; near-nullspace = 3 translations (no rotations), 3x3 blocks on every level"}
        del sol
        # aggregation on the device (MIS-2) against the host's greedy passes:
        # setup times side by side, then the MIS-2 hierarchy's FP64 solve
        setups = {"greedy": [], "mis2": []}
        for _ in range(3):
            for agg_name, code in (("greedy", amg.AGG_GREEDY), ("mis2", amg.AGG_MIS2)):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                sol = amg.AMG(rp, cl, val, B, aggregation=code)
                torch.cuda.synchronize()
                setups[agg_name].append(time.perf_counter() - t0)
                if agg_name == "greedy":
                    del sol
        sol.solve(f, tol=tol, maxiter=5000)
        times = []
        for _ in range(args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            u_p, it_p, res_p, st_p = sol.solve(f, tol=tol, maxiter=5000)
            e1.record(s)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        forms["mis2_fp64"] = {
            "value": float(np.mean(times)), "iterations": it_p, "rel_resid": res_p, "status": st_p,
            "setup_s": float(np.median(setups["mis2"])),
            "greedy_setup_s": float(np.median(setups["greedy"])), "levels": sol.nlevels,
            "err_vs_fp64_solution": float(torch.linalg.norm(u_p - u_ref) / torch.linalg.norm(u_ref)),
            "operator_bytes": int(sol.stats()["bytes_solve"]),
            "vcycle": "FP64; aggregates from a distance-2 maximal independent set on the device"}
        del sol
        # FP64 emulated on FP32 pairs: the whole solve phase's matrices as
        # hi + lo floats, FP64 vectors and CG; its fine SpMV against HBM
        sol = amg.AMG(rp, cl, val, B, precision=amg.PREC_DF64)
        t_df, it_df, res_df, st_df, u_df = _timed_solves(torch, sol, f, tol, args.steps, 5000, s)
        t_sp, algo_sp = _spmv_roofline(sol, torch, p.ndof, p.nnodes, p.nnzb, which=3)
        forms["df64"] = {
            "value": t_df, "iterations": it_df, "rel_resid": res_df, "status": st_df,
            "speedup_vs_fp64": forms["fp64"]["value"] / t_df,
            "err_vs_fp64_solution": float(torch.linalg.norm(u_df - u_ref) / torch.linalg.norm(u_ref)),
            "operator_bytes": int(sol.stats()["bytes_solve"]),
            "fine_spmv": {"kernel": "sell_spmv_kernel<3,3,df32,double,PLAIN,NONE>:G1:v1",
                          "traffic": NCU_TRAFFIC.get("sell_spmv_kernel<3,3,df32,double,PLAIN,NONE>:G1:v1"),
                          "algorithmic_bytes": algo_sp,
                          "launch_ms": t_sp * 1e3, "achieved_gbs": algo_sp / t_sp / 1e9,
                          "frac_of_measured_hbm": algo_sp / t_sp / 1e9 / peak,
                          "frac_of_nominal_8tbs": algo_sp / t_sp / 8e12},
            "vcycle": "V-cycle in FP64 emulated on FP32 pairs (hi + lo floats, ~2^-45 per "
                      "product), FP64 vectors; CG's A p, dots and true residual in FP64"}
        del sol
        forms["ilu0_fp64"] = ilu0_form(amg, torch, (rp, cl, val, B), f, tol, u_ref,
                                       forms["fp64"], p, s, args.steps)
        for name in ("fp64", "fp32", "bf16"):
            sc, bl = forms["scalar_" + name], forms[name]
            sc["block_speedup"] = sc["value"] / bl["value"]
            sc["block_memory_ratio"] = bl["operator_bytes"] / sc["operator_bytes"]
        # the setup side of the same comparison: each level's Galerkin product
        # R (A P) recomputed with block SpGEMMs and with scalar (1x1) SpGEMMs
        # on the unblocked operators (best of two, wall time incl. symbolic)
        gal = []
        for l in range(solver.nlevels - 1):
            tb = min(solver.galerkin_timing(l, amg.STORAGE_BLOCK)[0] for _ in range(2))
            ts, ds = min(solver.galerkin_timing(l, amg.STORAGE_SCALAR) for _ in range(2))
            gal.append({"level": l, "block_s": tb, "scalar_s": ts, "scalar_rel_diff": ds})
        tb_all, ts_all = sum(g["block_s"] for g in gal), sum(g["scalar_s"] for g in gal)
        forms["galerkin_block_vs_scalar"] = {"block_s": tb_all, "scalar_s": ts_all,
                                             "block_speedup": ts_all / tb_all, "levels": gal}
        if args.precision == "fp64":
            forms["learned"] = learned_form(amg, torch, solver, f, tol, u_ref,
                                            forms["fp64"]["value"], forms["fp64"]["iterations"],
                                            args.steps)
            w_learned = forms["learned"].pop("weights")
            forms["learned_fp32"] = learned_fp32_form(amg, torch, (rp, cl, val, B), w_learned, f,
                                                      tol, u_ref, forms["fp64"]["value"],
                                                      forms["fp32"], args.steps)
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
        "sell_padding": [list(solver.padding(l)) for l in range(stats["nlevels"])],
        "memory_mb": stats["bytes_matrices"] / 1e6,
        "clocks": clk.summary(),
        "e2e": {"value": e2e_t, "unit": "s", "h2d_bytes_per_step": 8 * p.ndof,
                "d2h_bytes_per_step": 8 * p.ndof},
        "gpu_launches": int(launches),
        "roofline": {"bound": "alu", "kernel": kernel_tag, "achieved": tflops,
                     "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": tflops / FP64_PEAK_TFLOPS,
                     "traffic": traffic, "peak_source": "derived: 152 SMs x 2 DFMA/clock x 2 flop x 2.07 GHz (FP64 pipe)",
                     "algorithmic_flops": flops, "launch_ms": 1e3 * t_spmv,
                     "hbm": {"achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "peak_source": peak_kind,
                             "frac_of_nominal_8tbs": achieved / 8000.0,
                             "algorithmic_bytes": algo}},
        "wall_s": wall,
        "precision": args.precision,
        "forms": forms,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.ref_sample, args.workload, p.nnzb)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
