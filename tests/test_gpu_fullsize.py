"""Parity with the oracle at the sizes the benchmark runs (GPU required).

The small-mesh parity tests never reach the setup kernels that only run on
large levels: the numeric Galerkin products switch to the row-per-lane-group
kernel at 16 384 block rows, and the smoothed-prolongation and transpose
kernels see different grids.  Here the whole hierarchy is compared with the
oracle's (Alg. 1 step by step, scalar CSR, FP64) on meshes beyond that
switch, and on the 80^3 inclusion benchmark itself (1 594 323 DOFs): every
level's aggregates, strength flags and patterns bit-exact, A, P, R, B values
within 1e-12, then the PCG solve (iterations +-1, solution within 1e-7), one
V-cycle, and sampled rows of the solve's own sliced kernels recomputed one by
one from the oracle's matrices.
"""
import numpy as np
import pytest

import oracle as o
import q1elasticity as q

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

amg = pytest.importorskip("paper_2202_09056_gb300")

from parity_util import compare_hierarchy, compare_levels, dev_args, vcycle_bound  # noqa: E402

ROW_KERNEL_SWITCH = 16384  # block rows from which the Galerkin products run row by row


def _pcg_parity(H, G, f):
    uo, ito, _ = H.solve(f, tol=1e-8, maxiter=2000)
    u, it, res, st = G.solve(torch.from_numpy(f).cuda(), tol=1e-8, maxiter=2000)
    u = u.cpu().numpy()
    assert st == amg.AMG_OK and res <= 1e-8
    assert abs(it - ito) <= 1, (it, ito)
    assert np.linalg.norm(u - uo) <= 1e-7 * np.linalg.norm(uo)
    return it, ito


@pytest.mark.parametrize("shape", [(26, 26, 26), (30, 24, 28)])
def test_hierarchy_and_pcg_beyond_row_kernel_switch(shape):
    """27^3 and 31x25x29 nodes (> 16 384 block rows): the fine A P and R (A P)
    products take the row-per-lane-group kernel; the hierarchy and the solve
    against the oracle."""
    p = q.make_problem(shape, traction=(0, 0, -1), inclusion_frac=0.2)
    assert p.nnodes > ROW_KERNEL_SWITCH
    H, G = compare_hierarchy(p, 3000, torch, amg)
    assert G.nlevels >= 3
    _pcg_parity(H, G, p.f)


def test_mis2_hierarchy_beyond_row_kernel_switch():
    p = q.make_problem((26, 26, 26), traction=(0, 0, -1), inclusion_frac=0.2)
    H, G = compare_hierarchy(p, 3000, torch, amg, aggregation="mis2")
    _pcg_parity(H, G, p.f)


# ------------------------------------------------------------------ 80^3 benchmark mesh
@pytest.fixture(scope="module")
def bench80():
    """The benchmark's workload: the oracle's hierarchy and solve (about 1.5
    minutes on one host core) and the CUDA hierarchy with default parameters."""
    p = q.inclusions(80)
    H = o.Hierarchy(o.from_problem(p), 3, p.B)
    rp, cl, val, B = dev_args(p, torch)
    G = amg.AMG(rp, cl, val, B)
    return p, H, G


@pytest.mark.slow
def test_bench80_hierarchy_matches_oracle(bench80):
    p, H, G = bench80
    assert p.ndof == 1594323 and p.nnzb == 13829839
    compare_levels(H, G, 6)


@pytest.mark.slow
def test_bench80_pcg_matches_oracle(bench80):
    """The benchmark solve itself: the CUDA path's iteration count (the
    number the benchmark reports) equals the oracle's within +-1, and the
    solutions agree to 1e-7."""
    p, H, G = bench80
    it, ito = _pcg_parity(H, G, p.f)
    assert it > 10


@pytest.mark.slow
def test_bench80_vcycle_matches_oracle(bench80):
    p, H, G = bench80
    r = np.random.default_rng(80).standard_normal(p.ndof)
    z = G.vcycle(torch.from_numpy(r).cuda()).cpu().numpy()
    zo = H.vcycle(r)
    assert np.linalg.norm(z - zo) <= vcycle_bound(H) * np.linalg.norm(zo)


def _sampled_rows(C, x, y, rows, what):
    """y's sampled rows against the oracle's CSR rows summed one by one; the
    bound is 1e-12 of sum |a_ij| |x_j| per row (the sum's rounding scale)."""
    for i in rows:
        s, e = C.ptr[i], C.ptr[i + 1]
        terms = C.val[s:e] * x[C.col[s:e]]
        ref = float(np.sum(terms))
        scale = float(np.sum(np.abs(terms)))
        assert abs(y[i] - ref) <= 1e-12 * max(scale, 1e-300), (what, i, y[i], ref)


@pytest.mark.slow
def test_bench80_solve_kernels_sampled(bench80):
    """The sliced kernels the PCG runs (not the BSR primitive): fine A, P and
    R, and the level-1 A, on 200 sampled rows each, against the oracle's
    operators of the same level."""
    p, H, G = bench80
    rng = np.random.default_rng(8080)
    for l in range(2):
        ol = H.level(l)
        nb = ol["n"] // ol["b"]
        nc = G.level_info(l)["nagg"] * 6
        ops = [(0, ol["A"], ol["n"], ol["n"]), (1, ol["P"], ol["n"], nc), (2, ol["R"], nc, ol["n"])]
        if l == 1:
            ops = ops[:1]
        for which, C, ny, nx in ops:
            x = rng.standard_normal(nx)
            y = torch.empty(ny, dtype=torch.float64, device="cuda")
            G.level_spmv(l, which, torch.from_numpy(x).cuda(), y)
            rows = rng.choice(ny, size=min(200, ny), replace=False)
            _sampled_rows(C, x, y.cpu().numpy(), rows, (l, "APR"[which]))
        assert nb == G.level_info(l)["nbrows"]


@pytest.mark.slow
def test_bench80_block_jacobi_pcg_matches_oracle(bench80):
    """The benchmark mesh with the block damped Jacobi smoother (the bench's
    bjacobi forms): the smoother blocks of every level within 1e-12 of the
    oracle's, the lambda estimates within 1e-10, and the PCG iterations
    within +-1 and the solution within 1e-7 of the oracle's block Jacobi
    solve (the hierarchy is the default one, compared above)."""
    p, _, _ = bench80
    H = o.Hierarchy(o.from_problem(p), 3, p.B, smoother="bjacobi")
    rp, cl, val, B = dev_args(p, torch)
    G = amg.AMG(rp, cl, val, B, smoother=amg.SMOOTH_BJACOBI)
    for l in range(H.nlevels - 1):
        ol, gi = H.level(l), G.level_info(l)
        assert abs(gi["smoother_lambda"] - ol["bj_lambda"]) <= 1e-10 * ol["bj_lambda"], l
        gMb = G.export(l)["Mb"]
        assert np.abs(gMb - ol["Mb"]).max() <= 1e-12 * np.abs(ol["Mb"]).max(), l
    it, ito = _pcg_parity(H, G, p.f)
    assert it > 10
