"""The scalar setup of Sec. 3/4's scalar and hybrid solvers (GPU required).

AMG_SETUP_SCALAR builds the hierarchy on scalar CSR rows (strength on the
node graph condensed from the scalar pattern, aggregation, tentative
prolongation, its smoothing, R = P^T, the Galerkin product and SPAI0 in
scalar arithmetic) and converts every level into blocks afterwards
(Listing 1).  With block storage the solve runs on those blocks ("NS
Hybrid1"); with scalar storage on the scalar matrices ("NS Scalar").  The
oracle is itself a scalar setup: both must match it level by level with the
same bars as the block setup, and solve to the same iterations.
"""
import numpy as np
import pytest

import oracle as o
import q1elasticity as q

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

amg = pytest.importorskip("paper_2202_09056_gb300")

from parity_util import compare_levels, dev_args  # noqa: E402

MESHES = [
    ((10, 10, 10), {"body": (0, 0, -1)}, 3000),
    ((7, 5, 9), {"traction": (0, 0, -1), "inclusion_frac": 0.2}, 200),
    ((12, 12, 12), {"traction": (0, 0, -1), "inclusion_frac": 0.2}, 300),
    ((26, 26, 26), {"traction": (0, 0, -1), "inclusion_frac": 0.2}, 3000),
]


def _pair(p, ce, aggregation="greedy", **gkw):
    H = o.Hierarchy(o.from_problem(p), 3, p.B, coarse_enough=ce, aggregation=aggregation)
    G = amg.AMG(*dev_args(p, torch), coarse_enough=ce, setup=amg.SETUP_SCALAR,
                aggregation={"greedy": amg.AGG_GREEDY, "mis2": amg.AGG_MIS2}[aggregation], **gkw)
    return H, G


def _pcg(H, G, f):
    uo, ito, _ = H.solve(f, tol=1e-8, maxiter=2000)
    u, it, res, st = G.solve(torch.from_numpy(f).cuda(), tol=1e-8, maxiter=2000)
    assert st == amg.AMG_OK and res <= 1e-8
    assert abs(it - ito) <= 1, (it, ito)
    assert np.linalg.norm(u.cpu().numpy() - uo) <= 1e-7 * np.linalg.norm(uo)
    return u, it


@pytest.mark.parametrize("shape,kw,ce", MESHES)
def test_hybrid1_hierarchy_and_solve_match_oracle(shape, kw, ce):
    """NS Hybrid1: scalar setup, block solve."""
    p = q.make_problem(shape, **kw)
    H, G = _pair(p, ce)
    compare_levels(H, G, 6)
    _pcg(H, G, p.f)


@pytest.mark.parametrize("shape,kw,ce", MESHES[1:3])
def test_ns_scalar_solve_matches_oracle_and_hybrid1(shape, kw, ce):
    """NS Scalar: scalar setup, scalar solve; the same iterations as the
    block solve of the same hierarchy, and the solve's scalar kernels against
    the oracle's operators."""
    p = q.make_problem(shape, **kw)
    H, G = _pair(p, ce, storage=amg.STORAGE_SCALAR)
    compare_levels(H, G, 6)
    u, it = _pcg(H, G, p.f)
    G1 = amg.AMG(*dev_args(p, torch), coarse_enough=ce, setup=amg.SETUP_SCALAR)
    u1, it1, _, _ = G1.solve(torch.from_numpy(p.f).cuda())
    assert it == it1 and torch.allclose(u, u1, rtol=0, atol=1e-9 * float(u1.abs().max()))
    rng = np.random.default_rng(3)
    for l in range(H.nlevels - 1):
        ol = H.level(l)
        nc = G.level_info(l)["nagg"] * 6
        for which, C, ny, nx in ((0, ol["A"], ol["n"], ol["n"]), (1, ol["P"], ol["n"], nc),
                                 (2, ol["R"], nc, ol["n"])):
            x = rng.standard_normal(nx)
            y = torch.empty(ny, dtype=torch.float64, device="cuda")
            G.level_spmv(l, which, torch.from_numpy(x).cuda(), y)
            ref = o.spmv(C, x)
            assert np.abs(y.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max(), (l, which)


def test_scalar_setup_equals_block_setup_bit_for_bit_patterns():
    """Both setups give the same hierarchy: aggregates, strength flags and
    patterns bit for bit, rho and omega on level 0 exactly (same sums in the
    same order), values to rounding."""
    p = q.make_problem((11, 9, 10), traction=(0, 0, -1), inclusion_frac=0.2)
    Gs = amg.AMG(*dev_args(p, torch), coarse_enough=200, setup=amg.SETUP_SCALAR)
    Gb = amg.AMG(*dev_args(p, torch), coarse_enough=200)
    assert Gs.nlevels == Gb.nlevels >= 3
    for l in range(Gb.nlevels):
        es, eb = Gs.export(l), Gb.export(l)
        for key in ("A", "P", "R"):
            if key in eb:
                assert np.array_equal(es[key][0], eb[key][0]) and np.array_equal(es[key][1], eb[key][1])
                scale = np.abs(eb[key][2]).max()
                assert np.abs(es[key][2] - eb[key][2]).max() <= 1e-12 * scale, (l, key)
        if "agg" in eb:
            assert np.array_equal(es["agg"], eb["agg"]) and np.array_equal(es["strong"], eb["strong"])
    i0s, i0b = Gs.level_info(0), Gb.level_info(0)
    assert i0s["rho"] == i0b["rho"] and i0s["omega"] == i0b["omega"]


def test_scalar_setup_with_mis2_matches_oracle():
    p = q.make_problem((12, 12, 12), traction=(0, 0, -1), inclusion_frac=0.2)
    H, G = _pair(p, 300, aggregation="mis2")
    compare_levels(H, G, 6)
    _pcg(H, G, p.f)


def test_scalar_setup_rejections():
    p = q.cube(4)
    args = dev_args(p, torch)
    with pytest.raises(amg.AmgError) as e:
        amg.AMG(*args, setup=amg.SETUP_SCALAR, smoother=amg.SMOOTH_ILU0)
    assert e.value.status == amg.AMG_ERR_ARG
    with pytest.raises(amg.AmgError) as e:
        amg.AMGBatch([args[:3]], [args[3]], [1], setup=amg.SETUP_SCALAR)
    assert e.value.status == amg.AMG_ERR_ARG
    with pytest.raises(amg.AmgError):
        amg.AMG(*args, setup=7)
