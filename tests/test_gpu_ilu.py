"""Block ILU(0) smoother on the GPU (the relaxation of Sec. 4's experiments)
against the oracle's block ILU(0) (GPU required).

Bars: the factor on every smoothing level within 1e-12 (level 0, identical
input bits) or 1e-10 (coarser levels, whose A_l carry the Galerkin rounding)
of its largest entry; the V-cycle within the coarse-solver bound used for
SPAI0; PCG solutions within 1e-7 with iteration counts within +-1; CG breaks
down on both sides where the oracle's does (too few sweeps, and the E = 1000
inclusion meshes, where ILU(0) itself is indefinite).
"""
import numpy as np
import pytest

import oracle as o
import q1elasticity as q

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

amg = pytest.importorskip("paper_2202_09056_gb300")


def _dev(p):
    d = torch.device("cuda:0")
    return (torch.from_numpy(p.row_ptr).to(d), torch.from_numpy(p.col).to(d),
            torch.from_numpy(p.val).to(d), torch.from_numpy(p.B).to(d))


def _pair(p, ce, sweeps):
    H = o.Hierarchy(o.from_problem(p), 3, p.B, coarse_enough=ce, smoother="ilu0",
                    ilu_sweeps=sweeps)
    G = amg.AMG(*_dev(p), coarse_enough=ce, smoother=amg.SMOOTH_ILU0, ilu_sweeps=sweeps)
    assert G.nlevels == H.nlevels
    return H, G


@pytest.mark.parametrize("shape,kw,ce", [
    ((8, 8, 8), {"body": (0, 0, -1)}, 300),
    ((7, 5, 9), {"traction": (0, 0, -1), "inclusion_frac": 0.2}, 200),
    ((12, 12, 12), {"body": (0, 0, -1)}, 300),
])
def test_ilu_factor_matches_oracle(shape, kw, ce):
    """The factor of every smoothing level (3x3 fine blocks, 6x6 coarse
    blocks, rows over many dependency levels and CTAs) against the oracle's
    factorisation of the oracle's own level matrix."""
    p = q.make_problem(shape, **kw)
    H, G = _pair(p, ce, 3)
    assert H.nlevels >= 2
    for l in range(H.nlevels - 1):
        ol = H.level(l)
        F = o.ILU0(ol["A"], ol["b"])
        ptr, col, val, dinv = F.factors()
        gA = G.export(l)["A"]
        assert np.array_equal(gA[0], ptr) and np.array_equal(gA[1], col), l
        gF, gD = G.ilu_factor(l)
        tol = 1e-12 if l == 0 else 1e-10
        assert np.abs(gF - val).max() <= tol * np.abs(val).max(), l
        assert np.abs(gD - dinv).max() <= tol * np.abs(dinv).max(), l


@pytest.mark.parametrize("sweeps", [0, 2, 3])
def test_ilu_vcycle_matches_oracle(sweeps):
    p = q.cube(8)
    H, G = _pair(p, 300, sweeps)
    rng = np.random.default_rng(sweeps)
    L, _ = H.coarse_factor()
    d = np.diag(L)
    cond_est = (d.max() / d[d > 0].min()) ** 2
    for _ in range(2):
        r = rng.standard_normal(p.ndof)
        z = G.vcycle(torch.from_numpy(r).cuda()).cpu().numpy()
        zo = H.vcycle(r)
        assert np.linalg.norm(z - zo) <= max(1e-12, 100 * cond_est * 1e-16) * np.linalg.norm(zo)


@pytest.mark.parametrize("shape,kw,ce", [
    ((8, 8, 8), {"body": (0, 0, -1)}, 300),
    ((10, 10, 10), {"body": (0, 0, -1)}, 3000),
    ((12, 12, 12), {"body": (0, 0, -1)}, 300),
])
def test_ilu_pcg_matches_oracle(shape, kw, ce):
    """Three sweeps per triangle on homogeneous cubes: the same iterations and
    solution as the oracle, and fewer iterations than SPAI0."""
    p = q.make_problem(shape, **kw)
    H, G = _pair(p, ce, 3)
    uo, ito, _ = H.solve(p.f, tol=1e-8, maxiter=1000)
    fb = torch.from_numpy(p.f).cuda()
    u, it, res, st = G.solve(fb, tol=1e-8, maxiter=1000)
    assert st == amg.AMG_OK and res <= 1e-8
    assert abs(it - ito) <= 1, (it, ito)
    assert np.linalg.norm(u.cpu().numpy() - uo) <= 1e-7 * np.linalg.norm(uo)
    _, it_spai0, _, _ = amg.AMG(*_dev(p), coarse_enough=ce).solve(fb)
    assert it < it_spai0


@pytest.mark.parametrize("p,sweeps", [
    (lambda: q.cube(8), 2),
    (lambda: q.make_problem((7, 5, 9), traction=(0, 0, -1), inclusion_frac=0.2), 3),
])
def test_ilu_breaks_down_where_the_oracle_does(p, sweeps):
    p = p()
    ce = 300 if p.nnodes > 400 else 200
    H, G = _pair(p, ce, sweeps)
    with pytest.raises(RuntimeError):
        H.solve(p.f, maxiter=3000)
    with pytest.raises(amg.AmgError) as e:
        G.solve(torch.from_numpy(p.f).cuda(), maxiter=3000)
    assert e.value.status == amg.AMG_ERR_BREAKDOWN


def test_ilu_is_rejected_outside_the_fp64_block_vcycle():
    p = q.cube(4)
    for kw in ({"precision": amg.PREC_FP32}, {"storage": amg.STORAGE_SCALAR},
               {"ilu_sweeps": 65}):
        with pytest.raises(amg.AmgError) as e:
            amg.AMG(*_dev(p), coarse_enough=30, smoother=amg.SMOOTH_ILU0, **kw)
        assert e.value.status == amg.AMG_ERR_ARG
    G = amg.AMG(*_dev(p), coarse_enough=30, smoother=amg.SMOOTH_ILU0)
    with pytest.raises(amg.AmgError):
        G.ilu_factor(G.nlevels - 1)  # the coarsest level has no smoother
