"""Block damped Jacobi smoother on the GPU against the oracle (GPU required).

Bars: the hierarchy as in the other parity tests (patterns, aggregates and
strength flags bit-exact, values within 1e-12); the level-0 undamped
inverse blocks within 1e-14 of the oracle's (the same Gauss-Jordan sequence,
each product and sum rounded on its own) and every level's damped blocks
within 1e-12 (the damping comes from a power iteration whose dot products
are reduced in another order); the lambda estimates within 1e-10; the
V-cycle within the bound set by the coarse solver; PCG iterations within +-1
and the solution within 1e-7; the reduced-precision V-cycles reach the same
true residual with no more iterations than FP64 (emulated FP64), at most two
more (FP32) or twelve more (BF16-stored values).
"""
import numpy as np
import pytest

import oracle as o
import q1elasticity as q

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
amg = pytest.importorskip("paper_2202_09056_gb300")

from parity_util import compare_levels, dev_args, rel, vcycle_bound  # noqa: E402


def _pair(p, ce, **kw):
    H = o.Hierarchy(o.from_problem(p), 3, p.B, coarse_enough=ce, smoother="bjacobi")
    G = amg.AMG(*dev_args(p, torch), coarse_enough=ce, smoother=amg.SMOOTH_BJACOBI, **kw)
    return H, G


CASES = [
    ((6, 5, 7), {"body": (0, 0, -1), "inclusion_frac": 0.2}, 150),
    ((12, 12, 12), {"traction": (0, 0, -1), "inclusion_frac": 0.2}, 300),
    ((9, 8, 10), {"body": (0, 0, -1), "nu": 0.45}, 200),
]


@pytest.mark.parametrize("shape,kw,ce", CASES)
def test_hierarchy_and_blocks_match_oracle(shape, kw, ce):
    p = q.make_problem(shape, **kw)
    H, G = _pair(p, ce)
    compare_levels(H, G, p.B.shape[1])
    for l in range(H.nlevels - 1):
        ol, gl = H.level(l), G.export(l)
        gi = G.level_info(l)
        assert abs(gi["smoother_lambda"] - ol["bj_lambda"]) <= 1e-10 * ol["bj_lambda"], l
        assert gl["Mb"].shape == ol["Mb"].shape, l
        assert rel(gl["Mb"], ol["Mb"]) <= 1e-12, l
        # undamped inverses: the same elimination sequence as the oracle's
        if l == 0:
            w_g = 2 * 0.8 / gi["smoother_lambda"]
            w_o = 2 * 0.8 / ol["bj_lambda"]
            Wo = o.block_jacobi(ol["A"], 3, 1.0)
            np.testing.assert_allclose(gl["Mb"] / w_g, Wo, rtol=1e-14, atol=0)
            np.testing.assert_allclose(ol["Mb"] / w_o, Wo, rtol=1e-14, atol=0)


@pytest.mark.parametrize("shape,kw,ce", CASES)
def test_vcycle_and_pcg_match_oracle(shape, kw, ce):
    p = q.make_problem(shape, **kw)
    H, G = _pair(p, ce)
    rng = np.random.default_rng(21)
    r = rng.standard_normal(p.ndof)
    z = G.vcycle(torch.from_numpy(r).cuda()).cpu().numpy()
    zo = H.vcycle(r)
    assert np.linalg.norm(z - zo) <= vcycle_bound(H) * np.linalg.norm(zo)
    uo, ito, _ = H.solve(p.f, tol=1e-8, maxiter=2000)
    u, it, res, st = G.solve(torch.from_numpy(p.f).cuda(), tol=1e-8, maxiter=2000)
    assert st == amg.AMG_OK and res <= 1e-8 and abs(it - ito) <= 1, (it, ito)
    assert np.linalg.norm(u.cpu().numpy() - uo) <= 1e-7 * np.linalg.norm(uo)
    # fewer iterations than SPAI0 on these meshes (oracle, same hierarchy)
    _, it0, _ = o.Hierarchy(o.from_problem(p), 3, p.B, coarse_enough=ce).solve(p.f, tol=1e-8)
    assert ito < it0, (ito, it0)


@pytest.mark.parametrize("prec", ["fp32", "bf16", "df64"])
def test_reduced_precision_vcycles_with_blocks(prec):
    p = q.make_problem((12, 12, 12), traction=(0, 0, -1), inclusion_frac=0.2)
    f = torch.from_numpy(p.f).cuda()
    _, G64 = _pair(p, 300)
    u64, it64, _, _ = G64.solve(f, tol=1e-8)
    pr = {"fp32": amg.PREC_FP32, "bf16": amg.PREC_BF16, "df64": amg.PREC_DF64}[prec]
    G = amg.AMG(*dev_args(p, torch), coarse_enough=300, smoother=amg.SMOOTH_BJACOBI, precision=pr)
    u, it, res, st = G.solve(f, tol=1e-8)
    A = o.from_problem(p).to_scipy()
    un = u.cpu().numpy()
    assert st == amg.AMG_OK and np.linalg.norm(p.f - A @ un) <= 1.0001e-8 * np.linalg.norm(p.f)
    assert it <= it64 + (0 if prec == "df64" else (12 if prec == "bf16" else 2)), (it, it64)
    assert np.linalg.norm(un - u64.cpu().numpy()) <= 1e-6 * np.linalg.norm(un)


def test_solve_is_reproducible_and_loop_mode_equal():
    p = q.make_problem((10, 9, 8), body=(0, 0, -1), inclusion_frac=0.2)
    f = torch.from_numpy(p.f).cuda()
    _, G = _pair(p, 200)
    u1, i1, r1, _ = G.solve(f)
    u2, i2, r2, _ = G.solve(f)
    assert i1 == i2 and r1 == r2 and torch.equal(u1, u2)
    _, G1 = _pair(p, 200, loop_mode=1)
    u3, i3, r3, _ = G1.solve(f)
    assert i3 == i1 and torch.equal(u3, u1)


def test_rejections():
    p = q.make_problem((5, 5, 5), body=(0, 0, -1))
    args = dev_args(p, torch)
    with pytest.raises(amg.AmgError) as e:
        amg.AMG(*args, coarse_enough=100, smoother=amg.SMOOTH_BJACOBI, storage=amg.STORAGE_SCALAR)
    assert e.value.status == amg.AMG_ERR_ARG
    with pytest.raises(amg.AmgError) as e:
        amg.AMG(*args, coarse_enough=100, smoother=amg.SMOOTH_BJACOBI, smooth_relax=0.0)
    assert e.value.status == amg.AMG_ERR_ARG
    G = amg.AMG(*args, coarse_enough=100, smoother=amg.SMOOTH_BJACOBI)
    with pytest.raises(amg.AmgError) as e:
        G.set_learned_smoother(amg.learned_init())
    assert e.value.status == amg.AMG_ERR_STATE
    with pytest.raises(amg.AmgError):  # the batch takes SPAI0 or block Jacobi only
        amg.AMGBatch([args[:3]], [args[3]], [1], coarse_enough=100, smoother=amg.SMOOTH_ILU0)


@pytest.mark.parametrize("variant", ["translations", "mis2"])
def test_block_jacobi_with_translations_or_mis2(variant):
    """Block Jacobi on the other hierarchies: the three translations as the
    near-nullspace (3x3 blocks on every level) and MIS-2 aggregation; PCG
    against the oracle's block Jacobi solve on the same hierarchy."""
    p = q.make_problem((11, 10, 12), traction=(0, 0, -1), inclusion_frac=0.2)
    if variant == "translations":
        B = np.zeros((p.ndof, 3))
        for c in range(3):
            B[c::3, c] = 1.0
        okw, gkw = {}, {}
    else:
        B = p.B
        okw, gkw = {"aggregation": "mis2"}, {"aggregation": amg.AGG_MIS2}
    H = o.Hierarchy(o.from_problem(p), 3, B, coarse_enough=200, smoother="bjacobi", **okw)
    rp, cl, val, _ = dev_args(p, torch)
    G = amg.AMG(rp, cl, val, torch.from_numpy(B).cuda(), coarse_enough=200,
                smoother=amg.SMOOTH_BJACOBI, **gkw)
    assert G.nlevels == H.nlevels >= 2
    for l in range(H.nlevels - 1):
        assert G.level_info(l)["bs"] == H.level(l)["b"]
        assert rel(G.export(l)["Mb"], H.level(l)["Mb"]) <= 1e-12, l
    uo, ito, _ = H.solve(p.f, tol=1e-8, maxiter=3000)
    u, it, res, st = G.solve(torch.from_numpy(p.f).cuda(), tol=1e-8, maxiter=3000)
    assert st == amg.AMG_OK and res <= 1e-8 and abs(it - ito) <= 1, (it, ito)
    assert np.linalg.norm(u.cpu().numpy() - uo) <= 1e-7 * np.linalg.norm(uo)
