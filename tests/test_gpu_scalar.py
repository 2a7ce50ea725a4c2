"""Scalar storage of the solve's operators (the "NS Scalar" solver of Sec. 4,
on the block hierarchy) against the oracle and against block storage.

Bars: every level operator's scalar sliced SpMV equals the oracle's scalar
CSR product (1e-12 relative) and the block kernel's result (1e-13); the
scalar-storage PCG solution is within 1e-7 of the oracle's with iterations
within +-1 of it and of the block-storage solve; the reduced-precision
V-cycles converge in scalar storage too; the forms that need blocks refuse
scalar storage.
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


def test_scalar_level_spmv_matches_oracle_and_block_storage():
    p = q.make_problem((13, 9, 11), traction=(0, 0, -1), inclusion_frac=0.2)
    args = _dev(p)
    Gb = amg.AMG(*args, coarse_enough=150)
    Gs = amg.AMG(*args, coarse_enough=150, storage=amg.STORAGE_SCALAR)
    assert Gs.nlevels == Gb.nlevels
    # a column index per value instead of per block
    assert Gs.stats()["bytes_solve"] > 1.2 * Gb.stats()["bytes_solve"] > 0
    rng = np.random.default_rng(11)
    for l in range(Gb.nlevels - 1):
        ex = Gb.export(l)
        b, nagg, nb = ex["info"]["bs"], ex["info"]["nagg"], ex["info"]["nbrows"]
        for which, (mat, br, bc, ncols) in enumerate([(ex["A"], b, b, nb), (ex["P"], b, 6, nagg),
                                                       (ex["R"], 6, b, nb)]):
            x = torch.from_numpy(rng.standard_normal(ncols * bc)).cuda()
            ys = torch.empty((len(mat[0]) - 1) * br, dtype=torch.float64, device="cuda")
            yb = torch.empty_like(ys)
            Gs.level_spmv(l, which, x, ys)
            Gb.level_spmv(l, which, x, yb)
            ref = o.spmv(o.unblock(mat[0], mat[1], mat[2].reshape(len(mat[1]), -1), br, bc,
                                   nbcols=ncols), x.cpu().numpy())
            scale = np.abs(ref).max()
            assert np.abs(ys.cpu().numpy() - ref).max() <= 1e-12 * scale, (l, which)
            assert torch.abs(ys - yb).max().item() <= 1e-13 * scale, (l, which)


def test_scalar_storage_solve_matches_oracle():
    p = q.make_problem((12, 11, 10), traction=(0, 0, -1), inclusion_frac=0.2)
    H = o.Hierarchy(o.from_problem(p), 3, p.B, coarse_enough=300)
    uo, ito, _ = H.solve(p.f, tol=1e-8, maxiter=2000)
    args = _dev(p)
    fb = torch.from_numpy(p.f).cuda()
    ub, itb, _, sb = amg.AMG(*args, coarse_enough=300).solve(fb)
    us, its, res, ss = amg.AMG(*args, coarse_enough=300, storage=amg.STORAGE_SCALAR).solve(fb)
    assert sb == ss == amg.AMG_OK and res <= 1e-8
    assert abs(its - ito) <= 1 and abs(its - itb) <= 1, (its, ito, itb)
    un = us.cpu().numpy()
    assert np.linalg.norm(un - uo) <= 1e-7 * np.linalg.norm(uo)
    A = o.from_problem(p).to_scipy()
    assert np.linalg.norm(p.f - A @ un) / np.linalg.norm(p.f) <= 1.0001e-8


@pytest.mark.parametrize("prec", [amg.PREC_FP32, amg.PREC_BF16])
def test_scalar_storage_reduced_precision_converges(prec):
    p = q.make_problem((11, 10, 12), traction=(0, 0, -1), inclusion_frac=0.2)
    args = _dev(p)
    fb = torch.from_numpy(p.f).cuda()
    ub, itb, _, _ = amg.AMG(*args, coarse_enough=300, precision=prec).solve(fb)
    us, its, res, st = amg.AMG(*args, coarse_enough=300, precision=prec,
                               storage=amg.STORAGE_SCALAR).solve(fb)
    assert st == amg.AMG_OK and res <= 1e-8
    assert abs(its - itb) <= max(2, itb // 10), (its, itb)
    assert torch.linalg.norm(us - ub) <= 1e-6 * torch.linalg.norm(ub)


def test_block_only_forms_refuse_scalar_storage():
    p = q.make_problem((6, 6, 6), traction=(0, 0, -1))
    G = amg.AMG(*_dev(p), coarse_enough=150, storage=amg.STORAGE_SCALAR)
    with pytest.raises(amg.AmgError) as e:
        G.set_learned_smoother(amg.learned_init(0))
    assert e.value.status == amg.AMG_ERR_ARG
    d = torch.device("cuda:0")
    mats = [tuple(t for t in _dev(p)[:3])]
    with pytest.raises(amg.AmgError) as e:
        amg.AMGBatch(mats, [_dev(p)[3]], [1], storage=amg.STORAGE_SCALAR)
    assert e.value.status == amg.AMG_ERR_ARG


def test_scalar_galerkin_matches_block_galerkin():
    """The setup-phase side of the Sec. 4 comparison: A_{l+1} = R (A P)
    recomputed from the unblocked operators with 1x1 SpGEMMs has the unblocked
    block product's pattern and its values within 1e-12 (only the summation
    order differs); the block recomputation reproduces the hierarchy's bits.
    Covers the lane-group row kernel, the CTA-per-row kernel and the
    upper-triangle product with its mirror, in both storages."""
    p = q.make_problem((13, 9, 11), traction=(0, 0, -1), inclusion_frac=0.2)
    G = amg.AMG(*_dev(p), coarse_enough=150)
    assert G.nlevels >= 3
    for l in range(G.nlevels - 1):
        tb, db = G.galerkin_timing(l, amg.STORAGE_BLOCK)
        ts, ds = G.galerkin_timing(l, amg.STORAGE_SCALAR)
        assert db == 0.0, l
        assert 0.0 <= ds <= 1e-12, (l, ds)
        assert tb > 0 and ts > 0
    with pytest.raises(amg.AmgError):
        G.galerkin_timing(G.nlevels - 1)


@pytest.mark.slow
def test_scalar_galerkin_full_size_fine_level():
    """80^3: the fine level's scalar Galerkin product (22 372 x 6 scalar rows
    of R, 124 M scalar entries of A) against the hierarchy's block product."""
    p = q.inclusions(80)
    G = amg.AMG(*_dev(p))
    ts, ds = G.galerkin_timing(0, amg.STORAGE_SCALAR)
    assert 0.0 <= ds <= 1e-12, ds
