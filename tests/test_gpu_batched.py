"""Batched form (GPU): independent instances with several load cases each.

Bars: every (instance, rhs) solution within 1e-7 of the FP64 oracle's
solution of that system, iterations within +-1; an instance solved inside a
batch is bitwise identical (iterations and solution) to the same instance and
right-hand side solved alone through the batched path; zero right-hand sides
give zero solutions.
"""
import numpy as np
import pytest

import oracle as o
import q1elasticity as q

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
amg = pytest.importorskip("paper_2202_09056_gb300")


def _instances():
    specs = [((6, 5, 7), 0.25, 3), ((9, 9, 9), 0.3, 1), ((8, 6, 10), 0.42, 5), ((5, 5, 5), 0.33, 2)]
    out = []
    for k, (shape, nu, nrhs) in enumerate(specs):
        dirs, _ = q.splitmix64_uniform(100 + k, 3 * nrhs)
        body = (dirs.reshape(nrhs, 3) - 0.5)
        p = q.make_problem(shape, nu=nu, body=body, inclusion_frac=0.2 if k % 2 else 0.0)
        out.append((p, nrhs))
    return out


def _dev(p):
    d = torch.device("cuda:0")
    return (torch.from_numpy(p.row_ptr).to(d), torch.from_numpy(p.col).to(d),
            torch.from_numpy(p.val).to(d)), torch.from_numpy(p.B).to(d)


def test_batch_matches_oracle_per_rhs():
    inst = _instances()
    mats, Bs, nrhs, F = [], [], [], []
    for p, k in inst:
        m, B = _dev(p)
        mats.append(m)
        Bs.append(B)
        nrhs.append(k)
        F.append(torch.from_numpy(np.atleast_2d(p.f).copy()).cuda())
    bat = amg.AMGBatch(mats, Bs, nrhs, coarse_enough=150)
    U, its, res, st = bat.solve(F, tol=1e-8)
    assert st == amg.AMG_OK
    info = bat.info()
    assert info["ninst"] == 4 and info["nrhs_total"] == sum(nrhs)
    assert all(t in (1, 2, 4) for lev in info["rhs_tile"] for t in lev)
    # the autotuned launch shape of every present operator (0: absent)
    assert all(c in (0, 64, 128, 256) for lev in info["cta_threads"] for c in lev)
    assert all(c in (0, 16, 32) for lev in info["ctas_per_sm"] for c in lev)
    assert info["cta_threads"][0][0] in (64, 128, 256)
    for i, (p, k) in enumerate(inst):
        H = o.Hierarchy(o.from_problem(p), 3, p.B, coarse_enough=150)
        fs = np.atleast_2d(p.f)
        for j in range(k):
            uo, ito, _ = H.solve(fs[j], tol=1e-8)
            u = U[i][j].cpu().numpy()
            assert res[i][j] <= 1e-8
            assert abs(its[i][j] - ito) <= 1, (i, j, its[i][j], ito)
            assert np.linalg.norm(u - uo) <= 1e-7 * np.linalg.norm(uo), (i, j)


@pytest.mark.parametrize("prec", ["fp64", "df64", "fp32", "fp64_bjacobi", "fp32_bjacobi"])
def test_instance_in_batch_equals_instance_alone(prec):
    """In every V-cycle precision (the coarse solve included) and with either
    smoother, an (instance, rhs) pair gives bitwise the same iterates in the
    batch as alone."""
    bj = {"smoother": amg.SMOOTH_BJACOBI}
    kw = {"fp64": {}, "df64": {"precision": amg.PREC_DF64},
          "fp32": {"precision": amg.PREC_FP32}, "fp64_bjacobi": bj,
          "fp32_bjacobi": dict(bj, precision=amg.PREC_FP32)}[prec]
    inst = _instances()
    mats, Bs, nrhs, F = [], [], [], []
    for p, k in inst:
        m, B = _dev(p)
        mats.append(m)
        Bs.append(B)
        nrhs.append(k)
        F.append(torch.from_numpy(np.atleast_2d(p.f).copy()).cuda())
    bat = amg.AMGBatch(mats, Bs, nrhs, coarse_enough=150, **kw)
    U, its, res, _ = bat.solve(F, tol=1e-8)
    for i in (0, 2):
        for j in range(nrhs[i]):
            one = amg.AMGBatch([mats[i]], [Bs[i]], [1], coarse_enough=150, **kw)
            U1, it1, res1, _ = one.solve([F[i][j:j + 1].clone()], tol=1e-8)
            assert it1[0][0] == its[i][j]
            assert torch.equal(U1[0][0], U[i][j]), (i, j)
            assert res1[0][0] == res[i][j]


def test_batch_with_block_jacobi_matches_oracle_per_rhs():
    """Block damped Jacobi in the batched V-cycle (block smoothing epilogue,
    block pre-smoothing in the restriction, level-0 block product): every
    (instance, rhs) within 1e-7 of the oracle's block Jacobi solve, iterations
    within +-1, and fewer iterations than the SPAI0 batch in total."""
    inst = _instances()
    mats, Bs, nrhs, F = [], [], [], []
    for p, k in inst:
        m, B = _dev(p)
        mats.append(m)
        Bs.append(B)
        nrhs.append(k)
        F.append(torch.from_numpy(np.atleast_2d(p.f).copy()).cuda())
    bat = amg.AMGBatch(mats, Bs, nrhs, coarse_enough=150, smoother=amg.SMOOTH_BJACOBI)
    U, its, res, st = bat.solve(F, tol=1e-8)
    assert st == amg.AMG_OK
    _, its0, _, _ = amg.AMGBatch(mats, Bs, nrhs, coarse_enough=150).solve(F, tol=1e-8)
    assert sum(map(sum, its)) < sum(map(sum, its0)), (its, its0)
    for i, (p, k) in enumerate(inst):
        H = o.Hierarchy(o.from_problem(p), 3, p.B, coarse_enough=150, smoother="bjacobi")
        fs = np.atleast_2d(p.f)
        for j in range(k):
            uo, ito, _ = H.solve(fs[j], tol=1e-8)
            u = U[i][j].cpu().numpy()
            assert res[i][j] <= 1e-8
            assert abs(its[i][j] - ito) <= 1, (i, j, its[i][j], ito)
            assert np.linalg.norm(u - uo) <= 1e-7 * np.linalg.norm(uo), (i, j)


def test_failing_instance_is_named():
    """Instances are set up by several host threads at once; a batch with two
    bad instances (a NaN in A) reports the lower-numbered one, every time."""
    mats, Bs = [], []
    for k, shape in enumerate(((5, 5, 5), (6, 5, 4), (4, 4, 6), (5, 6, 5), (4, 5, 4))):
        p = q.make_problem(shape, body=(0, 0, -1))
        (rp, cl, val), B = _dev(p)
        if k in (1, 3):
            val = val.clone()
            val[3, 1, 1] = float("nan")
        mats.append((rp, cl, val))
        Bs.append(B)
    for _ in range(3):
        with pytest.raises(amg.AmgError) as e:
            amg.AMGBatch(mats, Bs, [1] * 5, coarse_enough=100)
        assert e.value.status == amg.AMG_ERR_ARG
        assert str(e.value).count("instance 1: A or B holds a non-finite value") == 1, str(e.value)
    # the good instances alone still set up and solve
    good = [0, 2, 4]
    bat = amg.AMGBatch([mats[i] for i in good], [Bs[i] for i in good], [1] * 3, coarse_enough=100)
    assert bat.info()["ninst"] == 3


def test_batch_zero_rhs_and_cap():
    p = q.make_problem((5, 4, 6), body=[(0, 0, -1), (0, 0, 0), (1, 0, 0)])
    m, B = _dev(p)
    F = torch.from_numpy(p.f.copy()).cuda()
    bat = amg.AMGBatch([m], [B], [3], coarse_enough=100)
    U, its, res, st = bat.solve([F], tol=1e-8)
    assert st == amg.AMG_OK
    assert its[0][1] == 0 and not U[0][1].any()
    U, its, res, st = bat.solve([F], tol=1e-14, maxiter=2)
    assert st == amg.AMG_NOT_CONVERGED and its[0][0] == 2


def test_host_loop_mode_gives_identical_batch_results():
    """loop_mode 1 (one captured iteration per host launch, for profilers)
    runs the same kernels: the same bits as the device-side loop."""
    specs = q.batch_specs(3, seed=11, nmin=5, nmax=8, rhs_max=3)
    d = torch.device("cuda:0")
    mats, Bs, F, nrhs = [], [], [], []
    for sp in specs:
        p = q.make_problem(sp["n"], nu=sp["nu"], body=sp["body"])
        mats.append((torch.from_numpy(p.row_ptr).to(d), torch.from_numpy(p.col).to(d),
                     torch.from_numpy(p.val).to(d)))
        Bs.append(torch.from_numpy(p.B).to(d))
        F.append(torch.from_numpy(np.atleast_2d(p.f).copy()).to(d))
        nrhs.append(sp["nrhs"])
    U0, it0, r0, s0 = amg.AMGBatch(mats, Bs, nrhs, coarse_enough=150).solve(F)
    U1, it1, r1, s1 = amg.AMGBatch(mats, Bs, nrhs, coarse_enough=150, loop_mode=1).solve(F)
    assert s0 == s1 == amg.AMG_OK and it0 == it1 and r0 == r1
    assert all(torch.equal(a, b) for a, b in zip(U0, U1))


def test_emulated_fp64_batch_matches_oracle_and_fp64_batch():
    """PREC_DF64 batch: the V-cycle's SpMMs on FP32-pair values (the CG's A p
    and true residual stay FP64).  Every (instance, rhs) meets the oracle's
    bars; iterations within +-1 of the FP64 batch and solutions within 1e-9
    of it (the emulated V-cycle matches FP64 to about 1e-13)."""
    inst = _instances()
    mats, Bs, nrhs, F = [], [], [], []
    for p, k in inst:
        m, B = _dev(p)
        mats.append(m)
        Bs.append(B)
        nrhs.append(k)
        F.append(torch.from_numpy(np.atleast_2d(p.f).copy()).cuda())
    U, its, res, st = amg.AMGBatch(mats, Bs, nrhs, coarse_enough=150,
                                   precision=amg.PREC_DF64).solve(F, tol=1e-8)
    U64, its64, _, st64 = amg.AMGBatch(mats, Bs, nrhs, coarse_enough=150).solve(F, tol=1e-8)
    assert st == st64 == amg.AMG_OK
    for i, (p, k) in enumerate(inst):
        H = o.Hierarchy(o.from_problem(p), 3, p.B, coarse_enough=150)
        fs = np.atleast_2d(p.f)
        for j in range(k):
            uo, ito, _ = H.solve(fs[j], tol=1e-8)
            u = U[i][j].cpu().numpy()
            assert res[i][j] <= 1e-8
            assert abs(its[i][j] - ito) <= 1 and abs(its[i][j] - its64[i][j]) <= 1, (i, j)
            assert np.linalg.norm(u - uo) <= 1e-7 * np.linalg.norm(uo), (i, j)
            u64 = U64[i][j].cpu().numpy()
            assert np.linalg.norm(u - u64) <= 1e-9 * np.linalg.norm(u64), (i, j)
    with pytest.raises(amg.AmgError):
        amg.AMGBatch(mats, Bs, nrhs, coarse_enough=150, precision=amg.PREC_BF16)


def test_fp32_batch_solves_to_fp64_accuracy():
    """PREC_FP32 batch: the V-cycle's SpMMs on FP32 values with FP32 FMAs (x
    rounded to FP32, FP64 vectors), the CG in FP64.  Every (instance, rhs)
    reaches a host-checked true residual of 1e-8; against the oracle the bars
    of the single-instance FP32 form (solution within 1e-6, iterations at most
    1.5x + 5)."""
    inst = _instances()
    mats, Bs, nrhs, F = [], [], [], []
    for p, k in inst:
        m, B = _dev(p)
        mats.append(m)
        Bs.append(B)
        nrhs.append(k)
        F.append(torch.from_numpy(np.atleast_2d(p.f).copy()).cuda())
    U, its, res, st = amg.AMGBatch(mats, Bs, nrhs, coarse_enough=150,
                                   precision=amg.PREC_FP32).solve(F, tol=1e-8)
    assert st == amg.AMG_OK
    for i, (p, k) in enumerate(inst):
        H = o.Hierarchy(o.from_problem(p), 3, p.B, coarse_enough=150)
        A = o.from_problem(p).to_scipy()
        fs = np.atleast_2d(p.f)
        for j in range(k):
            uo, ito, _ = H.solve(fs[j], tol=1e-8)
            u = U[i][j].cpu().numpy()
            assert res[i][j] <= 1e-8
            assert np.linalg.norm(fs[j] - A @ u) <= 1.0001e-8 * np.linalg.norm(fs[j]), (i, j)
            assert its[i][j] <= 1.5 * ito + 5, (i, j, its[i][j], ito)
            assert np.linalg.norm(u - uo) <= 1e-6 * np.linalg.norm(uo), (i, j)
