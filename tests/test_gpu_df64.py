"""FP64 emulated on FP32 pairs (AMG_PREC_DF64) against the FP64 oracle (GPU
required).

Every solve-phase matrix is stored as hi + lo floats (the FP64 value with its
significand truncated to 48 bits), x is split the same way on the fly, each
product is formed in FP32 (error-free product of the his, the cross terms
added to its error) and summed in double-float arithmetic (two-sum of the
his, the los added to its error, fast two-sum renormalisation).  Per product
the relative error is below 2^-45 (two truncations of 2^-47, the dropped
lo*lo term and the FP32 roundings of the error terms); each addition rounds
the low part, at most 2^-46 of the running sum plus the term.  A row of n_i
terms therefore obeys the rigorous bound
    |y_i - (A x)_i| <= (n_i + 2) 2^-45 (|A| |x|)_i,
checked on every row, with |A| |x| from the oracle; the errors are random in
sign, so the median row sits far below it, at <= 2^-44 (|A| |x|)_i, which a
lost or misplaced low part (errors near 2^-24) cannot meet.  The V-cycle
runs on these copies while the CG's A p stays FP64; the solve then matches
the oracle like the FP64 path: iterations within +-1 and the solution within
1e-7.
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


def _check_rows(y, M, x):
    ref = o.spmv(M, x)
    absM = o.CSR(M.ptr, M.col, np.abs(M.val), M.shape)
    ax = o.spmv(absM, np.abs(x))
    nterms = np.diff(np.asarray(M.ptr))
    err = np.abs(y - ref)
    assert np.all(err <= (nterms + 2) * 2.0 ** -45 * ax), np.max(err / np.maximum(ax, 1e-300))
    live = ax > 0
    assert np.median(err[live] / ax[live]) <= 2.0 ** -44


def _x(rng, n):
    """Random signs and magnitudes over 40 binades, with exact zeros and
    values whose low part is zero (exactly representable in FP32)."""
    x = rng.standard_normal(n) * np.exp2(rng.integers(-20, 20, n))
    x[rng.choice(n, n // 10, replace=False)] = 0.0
    k = rng.choice(n, n // 10, replace=False)
    x[k] = np.float32(x[k]).astype(np.float64)
    return x


def test_df64_level_spmv_bound_on_every_operator():
    """A (3x3 and 6x6), P (3x6, 6x6) and R (6x3, 6x6) of every level, with the
    lane counts and multi-warp rows the solve uses."""
    p = q.make_problem((13, 9, 11), traction=(0, 0, -1), inclusion_frac=0.2)
    G = amg.AMG(*_dev(p), coarse_enough=150, precision=amg.PREC_DF64)
    assert G.nlevels >= 3
    rng = np.random.default_rng(11)
    for l in range(G.nlevels - 1):
        ex = G.export(l)
        b, nagg, nb = ex["info"]["bs"], ex["info"]["nagg"], ex["info"]["nbrows"]
        for which, (mat, br, bc, ncols) in enumerate([(ex["A"], b, b, nb), (ex["P"], b, 6, nagg),
                                                       (ex["R"], 6, b, nb)]):
            M = o.unblock(mat[0], mat[1], mat[2].reshape(len(mat[1]), -1), br, bc, nbcols=ncols)
            x = _x(rng, ncols * bc)
            y = torch.empty((len(mat[0]) - 1) * br, dtype=torch.float64, device="cuda")
            G.level_spmv(l, 3 + which, torch.from_numpy(x).cuda(), y)
            _check_rows(y.cpu().numpy(), M, x)


def test_df64_flushes_below_fp32_range():
    """Entries of x below 2^-126 in magnitude are flushed to zero by the split
    (the documented range of the emulation): the product equals the one with
    those entries zeroed, within the bound."""
    p = q.make_problem((6, 5, 7), traction=(0, 0, -1), inclusion_frac=0.2)
    G = amg.AMG(*_dev(p), coarse_enough=60, precision=amg.PREC_DF64)
    rng = np.random.default_rng(2)
    x = rng.standard_normal(p.ndof)
    tiny = rng.choice(p.ndof, 50, replace=False)
    x[tiny] = 1e-300
    y = torch.empty(p.ndof, dtype=torch.float64, device="cuda")
    G.level_spmv(0, 3, torch.from_numpy(x).cuda(), y)
    xz = x.copy()
    xz[tiny] = 0.0
    _check_rows(y.cpu().numpy(), o.from_problem(p), xz)


def test_df64_requires_its_precision():
    p = q.cube(4)
    G = amg.AMG(*_dev(p), coarse_enough=30)
    y = torch.empty(p.ndof, dtype=torch.float64, device="cuda")
    with pytest.raises(amg.AmgError) as e:
        G.level_spmv(0, 3, torch.zeros(p.ndof, dtype=torch.float64, device="cuda"), y)
    assert e.value.status == amg.AMG_ERR_STATE


@pytest.mark.parametrize("shape,kw,ce", [
    ((10, 10, 10), {"body": (0, 0, -1)}, 3000),
    ((12, 12, 12), {"traction": (0, 0, -1), "inclusion_frac": 0.2}, 300),
    ((11, 6, 8), {"traction": (0, 0, -1), "inclusion_frac": 0.2}, 150),
])
def test_df64_pcg_matches_oracle(shape, kw, ce):
    p = q.make_problem(shape, **kw)
    H = o.Hierarchy(o.from_problem(p), 3, p.B, coarse_enough=ce)
    uo, ito, _ = H.solve(p.f, tol=1e-8, maxiter=1000)
    G = amg.AMG(*_dev(p), coarse_enough=ce, precision=amg.PREC_DF64)
    u, it, res, st = G.solve(torch.from_numpy(p.f).cuda(), tol=1e-8, maxiter=1000)
    assert st == amg.AMG_OK and res <= 1e-8
    assert abs(it - ito) <= 1, (it, ito)
    un = u.cpu().numpy()
    assert np.linalg.norm(un - uo) <= 1e-7 * np.linalg.norm(uo)
    A = o.from_problem(p).to_scipy()
    assert np.linalg.norm(p.f - A @ un) / np.linalg.norm(p.f) <= 1.0001e-8
    # one V-cycle against the oracle's: the same bound as the FP64 path's
    # coarse-solver term plus the emulation's per-product error carried
    # through the smoothers and transfers (1e-11)
    r = np.random.default_rng(4).standard_normal(p.ndof)
    z = G.vcycle(torch.from_numpy(r).cuda()).cpu().numpy()
    zo = H.vcycle(r)
    L, _ = H.coarse_factor()
    d = np.diag(L)
    cond_est = (d.max() / d[d > 0].min()) ** 2
    assert np.linalg.norm(z - zo) <= max(1e-11, 100 * cond_est * 1e-16) * np.linalg.norm(zo)


@pytest.mark.slow
def test_df64_full_size_inclusions_80():
    """80^3 elements: 200 sampled rows of the fine FP32-pair SpMV recomputed
    on the host within the bound, and the DF64 solve (the same 92 iterations
    as FP64) confirmed with a host SpMV."""
    p = q.inclusions(80)
    G = amg.AMG(*_dev(p), precision=amg.PREC_DF64)
    rng = np.random.default_rng(80)
    x = rng.standard_normal(p.ndof)
    y = torch.empty(p.ndof, dtype=torch.float64, device="cuda")
    G.level_spmv(0, 3, torch.from_numpy(x).cuda(), y)
    y = y.cpu().numpy()
    for I in rng.choice(p.nnodes, 200, replace=False):
        s, e = p.row_ptr[I], p.row_ptr[I + 1]
        ref = sum(p.val[k] @ x[3 * p.col[k]:3 * p.col[k] + 3] for k in range(s, e))
        ax = sum(np.abs(p.val[k]) @ np.abs(x[3 * p.col[k]:3 * p.col[k] + 3]) for k in range(s, e))
        assert np.all(np.abs(y[3 * I:3 * I + 3] - ref) <= (3 * (e - s) + 2) * 2.0 ** -45 * ax)
    u, it, res, st = G.solve(torch.from_numpy(p.f).cuda(), tol=1e-8, maxiter=2000)
    assert st == amg.AMG_OK
    _, it64, _, _ = amg.AMG(*_dev(p)).solve(torch.from_numpy(p.f).cuda(), tol=1e-8, maxiter=2000)
    assert abs(it - it64) <= 1, (it, it64)
    import scipy.sparse as sp
    A = sp.bsr_matrix((p.val, p.col, p.row_ptr), shape=(p.ndof, p.ndof))
    un = u.cpu().numpy()
    assert np.linalg.norm(p.f - A @ un) / np.linalg.norm(p.f) <= 1.0001e-8


def test_df64_with_scalar_storage_and_learned_blocks():
    """The pair kernels in the other layouts the V-cycle uses: scalar (1x1)
    storage of every operator, and the learned 3x3 smoother blocks applied in
    the SpMV epilogue.  Each matches the FP64 V-cycle with the same setting:
    iterations within +-1, solutions within 1e-9."""
    p = q.make_problem((10, 9, 8), traction=(0, 0, -1), inclusion_frac=0.2)
    fb = torch.from_numpy(p.f).cuda()
    for kw in ({"storage": amg.STORAGE_SCALAR}, {}):
        G = amg.AMG(*_dev(p), coarse_enough=200, precision=amg.PREC_DF64, **kw)
        G64 = amg.AMG(*_dev(p), coarse_enough=200, **kw)
        if not kw:
            w = amg.learned_init(5)
            rng = np.random.default_rng(5)
            w[64 * 13:64 * 13 + 6 * 64] = 0.05 * rng.standard_normal(6 * 64)
            w = w.astype(np.float32)
            assert not G.set_learned_smoother(w)
            assert not G64.set_learned_smoother(w)
            np.testing.assert_array_equal(G.learned_blocks(), G64.learned_blocks())
        u, it, res, st = G.solve(fb)
        u64, it64, _, st64 = G64.solve(fb)
        assert st == st64 == amg.AMG_OK and res <= 1e-8
        assert abs(it - it64) <= 1, (kw, it, it64)
        assert torch.linalg.norm(u - u64) <= 1e-9 * torch.linalg.norm(u64), kw
