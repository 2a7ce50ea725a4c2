"""Parity of the CUDA path with the FP64 scalar-CSR oracle (GPU required).

Bars: aggregates, strength flags and every sparsity pattern bit-exact; FP64
SpMV within 1e-12 relative; setup values (P, R, A_c, B_c, smoother) within
1e-12 of the largest entry; the V-cycle within the bound set by the coarse
solver (dense inverse here, Cholesky solves in the oracle); the PCG solution
within 1e-7 relative with iteration counts within +-1.
"""
import numpy as np
import pytest

import oracle as o
import q1elasticity as q

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

amg = pytest.importorskip("paper_2202_09056_gb300")

from parity_util import compare_hierarchy, dev_args, rel, vcycle_bound  # noqa: E402


def _dev(p):
    return dev_args(p, torch)


def _rel(a, b):
    return rel(a, b)


def _random_bsr(nbr, nbc, br, bc, rng, density=0.3, empty_rows=()):
    rp, cl = [0], []
    for i in range(nbr):
        cols = [] if i in empty_rows else sorted(rng.choice(nbc, size=max(1, int(density * nbc)),
                                                            replace=False).tolist())
        cl += cols
        rp.append(len(cl))
    val = rng.standard_normal((len(cl), br, bc))
    return np.array(rp, np.int32), np.array(cl, np.int32), val


@pytest.mark.parametrize("br,bc", [(3, 3), (6, 6), (3, 6), (6, 3)])
def test_bsr_spmv_matches_oracle(br, bc):
    rng = np.random.default_rng(br * 10 + bc)
    nbr, nbc = 257, 131  # several CTAs, a ragged tail, empty rows
    rp, cl, val = _random_bsr(nbr, nbc, br, bc, rng, 0.1, empty_rows=(0, 5, 256))
    x = rng.standard_normal(nbc * bc)
    d = torch.device("cuda:0")
    y = amg.bsr_spmv(torch.from_numpy(rp).to(d), torch.from_numpy(cl).to(d),
                     torch.from_numpy(val).to(d), torch.from_numpy(x).to(d), nbcols=nbc)
    ref = o.spmv(o.unblock(rp, cl, val.reshape(len(cl), -1), br, bc, nbcols=nbc), x)
    assert np.abs(y.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()


def test_bsr_spmv_dot_is_deterministic_and_exact():
    p = q.inclusions(9)
    rp, cl, val, _ = _dev(p)
    x = torch.from_numpy(np.random.default_rng(1).standard_normal(p.ndof)).cuda()
    y1, d1 = amg.bsr_spmv_dot(rp, cl, val, x)
    y2, d2 = amg.bsr_spmv_dot(rp, cl, val, x)
    assert d1 == d2 and torch.equal(y1, y2)
    ref = o.spmv(o.from_problem(p), x.cpu().numpy())
    assert _rel(y1.cpu().numpy(), ref) <= 1e-12
    assert abs(d1 - x.cpu().numpy() @ ref) <= 1e-12 * abs(x.cpu().numpy() @ ref)


def test_spmv_empty_matrix():
    d = torch.device("cuda:0")
    rp = torch.zeros(1, dtype=torch.int32, device=d)
    y = amg.bsr_spmv(rp, torch.zeros(0, dtype=torch.int32, device=d),
                     torch.zeros((0, 3, 3), dtype=torch.float64, device=d),
                     torch.zeros(3, dtype=torch.float64, device=d), nbcols=1)
    assert y.numel() == 0


def _compare_hierarchy(p, coarse_enough, tol_val=1e-12, Bns=None, aggregation="greedy", **kw):
    return compare_hierarchy(p, coarse_enough, torch, amg, tol_val, Bns, aggregation, **kw)


@pytest.mark.parametrize("shape,kw,ce", [
    ((10, 10, 10), {"body": (0, 0, -1)}, 3000),
    ((7, 5, 9), {"traction": (0, 0, -1), "inclusion_frac": 0.2}, 200),
    ((12, 12, 12), {"traction": (0, 0, -1), "inclusion_frac": 0.2}, 300),
])
def test_setup_matches_oracle(shape, kw, ce):
    p = q.make_problem(shape, **kw)
    _compare_hierarchy(p, ce)


def _translations(ndof):
    T = np.zeros((ndof, 3))
    for c in range(3):
        T[c::3, c] = 1.0
    return T


@pytest.mark.parametrize("shape,kw,ce", [
    ((10, 10, 10), {"body": (0, 0, -1)}, 500),
    ((12, 11, 13), {"traction": (0, 0, -1), "inclusion_frac": 0.2}, 300),
])
def test_translations_only_setup_and_solve_match_oracle(shape, kw, ce):
    """The block solver without rotations (near-nullspace = the three
    translations, 3-DOF coarse nodes): hierarchy, then PCG, against the
    oracle; the rigid-body modes need fewer iterations."""
    p = q.make_problem(shape, **kw)
    T = _translations(p.ndof)
    H, G = _compare_hierarchy(p, ce, Bns=T)
    assert all(G.level_info(l)["bs"] == 3 for l in range(G.nlevels))
    uo, ito, _ = H.solve(p.f, tol=1e-8, maxiter=3000)
    fb = torch.from_numpy(p.f).cuda()
    u, it, res, st = G.solve(fb, tol=1e-8, maxiter=3000)
    assert st == amg.AMG_OK and res <= 1e-8 and abs(it - ito) <= 1, (it, ito)
    assert np.linalg.norm(u.cpu().numpy() - uo) <= 1e-7 * np.linalg.norm(uo)
    _, it6, _, _ = amg.AMG(*_dev(p), coarse_enough=ce).solve(fb)
    assert it6 < it


def test_vcycle_matches_oracle():
    p = q.make_problem((12, 12, 12), traction=(0, 0, -1), inclusion_frac=0.2)
    H, G = _compare_hierarchy(p, 300)
    rng = np.random.default_rng(5)
    for _ in range(2):
        r = rng.standard_normal(p.ndof)
        z = G.vcycle(torch.from_numpy(r).cuda()).cpu().numpy()
        zo = H.vcycle(r)
        assert np.linalg.norm(z - zo) <= vcycle_bound(H) * np.linalg.norm(zo)


@pytest.mark.parametrize("shape,kw,ce", [
    ((10, 10, 10), {"body": (0, 0, -1)}, 3000),
    ((11, 6, 8), {"traction": (0, 0, -1), "inclusion_frac": 0.2}, 150),
    ((16, 16, 16), {"traction": (0, 0, -1), "inclusion_frac": 0.2}, 3000),
])
def test_pcg_matches_oracle(shape, kw, ce):
    p = q.make_problem(shape, **kw)
    H = o.Hierarchy(o.from_problem(p), 3, p.B, coarse_enough=ce)
    uo, ito, reso = H.solve(p.f, tol=1e-8, maxiter=1000)
    rp, cl, val, B = _dev(p)
    G = amg.AMG(rp, cl, val, B, coarse_enough=ce)
    u, it, res, st = G.solve(torch.from_numpy(p.f).cuda(), tol=1e-8, maxiter=1000)
    u = u.cpu().numpy()
    assert st == amg.AMG_OK and res <= 1e-8
    assert abs(it - ito) <= 1, (it, ito)
    assert np.linalg.norm(u - uo) <= 1e-7 * np.linalg.norm(uo)
    # independent check of the returned residual
    A = o.from_problem(p).to_scipy()
    assert abs(np.linalg.norm(p.f - A @ u) / np.linalg.norm(p.f) - res) <= 1e-3 * res


def test_pcg_edge_cases():
    p = q.cube(6)
    rp, cl, val, B = _dev(p)
    G = amg.AMG(rp, cl, val, B, coarse_enough=100)
    f = torch.zeros(p.ndof, dtype=torch.float64, device="cuda")
    u, it, res, st = G.solve(f, u=torch.ones_like(f))
    assert it == 0 and st == amg.AMG_OK and not u.any()           # f = 0 gives u = 0
    fb = torch.from_numpy(p.f).cuda()
    us, _, _, _ = G.solve(fb, tol=1e-12)
    u, it, res, st = G.solve(fb, u=us.clone(), tol=1e-8)          # converged start
    assert it == 0 and st == amg.AMG_OK
    u, it, res, st = G.solve(fb, tol=1e-14, maxiter=3)            # iteration cap
    assert st == amg.AMG_NOT_CONVERGED and it == 3 and res > 1e-14
    G1 = amg.AMG(rp, cl, val, B, coarse_enough=10 ** 6)           # one level: exact solve
    assert G1.nlevels == 1
    u, it, res, st = G1.solve(fb, tol=1e-10)
    assert it == 1 and res <= 1e-10


@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 1, 1), (2, 2, 2), (5, 4, 3), (6, 6, 6),
                                   (9, 9, 9)])
def test_coarse_inverse_is_the_inverse(shape):
    """A one-level hierarchy's V-cycle is the dense coarse inverse applied to
    r: against a dense solve of the assembled matrix, within cond(A) times the
    unit roundoff.  Sizes from 24 to 3000 unknowns: a single partial panel of
    the 32-column blocked factor, then several panels with a ragged last one
    (4, 17, 8, 5 and 24 rows), up to 94 panels whose updates span from one
    tile row to thousands of tiles."""
    p = q.make_problem(shape, body=(0, 0, -1))
    A = o.from_problem(p).to_scipy().toarray()
    ev = np.linalg.eigvalsh(A)
    cond = ev[-1] / ev[0]
    rp, cl, val, B = _dev(p)
    G = amg.AMG(rp, cl, val, B, coarse_enough=10 ** 6)
    assert G.nlevels == 1
    rng = np.random.default_rng(11)
    for _ in range(2):
        r = rng.standard_normal(p.ndof)
        z = G.vcycle(torch.from_numpy(r).cuda()).cpu().numpy()
        ze = np.linalg.solve(A, r)
        assert np.linalg.norm(z - ze) <= 50 * cond * 2.2e-16 * np.linalg.norm(ze), shape


def test_solve_is_bitwise_reproducible():
    p = q.inclusions(10)
    rp, cl, val, B = _dev(p)
    G = amg.AMG(rp, cl, val, B, coarse_enough=300)
    fb = torch.from_numpy(p.f).cuda()
    u1, it1, r1, _ = G.solve(fb)
    u2, it2, r2, _ = G.solve(fb)
    assert it1 == it2 and r1 == r2 and torch.equal(u1, u2)


# ------------------------------------------------ MIS-2 aggregation on the device
@pytest.mark.parametrize("shape,kw,ce", [
    ((10, 10, 10), {"body": (0, 0, -1)}, 3000),
    ((7, 5, 9), {"traction": (0, 0, -1), "inclusion_frac": 0.2}, 200),
    ((12, 12, 12), {"traction": (0, 0, -1), "inclusion_frac": 0.2}, 300),
    ((21, 9, 14), {"traction": (0, 0, -1), "inclusion_frac": 0.2}, 100),
])
def test_mis2_setup_matches_oracle(shape, kw, ce):
    """Device MIS-2 aggregation: aggregates bit-exact with the oracle's
    sequential visit on every level (fine 3x3 graphs and coarse 6x6 ones,
    several CTAs of rows and ragged tails), then the whole hierarchy."""
    p = q.make_problem(shape, **kw)
    H, G = _compare_hierarchy(p, ce, aggregation="mis2")
    assert G.nlevels >= 2


@pytest.mark.parametrize("eps,levels", [(0.0, None), (10.0, 1)])
def test_mis2_degenerate_strength(eps, levels):
    """Every block strong (eps = 0) and no block strong (every node isolated:
    no aggregate, so the hierarchy keeps one level)."""
    p = q.make_problem((5, 4, 6), traction=(0, 0, -1), inclusion_frac=0.2)
    H, G = _compare_hierarchy(p, 40, aggregation="mis2", eps_strong=eps)
    if levels is not None:
        assert G.nlevels == levels


@pytest.mark.parametrize("shape,kw,ce", [
    ((10, 10, 10), {"body": (0, 0, -1)}, 3000),
    ((16, 16, 16), {"traction": (0, 0, -1), "inclusion_frac": 0.2}, 3000),
    ((11, 6, 8), {"traction": (0, 0, -1), "inclusion_frac": 0.2}, 150),
])
def test_mis2_pcg_matches_oracle(shape, kw, ce):
    p = q.make_problem(shape, **kw)
    H = o.Hierarchy(o.from_problem(p), 3, p.B, coarse_enough=ce, aggregation="mis2")
    uo, ito, _ = H.solve(p.f, tol=1e-8, maxiter=1000)
    G = amg.AMG(*_dev(p), coarse_enough=ce, aggregation=amg.AGG_MIS2)
    u, it, res, st = G.solve(torch.from_numpy(p.f).cuda(), tol=1e-8, maxiter=1000)
    assert st == amg.AMG_OK and res <= 1e-8
    assert abs(it - ito) <= 1, (it, ito)
    assert np.linalg.norm(u.cpu().numpy() - uo) <= 1e-7 * np.linalg.norm(uo)


@pytest.mark.slow
def test_mis2_full_size_inclusions_80():
    """80^3 elements: the fine-level aggregates of the device MIS-2 equal the
    oracle's (its strength and sequential visit on the scalar matrix), and
    the MIS-2 hierarchy solves to a host-checked 1e-8."""
    p = q.inclusions(80)
    rp, cl, val, B = _dev(p)
    G = amg.AMG(rp, cl, val, B, aggregation=amg.AGG_MIS2)
    agg = np.empty(p.nnodes, np.int32)
    amg._check(G._lib.amg_level_export(G._h, 0, 3, agg.ctypes.data, None, None))
    ago, nago = o.aggregate_mis2(o.from_problem(p), 3, 0.08)
    assert np.array_equal(agg, ago) and G.level_info(0)["nagg"] == nago
    u, it, res, st = G.solve(torch.from_numpy(p.f).cuda(), tol=1e-8, maxiter=2000)
    assert st == amg.AMG_OK
    import scipy.sparse as sp
    A = sp.bsr_matrix((p.val, p.col, p.row_ptr), shape=(p.ndof, p.ndof))
    un = u.cpu().numpy()
    assert np.linalg.norm(p.f - A @ un) / np.linalg.norm(p.f) <= 1.0001e-8


@pytest.mark.slow
def test_full_size_inclusions_80_sampled():
    """80^3 elements (1.59 M DOFs): sampled SpMV rows recomputed one by one on
    the host, and the solve's residual recomputed with a host SpMV."""
    p = q.inclusions(80)
    rp, cl, val, B = _dev(p)
    rng = np.random.default_rng(80)
    x = rng.standard_normal(p.ndof)
    y = amg.bsr_spmv(rp, cl, val, torch.from_numpy(x).cuda()).cpu().numpy()
    for I in rng.choice(p.nnodes, 200, replace=False):
        s, e = p.row_ptr[I], p.row_ptr[I + 1]
        ref = sum(p.val[k] @ x[3 * p.col[k]:3 * p.col[k] + 3] for k in range(s, e))
        assert np.abs(y[3 * I:3 * I + 3] - ref).max() <= 1e-12 * np.abs(ref).max()
    G = amg.AMG(rp, cl, val, B)
    u, it, res, st = G.solve(torch.from_numpy(p.f).cuda(), tol=1e-8, maxiter=2000)
    assert st == amg.AMG_OK
    import scipy.sparse as sp
    A = sp.bsr_matrix((p.val, p.col, p.row_ptr), shape=(p.ndof, p.ndof))
    un = u.cpu().numpy()
    assert np.linalg.norm(p.f - A @ un) / np.linalg.norm(p.f) <= 1.0001e-8


def test_level_spmv_sell_matches_oracle():
    """The solve's own sliced-ELL kernels for A, P and R of every level."""
    p = q.make_problem((13, 9, 11), traction=(0, 0, -1), inclusion_frac=0.2)
    rp, cl, val, B = _dev(p)
    G = amg.AMG(rp, cl, val, B, coarse_enough=150)
    rng = np.random.default_rng(7)
    for l in range(G.nlevels - 1):
        ex = G.export(l)
        b, nagg = ex["info"]["bs"], ex["info"]["nagg"]
        nb = ex["info"]["nbrows"]
        for which, (mat, br, bc, ncols) in enumerate([(ex["A"], b, b, nb), (ex["P"], b, 6, nagg),
                                                       (ex["R"], 6, b, nb)]):
            x = rng.standard_normal(ncols * bc)
            y = torch.empty((len(mat[0]) - 1) * br, dtype=torch.float64, device="cuda")
            G.level_spmv(l, which, torch.from_numpy(x).cuda(), y)
            ref = o.spmv(o.unblock(mat[0], mat[1], mat[2].reshape(len(mat[1]), -1), br, bc,
                                   nbcols=ncols), x)
            assert np.abs(y.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max(), (l, which)
        assert all(x >= 0 for x in G.padding(l))
    # the gather loads pairs of entries where the address allows: an x view
    # 8 bytes into an allocation (not 16-byte aligned) gives the same bits as
    # an aligned copy, on every operator of levels 0 and 1
    for l in range(min(2, G.nlevels - 1)):
        ex = G.export(l)
        b, nagg, nb = ex["info"]["bs"], ex["info"]["nagg"], ex["info"]["nbrows"]
        for which, (ny, nx) in enumerate(((nb * b, nb * b), (nb * b, nagg * 6), (nagg * 6, nb * b))):
            xs = torch.zeros(nx + 1, dtype=torch.float64, device="cuda")
            xs[1:] = torch.from_numpy(rng.standard_normal(nx)).cuda()
            x_al = xs[1:].clone()
            y_off = torch.empty(ny, dtype=torch.float64, device="cuda")
            y_al = torch.empty(ny, dtype=torch.float64, device="cuda")
            G.level_spmv(l, which, xs[1:], y_off)
            G.level_spmv(l, which, x_al, y_al)
            assert xs[1:].data_ptr() % 16 == 8 and torch.equal(y_off, y_al), (l, which)


def test_host_loop_mode_gives_identical_results():
    p = q.inclusions(9)
    rp, cl, val, B = _dev(p)
    fb = torch.from_numpy(p.f).cuda()
    u0, it0, r0, s0 = amg.AMG(rp, cl, val, B, coarse_enough=200).solve(fb)
    u1, it1, r1, s1 = amg.AMG(rp, cl, val, B, coarse_enough=200, loop_mode=1).solve(fb)
    assert (it0, r0, s0) == (it1, r1, s1) and torch.equal(u0, u1)


@pytest.mark.parametrize("prec", [amg.PREC_FP32, amg.PREC_BF16])
def test_reduced_precision_vcycle_solves_to_fp64_accuracy(prec):
    """Precision form: FP32 or BF16-stored V-cycle, FP64 CG.  The outer FP64
    recurrences still drive the true residual to 1e-8; the solution is
    compared with the FP64 oracle's."""
    p = q.make_problem((14, 12, 13), traction=(0, 0, -1), inclusion_frac=0.2)
    H = o.Hierarchy(o.from_problem(p), 3, p.B, coarse_enough=300)
    uo, ito, _ = H.solve(p.f, tol=1e-8, maxiter=2000)
    rp, cl, val, B = _dev(p)
    G = amg.AMG(rp, cl, val, B, coarse_enough=300, precision=prec)
    assert G.nlevels == H.nlevels
    fb = torch.from_numpy(p.f).cuda()
    u, it, res, st = G.solve(fb, tol=1e-8, maxiter=2000)
    assert st == amg.AMG_OK and res <= 1e-8
    A = o.from_problem(p).to_scipy()
    un = u.cpu().numpy()
    assert np.linalg.norm(p.f - A @ un) / np.linalg.norm(p.f) <= 1.0001e-8
    # both iterates have relative residual <= 1e-8; their difference is bounded
    # by the same residual bound amplified by the conditioning, which the FP64
    # parity test shows to stay below 1e-7 on these meshes
    assert np.linalg.norm(un - uo) <= 1e-6 * np.linalg.norm(uo)
    assert it <= 1.5 * ito + 5, (it, ito)
    # the V-cycle itself is close to the FP64 one
    r = np.random.default_rng(3).standard_normal(p.ndof)
    z = G.vcycle(torch.from_numpy(r).cuda()).cpu().numpy()
    zo = H.vcycle(r)
    tol = 1e-4 if prec == amg.PREC_FP32 else 5e-2
    assert np.linalg.norm(z - zo) <= tol * np.linalg.norm(zo)


def test_setup_rejects_malformed_patterns():
    """The input pattern is checked on the device before any kernel indexes
    with it; every malformed case returns AMG_ERR_ARG and names the row."""
    p = q.cube(3)
    rp0, cl0, val0, B0 = p.row_ptr.copy(), p.col.copy(), p.val, p.B

    def setup(rp, cl):
        d = torch.device("cuda:0")
        return amg.AMG(torch.from_numpy(rp).to(d), torch.from_numpy(cl).to(d),
                       torch.from_numpy(val0).to(d), torch.from_numpy(B0).to(d))

    # a valid pattern passes
    setup(rp0, cl0)
    # decreasing row pointer (row 5 ends before it starts); columns stay in range
    rp = rp0.copy()
    rp[6] = rp[5] - 1
    with pytest.raises(amg.AmgError) as e:
        setup(rp, cl0)
    assert e.value.status == amg.AMG_ERR_ARG and "row_ptr" in str(e.value)
    # unsorted columns in row 7
    cl = cl0.copy()
    a, b = rp0[7], rp0[8]
    cl[a], cl[a + 1] = cl[a + 1], cl[a]
    with pytest.raises(amg.AmgError) as e:
        setup(rp0, cl)
    assert "block row 7" in str(e.value) and "ascending" in str(e.value)
    # a column out of range in the last row
    cl = cl0.copy()
    cl[rp0[-1] - 1] = p.nnodes + 3
    with pytest.raises(amg.AmgError) as e:
        setup(rp0, cl)
    assert f"block row {p.nnodes - 1}" in str(e.value)
    # a row without its diagonal block: row 0's diagonal entry points at a
    # column absent from the row instead (columns kept ascending)
    cl = cl0.copy()
    row0 = list(cl0[rp0[0]:rp0[1]])
    free = next(c for c in range(p.nnodes) if c not in row0)
    d0 = rp0[0] + row0.index(0)
    cl[d0] = free
    cl[rp0[0]:rp0[1]] = np.sort(cl[rp0[0]:rp0[1]])
    with pytest.raises(amg.AmgError) as e:
        setup(rp0, cl)
    assert "block row 0 has no diagonal block" in str(e.value)
    # a non-symmetric pattern: row 7 loses its first block (column 2), row 2
    # keeps its block (2, 7)
    a = rp0[7]
    assert cl0[a] == 2 and 7 in cl0[rp0[2]:rp0[3]]
    cl = np.delete(cl0, a)
    rp = rp0.copy()
    rp[8:] -= 1
    d = torch.device("cuda:0")
    with pytest.raises(amg.AmgError) as e:
        amg.AMG(torch.from_numpy(rp).to(d), torch.from_numpy(cl).to(d),
                torch.from_numpy(np.delete(val0, a, axis=0)).to(d), torch.from_numpy(B0).to(d))
    assert "not symmetric" in str(e.value) and "block row 2" in str(e.value)


def test_non_finite_inputs_are_rejected():
    """A NaN or infinity in f or in the initial guess is an argument error
    before any iteration (a NaN norm must not read as a zero right-hand side),
    and the handle stays usable; a NaN in A or B fails the setup's input
    check; a NaN right-hand side in a batch names its pair."""
    p = q.make_problem((6, 5, 7), traction=(0, 0, -1), inclusion_frac=0.2)
    rp, cl, val, B = _dev(p)
    G = amg.AMG(rp, cl, val, B, coarse_enough=60)
    fb = torch.from_numpy(p.f).cuda()
    for bad_f, bad_u in ((float("nan"), None), (float("inf"), None), (None, float("nan"))):
        f, u = fb.clone(), torch.zeros_like(fb)
        if bad_f is not None:
            f[17] = bad_f
        if bad_u is not None:
            u[5] = bad_u
        with pytest.raises(amg.AmgError) as e:
            G.solve(f, u=u)
        assert e.value.status == amg.AMG_ERR_ARG
    u, it, res, st = G.solve(fb)
    assert st == amg.AMG_OK and res <= 1e-8
    for arr, idx in ((val, (int(rp[p.nnodes // 2]) + 1, 0, 0)), (B, (4, 2))):
        bad = arr.clone()
        bad[idx] = float("nan")
        args = (rp, cl, bad, B) if arr is val else (rp, cl, val, bad)
        with pytest.raises(amg.AmgError) as e:
            amg.AMG(*args, coarse_enough=60)
        assert e.value.status == amg.AMG_ERR_ARG
    bat = amg.AMGBatch([(rp, cl, val)], [B], [2], coarse_enough=60)
    F = torch.stack([fb, fb])
    F[1, 3] = float("nan")
    with pytest.raises(amg.AmgError) as e:
        bat.solve([F])
    assert e.value.status == amg.AMG_ERR_ARG and "right-hand side 1" in str(e.value)
