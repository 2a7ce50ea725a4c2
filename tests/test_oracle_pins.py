"""Pins of the FP64 scalar-CSR oracle against what the paper and the
mathematics fix.  Every oracle function is tied here to something other than
its own formula: the paper's worked example (Sec. 2), hand-worked
aggregations, closed forms, invariants of smoothed aggregation with rigid-body
modes (Sec. 2, Alg. 1), library routines for special cases, and dense direct
solves (Eq. 1).
"""
import json
import os

import numpy as np
import pytest

import oracle as o
import q1elasticity as q


# ---------------------------------------------------------------- Sec. 2 example
def test_worked_example_unblock_matches_paper(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "sec2_block_example.json")))
    b = g["block"]
    A = o.unblock(g["bsr"]["ptr"], g["bsr"]["col"], np.array(g["bsr"]["val"]).reshape(-1, b * b),
                  b, b)
    assert A.ptr.tolist() == g["csr"]["ptr"]
    assert A.col.tolist() == g["csr"]["col"]
    assert A.val.tolist() == g["csr"]["val"]
    assert np.array_equal(A.to_dense(), np.array(g["dense"]))
    # four times fewer logical values, half the rows (Sec. 2)
    assert len(g["bsr"]["col"]) * 4 == len(g["csr"]["col"])


def test_worked_example_spmv(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "sec2_block_example.json")))
    A = o.CSR(g["csr"]["ptr"], g["csr"]["col"], g["csr"]["val"], (6, 6))
    x = np.arange(1.0, 7.0)
    np.testing.assert_allclose(o.spmv(A, x), np.array(g["dense"]) @ x, rtol=1e-15)


def test_unblock_keeps_explicit_zeros():
    # a block with absent scalars: the scalar view keeps all of them as
    # explicit zeros (the block pattern stays the scalar pattern)
    val = np.array([[1.0, 0.0, 0.0, 2.0]])
    A = o.unblock([0, 1], [0], val, 2, 2)
    assert A.nnz == 4 and A.val.tolist() == [1.0, 0.0, 0.0, 2.0]


# ---------------------------------------------------------------- strength, aggregation
def _graph_matrix(case):
    n = case["n"]
    D = np.diag(case.get("diag", [1.0] * n))
    for i, j, v in case["sym"]:
        D[i, j] = D[j, i] = v
    for i, j, v in case["directed"]:
        D[i, j] = v
    ptr = [0]
    col, val = [], []
    for i in range(n):
        nz = np.nonzero(D[i])[0]
        col += nz.tolist()
        val += D[i, nz].tolist()
        ptr.append(len(col))
    return o.CSR(ptr, col, val, (n, n))


def test_aggregation_hand_worked(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "aggregation_graphs.json")))
    for case in g["cases"]:
        agg, nagg = o.aggregate(_graph_matrix(case), 1, 0.08)
        assert agg.tolist() == case["agg"], case["name"]
        assert nagg == case["nagg"], case["name"]


def test_strength_norms_and_eps_zero():
    p = q.cube(3)
    A = o.from_problem(p)
    G = o.strength(A, 3, 0.0)
    # node pattern = block pattern of the generator; norms = Frobenius^2
    assert np.array_equal(G["ptr"], p.row_ptr.astype(np.int64))
    assert np.array_equal(G["col"], p.col)
    np.testing.assert_allclose(G["norm2"], np.linalg.norm(p.val, axis=(1, 2)) ** 2, rtol=1e-14)
    rows = np.repeat(np.arange(p.nnodes), np.diff(p.row_ptr))
    # eps = 0: every present off-diagonal block with a non-zero entry is strong
    assert np.array_equal(G["strong"].astype(bool), (G["col"] != rows) & (G["norm2"] > 0))


def test_strength_monotone_in_eps():
    A = o.from_problem(q.inclusions(6))
    prev = None
    for eps in (0.0, 0.04, 0.08, 0.16, 0.5):
        s = o.strength(A, 3, eps)["strong"].astype(bool)
        if prev is not None:
            assert not (s & ~prev).any()
        prev = s


@pytest.mark.parametrize("shape", [(4, 4, 4), (5, 3, 7)])
def test_aggregates_partition_nonisolated_nodes(shape):
    p = q.make_problem(shape, traction=(0, 0, -1), inclusion_frac=0.2)
    A = o.from_problem(p)
    G = o.strength(A, 3, 0.08)
    agg, nagg = o.aggregate(A, 3, 0.08)
    rows = np.repeat(np.arange(p.nnodes), np.diff(G["ptr"]))
    has_strong = np.bincount(rows, weights=G["strong"], minlength=p.nnodes) > 0
    assert np.array_equal(agg >= 0, has_strong)        # isolated <=> no strong neighbour
    assert set(np.unique(agg[agg >= 0])) == set(range(nagg))  # ids 0..nagg-1 all used
    clamped = p.coords[:, 0] == 0.0
    assert (agg[clamped] == -1).all()                  # clamped nodes are isolated
    # every aggregate is connected through strong links (each pass grows an
    # aggregate only along strong connections)
    import scipy.sparse as sp
    import scipy.sparse.csgraph as cg
    S = sp.csr_matrix((G["strong"].astype(float), G["col"], G["ptr"]), shape=(p.nnodes,) * 2)
    S = S + S.T
    for k in range(nagg):
        m = np.nonzero(agg == k)[0]
        ncomp, _ = cg.connected_components(S[m][:, m], directed=False)
        assert ncomp == 1


# ---------------------------------------------------------------- tentative prolongation
def test_tentative_orthonormal_and_reproduces_B():
    p = q.make_problem((4, 3, 3), clamp=False, body=(0, 0, -1))
    A = o.from_problem(p)
    agg, nagg = o.aggregate(A, 3, 0.08)
    Pt, Bc = o.tentative(p.nnodes, 3, agg, nagg, p.B)
    Pd = Pt.to_dense()
    rows = np.repeat(agg >= 0, 3)
    np.testing.assert_allclose(Pd[rows] @ Bc, p.B[rows], atol=1e-13)
    for a in range(nagg):
        m = np.repeat(agg == a, 3)
        Q = Pd[np.ix_(m, np.arange(6 * a, 6 * a + 6))]
        keep = np.abs(Q).sum(0) > 0
        np.testing.assert_allclose(Q[:, keep].T @ Q[:, keep], np.eye(keep.sum()), atol=1e-13)
        Ra = Bc[6 * a:6 * a + 6]
        assert np.allclose(np.tril(Ra, -1), 0.0)
        # thin QR is unique for full column rank with R_kk > 0: compare to LAPACK
        if keep.all():
            Qn, Rn = np.linalg.qr(p.B[m])
            s = np.sign(np.diag(Rn))
            np.testing.assert_allclose(Q, Qn * s, atol=1e-12)
            np.testing.assert_allclose(Ra, s[:, None] * Rn, atol=1e-12 * np.abs(Rn).max())


def test_tentative_single_node_aggregate_is_rank_three():
    # one node: translations span its three rows, rotations are dependent
    B = np.array([[1, 0, 0, 0, 0.3, -0.2], [0, 1, 0, -0.3, 0, 0.1], [0, 0, 1, 0.2, -0.1, 0]], float)
    Pt, Bc = o.tentative(1, 3, np.array([0], np.int32), 1, B)
    Q = Pt.to_dense()
    assert np.count_nonzero(np.abs(Q).sum(0)) == 3
    np.testing.assert_allclose(Q @ Bc, B, atol=1e-14)
    assert np.count_nonzero(np.abs(Bc).sum(1)) == 3


def _translations(ndof):
    T = np.zeros((ndof, 3))
    for c in range(3):
        T[c::3, c] = 1.0
    return T


def test_tentative_translations_is_normalised_block_identity():
    # Without rotations (the block solver with no near-nullspace) the stacked
    # member rows of an aggregate of n_a nodes are n_a identity blocks: Q is
    # the block identity over sqrt(n_a) and R = sqrt(n_a) I, in closed form.
    p = q.make_problem((4, 3, 3), clamp=False, body=(0, 0, -1))
    A = o.from_problem(p)
    agg, nagg = o.aggregate(A, 3, 0.08)
    Pt, Bc = o.tentative(p.nnodes, 3, agg, nagg, _translations(p.ndof))
    Pd = Pt.to_dense()
    assert Pd.shape == (p.ndof, 3 * nagg) and Bc.shape == (3 * nagg, 3)
    for a in range(nagg):
        na = int((agg == a).sum())
        np.testing.assert_allclose(Bc[3 * a:3 * a + 3], np.sqrt(na) * np.eye(3), rtol=1e-15)
        for I in np.nonzero(agg == a)[0]:
            np.testing.assert_allclose(Pd[3 * I:3 * I + 3, 3 * a:3 * a + 3], np.eye(3) / np.sqrt(na),
                                       rtol=1e-15, atol=0)
    assert np.count_nonzero(Pd) == 3 * int((agg >= 0).sum())


@pytest.mark.parametrize("eps", [0.0, 0.08])
def test_smoothed_prolongation_keeps_translations(eps):
    # The same chain as for the rigid modes with B = the three translations
    # (A T = 0 on the unconstrained operator too); coarse nodes carry 3 DOFs.
    p = q.make_problem((6, 5, 4), clamp=False, body=(0, 0, -1))
    A, B, b = o.from_problem(p), _translations(p.ndof), 3
    for level in range(3):
        nn = A.shape[0] // b
        agg, nagg = o.aggregate(A, b, eps * 0.5 ** level)
        assert nagg < nn
        rows = np.repeat(agg >= 0, b)
        Pt, Bc = o.tentative(nn, b, agg, nagg, B)
        assert Bc.shape == (3 * nagg, 3)
        d, rho = o.jacobi_rho(A)
        P = o.smooth_prolongation(A, d, (4.0 / 3.0) / rho, Pt)
        assert np.abs((P.to_scipy() @ Bc - B)[rows]).max() <= 1e-10
        Ac = o.spgemm(o.transpose(P), o.spgemm(A, P))
        As = Ac.to_scipy()
        scale = max(abs(As).max(), abs(A.to_scipy()).max())
        assert np.abs(As @ Bc).max() <= 1e-10 * scale * np.abs(Bc).max()
        A, B = Ac, Bc
        if nagg < 2:
            break


def test_translations_only_hierarchy_solves_and_is_weaker():
    # The block solver without a near-nullspace: 3-DOF coarse nodes, PCG to a
    # dense direct solve's answer; the rigid-body modes cut the iterations.
    p = q.make_problem((5, 4, 6), traction=(0, 0, -1), inclusion_frac=0.2)
    H3 = o.Hierarchy(o.from_problem(p), 3, _translations(p.ndof), coarse_enough=150)
    H6 = o.Hierarchy(o.from_problem(p), 3, p.B, coarse_enough=150)
    assert H3.nlevels >= 2 and all(H3.level(l)["b"] == 3 for l in range(H3.nlevels))
    assert H3.level(1)["n"] == 3 * H3.level(0)["nagg"]
    u3, it3, res3 = H3.solve(p.f, tol=1e-8, maxiter=3000)
    u6, it6, _ = H6.solve(p.f, tol=1e-8)
    ud = np.linalg.solve(q.bsr_to_dense(p), p.f)
    assert res3 <= 1e-8
    assert np.linalg.norm(u3 - ud) <= 1e-7 * np.linalg.norm(ud)
    assert it6 < it3


# ---------------------------------------------------------------- Jacobi rho, omega, P
def test_jacobi_diagonal_and_gershgorin_bound():
    p = q.inclusions(5)
    A = o.from_problem(p)
    d, rho = o.jacobi_rho(A)
    Ad = A.to_dense()
    np.testing.assert_array_equal(d, np.diag(Ad))
    # Gershgorin: rho bounds the spectrum of D^-1 A from above, and is attained
    # by a row sum of |D^-1 A|
    lam = np.abs(np.linalg.eigvals(Ad / d[:, None])).max()
    assert rho >= lam * (1 - 1e-12)
    assert np.isclose(rho, (np.abs(Ad).sum(1) / np.abs(d)).max(), rtol=1e-14)


def test_gershgorin_closed_form_on_laplacian():
    # tridiag(-1, 2, -1): interior rows give (1 + 2 + 1) / 2 = 2 exactly
    n = 9
    ptr, col, val = [0], [], []
    for i in range(n):
        for j, v in ((i - 1, -1.0), (i, 2.0), (i + 1, -1.0)):
            if 0 <= j < n:
                col.append(j)
                val.append(v)
        ptr.append(len(col))
    d, rho = o.jacobi_rho(o.CSR(ptr, col, val, (n, n)))
    assert rho == 2.0 and (d == 2.0).all()


def test_default_stop_rule_on_ten_cube():
    # 3993 DOFs > 3000 coarsens once; 6 x (aggregates) < 3000 stops
    H = o.Hierarchy(o.from_problem(q.cube(10)), 3, q.cube(10).B)
    assert H.nlevels == 2
    L1 = H.level(1)
    assert L1["b"] == 6 and L1["n"] == 6 * H.level(0)["nagg"] <= 3000


@pytest.mark.parametrize("shape,ce", [((16, 16, 16), 300), ((14, 12, 13), 200),
                                      ((18, 18, 18), 400), ((20, 20, 20), 600)])
def test_stop_rule_against_separate_aggregation(shape, ce):
    """The coarsening stop rule, level by level, against the aggregation
    function called on its own for every level: a level below the finest is
    coarsened only if it holds more than coarse_enough rows and is not small
    (<= 2 ce rows) with a tiny aggregation (< ce / 4 coarse rows); the
    coarsest level is there because one of the stop conditions holds; the
    finest level above ce is always coarsened."""
    p = q.make_problem(shape, traction=(0, 0, -1), inclusion_frac=0.2)
    H = _hierarchy(p, coarse_enough=ce)
    assert H.nlevels >= 2
    triggered = False
    for l in range(1, H.nlevels):
        L = H.level(l)
        agg, nagg = o.aggregate(L["A"], L["b"], L["eps"])
        nn = L["n"] // L["b"]
        small, tiny = L["n"] <= 2 * ce, 4 * nagg * 6 < ce
        if l < H.nlevels - 1:
            assert L["n"] > ce and not (small and tiny) and nagg == L["nagg"]
            assert np.array_equal(agg, L["agg"])
        else:
            assert L["n"] <= ce or (small and tiny) or nagg == 0 or nagg >= 0.9 * nn
            triggered = L["n"] > ce
    if shape == (16, 16, 16):
        assert triggered  # 1842 -> 342 rows; 342 <= 600 and 6 x 11 < 75 stops there


def test_default_omega_is_twice_the_gershgorin_textbook_value():
    """omega = relax (4/3) / rho with relax = 2 by default: exactly twice the
    relax = 1 value, with rho the Gershgorin bound of the level's matrix."""
    p = q.make_problem((9, 8, 10), traction=(0, 0, -1), inclusion_frac=0.2)
    H2, H1 = _hierarchy(p, coarse_enough=100), _hierarchy(p, coarse_enough=100, relax=1.0)
    L2, L1 = H2.level(0), H1.level(0)
    _, rho = o.jacobi_rho(L2["A"])
    assert L2["rho"] == rho and L2["omega"] == 2.0 * (4.0 / 3.0) / rho
    assert L2["omega"] == 2.0 * L1["omega"]


def _hierarchy(p, **kw):
    return o.Hierarchy(o.from_problem(p), 3, p.B, **kw)


@pytest.mark.parametrize("eps", [0.0, 0.08])
def test_smoothed_prolongation_keeps_rigid_modes(eps):
    # On the unconstrained (singular) operator A B = 0, so the smoothed
    # prolongation reproduces the modes, P B_c = (I - w D^-1 A) P_tent B_c =
    # B - w D^-1 A B = B, whatever aggregates the threshold produces, and every
    # Galerkin operator annihilates its restricted rigid-body modes.  The
    # coarsening steps are chained by hand (a singular coarsest matrix has no
    # Cholesky factor, so the full setup does not apply).
    p = q.make_problem((6, 5, 4), clamp=False, body=(0, 0, -1))
    A, B, b = o.from_problem(p), p.B, 3
    for level in range(3):
        nn = A.shape[0] // b
        agg, nagg = o.aggregate(A, b, eps * 0.5 ** level)
        assert nagg < nn
        rows = np.repeat(agg >= 0, b)
        Pt, Bc = o.tentative(nn, b, agg, nagg, B)
        d, rho = o.jacobi_rho(A)
        P = o.smooth_prolongation(A, d, (4.0 / 3.0) / rho, Pt)
        Ps = P.to_scipy()
        scale = np.abs(B).max()
        assert np.abs((Ps @ Bc - B)[rows]).max() <= 1e-10 * scale
        Ac = o.spgemm(o.transpose(P), o.spgemm(A, P))
        As = Ac.to_scipy()
        scale = max(abs(As).max(), abs(A.to_scipy()).max())  # A_c may vanish entirely
        assert np.abs(As @ Bc).max() <= 1e-10 * scale * np.abs(Bc).max()
        A, B, b = Ac, Bc, 6
        if nagg < 2:
            break


def test_prolongation_and_galerkin_against_dense_algebra():
    p = q.make_problem((4, 4, 3), traction=(0, 0, -1), inclusion_frac=0.2)
    A = o.from_problem(p)
    agg, nagg = o.aggregate(A, 3, 0.08)
    Pt, Bc = o.tentative(p.nnodes, 3, agg, nagg, p.B)
    d, rho = o.jacobi_rho(A)
    w = (4.0 / 3.0) / rho
    P = o.smooth_prolongation(A, d, w, Pt)
    Pd, Ptd, Ad = P.to_dense(), Pt.to_dense(), A.to_dense()
    dense = Ptd - w * (Ad / d[:, None]) @ Ptd
    np.testing.assert_allclose(Pd, dense, atol=1e-14)
    R = o.transpose(P)
    np.testing.assert_array_equal(R.to_dense(), Pd.T)
    Ac = o.spgemm(R, o.spgemm(A, P))
    Acd = Ac.to_dense()
    np.testing.assert_allclose(Acd, Pd.T @ A.to_dense() @ Pd, atol=1e-13 * np.abs(Acd).max())
    assert np.abs(Acd - Acd.T).max() <= 1e-13 * np.abs(Acd).max()
    # symbolic pattern: every P row of an aggregated node has whole 6-column groups
    cnt = np.diff(P.ptr)
    assert (cnt % 6 == 0).all()


def test_spgemm_symbolic_pattern_keeps_cancellation():
    A = o.CSR([0, 2, 4], [0, 1, 0, 1], [1.0, 1.0, 1.0, 1.0], (2, 2))
    B = o.CSR([0, 1, 2], [0, 0], [1.0, -1.0], (2, 1))
    C = o.spgemm(A, B)  # exact cancellation: entries stay, value 0
    assert C.col.tolist() == [0, 0] and C.val.tolist() == [0.0, 0.0]


# ---------------------------------------------------------------- smoother, coarse solver
def test_spai0_diagonal_matrix_is_exact_inverse_and_minimal():
    d = np.array([2.0, 4.0, 0.5])
    A = o.CSR([0, 1, 2, 3], [0, 1, 2], d, (3, 3))
    np.testing.assert_allclose(o.spai0(A), 1.0 / d, rtol=1e-15)
    A = o.from_problem(q.cube(3))
    m = o.spai0(A)
    Ad = A.to_dense()
    f0 = np.linalg.norm(np.eye(len(m)) - m[:, None] * Ad)
    rng = np.random.default_rng(1)
    for _ in range(5):
        dm = 1e-3 * rng.standard_normal(len(m)) * np.abs(m)
        assert np.linalg.norm(np.eye(len(m)) - (m + dm)[:, None] * Ad) > f0


def _block_diag_csr(blocks):
    """Scalar CSR of a block-diagonal matrix with the given dense blocks
    (explicit zeros kept inside each block)."""
    b = blocks.shape[1]
    n = len(blocks) * b
    ptr, col, val = [0], [], []
    for I, B in enumerate(blocks):
        for r in range(b):
            col += list(range(I * b, I * b + b))
            val += list(B[r])
            ptr.append(len(col))
    return o.CSR(ptr, col, np.array(val), (n, n))


@pytest.mark.parametrize("b", [3, 6])
def test_block_jacobi_inverts_blocks_and_drops_zero_rows(b):
    """Block damped Jacobi blocks: M_I A_II = w I on each SPD block, exactly
    symmetric; a zero row and column of A_II (a dropped near-nullspace column
    below the finest level) gives a zero row and column of M_I and M is the
    inverse on the other rows and columns; a non-positive pivot is an error."""
    rng = np.random.default_rng(b)
    blocks = []
    for _ in range(4):
        X = rng.standard_normal((b, b))
        blocks.append(X @ X.T + b * np.eye(b))
    blocks = np.array(blocks)
    blocks[2][1, :] = blocks[2][:, 1] = 0.0
    w = 0.7
    M = o.block_jacobi(_block_diag_csr(blocks), b, w)
    for I in range(4):
        assert np.array_equal(M[I], M[I].T)
        keep = np.ones(b, bool)
        if I == 2:
            keep[1] = False
            assert not M[I][1].any() and not M[I][:, 1].any()
        k = np.ix_(keep, keep)
        np.testing.assert_allclose(M[I][k] @ blocks[I][k], w * np.eye(keep.sum()), atol=1e-13)
    blocks[3] = -blocks[3]
    with pytest.raises(ValueError):
        o.block_jacobi(_block_diag_csr(blocks), b, w)


def test_block_jacobi_lambda_is_a_tight_lower_bound():
    """The Rayleigh-quotient estimate of lambda_max(D_b^{-1} A): exactly 1 on
    a block-diagonal A (D_b^{-1} A = I); on Q1 elasticity at most the dense
    eigenvalue and within 10 % of it after 20 power iterations."""
    rng = np.random.default_rng(9)
    blocks = []
    for _ in range(5):
        X = rng.standard_normal((3, 3))
        blocks.append(X @ X.T + 3 * np.eye(3))
    A = _block_diag_csr(np.array(blocks))
    W = o.block_jacobi(A, 3, 1.0)
    assert abs(o.block_jacobi_lambda(A, 3, W) - 1.0) <= 1e-13
    for shape, kw in [((4, 4, 4), {}), ((5, 4, 6), {"inclusion_frac": 0.2}),
                      ((5, 5, 5), {"nu": 0.45})]:
        p = q.make_problem(shape, body=(0, 0, -1), **kw)
        A = o.from_problem(p)
        W = o.block_jacobi(A, 3, 1.0)
        lam = o.block_jacobi_lambda(A, 3, W)
        Ad = A.to_dense()
        D = np.zeros_like(Ad)
        for I in range(Ad.shape[0] // 3):
            D[3 * I:3 * I + 3, 3 * I:3 * I + 3] = Ad[3 * I:3 * I + 3, 3 * I:3 * I + 3]
        top = np.linalg.eigvals(np.linalg.solve(D, Ad)).real.max()
        assert 0.9 * top <= lam <= top * (1 + 1e-12), (shape, lam, top)


def test_block_jacobi_hierarchy_damping_vcycle_and_solve():
    """The block damped Jacobi smoother of every level is (2 w_s / lambda)
    A_II^{-1} with lambda the level's estimate, so the damped operator M A
    peaks between 2 w_s and 2 w_s / 0.9; the V-cycle stays symmetric; PCG
    meets the dense direct solve and needs fewer iterations than SPAI0 on
    this inclusions mesh."""
    p = q.make_problem((6, 5, 7), body=(0, 0, -1), inclusion_frac=0.2)
    A = o.from_problem(p)
    H = o.Hierarchy(A, 3, p.B, coarse_enough=150, smoother="bjacobi")
    assert H.nlevels >= 2
    for l in range(H.nlevels - 1):
        L = H.level(l)
        b = L["b"]
        lam = L["bj_lambda"]
        W = o.block_jacobi(L["A"], b, 1.0)
        np.testing.assert_allclose(L["Mb"], (2 * 0.8 / lam) * W, rtol=1e-14, atol=0)
        if l == 0:
            Ad = L["A"].to_dense()
            Md = np.zeros_like(Ad)
            for I in range(len(W)):
                Md[b * I:b * I + b, b * I:b * I + b] = L["Mb"][I]
            top = np.linalg.eigvals(Md @ Ad).real.max()
            assert 1.6 * (1 - 1e-12) <= top <= 1.6 / 0.9, top
    rng = np.random.default_rng(12)
    x, y = rng.standard_normal(p.ndof), rng.standard_normal(p.ndof)
    a, c = x @ H.vcycle(y), y @ H.vcycle(x)
    assert abs(a - c) <= 1e-12 * abs(a)
    u, it, rel = H.solve(p.f, tol=1e-8)
    us = np.linalg.solve(q.bsr_to_dense(p), p.f)
    assert rel <= 1e-8 and np.linalg.norm(u - us) <= 1e-7 * np.linalg.norm(us)
    _, it0, _ = o.Hierarchy(A, 3, p.B, coarse_enough=150).solve(p.f, tol=1e-8)
    assert it < it0, (it, it0)


def test_cholesky_against_lapack_and_zero_rows():
    rng = np.random.default_rng(2)
    X = rng.standard_normal((12, 12))
    S = X @ X.T + 12 * np.eye(12)
    S[4, :] = S[:, 4] = 0.0
    L, z, rc = o.cholesky(S)
    assert rc == 0 and z.tolist() == [1 if i == 4 else 0 for i in range(12)]
    f = rng.standard_normal(12)
    u = o.cholesky_solve(L, z, f)
    keep = np.arange(12) != 4
    np.testing.assert_allclose(u[keep], np.linalg.solve(S[np.ix_(keep, keep)], f[keep]), rtol=1e-12)
    assert u[4] == 0.0
    L, z, rc = o.cholesky(-np.eye(3))
    assert rc < 0


# ---------------------------------------------------------------- V-cycle, CG
def test_vcycle_is_symmetric():
    p = q.inclusions(6)
    H = _hierarchy(p, coarse_enough=200)
    assert H.nlevels >= 2
    rng = np.random.default_rng(3)
    x, y = rng.standard_normal(p.ndof), rng.standard_normal(p.ndof)
    a, b = x @ H.vcycle(y), y @ H.vcycle(x)
    assert abs(a - b) <= 1e-12 * abs(a)


def test_coarse_correction_is_a_projection():
    # no smoothing, two levels: V = P A_c^-1 P^T, so (V A)^2 = V A
    p = q.cube(6)
    H = _hierarchy(p, coarse_enough=400, npre=0, npost=0)
    assert H.nlevels == 2
    A = o.from_problem(p).to_scipy()
    x = np.random.default_rng(4).standard_normal(p.ndof)
    vx = H.vcycle(A @ x)
    np.testing.assert_allclose(H.vcycle(A @ vx), vx, atol=1e-9 * np.abs(vx).max())


def test_one_level_hierarchy_is_a_direct_solve():
    p = q.cube(3)
    H = _hierarchy(p, coarse_enough=10 ** 6)
    assert H.nlevels == 1
    u, it, rel = H.solve(p.f, tol=1e-10)
    assert it == 1 and rel <= 1e-10


@pytest.mark.parametrize("shape,kw", [((4, 4, 4), {}), ((6, 3, 5), {"inclusion_frac": 0.2}),
                                      ((8, 8, 8), {"inclusion_frac": 0.2})])
def test_pcg_matches_dense_direct_solve(shape, kw):
    p = q.make_problem(shape, traction=(0, 0, -1), **kw)
    H = _hierarchy(p, coarse_enough=150)
    assert H.nlevels >= 2
    u, it, rel = H.solve(p.f, tol=1e-8)
    us = np.linalg.solve(q.bsr_to_dense(p), p.f)
    assert rel <= 1e-8
    assert np.linalg.norm(u - us) <= 1e-7 * np.linalg.norm(us)
    assert 1 <= it < 400


def test_pcg_zero_rhs_and_warm_start():
    p = q.cube(4)
    H = _hierarchy(p, coarse_enough=150)
    u, it, rel = H.solve(np.zeros(p.ndof))
    assert it == 0 and not u.any()
    us, _, _ = H.solve(p.f, tol=1e-12)
    u, it, rel = H.solve(p.f, u0=us, tol=1e-8)
    assert it == 0 and rel <= 1e-8
