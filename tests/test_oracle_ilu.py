"""Pins of the oracle's block ILU(0) (the smoother of Sec. 4's experiments)
and the measured reason it has no GPU path here.

* L U equals A on A's block pattern (dense products; a wrong update index or
  block order breaks it), U's diagonal inverses are inverses;
* on a block-tridiagonal matrix (a chain of nodes) ILU(0) has no dropped fill,
  so it is the exact LU: applying it with enough Jacobi sweeps solves A x = r;
* the Jacobi sweeps of a triangular solve converge to the exact substitution
  (they are exact after as many sweeps as the triangle's depth);
* for symmetric A the factors give a symmetric M^-1 = (L U)^-1;
* findings: on a homogeneous cube the ILU(0) V(1,1) needs about half the
  iterations of SPAI0, but with fewer than three Jacobi sweeps per triangle
  the smoother amplifies errors and CG breaks down; on the E = 1000
  inclusion meshes ILU(0) itself is indefinite (a negative eigenvalue of
  M^-1 A), so it cannot precondition CG there.
"""
import numpy as np
import pytest

import oracle as o
import q1elasticity as q


def _dense_factors(F, n):
    ptr, col, val, dinv = F.factors()
    b = F.b
    L, U = np.eye(n), np.zeros((n, n))
    for I in range(F.nb):
        for k in range(ptr[I], ptr[I + 1]):
            J = col[k]
            blk = (slice(b * I, b * I + b), slice(b * J, b * J + b))
            if J < I:
                L[blk] = val[k]
            else:
                U[blk] = val[k]
    return L, U, dinv


def test_lu_matches_a_on_the_block_pattern():
    p = q.make_problem((4, 3, 3), traction=(0, 0, -1), inclusion_frac=0.2)
    A = o.from_problem(p)
    F = o.ILU0(A, 3)
    Ad = A.to_dense()
    L, U, dinv = _dense_factors(F, Ad.shape[0])
    on = Ad != 0
    assert np.abs((L @ U - Ad)[on]).max() <= 1e-13 * np.abs(Ad).max()
    for I in range(F.nb):
        np.testing.assert_allclose(dinv[I] @ U[3 * I:3 * I + 3, 3 * I:3 * I + 3], np.eye(3),
                                   atol=1e-12)


def _chain(nb, b=3, seed=0):
    """Block tridiagonal SPD matrix (a chain of nb nodes)."""
    rng = np.random.default_rng(seed)
    n = nb * b
    A = np.zeros((n, n))
    for I in range(nb - 1):
        C = 0.3 * rng.standard_normal((b, b))
        A[b * I:b * I + b, b * I + b:b * I + 2 * b] = C
        A[b * I + b:b * I + 2 * b, b * I:b * I + b] = C.T
    for I in range(nb):
        G = rng.standard_normal((b, b))
        A[b * I:b * I + b, b * I:b * I + b] = G @ G.T + 3 * np.eye(b)
    ptr, col, val = [0], [], []
    for i in range(n):
        for j in range(n):
            if abs(i // b - j // b) <= 1:
                col.append(j)
                val.append(A[i, j])
        ptr.append(len(col))
    return A, o.CSR(ptr, col, val, (n, n))


def test_tridiagonal_ilu0_is_exact_lu():
    A, Acsr = _chain(7)
    F = o.ILU0(Acsr, 3)
    r = np.random.default_rng(1).standard_normal(A.shape[0])
    x = F.apply(r, 7)  # the triangles have depth 7: exact after 7 sweeps
    np.testing.assert_allclose(A @ x, r, atol=1e-11 * np.abs(r).max())


def test_jacobi_sweeps_converge_to_the_substitution():
    A, Acsr = _chain(6, seed=2)
    F = o.ILU0(Acsr, 3)
    L, U, _ = _dense_factors(F, A.shape[0])
    r = np.random.default_rng(3).standard_normal(A.shape[0])
    exact = np.linalg.solve(U, np.linalg.solve(L, r))
    errs = [np.linalg.norm(F.apply(r, k) - exact) for k in range(7)]
    assert errs[-1] <= 1e-12 * np.linalg.norm(exact)
    assert errs[0] > 1e-6 * np.linalg.norm(exact)


def test_symmetric_a_gives_symmetric_preconditioner():
    p = q.make_problem((3, 3, 3), body=(0, 0, -1))
    A = o.from_problem(p)
    F = o.ILU0(A, 3)
    n = p.ndof
    Minv = np.stack([F.apply(e, 40) for e in np.eye(n)], 1)
    assert np.abs(Minv - Minv.T).max() <= 1e-12 * np.abs(Minv).max()


def test_findings_homogeneous_cube_and_inclusions():
    p = q.cube(8)
    it = {}
    for sm, sw in (("spai0", 0), ("ilu0", 3), ("ilu0", 40)):
        H = o.Hierarchy(o.from_problem(p), 3, p.B, coarse_enough=300, smoother=sm, ilu_sweeps=sw)
        it[(sm, sw)] = H.solve(p.f, maxiter=3000)[1]
    assert it[("ilu0", 40)] * 1.6 < it[("spai0", 0)] and it[("ilu0", 3)] < it[("spai0", 0)]
    H1 = o.Hierarchy(o.from_problem(p), 3, p.B, coarse_enough=300, smoother="ilu0", ilu_sweeps=1)
    with pytest.raises(RuntimeError):
        H1.solve(p.f, maxiter=3000)
    # inclusions: the exact ILU(0) preconditioner is indefinite
    pi = q.inclusions(6)
    A = o.from_problem(pi)
    F = o.ILU0(A, 3)
    Ad = A.to_dense()
    Minv = np.stack([F.apply(e, 60) for e in np.eye(pi.ndof)], 1)
    lam = np.linalg.eigvals(Minv @ Ad).real
    assert lam.min() < -0.1


def test_zero_dof_row_gets_unit_pivot_and_zero_output():
    """A DOF whose whole row and column are zero (a coarse DOF whose
    near-nullspace column was dropped in the QR) gets a unit pivot in its
    diagonal block's inverse, a zero row and column there, and a zero
    component in every application; the other DOFs are solved as if it were
    absent."""
    A, _ = _chain(5, b=3, seed=4)
    z = 7                                   # DOF 1 of node 2
    A[z, :] = 0.0
    A[:, z] = 0.0
    n = A.shape[0]
    ptr, col, val = [0], [], []
    for i in range(n):
        for j in range(n):
            if abs(i // 3 - j // 3) <= 1:
                col.append(j)
                val.append(A[i, j])
        ptr.append(len(col))
    F = o.ILU0(o.CSR(ptr, col, val, (n, n)), 3)
    _, _, _, dinv = F.factors()
    assert np.all(dinv[z // 3][z % 3, :] == 0.0) and np.all(dinv[z // 3][:, z % 3] == 0.0)
    r = np.random.default_rng(6).standard_normal(n)
    x = F.apply(r, 5)                       # tridiagonal blocks: exact after 5 sweeps
    assert x[z] == 0.0
    keep = np.arange(n) != z
    np.testing.assert_allclose(A[np.ix_(keep, keep)] @ x[keep], r[keep], atol=1e-11 * np.abs(r).max())
