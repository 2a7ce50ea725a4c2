"""Pins of the synthetic input generator (Q1 hexahedral linear elasticity).

The generator builds the system of Eq. 1 and the n x 6 rigid-body-mode matrix
B of Sec. 2.  These tests tie it to facts of the continuum problem rather
than to its own formulas.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as sla

import q1elasticity as q


def _scipy(p):
    n = p.nnodes
    return sp.bsr_matrix((p.val, p.col, p.row_ptr), shape=(3 * n, 3 * n)).tocsr()


def test_splitmix64_reference_vector():
    # First output of SplitMix64 from state 0, as published with the generator.
    assert q.splitmix64(0)[0] == 0xE220A8397B1DCDAF


@pytest.mark.parametrize("nu", [0.2, 0.3, 0.45])
def test_element_stiffness_rigid_modes(nu):
    Ke = q.element_stiffness(0.5, nu)
    assert np.array_equal(Ke, Ke.T)
    ev = np.linalg.eigvalsh(Ke)
    scale = ev[-1]
    # exactly six zero-energy modes (3 translations, 3 rotations), rest positive
    assert np.sum(np.abs(ev) < 1e-12 * scale) == 6
    assert ev[6] > 1e-6 * scale
    # they are the rigid-body motions of the 8 element nodes
    X = np.array([[(a & 1) * 0.5, ((a >> 1) & 1) * 0.5, ((a >> 2) & 1) * 0.5] for a in range(8)])
    X -= X.mean(0)
    R = np.zeros((24, 6))
    for a, (x, y, z) in enumerate(X):
        R[3 * a:3 * a + 3] = [[1, 0, 0, 0, z, -y], [0, 1, 0, -z, 0, x], [0, 0, 1, y, -x, 0]]
    assert np.abs(Ke @ R).max() <= 1e-13 * scale


def test_element_stiffness_uniaxial_strain_energy():
    # A homogeneous strain eps_xx = 1 on a unit cube stores energy
    # (lambda + 2 mu) / 2 per unit volume (closed form of linear elasticity).
    nu = 0.3
    lam = nu / ((1 + nu) * (1 - 2 * nu))
    mu = 1 / (2 * (1 + nu))
    Ke = q.element_stiffness(1.0, nu)
    u = np.zeros(24)
    for a in range(8):
        u[3 * a] = float(a & 1)  # u_x = x
    assert abs(0.5 * u @ Ke @ u - 0.5 * (lam + 2 * mu)) < 1e-14


def test_unconstrained_matrix_annihilates_rigid_modes():
    p = q.make_problem((4, 3, 5), clamp=False, body=(0, 0, -1))
    A = _scipy(p)
    KB = A @ p.B
    assert np.abs(KB).max() <= 1e-13 * abs(A).max() * np.abs(p.B).max()


def test_symmetric_and_positive_definite_when_clamped():
    p = q.make_problem((3, 2, 4), body=(0, 0, -1))
    A = q.bsr_to_dense(p)
    assert np.array_equal(A, A.T)
    assert np.linalg.eigvalsh(A)[0] > 0


def test_patch_test_reproduces_linear_field():
    # Q1 elements reproduce any linear displacement exactly: prescribe
    # u = a + G x on the boundary, solve for the interior, compare.
    p = q.make_problem((4, 4, 4), clamp=False, body=None)
    A = _scipy(p).tocsr()
    rng = np.random.default_rng(0)
    a, G = rng.standard_normal(3), rng.standard_normal((3, 3))
    u_exact = (a[None, :] + p.coords @ G.T).ravel()
    x = p.coords
    hmax = x.max(0)
    bnd = np.any((x <= 1e-12) | (x >= hmax - 1e-12), axis=1)
    bd = np.repeat(bnd, 3)
    inn = ~bd
    rhs = -A[inn][:, bd] @ u_exact[bd]
    u_in = sla.spsolve(A[inn][:, inn].tocsc(), rhs)
    assert np.abs(u_in - u_exact[inn]).max() <= 1e-10 * np.abs(u_exact).max()


def test_loads_sum_to_resultants():
    p = q.make_problem((3, 4, 2), clamp=False, body=(0.5, 0.0, -1.0))
    V = 3 * 4 * 2 * p.h ** 3
    np.testing.assert_allclose(p.f.reshape(-1, 3).sum(0), [0.5 * V, 0.0, -V], rtol=1e-14, atol=1e-15)
    p = q.make_problem((3, 4, 2), clamp=False, traction=(0.0, 0.0, -1.0))
    area = 4 * 2 * p.h ** 2
    np.testing.assert_allclose(p.f.reshape(-1, 3).sum(0), [0.0, 0.0, -area], rtol=1e-14, atol=1e-15)


def test_clamped_rows_are_identity_and_decoupled():
    p = q.make_problem((3, 2, 2), body=(0, 0, -1))
    A = q.bsr_to_dense(p)
    clamped = np.repeat(p.coords[:, 0] == 0.0, 3)
    assert np.array_equal(A[clamped][:, clamped], np.eye(clamped.sum()))
    assert not A[clamped][:, ~clamped].any()
    assert not p.f[clamped].any()


def test_inclusion_volume_fraction():
    E = q.material((16, 16, 16), 1 / 16, inclusion_frac=0.2, seed=2202)
    frac = np.mean(E == 1000.0)
    assert 0.2 <= frac < 0.3
    assert set(np.unique(E)) == {1.0, 1000.0}
    E2 = q.material((16, 16, 16), 1 / 16, inclusion_frac=0.2, seed=2202)
    assert np.array_equal(E, E2)


def test_matrix_scales_with_material():
    p1 = q.make_problem(3, body=(0, 0, -1))
    p2 = q.make_problem(3, body=(0, 0, -1), E_el=np.full(27, 7.0))
    free = p1.val[:, 0, 0] != 1.0
    np.testing.assert_allclose(p2.val[free], 7.0 * p1.val[free], rtol=1e-14,
                               atol=1e-14 * np.abs(p2.val).max())


def test_batch_specs_ranges_and_determinism():
    s = q.batch_specs(64)
    assert len(s) == 64
    assert all(20 <= x["n"] <= 60 and 0.2 <= x["nu"] < 0.45 and 1 <= x["nrhs"] <= 16 for x in s)
    assert all(np.allclose(np.linalg.norm(x["body"], axis=1), 1.0) for x in s)
    assert [x["n"] for x in s] == [x["n"] for x in q.batch_specs(64)]
