"""Pins of the FP64 learned-smoother reference (oracle/learned.py) and of the
oracle's block smoother.

* the analytic gradient equals central finite differences (h = 1e-6);
* dL/dM equals the derivative of the loss written densely;
* a zero output layer reproduces SPAI0: same blocks, same V-cycle, same CG
  iterations as the scalar SPAI0 hierarchy;
* features are unit-free (scaling A leaves them unchanged).
"""
import numpy as np
import pytest

import oracle as o
import oracle.learned as lo
import q1elasticity as q


def _setup(shape=(5, 4, 6)):
    p = q.make_problem(shape, traction=(0, 0, -1), inclusion_frac=0.2)
    A = o.from_problem(p).to_scipy()
    H = o.Hierarchy(o.from_problem(p), 3, p.B, coarse_enough=100)
    m = H.level(0)["M"]
    X = lo.features(p.row_ptr, p.col, p.val)
    rng = np.random.default_rng(0)
    R = rng.standard_normal((3, p.ndof))
    return p, A, H, m, X, R


def test_features_are_unit_free():
    p = q.make_problem((4, 3, 4), traction=(0, 0, -1), inclusion_frac=0.2)
    X1 = lo.features(p.row_ptr, p.col, p.val)
    X2 = lo.features(p.row_ptr, p.col, 37.5 * p.val)
    np.testing.assert_allclose(X1, X2, rtol=1e-14, atol=1e-15)
    clamped = p.coords[:, 0] == 0.0
    np.testing.assert_allclose(X1[clamped, :9], np.tile(np.eye(3).ravel() / np.sqrt(3), (clamped.sum(), 1)))
    assert (X1[clamped, 9:11] == 0).all()


def test_gradient_matches_finite_differences():
    p, A, H, m, X, R = _setup()
    prm = lo.init_params(seed=1)
    prm["W2"] = 0.05 * np.random.default_rng(2).standard_normal(prm["W2"].shape)
    prm["b2"] = 0.02 * np.random.default_rng(3).standard_normal(6)
    L, g = lo.grad_params(prm, X, m, A, R)
    v = lo.flatten(prm)
    rng = np.random.default_rng(4)
    idx = rng.choice(lo.NPARAM, 25, replace=False)
    h = 1e-6
    for i in idx:
        vp, vm = v.copy(), v.copy()
        vp[i] += h
        vm[i] -= h
        fd = (lo.loss(lo.unflatten(vp), X, m, A, R) - lo.loss(lo.unflatten(vm), X, m, A, R)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(g).max(), 1e-12) + 1e-6 * abs(fd), (i, fd, g[i])


def test_grad_M_matches_dense_derivative():
    p, A, H, m, X, R = _setup((3, 3, 3))
    prm = lo.init_params(seed=1)
    o_, _, _ = lo.forward(prm, X)
    M = lo.smoother_blocks(m, o_)
    L, G = lo.loss_and_grad_M(A, M, R[:1])
    Ad = A.toarray()
    e = R[0]
    # dense: L(Mb) = e'^T A e' / e^T A e with e' = (I - Mb A) e, Mb block diagonal
    n = len(e)
    Mb = np.zeros((n, n))
    for I in range(n // 3):
        Mb[3 * I:3 * I + 3, 3 * I:3 * I + 3] = M[I]
    ep = e - Mb @ Ad @ e
    assert np.isclose(L, ep @ Ad @ ep / (e @ Ad @ e), rtol=1e-12)
    Gd = -2.0 * np.outer(Ad @ ep, Ad @ e) / (e @ Ad @ e)
    for I in range(n // 3):
        np.testing.assert_allclose(G[I], Gd[3 * I:3 * I + 3, 3 * I:3 * I + 3], rtol=1e-10, atol=1e-14)


def test_loss_penalises_an_unstable_smoother():
    # scaling SPAI0 up until lambda_max(M A) passes 2 makes the energy-norm
    # loss on white-noise errors exceed 1 (some errors grow)
    p, A, H, m, X, R = _setup((5, 5, 5))
    base = np.einsum("ni,ij->nij", m.reshape(-1, 3), np.eye(3))
    L1, _ = lo.loss_and_grad_M(A, base, R)
    L3, _ = lo.loss_and_grad_M(A, 3.0 * base, R)
    assert L1 < 1.0 < L3


def test_zero_output_layer_is_spai0():
    p, A, H, m, X, R = _setup((8, 7, 6))
    prm = lo.init_params(seed=5)
    o_, _, _ = lo.forward(prm, X)
    M = lo.smoother_blocks(m, o_)
    np.testing.assert_allclose(M, np.einsum("ni,ij->nij", m.reshape(-1, 3), np.eye(3)), atol=0)
    u0, it0, _ = H.solve(p.f, tol=1e-8)
    z0 = H.vcycle(R[0])
    H.set_block_smoother(0, M)
    u1, it1, _ = H.solve(p.f, tol=1e-8)
    assert it1 == it0
    np.testing.assert_allclose(H.vcycle(R[0]), z0, rtol=1e-14, atol=1e-14 * np.abs(z0).max())


def test_block_smoother_vcycle_stays_symmetric():
    p, A, H, m, X, R = _setup((6, 5, 5))
    prm = lo.init_params(seed=5)
    prm["W2"] = 0.05 * np.random.default_rng(6).standard_normal(prm["W2"].shape)
    o_, _, _ = lo.forward(prm, X)
    H.set_block_smoother(0, lo.smoother_blocks(m, o_))
    x, y = R[0], R[1]
    a, b = x @ H.vcycle(y), y @ H.vcycle(x)
    assert abs(a - b) <= 1e-12 * abs(a)
