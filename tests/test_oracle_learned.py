"""Pins of the FP64 learned-smoother reference (oracle/learned.py) and of the
oracle's block smoother.

* the analytic gradient equals central finite differences (h = 1e-6);
* dL/dM equals the derivative of the loss written densely;
* a zero output layer reproduces SPAI0: same blocks, same V-cycle, same CG
  iterations as the scalar SPAI0 hierarchy;
* features are unit-free (scaling A leaves them unchanged);
* the output-to-block map puts each output in its place of the lower
  triangular factor (closed forms for single outputs) and gives symmetric
  positive semidefinite blocks for any output.
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


def test_factor_mapping_and_definiteness():
    m = np.array([4.0, 9.0, 16.0])          # S = diag(2, 3, 4)
    S = np.diag([2.0, 3.0, 4.0])
    t = 0.7
    # o3 sits at L[1, 0]: K = [[1, t, 0], [t, 1 + t^2, 0], [0, 0, 1]]
    o3 = np.zeros((1, 6))
    o3[0, 3] = t
    K = np.array([[1, t, 0], [t, 1 + t * t, 0], [0, 0, 1]])
    np.testing.assert_allclose(lo.smoother_blocks(m, o3)[0], S @ K @ S, rtol=1e-15)
    # o5 sits at L[2, 1] and o1 on L[1, 1]
    o = np.zeros((1, 6))
    o[0, 1], o[0, 5] = -0.5, t
    K = np.array([[1, 0, 0], [0, 0.25, 0.5 * t], [0, 0.5 * t, t * t + 1]])
    np.testing.assert_allclose(lo.smoother_blocks(m, o)[0], S @ K @ S, rtol=1e-15)
    # any output: symmetric, eigenvalues >= 0; singular exactly when 1 + o_k = 0
    rng = np.random.default_rng(1)
    o = 3.0 * rng.standard_normal((200, 6))
    M = lo.smoother_blocks(np.tile(m, 200), o)
    np.testing.assert_array_equal(M, np.transpose(M, (0, 2, 1)))
    assert np.linalg.eigvalsh(M).min() >= -1e-12 * np.abs(M).max()
    o[0, :3] = [-1.0, 0.3, 0.2]
    assert abs(np.linalg.det(lo.smoother_blocks(m, o[:1])[0])) == 0.0


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
