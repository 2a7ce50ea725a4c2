"""ORACLE -- test infrastructure only.  FP64 reference of the learned smoother.

The learned smoother replaces the fine-level SPAI0 diagonal by a 3x3 block per
node, produced by a small MLP from unit-free features of the node's block row:

  features x_I (12): A_II / ||A_II||_F (9, row-major),
                     sum_{J != I} ||A_IJ||_F^2 / ||A_II||_F^2,
                     max_{J != I} ||A_IJ||_F / ||A_II||_F,
                     (number of blocks in row I) / 27;
  network:           h = relu(W1 x + b1) (64), o = W2 h + b2 (6);
  smoother block:    M_I = S_I L_I L_I^T S_I, S_I = diag(sqrt(m)) with m the
                     damped SPAI0 diagonal of the node's three scalar rows and
                     L_I the lower-triangular factor
                     [[1 + o0, 0, 0], [o3, 1 + o1, 0], [o4, o5, 1 + o2]].

M_I is symmetric positive semidefinite for every output, and definite unless
a diagonal entry of L_I is zero.  A zero output layer gives M_I = diag(m):
plain SPAI0.  The training loss is
the energy-norm error reduction of one smoothing step over error samples e_s,
L = (1/S) sum_s ||e_s - M A e_s||_A^2 / ||e_s||_A^2; with r = A e and
e' = e - M r its gradient with respect to M_I is
-(2/S) sum_s (A e'_s)_I r_{s,I}^T / (e_s . r_s) (A is symmetric).  A step that
amplifies some error (lambda(M A) > 2) raises the loss, so minimising it keeps
the smoother convergent.  Everything here is plain numpy in FP64; only tests
and the benchmark's CPU leg use it.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

NF = 12        # features
NH = 64        # hidden units
NO = 6         # outputs (symmetric 3x3)
TRI = [(0, 0), (1, 1), (2, 2), (1, 0), (2, 0), (2, 1)]   # entry of L_I set by o_k


def features(row_ptr, col, val):
    """Unit-free features of every block row of a 3x3 BSR matrix, [N, 12]."""
    n = row_ptr.shape[0] - 1
    X = np.zeros((n, NF))
    for I in range(n):
        s, e = row_ptr[I], row_ptr[I + 1]
        nrm = np.linalg.norm(val[s:e].reshape(e - s, 9), axis=1)
        d = np.nonzero(col[s:e] == I)[0][0] + s
        nI = np.linalg.norm(val[d])
        X[I, :9] = (val[d] / nI).ravel()
        off = [k for k in range(s, e) if k != d]
        if off:
            X[I, 9] = np.sum(nrm[np.array(off) - s] ** 2) / nI ** 2
            X[I, 10] = np.max(nrm[np.array(off) - s]) / nI
        X[I, 11] = (e - s) / 27.0
    return X


def init_params(seed=0, scale=0.3):
    """W1 small seeded Gaussian, W2 = 0 and biases 0: the start is SPAI0."""
    rng = np.random.default_rng(seed)
    return {"W1": scale * rng.standard_normal((NH, NF)) / np.sqrt(NF), "b1": np.zeros(NH),
            "W2": np.zeros((NO, NH)), "b2": np.zeros(NO)}


def flatten(p):
    return np.concatenate([p["W1"].ravel(), p["b1"], p["W2"].ravel(), p["b2"]])


def unflatten(v):
    v = np.asarray(v, dtype=np.float64)
    i = 0
    out = {}
    for k, shape in (("W1", (NH, NF)), ("b1", (NH,)), ("W2", (NO, NH)), ("b2", (NO,))):
        size = int(np.prod(shape))
        out[k] = v[i:i + size].reshape(shape)
        i += size
    return out


NPARAM = NH * NF + NH + NO * NH + NO


def forward(p, X):
    pre = X @ p["W1"].T + p["b1"]
    h = np.maximum(pre, 0.0)
    o = h @ p["W2"].T + p["b2"]
    return o, h, pre


def factor_from_output(o):
    """L_I = I + the lower-triangular matrix holding the six outputs, [N, 3, 3]."""
    L = np.zeros((o.shape[0], 3, 3))
    L[:] = np.eye(3)
    for k, (a, b) in enumerate(TRI):
        L[:, a, b] += o[:, k]
    return L


def smoother_blocks(m, o):
    """M_I = S L L^T S with S = diag(sqrt(m_I)), [N, 3, 3]."""
    S = np.sqrt(np.asarray(m).reshape(-1, 3))
    L = factor_from_output(o)
    K = L @ np.transpose(L, (0, 2, 1))
    return S[:, :, None] * K * S[:, None, :]


def apply_blocks(M, r):
    return np.einsum("nab,nb->na", M, r.reshape(-1, 3)).ravel()


def loss_and_grad_M(A: sp.spmatrix, M, E):
    """L and dL/dM (unsymmetrised, [N, 3, 3]) for error samples E [S, n]."""
    S = E.shape[0]
    L = 0.0
    G = np.zeros_like(M)
    for e in E:
        r = A @ e
        den = e @ r
        ep = e - apply_blocks(M, r)
        g = A @ ep
        L += (ep @ g) / den
        G += np.einsum("na,nb->nab", (-2.0 / den) * g.reshape(-1, 3), r.reshape(-1, 3))
    return L / S, G / S


def grad_params(p, X, m, A, R):
    """(L, flat gradient) of the loss over error samples R with respect to
    (W1, b1, W2, b2)."""
    o, h, pre = forward(p, X)
    M = smoother_blocks(m, o)
    L, GM = loss_and_grad_M(A, M, R)
    S = np.sqrt(np.asarray(m).reshape(-1, 3))
    GK = S[:, :, None] * GM * S[:, None, :]          # dL/dK, K = L L^T
    GL = (GK + np.transpose(GK, (0, 2, 1))) @ factor_from_output(o)   # dL/dL
    do = np.zeros((X.shape[0], NO))
    for k, (a, b) in enumerate(TRI):
        do[:, k] = GL[:, a, b]
    gW2 = do.T @ h
    gb2 = do.sum(0)
    dh = (do @ p["W2"]) * (pre > 0)
    gW1 = dh.T @ X
    gb1 = dh.sum(0)
    return L, np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2])


def loss(p, X, m, A, R):
    o, _, _ = forward(p, X)
    return loss_and_grad_M(A, smoother_blocks(m, o), R)[0]
