"""Learned smoother (GPU) against the FP64 reference in oracle/learned.py.

Bars: the tensor-core forward gives the oracle's smoother blocks to BF16
accuracy; the device gradient of the training loss matches the oracle's
analytic (finite-difference-pinned) gradient to BF16 accuracy; with a zero
output layer the solve is the SPAI0 solve; a solve with learned blocks
matches the oracle run with the same blocks (iterations +-1, solution 1e-7);
a singular block, or a smoother with lambda_max(M A) >= max(1.9, SPAI0's),
falls back to SPAI0; training lowers
the energy-norm loss, the result passes the stability check, and the CG
iteration count drops on a mesh it has not seen.
"""
import numpy as np
import pytest

import oracle as o
import oracle.learned as lo
import q1elasticity as q

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
amg = pytest.importorskip("paper_2202_09056_gb300")


def _dev(p):
    d = torch.device("cuda:0")
    return (torch.from_numpy(p.row_ptr).to(d), torch.from_numpy(p.col).to(d),
            torch.from_numpy(p.val).to(d), torch.from_numpy(p.B).to(d))


def _params(seed=3, w2=0.08, bdiag=0.0):
    rng = np.random.default_rng(seed)
    w = amg.learned_init(seed)
    w[64 * 12:64 * 12 + 64] = 0.05 * rng.standard_normal(64)
    w[64 * 13:64 * 13 + 6 * 64] = w2 * rng.standard_normal(6 * 64)
    w[-6:] = 0.02 * rng.standard_normal(6)
    w[-6:-3] += bdiag   # shrink the factor's diagonal: lambda_max(M A) below SPAI0's
    return w.astype(np.float32)


def test_forward_matches_oracle_blocks():
    p = q.make_problem((7, 6, 8), traction=(0, 0, -1), inclusion_frac=0.2)
    G = amg.AMG(*_dev(p), coarse_enough=150)
    w = _params(bdiag=-0.15)
    assert not G.set_learned_smoother(w)
    Mb = G.learned_blocks()
    m = G.export(0)["M"]
    X = lo.features(p.row_ptr, p.col, p.val)
    out, _, _ = lo.forward(lo.unflatten(w.astype(np.float64)), X)
    S = np.sqrt(m.reshape(-1, 3))
    Kg = Mb / (S[:, :, None] * S[:, None, :])
    Lo = lo.factor_from_output(out)
    Ko = Lo @ np.transpose(Lo, (0, 2, 1))
    assert np.abs(Kg - Ko).max() <= 3e-2 * np.abs(Ko - np.eye(3)).max() + 1e-4
    np.testing.assert_allclose(Mb, np.transpose(Mb, (0, 2, 1)), rtol=0, atol=0)


def test_gradient_matches_oracle():
    p = q.make_problem((6, 5, 7), traction=(0, 0, -1), inclusion_frac=0.2)
    G = amg.AMG(*_dev(p), coarse_enough=120)
    H = o.Hierarchy(o.from_problem(p), 3, p.B, coarse_enough=120)
    rng = np.random.default_rng(9)
    A = o.from_problem(p).to_scipy()
    E0 = rng.standard_normal((3, p.ndof))
    R = np.stack([E0[0] - H.vcycle(A @ E0[0]), E0[1], E0[2]])  # error samples
    w = _params(seed=5)
    T = amg.Trainer(w)
    T.add_samples(G, torch.from_numpy(R).cuda())
    loss, g = T.eval()
    m = G.export(0)["M"]
    X = lo.features(p.row_ptr, p.col, p.val)
    Lo, go = lo.grad_params(lo.unflatten(w.astype(np.float64)), X, m, A, R)
    assert abs(loss - Lo) <= 2e-2 * Lo
    assert np.linalg.norm(g - go) <= 5e-2 * np.linalg.norm(go)


def test_zero_output_layer_is_spai0_solve():
    p = q.make_problem((9, 8, 7), traction=(0, 0, -1), inclusion_frac=0.2)
    G = amg.AMG(*_dev(p), coarse_enough=150)
    fb = torch.from_numpy(p.f).cuda()
    u0, it0, _, _ = G.solve(fb)
    assert not G.set_learned_smoother(amg.learned_init(1))
    u1, it1, res1, st = G.solve(fb)
    assert st == amg.AMG_OK and abs(it1 - it0) <= 1
    assert torch.linalg.norm(u1 - u0) <= 1e-7 * torch.linalg.norm(u0)


def test_learned_solve_matches_oracle_with_same_blocks():
    p = q.make_problem((10, 9, 8), traction=(0, 0, -1), inclusion_frac=0.2)
    G = amg.AMG(*_dev(p), coarse_enough=200)
    H = o.Hierarchy(o.from_problem(p), 3, p.B, coarse_enough=200)
    assert not G.set_learned_smoother(_params(seed=7, w2=0.05))
    H.set_block_smoother(0, G.learned_blocks())
    uo, ito, _ = H.solve(p.f, tol=1e-8)
    u, it, res, st = G.solve(torch.from_numpy(p.f).cuda(), tol=1e-8)
    assert st == amg.AMG_OK and abs(it - ito) <= 1, (it, ito)
    assert np.linalg.norm(u.cpu().numpy() - uo) <= 1e-7 * np.linalg.norm(uo)
    r = np.random.default_rng(2).standard_normal(p.ndof)
    z = G.vcycle(torch.from_numpy(r).cuda()).cpu().numpy()
    assert np.linalg.norm(z - H.vcycle(r)) <= 1e-9 * np.linalg.norm(z)


def test_fallback_to_spai0_when_singular_or_unstable():
    p = q.make_problem((6, 6, 6), traction=(0, 0, -1))
    G = amg.AMG(*_dev(p), coarse_enough=150)
    fb = torch.from_numpy(p.f).cuda()
    _, it0, _, _ = G.solve(fb)
    w = amg.learned_init(2)           # W2 = 0: o = b2 on every node
    w[-6] = -1.0                      # 1 + o0 = 0: every block singular
    assert G.set_learned_smoother(w) == 1
    assert G.stats()["learned"] == 0
    _, it1, _, st = G.solve(fb)
    assert st == amg.AMG_OK and it1 == it0
    w[-6:-3] = 2.0                    # L = 3 I: M = 9 x SPAI0, lambda_max(M A) > 2
    assert G.set_learned_smoother(w) == 2
    assert G.stats()["learned_lambda"] > 2.0
    _, it2, _, st = G.solve(fb)
    assert st == amg.AMG_OK and it2 == it0


def test_training_lowers_loss_and_iterations():
    meshes = [q.make_problem(n, traction=(0, 0, -1), inclusion_frac=0.2, seed=s)
              for n, s in ((10, 1), (12, 2))]
    solvers = [amg.AMG(*_dev(p), coarse_enough=300) for p in meshes]
    T = amg.Trainer(amg.learned_init(0), lr=3e-3)
    for k, G in enumerate(solvers):
        T.add_generated(G, 4, seed=10 + k)
    l0, _ = T.eval()
    for _ in range(6):
        T.step(25)
    l1, _ = T.eval()
    assert l1 < 0.9 * l0, (l0, l1)
    test = q.make_problem(14, traction=(0, 0, -1), inclusion_frac=0.2, seed=3)
    G = amg.AMG(*_dev(test), coarse_enough=300)
    fb = torch.from_numpy(test.f).cuda()
    _, it_spai0, _, _ = G.solve(fb)
    assert not G.set_learned_smoother(T.params())
    info = G.stats()
    assert info["learned"] == 1 and 0.5 < info["learned_lambda"] < max(1.9, info["spai0_lambda"]), info
    _, it_learned, res, st = G.solve(fb)
    assert st == amg.AMG_OK and res <= 1e-8
    assert it_learned < it_spai0, (it_learned, it_spai0)
    G.clear_learned_smoother()
    assert G.stats()["learned"] == 0


@pytest.mark.parametrize("prec", [amg.PREC_FP32, amg.PREC_BF16])
def test_learned_blocks_in_reduced_precision_vcycle(prec):
    """The FP32 / BF16 V-cycles apply the learned blocks in FP32: a zero
    output layer gives the SPAI0 solve of that precision, and blocks from a
    random network solve to 1e-8 with iterations close to the FP64 V-cycle
    with the same blocks."""
    p = q.make_problem((10, 9, 8), traction=(0, 0, -1), inclusion_frac=0.2)
    fb = torch.from_numpy(p.f).cuda()
    G = amg.AMG(*_dev(p), coarse_enough=200, precision=prec)
    u0, it0, _, _ = G.solve(fb)
    assert not G.set_learned_smoother(amg.learned_init(1))
    u1, it1, _, st = G.solve(fb)
    assert st == amg.AMG_OK and abs(it1 - it0) <= 1
    assert torch.linalg.norm(u1 - u0) <= 1e-7 * torch.linalg.norm(u0)
    w = _params(seed=7, w2=0.05)
    assert not G.set_learned_smoother(w)
    u2, it2, res2, st2 = G.solve(fb)
    G64 = amg.AMG(*_dev(p), coarse_enough=200)
    assert not G64.set_learned_smoother(w)
    u3, it3, _, _ = G64.solve(fb)
    assert st2 == amg.AMG_OK and res2 <= 1e-8
    assert abs(it2 - it3) <= max(2, it3 // 10), (it2, it3)
    assert torch.linalg.norm(u2 - u3) <= 1e-6 * torch.linalg.norm(u3)
