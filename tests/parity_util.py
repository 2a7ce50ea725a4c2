"""Helpers shared by the GPU parity tests: device copies of a generated
problem and the level-by-level comparison of a CUDA hierarchy with the
oracle's (aggregates, strength flags and patterns bit-exact, values within a
relative bound)."""
import numpy as np

import oracle as o


def dev_args(p, torch):
    d = torch.device("cuda:0")
    return (torch.from_numpy(p.row_ptr).to(d), torch.from_numpy(p.col).to(d),
            torch.from_numpy(p.val).to(d), torch.from_numpy(p.B).to(d))


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def compare_levels(H, G, ns, tol_val=1e-12):
    """Every level of the CUDA hierarchy G against the oracle's H: A, P, R
    patterns and strength flags and aggregates bit-exact; A, P, R, B values
    within tol_val of the largest entry; rho and omega exact on level 0 (same
    input bits, same summation order) and within 1e-12 below (the coarse
    operators inherit rounding differences of the Galerkin products); the
    smoother within 1e-14 on level 0."""
    assert G.nlevels == H.nlevels
    for l in range(H.nlevels):
        ol, gl = H.level(l), G.export(l)
        b = ol["b"]
        gA = gl["A"]
        cA = o.unblock(gA[0], gA[1], gA[2].reshape(len(gA[1]), -1), b, b)
        assert np.array_equal(cA.ptr, ol["A"].ptr) and np.array_equal(cA.col, ol["A"].col), l
        assert rel(cA.val, ol["A"].val) <= tol_val, l
        assert rel(gl["B"], ol["B"]) <= tol_val, l
        del cA, gA
        if l == H.nlevels - 1:
            continue
        og = H.graph(l)
        assert np.array_equal(gl["strong"], og["strong"]), l
        assert np.array_equal(gl["agg"], ol["agg"]), l
        info = gl["info"]
        assert info["nagg"] == ol["nagg"], l
        rtol = 0.0 if l == 0 else 1e-12
        assert abs(info["rho"] - ol["rho"]) <= rtol * ol["rho"], l
        assert abs(info["omega"] - ol["omega"]) <= rtol * ol["omega"], l
        gP, gR = gl["P"], gl["R"]
        cP = o.unblock(gP[0], gP[1], gP[2].reshape(len(gP[1]), -1), b, ns, nbcols=info["nagg"])
        cR = o.unblock(gR[0], gR[1], gR[2].reshape(len(gR[1]), -1), ns, b, nbcols=info["nbrows"])
        assert np.array_equal(cP.ptr, ol["P"].ptr) and np.array_equal(cP.col, ol["P"].col), l
        assert np.array_equal(cR.ptr, ol["R"].ptr) and np.array_equal(cR.col, ol["R"].col), l
        assert rel(cP.val, ol["P"].val) <= tol_val, l
        assert rel(cR.val, ol["R"].val) <= tol_val, l
        assert rel(gl["M"], ol["M"]) <= (1e-14 if l == 0 else tol_val), l


def compare_hierarchy(p, coarse_enough, torch, amg, tol_val=1e-12, Bns=None,
                      aggregation="greedy", **kw):
    """Build the oracle's and the CUDA hierarchy of problem p and compare them."""
    Bns = p.B if Bns is None else Bns
    H = o.Hierarchy(o.from_problem(p), 3, Bns, coarse_enough=coarse_enough,
                    aggregation=aggregation, **kw)
    rp, cl, val, _ = dev_args(p, torch)
    G = amg.AMG(rp, cl, val, torch.from_numpy(Bns).cuda(), coarse_enough=coarse_enough,
                aggregation={"greedy": amg.AGG_GREEDY, "mis2": amg.AGG_MIS2}[aggregation], **kw)
    compare_levels(H, G, Bns.shape[1], tol_val)
    return H, G


def vcycle_bound(H):
    """Relative bound on the difference of the two V-cycles: the coarsest
    level is solved with a dense inverse on the GPU and with Cholesky
    substitutions in the oracle, which agree to about cond(A_L) 1e-16; the
    smoothers and prolongations carry that to the fine level."""
    L, _ = H.coarse_factor()
    d = np.diag(L)
    cond_est = (d.max() / d[d > 0].min()) ** 2
    return max(1e-12, 100 * cond_est * 1e-16)
