"""Pins of the oracle's MIS-2 aggregation (the parallel alternative to the
greedy passes of the point-wise aggregation, Sec. 4 / Alg. 1).

The oracle visits nodes one by one in descending priority (the greedy
distance-2 independent set).  These tests tie it to: the published test
vectors of the priority hash, hand-worked graphs, and, on random graphs and
the strength graphs of elasticity meshes, a brute-force check of the property
that defines that set uniquely (no two roots within two edges; every other
node with a neighbour has a root of higher priority within two edges),
found here by synchronous rounds of local maxima instead of the oracle's
sequential visit.
"""
import json
import os

import numpy as np
import pytest

import oracle as o
import q1elasticity as q


def _graph_matrix(case):
    n = case["n"]
    D = np.diag([1.0] * n)
    for i, j, v in case["sym"]:
        D[i, j] = D[j, i] = v
    for i, j, v in case["directed"]:
        D[i, j] = v
    ptr, col, val = [0], [], []
    for i in range(n):
        nz = np.nonzero(D[i])[0]
        col += nz.tolist()
        val += D[i, nz].tolist()
        ptr.append(len(col))
    return o.CSR(ptr, col, val, (n, n))


def test_fmix32_published_vectors(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "mis2_graphs.json")))
    for x, y in g["fmix32_vectors"]["pairs"]:
        assert o.fmix32(int(x, 16)) == int(y, 16)


def test_fmix32_is_a_bijection_on_a_range():
    xs = list(range(0, 1 << 16)) + [0xFFFFFFFF - k for k in range(1 << 12)]
    assert len({o.fmix32(x) for x in xs}) == len(xs)


def test_mis2_hand_worked(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "mis2_graphs.json")))
    for case in g["cases"]:
        agg, nagg = o.aggregate_mis2(_graph_matrix(case), 1, 0.08)
        assert agg.tolist() == case["agg"], case["name"]
        assert nagg == case["nagg"], case["name"]


# ---------------------------------------------------------------- brute force
def _adjacency(G, n):
    """Undirected strong adjacency (dense bool) from an oracle strength graph."""
    adj = np.zeros((n, n), dtype=bool)
    for i in range(n):
        for p in range(G["ptr"][i], G["ptr"][i + 1]):
            if G["strong"][p]:
                adj[i, G["col"][p]] = adj[G["col"][p], i] = True
    np.fill_diagonal(adj, False)
    return adj


def _rounds_roots(adj, prio):
    """Roots by synchronous rounds: an undecided node becomes a root when no
    root is within two edges and it has the highest priority among the
    undecided nodes within two edges; it is excluded when a root is."""
    n = len(prio)
    near = adj | ((adj.astype(np.int64) @ adj.astype(np.int64)) > 0)
    np.fill_diagonal(near, False)
    isolated = ~adj.any(axis=1)
    state = np.where(isolated, 0, 1)          # 0 excluded, 1 undecided, 2 root
    while (state == 1).any():
        new = state.copy()
        for i in np.nonzero(state == 1)[0]:
            nb = np.nonzero(near[i])[0]
            if (state[nb] == 2).any():
                new[i] = 0
            elif all(prio[k] < prio[i] for k in nb if state[k] == 1):
                new[i] = 2
        assert not np.array_equal(new, state)
        state = new
    return state == 2, near, isolated


def _check_and_aggregate(adj, prio):
    roots, near, isolated = _rounds_roots(adj, prio)
    n = len(prio)
    r = np.nonzero(roots)[0]
    # independent in the squared graph
    assert not near[np.ix_(r, r)].any()
    # every other connected node has a higher-priority root within two edges
    for v in range(n):
        if roots[v] or isolated[v]:
            continue
        assert any(prio[u] > prio[v] for u in r if near[v, u])
    # aggregates from the roots
    rid = -np.ones(n, dtype=np.int64)
    rid[r] = np.arange(len(r))
    step1 = rid.copy()
    for v in range(n):
        if not roots[v]:
            rs = [u for u in np.nonzero(adj[v])[0] if roots[u]]
            assert len(rs) <= 1
            if rs:
                step1[v] = rid[rs[0]]
    agg = step1.copy()
    for v in range(n):
        if agg[v] < 0 and not isolated[v]:
            agg[v] = next(step1[u] for u in np.nonzero(adj[v])[0] if step1[u] >= 0)
    return agg, len(r)


def _random_graph_matrix(n, p_edge, p_one_way, seed):
    rng = np.random.default_rng(seed)
    D = np.eye(n)
    for i in range(n):
        for j in range(i + 1, n):
            if rng.random() < p_edge:
                D[i, j] = D[j, i] = -0.5
                if rng.random() < p_one_way:
                    D[j, i] = -0.01          # strong in one direction only
            elif rng.random() < p_edge:
                D[i, j] = D[j, i] = -0.01    # weak link
    ptr, col, val = [0], [], []
    for i in range(n):
        nz = np.nonzero(D[i])[0]
        col += nz.tolist()
        val += D[i, nz].tolist()
        ptr.append(len(col))
    return o.CSR(ptr, col, val, (n, n))


@pytest.mark.parametrize("n,p_edge,seed", [(12, 0.25, 1), (30, 0.08, 2), (60, 0.04, 3),
                                          (60, 0.12, 4), (90, 0.03, 5)])
def test_mis2_random_graphs_brute_force(n, p_edge, seed):
    A = _random_graph_matrix(n, p_edge, 0.3, seed)
    G = o.strength(A, 1, 0.08)
    adj = _adjacency(G, n)
    prio = [o.fmix32(i) for i in range(n)]
    want, nwant = _check_and_aggregate(adj, prio)
    agg, nagg = o.aggregate_mis2(A, 1, 0.08)
    assert nagg == nwant
    assert np.array_equal(agg, want)


@pytest.mark.parametrize("mesh", ["cube5", "inclusions6"])
def test_mis2_elasticity_strength_graph_brute_force(mesh):
    p = q.cube(5) if mesh == "cube5" else q.inclusions(6)
    A = o.from_problem(p)
    G = o.strength(A, 3, 0.08)
    n = p.nnodes
    adj = _adjacency(G, n)
    want, nwant = _check_and_aggregate(adj, [o.fmix32(i) for i in range(n)])
    agg, nagg = o.aggregate_mis2(A, 3, 0.08)
    assert nagg == nwant and np.array_equal(agg, want)
    # a node is aggregated iff it has a neighbour (clamped nodes have none);
    # aggregates are much larger than single nodes
    assert np.array_equal(agg >= 0, adj.any(axis=1))
    assert (agg >= 0).sum() / nagg > 4


def test_mis2_hierarchy_solves_and_keeps_rigid_modes():
    p = q.inclusions(8)
    A = o.from_problem(p)
    H = o.Hierarchy(A, 3, p.B, aggregation="mis2", coarse_enough=500)
    L0 = H.level(0)
    want, nagg = o.aggregate_mis2(A, 3, 0.08)
    assert np.array_equal(L0["agg"], want) and L0["nagg"] == nagg
    # Alg. 1 with any aggregation: P_tent B_c = B on the rows of aggregated
    # nodes (clamped nodes have no neighbour and a zero row)
    Pt, Bc = o.tentative(p.nnodes, 3, want, nagg, p.B)
    rows = np.repeat(want >= 0, 3)
    np.testing.assert_allclose((Pt.to_dense() @ Bc)[rows], p.B[rows], atol=1e-12)
    assert not Pt.to_dense()[~rows].any()
    u, it, res = H.solve(p.f)
    assert res <= 1e-8 and it < 200
    r = p.f - o.spmv(A, u)
    assert np.linalg.norm(r) <= 1.01e-8 * np.linalg.norm(p.f)
    Hg = o.Hierarchy(A, 3, p.B, coarse_enough=500)
    _, itg, _ = Hg.solve(p.f)
    assert abs(it - itg) <= max(5, itg // 3)
