"""Pins of the symbolic-support oracle (Sections 2 and 5: a symbolic support
set with a given symbol-to-symbol dissimilarity; the support is fixed).

  * with D the squared distances of points standing behind the symbols, the
    cost, W^2 and B-ADMM reduce to the coordinate oracle with a fixed
    support (a reduction to an independently pinned function);
  * with the 0/1 discrete metric on a common symbol set, W is the total
    variation distance 1/2 sum |a - b| (closed form of that LP);
  * the projection of a seed onto the centroid symbols: hand-derived example,
    mass conservation;
  * the initial picks: distinct, seeded, the shuffle of cluster.init_pick's
    generator over every id.
"""
import numpy as np

from oracle import badmm_barycenter, cost_matrix, w2_exact
from oracle.cluster import splitmix64
from oracle.symbolic import (badmm_sym, d2_cluster_sym, project_to_symbols, sym_cost, sym_init_pick,
                             w2_sym)


def points_and_table(seed, V=9, q=3):
    rng = np.random.default_rng(seed)
    P = rng.normal(size=(V, q)) * 2.0
    return P, cost_matrix(P, P)


def test_sym_cost_reduces_to_coordinates():
    P, D = points_and_table(1)
    s, t = [0, 3, 5], [8, 1, 3, 2]
    np.testing.assert_array_equal(sym_cost(D, s, t), cost_matrix(P[s], P[t]))


def test_w2_sym_reduces_to_coordinates():
    P, D = points_and_table(2)
    rng = np.random.default_rng(3)
    for _ in range(5):
        s = rng.choice(9, 4, replace=False)
        t = rng.choice(9, 5, replace=False)
        ws, wt = rng.dirichlet(np.ones(4)), rng.dirichlet(np.ones(5))
        assert abs(w2_sym(D, s, ws, t, wt) - w2_exact(P[s], ws, P[t], wt)) <= 1e-9


def test_w2_sym_discrete_metric_is_total_variation():
    V = 7
    D = 1.0 - np.eye(V)
    rng = np.random.default_rng(4)
    for _ in range(6):
        a, b = rng.dirichlet(np.ones(V)), rng.dirichlet(np.ones(V))
        assert abs(w2_sym(D, np.arange(V), a, np.arange(V), b) - 0.5 * np.abs(a - b).sum()) <= 1e-9


def test_badmm_sym_reduces_to_fixed_support_badmm():
    P, D = points_and_table(5, V=12)
    rng = np.random.default_rng(6)
    s = [1, 4, 7, 10]
    members = []
    for _ in range(6):
        t = rng.choice(12, int(rng.integers(2, 8)), replace=False)
        members.append((t, rng.dirichlet(np.ones(len(t)))))
    w0 = rng.dirichlet(np.ones(4))
    ref = badmm_barycenter([(P[t], wt) for t, wt in members], P[s], w0, T=40, tau=10, fix_x=True)
    got = badmm_sym(D, members, s, w0, T=40, tau=10)
    np.testing.assert_allclose(got["w"], ref["w"], atol=1e-14)
    for a, b in zip(got["P2"], ref["P2"]):
        np.testing.assert_allclose(a, b, atol=1e-14)
    assert abs(got["obj"] - ref["obj"]) <= 1e-12 * ref["obj"]
    assert abs(got["rho"] - ref["rho"]) <= 1e-12 * ref["rho"]


def test_project_to_symbols_hand_example():
    # symbols on a line at 0, 1, 2, 5, 9 (squared distances); centroid symbols
    # {0, 3} (at 0 and 5): 1 -> 0 (1 < 16), 2 -> 0 (4 < 9), 9 -> 5 (16 < 81);
    # a tie is impossible here.  Masses 0.2 (at 1), 0.3 (at 2), 0.5 (at 9).
    x = np.array([[0.0], [1.0], [2.0], [5.0], [9.0]])
    D = cost_matrix(x, x)
    w = project_to_symbols(D, [0, 3], [1, 2, 4], np.array([0.2, 0.3, 0.5]))
    np.testing.assert_allclose(w, [0.5, 0.5], atol=1e-15)
    # a distribution already on the centroid symbols is returned as it is
    w2 = project_to_symbols(D, [0, 3, 4], [4, 0], np.array([0.25, 0.75]))
    np.testing.assert_allclose(w2, [0.75, 0.0, 0.25], atol=1e-15)


def test_sym_init_pick_is_the_seeded_shuffle():
    N, K, seed = 11, 4, 77
    ids = list(range(N))
    state = seed
    for t in range(K):
        state, z = splitmix64(state)
        j = t + z % (N - t)
        ids[t], ids[j] = ids[j], ids[t]
    assert sym_init_pick(N, K, seed) == ids[:K]
    assert len(set(sym_init_pick(N, 6, 3))) == 6


def test_d2_cluster_sym_one_symbol_and_first_round():
    """With a single centroid symbol every centroid is the point mass on it, so
    every W^2 is the same and all labels go to centroid 0 (ties -> lowest
    index), with the closed-form objective; with several symbols the first
    round's labels are the brute-force argmin of the LP values against the
    projected seeds."""
    rng = np.random.default_rng(9)
    _, D = points_and_table(10, V=8)
    bags = []
    for _ in range(14):
        t = rng.choice(8, int(rng.integers(2, 6)), replace=False)
        bags.append((t, rng.dirichlet(np.ones(len(t)))))
    res = d2_cluster_sym(D, bags, 3, [2], seed=5, rounds=2, T=10)
    assert (res["labels"] == 0).all()
    closed = np.mean([float(wt @ D[2, t]) for t, wt in bags])
    assert abs(res["obj_per_round"][0] - closed) <= 1e-9
    s = [0, 3, 6]
    res = d2_cluster_sym(D, bags, 3, s, seed=6, rounds=1, T=10)
    seeds = [project_to_symbols(D, s, *bags[k]) for k in res["picks"]]
    Dm = np.array([[w2_sym(D, s, w, *b) for w in seeds] for b in bags])
    np.testing.assert_array_equal(res["labels_per_round"][0], np.argmin(Dm, axis=1))
    assert abs(res["obj_per_round"][0] - Dm.min(axis=1).mean()) <= 1e-12
