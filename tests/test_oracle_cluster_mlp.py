"""Pins of the oracle's merge initialisation, D2-clustering loop and pruning MLP.

  * Eq. (merge): hand-derived golden example; brute-force re-derivation of the
    chosen pair; merging preserves total weight and the weighted mean (first
    moment) exactly; m >= m_k is the identity; m = 1 gives the weighted mean;
  * Algorithm 1 with m = 1 is exactly Lloyd's K-means on the distribution
    means (Section 1 and Section 7 make this reduction): labels and centroids
    are compared with an independent K-means written here;
  * SplitMix64 against the published reference outputs for seed 1234567;
  * MLP: finite-difference gradients, a hand-worked 1-D example, translation
    invariance of the centred embedding.
"""
import json
import os

import numpy as np
import pytest

from oracle import merge_reduce, d2_cluster, splitmix64, init_pick, w2_exact
from oracle import mlp

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_merge_golden():
    g = json.load(open(os.path.join(GOLD, "merge_three_points.json")))
    x, w = merge_reduce(np.array(g["x"]), np.array(g["w"]), g["m"])
    np.testing.assert_allclose(x, np.array(g["x_out"]), atol=1e-15)
    np.testing.assert_allclose(w, np.array(g["w_out"]), atol=1e-15)


@pytest.mark.parametrize("seed", range(4))
def test_merge_invariants(seed):
    rng = np.random.default_rng(seed)
    mk = int(rng.integers(5, 12))
    y = rng.normal(size=(mk, 3))
    w = rng.dirichlet(np.ones(mk))
    for m in (1, 2, mk - 1, mk, mk + 3):
        x, v = merge_reduce(y, w, m)
        assert x.shape[0] == min(m, mk)
        assert abs(v.sum() - w.sum()) < 1e-14
        np.testing.assert_allclose(v @ x, w @ y, atol=1e-13)
        if m >= mk:
            np.testing.assert_array_equal(x, y)
    # the first merge is the brute-force minimiser of the criterion
    best = min(((w[i] * w[j] * np.sum((y[i] - y[j]) ** 2) / (w[i] + w[j]), i, j)
                for i in range(mk) for j in range(i + 1, mk)))
    _, i, j = best
    x, v = merge_reduce(y, w, mk - 1)
    np.testing.assert_allclose(x[i], (w[i] * y[i] + w[j] * y[j]) / (w[i] + w[j]), atol=1e-14)
    assert abs(v[i] - (w[i] + w[j])) < 1e-15


def test_splitmix64_reference_vector():
    # outputs of the reference splitmix64.c (Vigna) for state 1234567
    expect = [6457827717110365317, 3203168211198807973, 9817491932198370423,
              4593380528125082431, 16408922859458223821]
    s = 1234567
    got = []
    for _ in range(5):
        s, z = splitmix64(s)
        got.append(z)
    assert got == expect


def lloyd_on_means(means, init_means, rounds):
    c = init_means.copy()
    labels_all = []
    for _ in range(rounds):
        d = ((means[:, None, :] - c[None, :, :]) ** 2).sum(-1)
        lab = np.argmin(d, axis=1)
        labels_all.append(lab)
        for i in range(len(c)):
            if (lab == i).any():
                c[i] = means[lab == i].mean(0)
    return labels_all, c


def test_d2_with_m1_is_kmeans_on_means():
    rng = np.random.default_rng(21)
    bags = []
    centers = rng.normal(size=(3, 2)) * 4
    for k in range(24):
        mk = int(rng.integers(2, 5))
        y = centers[k % 3] + rng.normal(size=(mk, 2))
        bags.append((y, rng.dirichlet(np.ones(mk))))
    K, rounds = 3, 3
    res = d2_cluster(bags, K, 1, seed=99, rounds=rounds, T=25, tau=10)
    means = np.array([w @ y for y, w in bags])
    picks = init_pick([y.shape[0] for y, _ in bags], K, 1, 99)
    labels_ref, cent_ref = lloyd_on_means(means, means[picks], rounds)
    for r in range(rounds):
        np.testing.assert_array_equal(res["labels_per_round"][r], labels_ref[r])
    np.testing.assert_allclose(res["x"][:, 0, :], cent_ref, atol=1e-10)
    # the objective is the mean of W^2 = ||mean - c||^2 + variance
    var = np.array([w @ np.sum((y - w @ y) ** 2, 1) for y, w in bags])
    assert res["obj_per_round"][0] >= var.mean() - 1e-12


def small_params(seed, d, H=6, E=4):
    rng = np.random.default_rng(seed)
    return dict(W1=rng.normal(size=(H, d)) * 0.7, b1=rng.normal(size=H) * 0.1,
                W2=rng.normal(size=(H, H)) * 0.5, b2=rng.normal(size=H) * 0.1,
                W3=rng.normal(size=(E, H)) * 0.5)


def test_mlp_gradient_finite_differences():
    rng = np.random.default_rng(3)
    d = 3
    params = small_params(4, d)
    bags = [(rng.normal(size=(int(rng.integers(2, 6)), d)), None) for _ in range(4)]
    bags = [(y, rng.dirichlet(np.ones(len(y)))) for y, _ in bags]
    cents = [(rng.normal(size=(3, d)), rng.dirichlet(np.ones(3))) for _ in range(2)]
    pairs = [(0, 0), (1, 1), (2, 0), (3, 1), (0, 1)]
    targets = [w2_exact(cents[q][0], cents[q][1], *bags[a]) for a, q in pairs]
    L, g = mlp.pair_loss_and_grad(params, bags, cents, pairs, targets)
    h = 1e-6
    for name in mlp.PARAM_NAMES:
        P = params[name]
        flat = P.reshape(-1)
        for idx in range(0, flat.size, max(1, flat.size // 7)):
            old = flat[idx]
            flat[idx] = old + h
            Lp, _ = mlp.pair_loss_and_grad(params, bags, cents, pairs, targets)
            flat[idx] = old - h
            Lm, _ = mlp.pair_loss_and_grad(params, bags, cents, pairs, targets)
            flat[idx] = old
            fd = (Lp - Lm) / (2 * h)
            assert abs(fd - g[name].reshape(-1)[idx]) <= 1e-6 * max(1.0, abs(fd))


def test_mlp_hand_example():
    # d = 1, H = 1, E = 1: W1 = 2, b1 = 0.5, W2 = 3, b2 = -1, W3 = 0.5.
    # P = {(0.25, -1), (0.75, 3)}: mean 2, centred u = (-3, 1);
    # a1 = (-5.5, 2.5) -> h1 = (0, 2.5); a2 = (-1, 6.5) -> h2 = (0, 6.5);
    # g = 0.75 * 6.5 = 4.875; f = 0.5 * 4.875 = 2.4375.
    params = dict(W1=np.array([[2.0]]), b1=np.array([0.5]), W2=np.array([[3.0]]),
                  b2=np.array([-1.0]), W3=np.array([[0.5]]))
    f = mlp.embed(params, np.array([[-1.0], [3.0]]), np.array([0.25, 0.75]))
    assert abs(f[0] - 2.4375) < 1e-15


def test_mlp_translation_invariant_and_predictor_bound():
    rng = np.random.default_rng(5)
    params = small_params(6, 2)
    y = rng.normal(size=(5, 2))
    w = rng.dirichlet(np.ones(5))
    np.testing.assert_allclose(mlp.embed(params, y + 7.0, w), mlp.embed(params, y, w), atol=1e-12)
    cents = [(rng.normal(size=(3, 2)), rng.dirichlet(np.ones(3))) for _ in range(4)]
    pred, mt = mlp.predict(params, (y, w), cents)
    assert (pred >= mt - 1e-15).all()
    for i, (x, wx) in enumerate(cents):
        assert w2_exact(x, wx, y, w) >= mt[i] - 1e-12


def test_prune_assign_exact_when_margin_holds_and_falls_back():
    exact = [5.0, 1.0, 3.0, 0.5]
    # predictions rank centroid 3 and 1 first; bounds of 0 and 2 exceed b = 0.5
    lab, b, fb, n = mlp.prune_assign_one(np.array([6.0, 1.1, 3.5, 0.6]), np.array([4.0, 0.2, 2.0, 0.1]),
                                         lambda i: exact[i], r=2, delta=0.1)
    assert (lab, b, fb, n) == (3, 0.5, False, 2)
    # the true best (3) is outside the candidates {0, 1}; its bound
    # max(0.1, 1.5 - 1.0) = 0.5 does not exceed b = 1.0, so all K are solved
    lab, b, fb, n = mlp.prune_assign_one(np.array([0.4, 1.1, 3.5, 1.5]), np.array([0.1, 0.2, 2.0, 0.1]),
                                         lambda i: exact[i], r=2, delta=1.0)
    assert (lab, b, fb, n) == (3, 0.5, True, 4)


def test_init_pick_falls_back_to_the_largest():
    """With fewer than K distributions of m points, the picks are the largest
    distributions (threshold = the K-th largest m_k), distinct, seeded; with
    enough of them the threshold is m itself."""
    sizes = [3, 9, 5, 9, 2, 7, 8, 4, 6, 9]
    for seed in range(20):
        p = init_pick(sizes, 4, 12, seed)          # nobody has 12 points
        assert len(set(p)) == 4 and all(sizes[k] >= 8 for k in p)   # 4th largest size is 8
        q = init_pick(sizes, 3, 6, seed)           # 7 bags have >= 6 points
        assert len(set(q)) == 3 and all(sizes[k] >= 6 for k in q)
    # the fallback threshold equals m when exactly K bags qualify
    assert sorted(init_pick(sizes, 3, 9, 1)) == [1, 3, 9]


def test_pad_support_golden():
    """Padding reading (Section 5 assumes m_k >= m): hand-derived golden values,
    and padding leaves the distribution unchanged (W^2 to the seed is 0)."""
    from oracle.cluster import pad_support
    g = json.load(open(os.path.join(GOLD, "pad_support.json")))
    x, w = pad_support(np.array(g["x"]), np.array(g["w"]), g["m"])
    np.testing.assert_array_equal(x, np.array(g["x_out"]))
    np.testing.assert_array_equal(w, np.array(g["w_out"]))
    np.testing.assert_allclose(w @ x, np.array(g["mean"]), atol=1e-15)
    assert w2_exact(x, w, np.array(g["x"]), np.array(g["w"])) <= 1e-12
    # a seed that already has m points (or more) is returned as it is
    x2, w2 = pad_support(np.array(g["x"]), np.array(g["w"]), 2)
    np.testing.assert_array_equal(x2, np.array(g["x"]))
    np.testing.assert_array_equal(w2, np.array(g["w"]))


def test_d2_cluster_pads_small_seeds():
    """With m above every m_k each seed is the (unmerged) bag plus zero-weight
    copies of its last point: the first round's W^2 to that seed's own bag is 0."""
    rng = np.random.default_rng(8)
    bags = [(rng.normal(size=(int(rng.integers(2, 5)), 2)), None) for _ in range(7)]
    bags = [(y, rng.dirichlet(np.ones(len(y)))) for y, _ in bags]
    K, m = 2, 6
    res = d2_cluster(bags, K, m, seed=4, rounds=1, T=5, tau=10)
    picks = res["picks"]
    from oracle.cluster import d2_assign as oracle_assign
    # recompute the round-1 distances to the padded seeds directly
    seeds = []
    for k in picks:
        y, wy = bags[k]
        q = y.shape[0]
        seeds.append((np.vstack([y] + [y[-1:]] * (m - q)), np.concatenate([wy, np.zeros(m - q)])))
    _, dists, D = oracle_assign(bags, seeds)
    for i, k in enumerate(picks):
        assert D[k, i] <= 1e-12
    assert abs(res["obj_per_round"][0] - dists.mean()) <= 1e-12


def test_d2_cluster_warm_start_selection(monkeypatch):
    """Section 5, warm start: in round r > 0 a member starts from its cached
    Pi^(k,2) exactly when its label equals its label of round r - 1 (the most
    recent assignment); every other member, and every member in round 0,
    starts from w_i w_j^(k).  Labels are teacher-forced so that the expected
    sequence of barycenter calls can be written out by hand:

      labels  round 0: 0 0 0 1 1 1
              round 1: 0 1 0 1 0 1   (members 1 and 4 move)
              round 2: 1 1 0 1 0 1   (member 0 moves; 1 and 4 stay where round 1 put them)

      round 0: cluster 0 <- [0, 1, 2] all cold;  cluster 1 <- [3, 4, 5] all cold
      round 1: cluster 0 <- [0, 2, 4] warm T T F; cluster 1 <- [1, 3, 5] warm F T T
      round 2: cluster 0 <- [2, 4]    warm T T;   cluster 1 <- [0, 1, 3, 5] warm F T T T

    and a warm member's plan0 is the Pi^(k,2) that its previous round's call
    returned for it (member 1's in round 2 comes from round 1's cluster 1
    call, not from round 0)."""
    import oracle.cluster as oc
    rng = np.random.default_rng(12)
    bags = [(rng.normal(size=(3 + (k % 3), 2)) + (k // 3) * 3.0, None) for k in range(6)]
    bags = [(y, rng.dirichlet(np.ones(len(y)))) for y, _ in bags]
    ids_of = {id(b[0]): k for k, b in enumerate(bags)}
    calls = []
    real = oc.badmm_barycenter

    def recorder(members, x0, w0, **kw):
        res = real(members, x0, w0, **kw)
        ids = [ids_of[id(y)] for y, _ in members]
        warm = kw.get("warm")
        plan0 = kw.get("plan0")
        calls.append(dict(ids=ids, warm=[bool(v) for v in warm],
                          plan0={k: (None if p is None else p.copy()) for k, p in zip(ids, plan0)},
                          P2={k: res["P2"][t].copy() for t, k in enumerate(ids)}))
        return res

    monkeypatch.setattr(oc, "badmm_barycenter", recorder)
    L = [[0, 0, 0, 1, 1, 1], [0, 1, 0, 1, 0, 1], [1, 1, 0, 1, 0, 1]]
    oc.d2_cluster(bags, 2, 2, seed=1, rounds=3, T=4, tau=10, labels_in=L)
    expect = [([0, 1, 2], [False] * 3), ([3, 4, 5], [False] * 3),
              ([0, 2, 4], [True, True, False]), ([1, 3, 5], [False, True, True]),
              ([2, 4], [True, True]), ([0, 1, 3, 5], [False, True, True, True])]
    assert [(c["ids"], c["warm"]) for c in calls] == expect
    # plan0 of each warm member is what the previous round returned for it
    r0 = {**calls[0]["P2"], **calls[1]["P2"]}
    r1 = {**calls[2]["P2"], **calls[3]["P2"]}
    for k in (0, 2):
        np.testing.assert_array_equal(calls[2]["plan0"][k], r0[k])
    for k in (3, 5):
        np.testing.assert_array_equal(calls[3]["plan0"][k], r0[k])
    for k in (2, 4):
        np.testing.assert_array_equal(calls[4]["plan0"][k], r1[k])
    for k in (1, 3, 5):
        np.testing.assert_array_equal(calls[5]["plan0"][k], r1[k])
    # member 1's round-0 plan (cluster 0) differs from its round-1 plan: the
    # check above really distinguishes the two rounds' caches
    assert r0[1].shape == r1[1].shape and not np.array_equal(r0[1], r1[1])
