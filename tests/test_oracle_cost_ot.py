"""Pins of the oracle's cost and exact W^2 against facts independent of it.

Cost: brute-force loops, the norm-expansion identity, symmetry.
W^2 (Eq. primal): 1-D closed form (quantile coupling), permutation brute force
(Birkhoff: uniform equal-size problems have a permutation optimum), W(P,P)=0,
symmetry, the translation identity, hand-derived golden values.
"""
import itertools
import json
import os

import numpy as np
import pytest

from oracle import cost_matrix, w2_exact

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_cost_brute_force_and_identities():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(5, 3))
    y = rng.normal(size=(7, 3))
    C = cost_matrix(x, y)
    B = np.zeros((5, 7))
    for i in range(5):
        for j in range(7):
            s = 0.0
            for t in range(3):
                s += (x[i, t] - y[j, t]) ** 2
            B[i, j] = s
    np.testing.assert_allclose(C, B, rtol=0, atol=1e-13)
    # ||x||^2 + ||y||^2 - 2 x.y
    N = (x * x).sum(1)[:, None] + (y * y).sum(1)[None, :] - 2 * x @ y.T
    np.testing.assert_allclose(C, N, atol=1e-12)
    np.testing.assert_allclose(cost_matrix(y, x), C.T, atol=0)
    assert (C >= 0).all()


def quantile_w2_1d(a, wa, b, wb):
    """Closed form in 1-D: integral over t of (F_a^-1(t) - F_b^-1(t))^2."""
    ia, ib = np.argsort(a), np.argsort(b)
    a, wa, b, wb = a[ia], wa[ia] / wa.sum(), b[ib], wb[ib] / wb.sum()
    i = j = 0
    ra, rb = wa[0], wb[0]
    tot = 0.0
    while i < len(a) and j < len(b):
        t = min(ra, rb)
        tot += t * (a[i] - b[j]) ** 2
        ra -= t
        rb -= t
        if ra <= 1e-15:
            i += 1
            ra = wa[i] if i < len(a) else 0
        if rb <= 1e-15:
            j += 1
            rb = wb[j] if j < len(b) else 0
    return tot


@pytest.mark.parametrize("seed", range(6))
def test_w2_matches_1d_closed_form(seed):
    rng = np.random.default_rng(seed)
    ma, mb = rng.integers(1, 9, size=2)
    a = rng.normal(size=ma) * 3
    b = rng.normal(size=mb) * 3 + 1
    wa = rng.dirichlet(np.ones(ma))
    wb = rng.dirichlet(np.ones(mb))
    got = w2_exact(a[:, None], wa, b[:, None], wb)
    ref = quantile_w2_1d(a, wa, b, wb)
    assert abs(got - ref) <= 1e-9 * max(1.0, ref)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 6])
def test_w2_uniform_equal_size_is_assignment(n):
    rng = np.random.default_rng(10 + n)
    x = rng.normal(size=(n, 3))
    y = rng.normal(size=(n, 3)) + 0.5
    C = cost_matrix(x, y)
    best = min(sum(C[i, p[i]] for i in range(n)) for p in itertools.permutations(range(n))) / n
    got = w2_exact(x, np.full(n, 1.0 / n), y, np.full(n, 1.0 / n))
    assert abs(got - best) <= 1e-9 * max(1.0, best)


def test_w2_self_zero_symmetry_translation():
    rng = np.random.default_rng(3)
    x = rng.normal(size=(6, 4))
    y = rng.normal(size=(9, 4)) * 2
    wx = rng.dirichlet(np.ones(6))
    wy = rng.dirichlet(np.ones(9))
    assert abs(w2_exact(x, wx, x, wx)) < 1e-10
    d1 = w2_exact(x, wx, y, wy)
    d2 = w2_exact(y, wy, x, wx)
    assert abs(d1 - d2) < 1e-9
    mx, my = wx @ x, wy @ y
    centred = w2_exact(x - mx, wx, y - my, wy)
    assert abs(d1 - (np.sum((mx - my) ** 2) + centred)) < 1e-9
    # the mean term is a lower bound (Jensen)
    assert d1 >= np.sum((mx - my) ** 2) - 1e-12


@pytest.mark.parametrize("name", ["w2_two_point.json", "w2_1d_staircase.json"])
def test_w2_golden(name):
    g = json.load(open(os.path.join(GOLD, name)))
    got = w2_exact(np.array(g["P"]["x"]), np.array(g["P"]["w"]),
                   np.array(g["Q"]["x"]), np.array(g["Q"]["w"]))
    assert abs(got - g["W2"]) < 1e-10
