"""The entropic dual bound used by the bounded assignment, restated in FP64 on
the CPU and checked against the exact transportation LP of Eq. (primal)
(HiGHS through the oracle):

  * the dual of the LP is max sum_i v_i f_i + sum_j u_j g_j subject to
    f_i + g_j <= C_ij; Sinkhorn iterations of the entropy-regularised problem
    give potentials that the c-transform g'_j = min_i (C_ij - f_i) (or
    f'_i = min_j (C_ij - g_j)) makes feasible, so the dual objective is a
    lower bound of W^2 for ANY number of iterations, any eps and any starting
    potentials, including zero-weight points on either side;
  * it is never weaker than the one-sided relaxations it starts from (the
    c-transforms of zero potentials), and after a few dozen iterations it is
    within a few percent of W^2 on document-like problems;
  * log2-domain iterations with each log-sum-exp shifted by the previous
    value of its potential give the same potentials as the plain form."""
import numpy as np
import pytest

from oracle.ot import transport_lp


def lse2(x):
    mx = np.max(x)
    return mx + np.log2(np.sum(np.exp2(x - mx)))


def sinkhorn_log2(C, a, b, eps, iters, shifted=False):
    """Potentials F, G in log2 units (f = F eps ln 2) after `iters` iterations."""
    sc = 1.0 / (eps * np.log(2.0))
    la = np.where(a > 0, np.log2(np.where(a > 0, a, 1.0)), -np.inf)
    lb = np.where(b > 0, np.log2(np.where(b > 0, b, 1.0)), -np.inf)
    F = np.zeros(len(a))
    G = np.zeros(len(b))
    for _ in range(iters):
        for i in range(len(a)):
            x = G + lb - sc * C[i]
            if shifted:
                sh = -F[i]
                s = np.sum(np.exp2(x - sh))
                F[i] = -(sh + np.log2(s)) if 2.0 ** -100 <= s <= 2.0 ** 100 else -lse2(x)
            else:
                F[i] = -lse2(x)
        for j in range(len(b)):
            if b[j] > 0:
                G[j] = -lse2(F + la - sc * C[:, j])
    return F / sc, G / sc


def dual_bound(C, a, b, f, g):
    g2 = np.min(C - f[:, None], axis=0)
    f2 = np.min(C - g[None, :], axis=1)
    with np.errstate(invalid="ignore"):
        lb_a = a @ f + b @ g2
        lb_b = a @ f2 + np.sum(np.where(b > 0, b * np.where(np.isfinite(g), g, 0.0), 0.0))
    return max(lb_a, lb_b)


def problem(rng, m, n, d, zero_a=0, zero_b=0):
    x = rng.normal(size=(m, d))
    y = rng.normal(size=(n, d))
    C = ((x[:, None, :] - y[None, :, :]) ** 2).sum(-1)
    a = rng.dirichlet(np.ones(m))
    b = rng.dirichlet(np.ones(n))
    a[:zero_a] = 0.0
    b[:zero_b] = 0.0
    return C, a / a.sum(), b / b.sum()


@pytest.mark.parametrize("seed", range(6))
def test_bound_never_exceeds_the_lp(seed):
    rng = np.random.default_rng(seed)
    C, a, b = problem(rng, 9, 7, 4, zero_a=seed % 3, zero_b=seed % 2)
    w2, _ = transport_lp(C, a, b)
    for eps_rel, iters in ((0.05, 0), (0.05, 1), (0.05, 30), (0.01, 60), (1.0, 5)):
        f, g = sinkhorn_log2(C, a, b, eps_rel * C.mean(), iters)
        lb = dual_bound(C, a, b, f, g)
        assert lb <= w2 + 1e-9 * max(1.0, w2), (eps_rel, iters, lb, w2)
    # arbitrary (even absurd) potentials stay valid after the c-transform
    f = rng.normal(size=C.shape[0]) * 50.0
    g = rng.normal(size=C.shape[1]) * 50.0
    assert dual_bound(C, a, b, f, g) <= w2 + 1e-9 * max(1.0, w2)


def test_bound_dominates_the_one_sided_relaxations_and_is_tight():
    rng = np.random.default_rng(11)
    gaps = []
    for _ in range(8):
        C, a, b = problem(rng, 16, 12, 6)
        w2, _ = transport_lp(C, a, b)
        lb1 = b @ C.min(axis=0)   # each bag point to its nearest centroid point
        lb2 = a @ C.min(axis=1)
        f, g = sinkhorn_log2(C, a, b, 0.05 * C.mean(), 30)
        lb = dual_bound(C, a, b, f, g)
        zero = dual_bound(C, a, b, np.zeros(16), np.zeros(12))
        assert abs(zero - max(lb1, lb2)) <= 1e-12 * w2
        assert lb >= max(lb1, lb2) - 1e-12 * w2
        assert lb <= w2 + 1e-9 * w2
        gaps.append((w2 - lb) / w2)
    assert np.median(gaps) < 0.05, gaps


def test_shifted_log_sum_exp_gives_the_same_potentials():
    rng = np.random.default_rng(5)
    C, a, b = problem(rng, 10, 8, 3, zero_b=1)
    f1, g1 = sinkhorn_log2(C, a, b, 0.05 * C.mean(), 25)
    f2, g2 = sinkhorn_log2(C, a, b, 0.05 * C.mean(), 25, shifted=True)
    np.testing.assert_allclose(f1, f2, rtol=0, atol=1e-9 * np.abs(C).max())
    ok = b > 0
    np.testing.assert_allclose(g1[ok], g2[ok], rtol=0, atol=1e-9 * np.abs(C).max())
