"""Pins of the oracle's B-ADMM (Algorithm badmm) against facts independent of it.

  * marginal invariants that hold by construction of Eqs. badmmc0 / badmmc1 and
    the conservation of dual mass (Eq. badmm2);
  * m = 1 closed form (w = 1, Pi^(k,1) = w^(k), x = mean of member means,
    objective = weighted variance around x);
  * fixed w and x: each member's plan tends to the exact OT (1-D closed form);
  * N = 1 with m = m_1 started at the member: the barycenter is the member;
  * 1-D barycenter: the averaged quantile function is optimal, so it lower-bounds
    the B-ADMM barycenter's exact objective, which stays within a small band;
  * fixed support: the full-batch LP (Eq. fullbatch-lp) optimum is within a few
    per cent (the paper's Table 1 gap is 0.04-0.8%);
  * translation / scaling / member-permutation invariances;
  * a planted mistake (a transposed normalisation) breaks the invariants.
"""
import numpy as np
import pytest
from scipy.optimize import linprog

from oracle import badmm_barycenter, cost_matrix, w2_exact


def make_members(seed, N, d, mk=(2, 6), scale=1.0):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(N):
        k = int(rng.integers(mk[0], mk[1] + 1))
        y = rng.normal(size=(k, d)) * scale + rng.normal(size=d) * 2 * scale
        w = rng.dirichlet(np.ones(k))
        out.append((y, w))
    return out


def start(members, m, seed=5):
    rng = np.random.default_rng(seed)
    pool = np.concatenate([y for y, _ in members])
    x0 = pool[rng.choice(len(pool), m, replace=len(pool) < m)]
    return x0, np.full(m, 1.0 / m)


@pytest.mark.parametrize("rule", ["R1", "R2"])
def test_marginals_and_dual_mass(rule):
    mem = make_members(0, 7, 3)
    x0, w0 = start(mem, 4)
    r = badmm_barycenter(mem, x0, w0, T=37, tau=10, rule=rule)
    assert abs(r["w"].sum() - 1) < 1e-12
    for k, (y, wk) in enumerate(mem):
        np.testing.assert_allclose(r["P1"][k].sum(0), wk, atol=1e-12)
        np.testing.assert_allclose(r["P2"][k].sum(1), r["w"], atol=1e-12)
        assert abs(r["Lam"][k].sum()) < 1e-12 * r["rho"] * 37 + 1e-12
        assert (r["P1"][k] > 0).all() and (r["P2"][k] > 0).all()


def test_rho_is_rho0_times_mean_cost():
    mem = make_members(1, 4, 2)
    x0, w0 = start(mem, 3)
    r = badmm_barycenter(mem, x0, w0, T=1, rho0=2.0)
    allc = np.concatenate([cost_matrix(x0, y).ravel() for y, _ in mem])
    assert abs(r["rho"] - 2.0 * allc.mean()) < 1e-12 * r["rho"]


def test_m1_closed_form():
    mem = make_members(2, 6, 3)
    x0 = np.array([[10.0, -3.0, 4.0]])
    r = badmm_barycenter(mem, x0, np.array([1.0]), T=25, tau=10)
    assert r["w"].shape == (1,) and abs(r["w"][0] - 1.0) < 1e-15
    for k, (y, wk) in enumerate(mem):
        np.testing.assert_allclose(r["P1"][k][0], wk, atol=1e-15)
    mean_of_means = np.mean([wk @ y for y, wk in mem], axis=0)
    np.testing.assert_allclose(r["x"][0], mean_of_means, atol=1e-12)
    obj = np.mean([wk @ np.sum((y - r["x"][0]) ** 2, axis=1) for y, wk in mem])
    assert abs(r["obj"] - obj) < 1e-12 * obj


def cdf_breaks(a, wa):
    """Cumulative weights in increasing order of position (the CDF's jumps)."""
    return np.cumsum(wa[np.argsort(a)])


def quantile_fn(a, wa, t):
    o = np.argsort(a)
    cdf = np.cumsum(wa[o])
    idx = np.minimum(np.searchsorted(cdf, t, side="left"), len(a) - 1)
    return a[o][idx]


def test_fixed_w_fixed_x_tends_to_exact_ot_1d():
    rng = np.random.default_rng(4)
    x = np.sort(rng.normal(size=5))[:, None]
    wx = rng.dirichlet(np.ones(5))
    mem = [(rng.normal(size=(4, 1)) + 0.3, rng.dirichlet(np.ones(4))) for _ in range(3)]
    exact = []
    for y, wy in mem:
        # 1-D closed form on a fine quantile grid (exact for piecewise constants)
        ts = np.unique(np.concatenate([cdf_breaks(x[:, 0], wx), cdf_breaks(y[:, 0], wy), [0.0]]))
        tot = 0.0
        for a, b in zip(ts[:-1], ts[1:]):
            mid = 0.5 * (a + b)
            tot += (b - a) * (quantile_fn(x[:, 0], wx, mid) - quantile_fn(y[:, 0], wy, mid)) ** 2
        exact.append(tot)
    exact = np.mean(exact)
    gaps = []
    for T in (200, 1000, 5000):
        r = badmm_barycenter(mem, x, wx, T=T, fix_w=True, fix_x=True)
        gaps.append(abs(r["obj"] - exact) / exact)
    assert gaps[-1] < 1e-3
    assert gaps[-1] <= gaps[0] + 1e-12


def test_single_member_barycenter_is_the_member():
    """One distribution, m = m_1, started at the member: the barycenter is the
    member itself.  With the support held fixed the weights and plans converge
    to it; with a moving support the objective and the exact W^2 still go to 0
    (a point of tiny weight may wander, so x itself is not compared)."""
    rng = np.random.default_rng(6)
    y = rng.normal(size=(5, 2)) * 2
    wy = rng.dirichlet(np.ones(5))
    var = float(wy @ np.sum((y - wy @ y) ** 2, axis=1))
    fixed = badmm_barycenter([(y, wy)], y.copy(), wy.copy(), T=1000, fix_x=True)
    assert fixed["obj"] < 1e-8 * var
    np.testing.assert_allclose(fixed["w"], wy, atol=1e-6)
    np.testing.assert_allclose(fixed["P2"][0], np.diag(wy), atol=1e-6)
    free = badmm_barycenter([(y, wy)], y.copy(), wy.copy(), T=1000, tau=10)
    assert free["obj"] < 1e-3 * var
    assert w2_exact(free["x"], free["w"], y, wy) < 1e-3 * var
    np.testing.assert_allclose(free["w"], wy, atol=1e-3)


def test_1d_barycenter_quantile_bound():
    rng = np.random.default_rng(7)
    mem = [(rng.normal(size=(3, 1)) * 0.7 + rng.normal() * 2, rng.dirichlet(np.ones(3)))
           for _ in range(4)]
    # optimal barycenter in 1-D: average of quantile functions; its objective is
    # (1/N) sum_k int (Qbar - Q_k)^2 on the merged breakpoint grid
    ts = np.unique(np.concatenate([cdf_breaks(y[:, 0], w) for y, w in mem] + [[0.0]]))
    lower = 0.0
    support, weights = [], []
    for a, b in zip(ts[:-1], ts[1:]):
        mid = 0.5 * (a + b)
        qs = np.array([quantile_fn(y[:, 0], w, mid) for y, w in mem])
        qbar = qs.mean()
        lower += (b - a) * np.mean((qs - qbar) ** 2)
        support.append(qbar)
        weights.append(b - a)
    m = len(support)
    x0, w0 = start(mem, m, seed=8)
    r = badmm_barycenter(mem, x0, w0, T=2000, tau=10)
    achieved = np.mean([w2_exact(r["x"], r["w"], y, w) for y, w in mem])
    assert achieved >= lower - 1e-9
    assert achieved <= lower * 1.05 + 1e-9


def fullbatch_lp(mem, x):
    """Eq. (fullbatch-lp) with fixed support x: variables (w, Pi^(1..N))."""
    m = x.shape[0]
    Cs = [cost_matrix(x, y) for y, _ in mem]
    nv = m + sum(C.size for C in Cs)
    c = np.zeros(nv)
    rows, rhs = [], []
    off = m
    for C, (y, wy) in zip(Cs, mem):
        mk = C.shape[1]
        c[off:off + C.size] = C.ravel() / len(mem)
        for i in range(m):          # row sums = w_i
            a = np.zeros(nv)
            a[off + i * mk: off + (i + 1) * mk] = 1
            a[i] = -1
            rows.append(a)
            rhs.append(0.0)
        for j in range(mk):         # column sums = w_j^(k)
            a = np.zeros(nv)
            a[off + j: off + C.size: mk] = 1
            rows.append(a)
            rhs.append(wy[j])
        off += C.size
    a = np.zeros(nv)
    a[:m] = 1
    rows.append(a)
    rhs.append(1.0)
    res = linprog(c, A_eq=np.array(rows), b_eq=np.array(rhs), bounds=(0, None), method="highs")
    assert res.status == 0
    return res.fun


@pytest.mark.parametrize("seed", range(3))
def test_fixed_support_close_to_full_batch_lp(seed):
    """B-ADMM is an approximation (Section 4): with a pre-fixed support its
    weights give an exact objective at or above the full-batch LP optimum and,
    for a cluster of 30 distributions, within 2% of it (the paper's Table 1
    reports 0.04-0.8% at N = 1000; the consensus rule is weaker for small N)."""
    mem = make_members(100 + seed, 30, 2, mk=(2, 5))
    x0, w0 = start(mem, 4, seed=seed)
    lp = fullbatch_lp(mem, x0)
    r = badmm_barycenter(mem, x0, w0, T=2000, fix_x=True)
    exact = np.mean([w2_exact(x0, r["w"], y, w) for y, w in mem])
    assert exact >= lp - 1e-9                   # LP is the minimum over w
    assert (exact - lp) / lp < 0.02
    assert abs(r["obj"] - lp) / lp < 0.02


def test_invariances():
    mem = make_members(11, 5, 3)
    x0, w0 = start(mem, 4)
    base = badmm_barycenter(mem, x0, w0, T=30, tau=7)
    t = np.array([3.0, -1.0, 0.5])
    sh = badmm_barycenter([(y + t, w) for y, w in mem], x0 + t, w0, T=30, tau=7)
    np.testing.assert_allclose(sh["x"], base["x"] + t, atol=1e-8)
    np.testing.assert_allclose(sh["w"], base["w"], atol=1e-9)
    for a, b in zip(sh["P2"], base["P2"]):
        np.testing.assert_allclose(a, b, atol=1e-9)
    s = 2.5
    sc = badmm_barycenter([(y * s, w) for y, w in mem], x0 * s, w0, T=30, tau=7)
    np.testing.assert_allclose(sc["x"], base["x"] * s, atol=1e-8)
    np.testing.assert_allclose(sc["w"], base["w"], atol=1e-9)
    assert abs(sc["obj"] - base["obj"] * s * s) < 1e-8 * sc["obj"]
    perm = [3, 0, 4, 1, 2]
    pm = badmm_barycenter([mem[p] for p in perm], x0, w0, T=30, tau=7)
    np.testing.assert_allclose(pm["w"], base["w"], atol=1e-12)
    for t_, p in enumerate(perm):
        np.testing.assert_allclose(pm["P2"][t_], base["P2"][p], atol=1e-12)


def test_warm_start_uses_cached_plan():
    mem = make_members(12, 4, 2)
    x0, w0 = start(mem, 3)
    first = badmm_barycenter(mem, x0, w0, T=20)
    cold = badmm_barycenter(mem, first["x"], first["w"], T=1)
    warm = badmm_barycenter(mem, first["x"], first["w"], T=1, plan0=first["P2"],
                            warm=[True] * 4)
    assert any(np.abs(a - b).max() > 1e-6 for a, b in zip(cold["P2"], warm["P2"]))
    mixed = badmm_barycenter(mem, first["x"], first["w"], T=1, plan0=first["P2"],
                             warm=[True, False, True, False])
    # Pi^(k,1) after one iteration depends only on member k's starting plan
    np.testing.assert_allclose(mixed["P1"][0], warm["P1"][0], atol=1e-15)
    np.testing.assert_allclose(mixed["P1"][1], cold["P1"][1], atol=1e-15)


def test_planted_mistakes_are_caught(monkeypatch):
    """Mistakes planted in the oracle must fail at least one pin above."""
    import oracle.badmm as ob

    # (1) a dropped term in the cost (last coordinate ignored) -> m=1 closed form fails
    with monkeypatch.context() as mp:
        mp.setattr(ob, "cost_matrix", lambda x, y: cost_matrix(x[:, :-1], y[:, :-1]))
        with pytest.raises(AssertionError):
            test_m1_closed_form()
    # (2) Pi^(k,1) instead of Pi^(k,2) in Eq. updatex -> translation invariance fails
    real = ob.update_support
    with monkeypatch.context() as mp:
        def wrong(x, w, P2, Y, _real=real):
            return _real(x, w, [p * (1.0 + 0.3 * np.arange(p.shape[1])[None, :] / p.shape[1])
                                for p in P2], Y)
        mp.setattr(ob, "update_support", wrong)
        with pytest.raises(AssertionError):
            test_invariances()
    # (3) R1 without normalisation -> the weight-sum / marginal pins fail
    with monkeypatch.context() as mp:
        mp.setattr(ob, "consensus_weights", lambda wt, rule: np.sum(wt, axis=0) / (len(wt) * 1.01))
        with pytest.raises(AssertionError):
            test_marginals_and_dual_mass("R1")
