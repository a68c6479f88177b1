"""Symbolic supports (oracle; test infrastructure only).

Section 2 allows the support space to be a symbolic set with a given
symbol-to-symbol dissimilarity instead of R^d; Section 5 notes that the
support-update step of D2-clustering is then skipped, since the set of
symbols is fixed.  A distribution is (symbol ids, weights); a centroid is m
symbols and their weights; the cost between symbol s and symbol t is D[s, t].

Readings where the paper is silent (each listed in the design notes):
  * every centroid is supported on the same m symbols (the caller's set);
  * initialisation: K distinct distributions drawn by the SplitMix64 partial
    Fisher-Yates shuffle of all ids (no size condition: nothing is merged);
    centroid weights are the drawn distribution's masses moved to the nearest
    centroid symbol (smallest D[s_i, t], first minimum);
  * the rounds are those of the coordinate loop (cluster.cluster_rounds).
"""
import numpy as np

from .badmm import badmm_barycenter
from .cluster import MASK64, cluster_rounds, splitmix64
from .ot import transport_lp


def sym_cost(D, s, t):
    """C[i, j] = D[s_i, t_j]: the cost matrix between symbols s (m) and t (m_k)
    (Section 2: the given symbol-to-symbol dissimilarity as the ground cost)."""
    D = np.asarray(D, dtype=np.float64)
    return D[np.ix_(np.asarray(s, dtype=np.int64), np.asarray(t, dtype=np.int64))]


def w2_sym(D, s, ws, t, wt):
    """Optimal value of the transportation LP of Eq. (primal) with the given costs."""
    val, _ = transport_lp(sym_cost(D, s, t), ws, wt)
    return val


def badmm_sym(D, members, s, w0, **kw):
    """Algorithm badmm with fixed symbolic support s: members are (t_k, w_k)."""
    costs = [sym_cost(D, s, t) for t, _ in members]
    return badmm_barycenter(members, None, w0, costs=costs, **kw)


def project_to_symbols(D, s, t, wt):
    """Weights on the symbols s of a distribution (t, wt): each t_j's mass goes
    to its nearest symbol in s (first minimum of D[s_i, t_j] over i); the
    initialisation reading for symbolic supports of the module header."""
    C = sym_cost(D, s, t)
    w = np.zeros(len(s))
    for j in range(len(t)):
        w[int(np.argmin(C[:, j]))] += float(wt[j])
    return w / w.sum()


def sym_init_pick(N, K, seed):
    """K distinct ids of 0..N-1 by the partial Fisher-Yates shuffle driven by
    SplitMix64: the random initialisation of Algorithm 1 (module header)."""
    ids = list(range(N))
    state = seed & MASK64
    for t in range(K):
        state, z = splitmix64(state)
        j = t + int(z % (N - t))
        ids[t], ids[j] = ids[j], ids[t]
    return ids[:K]


def d2_cluster_sym(D, bags, K, s, seed, rounds, *, rho0=2.0, T=100, tau=10, eps=1e-16, rule="R1",
                   labels_in=None):
    """Algorithm 1 on symbolic distributions, every centroid on the symbols s.
    bags: list of (t, wt).  Returns dict(w (K, m), labels, obj_per_round, picks)."""
    N = len(bags)
    picks = sym_init_pick(N, K, seed)
    cents = [project_to_symbols(D, s, *bags[k]) for k in picks]

    def assign(ws):
        Dm = np.array([[w2_sym(D, s, w, *bags[k]) for w in ws] for k in range(N)])
        labels = np.argmin(Dm, axis=1)
        return labels, Dm[np.arange(N), labels]

    def update(i, ids, w, plan0, warm):
        res = badmm_sym(D, [bags[k] for k in ids], s, w, rho0=rho0, T=T, tau=tau, eps=eps, rule=rule,
                        plan0=plan0, warm=warm)
        return res["w"], res["P2"]

    cents, labels, objs, all_labels = cluster_rounds(N, cents, rounds, assign, update, labels_in)
    return dict(w=np.array(cents), labels=labels, obj_per_round=objs, labels_per_round=all_labels,
                picks=picks)
