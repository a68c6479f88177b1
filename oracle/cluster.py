"""D2-clustering outer loop (oracle; test infrastructure only).

Algorithm 1 (D2 Clustering) of Section 2 with the implementation choices of
Section 5: centroids initialised from randomly chosen distributions reduced by
Eq. (merge); the assignment step by exact W (Eq. primal); the update step by
B-ADMM (Algorithm badmm) with a fixed iteration count, warm-starting the plan
of every member whose label did not change.

Readings where the paper is silent:
  * random choices use SplitMix64 (Steele, Lea & Flood, OOPSLA 2014), seeded by
    the caller: K distinct members with m_k >= m are drawn by a partial
    Fisher-Yates shuffle of the eligible member ids (ascending), index
    t + (next() mod (E - t)) at step t;
  * argmin ties go to the lowest centroid index;
  * an empty cluster keeps its previous centroid;
  * a fixed number of rounds replaces the label-change stopping rule;
  * obj_per_round[r] = (1/N) sum_k W^2(Q_{l_k}, P^(k)) at the assignment of
    round r (the within-cluster variation of Section 2).
"""
import numpy as np

from .badmm import badmm_barycenter
from .merge import merge_reduce
from .ot import w2_exact

MASK64 = (1 << 64) - 1


def splitmix64(state):
    """One SplitMix64 step (Steele, Lea & Flood, OOPSLA 2014): returns
    (new_state, output), all arithmetic mod 2^64.  The generator of the random
    initialisation of Algorithm 1 (a reading: the paper names none)."""
    state = (state + 0x9E3779B97F4A7C15) & MASK64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return state, z ^ (z >> 31)


def init_pick(sizes, K, m, seed):
    """Ids of the K members whose merged supports seed the centroids.

    Eligible: the ids with m_k >= m (the merge of Eq. (merge) then reduces each
    to m points).  The paper leaves the case of fewer than K such members
    open; the reading taken is to lower the threshold to the K-th largest m_k,
    so the K picks are drawn among the largest distributions (those with fewer
    than m points are later padded with zero-weight copies)."""
    if K > len(sizes):
        raise ValueError("fewer than K distributions")
    thr = min(m, sorted(sizes, reverse=True)[K - 1])
    eligible = [k for k, s in enumerate(sizes) if s >= thr]
    state = seed & MASK64
    E = len(eligible)
    for t in range(K):
        state, z = splitmix64(state)
        j = t + int(z % (E - t))
        eligible[t], eligible[j] = eligible[j], eligible[t]
    return eligible[:K]


def pad_support(x, w, m):
    """A centroid seeded by a distribution with fewer than m points keeps m
    support points: the missing ones are zero-weight copies of its last point
    (reading taken where the paper assumes m_k >= m)."""
    q = x.shape[0]
    if q >= m:
        return x, w
    return (np.vstack([x, np.repeat(x[-1:], m - q, axis=0)]),
            np.concatenate([w, np.zeros(m - q)]))


def d2_assign(bags_list, cents):
    """Assignment step of Algorithm 1: l_k = argmin_i W(Q_i, P_k) (ties -> lowest i).

    bags_list: list of (y, w); cents: list of (x, w).  Returns (labels, dists, D)
    with D the full N x K matrix of W^2.
    """
    N, K = len(bags_list), len(cents)
    D = np.empty((N, K))
    for k, (y, wy) in enumerate(bags_list):
        for i, (x, wx) in enumerate(cents):
            D[k, i] = w2_exact(x, wx, y, wy)
    labels = np.argmin(D, axis=1)            # first minimum = lowest index
    return labels, D[np.arange(N), labels], D


def cluster_rounds(N, cents, rounds, assign, update, labels_in=None):
    """The rounds of Algorithm 1 with the Section 5 warm start, for any kind of
    centroid: assign(cents) -> (labels, dists); update(i, ids, cent, plan0,
    warm) -> (new centroid, that call's Pi^(k,2) list).  A member starts from
    its cached Pi^(k,2) exactly when its label equals its label at the
    previous round's assignment; an empty cluster keeps its centroid.
    labels_in: optional per-round labels used instead of the assignment
    (teacher forcing).  Returns (cents, labels, objs, labels_per_round)."""
    K = len(cents)
    prev_labels = None
    cache = [None] * N
    objs, all_labels = [], []
    for r in range(rounds):
        labels, dists = assign(cents)
        objs.append(float(np.mean(dists)))
        if labels_in is not None:
            labels = np.asarray(labels_in[r])
        all_labels.append(labels.copy())
        new_cents = []
        for i in range(K):
            ids = [k for k in range(N) if labels[k] == i]
            if not ids:
                new_cents.append(cents[i])
                continue
            warm = [prev_labels is not None and prev_labels[k] == i and cache[k] is not None
                    for k in ids]
            cent, P2 = update(i, ids, cents[i], [cache[k] for k in ids], warm)
            for t, k in enumerate(ids):
                cache[k] = P2[t]
            new_cents.append(cent)
        cents = new_cents
        prev_labels = labels
    return cents, prev_labels, objs, all_labels


def d2_cluster(bags_list, K, m, seed, rounds, *, rho0=2.0, T=100, tau=10, eps=1e-16,
               rule="R1", labels_in=None):
    """Algorithm 1 with the Section 5 choices.

    labels_in: optional list of per-round label arrays; when given, round r uses
    labels_in[r] instead of its own assignment (teacher forcing, so a single
    near-tie flip does not make later rounds incomparable).
    Returns dict(x (K,m,d), w (K,m), labels, obj_per_round, dists).
    """
    sizes = [y.shape[0] for y, _ in bags_list]
    picks = init_pick(sizes, K, m, seed)
    cents = [pad_support(*merge_reduce(bags_list[k][0], bags_list[k][1], m), m) for k in picks]

    def assign(cs):
        labels, dists, _ = d2_assign(bags_list, cs)
        return labels, dists

    def update(i, ids, cent, plan0, warm):
        res = badmm_barycenter([bags_list[k] for k in ids], cent[0], cent[1], rho0=rho0, T=T, tau=tau,
                               eps=eps, rule=rule, plan0=plan0, warm=warm)
        return (res["x"], res["w"]), res["P2"]

    cents, labels, objs, all_labels = cluster_rounds(len(bags_list), cents, rounds, assign, update, labels_in)
    return dict(x=np.array([c[0] for c in cents]), w=np.array([c[1] for c in cents]),
                labels=labels, obj_per_round=objs, labels_per_round=all_labels,
                picks=picks)
