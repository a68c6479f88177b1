"""Learned candidate pruning for the assignment step (oracle; test infrastructure only).

The paper has no learned component: its own assignment accelerator is the
triangle-inequality skipping of Section 5.  This module is the FP64 reference
for the pruning network the library adds in front of the exact assignment of
Algorithm 1.  Design (stated, not from the paper):

  * translation identity of squared-Euclidean OT: for means mu_P, mu_Q,
        W^2(P, Q) = ||mu_P - mu_Q||^2 + W^2(P - mu_P, Q - mu_Q),
    so the mean term is exact and a certified lower bound of W^2;
  * embedding of a distribution P = {(w_j, y_j)} with centred points
    u_j = y_j - mu_P:
        h1_j = relu(W1 u_j + b1),  h2_j = relu(W2 h1_j + b2),
        g = sum_j w_j h2_j,        f(P) = W3 g;
  * predictor  What^2(P, Q) = ||mu_P - mu_Q||^2 + ||f(P) - f(Q)||^2;
  * training loss over pairs (a, q) with exact targets t = W^2 - ||mu_a - mu_q||^2:
        L = (1/B) sum_b (||f(P_a) - f(Q_q)||^2 - t_b)^2;
  * assignment: the r centroids with the smallest predictions are solved
    exactly; with b the best exact value among them, every other centroid i
    must satisfy max(||mu_P - mu_Qi||^2, What^2_i - delta) > b, otherwise all
    K centroids are solved exactly.
"""
import numpy as np

PARAM_NAMES = ("W1", "b1", "W2", "b2", "W3")


def mean_of(y, w):
    """mu_P = sum_j w_j y_j, the mean of the translation identity (module header)."""
    return np.asarray(w, np.float64) @ np.asarray(y, np.float64)


def embed(params, y, w, want_cache=False):
    """f(P) for one distribution (the embedding of the module header; no paper
    passage); params hold float arrays W1 (H,d) b1 (H) W2 (H,H) b2 (H) W3 (E,H)."""
    y = np.asarray(y, np.float64)
    w = np.asarray(w, np.float64)
    W1, b1, W2, b2, W3 = (np.asarray(params[k], np.float64) for k in PARAM_NAMES)
    mu = w @ y
    u = y - mu[None, :]
    a1 = u @ W1.T + b1[None, :]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2[None, :]
    h2 = np.maximum(a2, 0.0)
    g = w @ h2
    f = W3 @ g
    if want_cache:
        return f, dict(u=u, a1=a1, h1=h1, a2=a2, h2=h2, g=g, w=w)
    return f


def embed_backward(params, cache, df):
    """Gradients of <df, f(P)> with respect to the parameters (same names), by
    the chain rule through the embedding of the module header."""
    W1, b1, W2, b2, W3 = (np.asarray(params[k], np.float64) for k in PARAM_NAMES)
    g, w, h2, a2, h1, a1, u = (cache[k] for k in ("g", "w", "h2", "a2", "h1", "a1", "u"))
    gW3 = np.outer(df, g)
    dg = W3.T @ df
    dh2 = w[:, None] * dg[None, :]
    da2 = dh2 * (a2 > 0)
    gW2 = da2.T @ h1
    gb2 = da2.sum(0)
    dh1 = da2 @ W2
    da1 = dh1 * (a1 > 0)
    gW1 = da1.T @ u
    gb1 = da1.sum(0)
    return dict(W1=gW1, b1=gb1, W2=gW2, b2=gb2, W3=gW3)


def pair_loss_and_grad(params, bags, cents, pairs, targets):
    """Loss L of the module header and its gradient for pairs (bag index a,
    centroid index q).

    bags, cents: lists of (y, w); targets: exact W^2 values of the pairs.
    """
    fb, cb = {}, {}
    for a, q in pairs:
        if ("b", a) not in fb:
            fb[("b", a)] = embed(params, bags[a][0], bags[a][1], want_cache=True)
        if ("c", q) not in fb:
            fb[("c", q)] = embed(params, cents[q][0], cents[q][1], want_cache=True)
    B = len(pairs)
    L = 0.0
    dfs = {}
    for (a, q), t in zip(pairs, targets):
        fa = fb[("b", a)][0]
        fq = fb[("c", q)][0]
        mu2 = float(np.sum((mean_of(*bags[a]) - mean_of(*cents[q])) ** 2))
        diff = fa - fq
        res = float(diff @ diff) - (float(t) - mu2)
        L += res * res / B
        gdiff = (2.0 * res / B) * 2.0 * diff
        dfs[("b", a)] = dfs.get(("b", a), 0.0) + gdiff
        dfs[("c", q)] = dfs.get(("c", q), 0.0) - gdiff
    grads = {k: np.zeros_like(np.asarray(params[k], np.float64)) for k in PARAM_NAMES}
    for key, df in dfs.items():
        gk = embed_backward(params, fb[key][1], df)
        for k in PARAM_NAMES:
            grads[k] += gk[k]
    return L, grads


def predict(params, bag, cents):
    """What^2(P, Q_i) for every centroid (the predictor of the module header),
    and the exact mean terms."""
    fP = embed(params, *bag)
    muP = mean_of(*bag)
    pred, mean_term = [], []
    for (x, wx) in cents:
        fQ = embed(params, x, wx)
        mt = float(np.sum((muP - mean_of(x, wx)) ** 2))
        d = fP - fQ
        mean_term.append(mt)
        pred.append(mt + float(d @ d))
    return np.array(pred), np.array(mean_term)


def prune_assign_one(pred, mean_term, exact_fn, r, delta):
    """Label of one distribution by the pruned rule of the module header (exact
    W^2 of Eq. primal on the candidates, the margin test, else all K);
    exact_fn(i) gives W^2 to centroid i.

    Returns (label, W^2 to it, fell_back, number of exact solves).
    """
    K = len(pred)
    order = np.argsort(pred, kind="stable")
    cand = sorted(int(i) for i in order[:min(r, K)])
    vals = {i: exact_fn(i) for i in cand}
    best = min(cand, key=lambda i: (vals[i], i))
    b = vals[best]
    others = [i for i in range(K) if i not in vals]
    ok = all(max(mean_term[i], pred[i] - delta) > b for i in others)
    if ok:
        return best, b, False, len(cand)
    for i in others:
        vals[i] = exact_fn(i)
    best = min(range(K), key=lambda i: (vals[i], i))
    return best, vals[best], True, K
