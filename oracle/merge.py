"""Centroid initialisation by greedy merging (oracle; test infrastructure only).

Section 5, initialisation paragraph and Eq. (merge): while a distribution has
more support points than m, merge the pair (i, j) minimising
    w_i w_j ||x_i - x_j||^2 / (w_i + w_j)
into one point at the weighted mean (w_i x_i + w_j x_j) / (w_i + w_j) with
weight w_i + w_j.  Ties (paper silent): pairs are scanned in lexicographic
(i, j), i < j, order and the first minimum wins; the merged point takes the
smaller index i, the point j is removed and later points shift down by one.
"""
import numpy as np


def merge_reduce(y, w, m):
    """Reduce (y (m_k, d), w (m_k,)) to at most m support points by Eq. (merge)."""
    pts = [np.array(v, dtype=np.float64) for v in np.asarray(y, dtype=np.float64)]
    wts = [float(v) for v in np.asarray(w, dtype=np.float64)]
    while len(pts) > m:
        best, bi, bj = None, -1, -1
        for i in range(len(pts)):
            for j in range(i + 1, len(pts)):
                den = wts[i] + wts[j]
                diff = pts[i] - pts[j]
                crit = wts[i] * wts[j] * float(diff @ diff) / den if den > 0 else 0.0
                if best is None or crit < best:
                    best, bi, bj = crit, i, j
        wbar = wts[bi] + wts[bj]
        if wbar > 0:
            xbar = (wts[bi] * pts[bi] + wts[bj] * pts[bj]) / wbar
        else:
            xbar = 0.5 * (pts[bi] + pts[bj])
        pts[bi] = xbar
        wts[bi] = wbar
        del pts[bj]
        del wts[bj]
    return np.array(pts), np.array(wts)
