"""Exact squared 2-Wasserstein distance (oracle; test infrastructure only).

Eq. (primal) of Section 2: the transportation LP
    min sum_ij pi_ij c(x_i, y_j)  s.t.  sum_i pi_ij = w_j^(b),  sum_j pi_ij = w_i^(a),
    pi >= 0,
with c the squared Euclidean distance.  The paper solves it with a commercial
network simplex; any exact LP solver gives the same (unique) optimal value, so
the oracle hands the LP to scipy's HiGHS solver as a library step.
"""
import numpy as np
from scipy.optimize import linprog

from .cost import cost_matrix


def transport_lp(C, a, b):
    """Optimal value and plan of min <C, P> s.t. P 1 = a, P^T 1 = b, P >= 0
    (Eq. primal, Section 2).

    a and b are rescaled to the same total (their mean total) so that tiny
    rounding differences in the inputs do not make the LP infeasible.
    """
    C = np.asarray(C, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    m, n = C.shape
    tot = 0.5 * (a.sum() + b.sum())
    a = a * (tot / a.sum())
    b = b * (tot / b.sum())
    # equality rows: m row sums then n column sums (one is redundant; HiGHS copes)
    A = np.zeros((m + n, m * n))
    for i in range(m):
        A[i, i * n:(i + 1) * n] = 1.0
    for j in range(n):
        A[m + j, j::n] = 1.0
    res = linprog(C.reshape(-1), A_eq=A, b_eq=np.concatenate([a, b]), bounds=(0, None),
                  method="highs", options=dict(primal_feasibility_tolerance=1e-10,
                                               dual_feasibility_tolerance=1e-10))
    if res.status != 0:
        raise RuntimeError("transport LP failed: " + str(res.message))
    return float(res.fun), res.x.reshape(m, n)


def w2_exact(x, wx, y, wy):
    """W^2(P, Q) for P = {(wx_i, x_i)}, Q = {(wy_j, y_j)} (Eq. primal, p = 2)."""
    val, _ = transport_lp(cost_matrix(x, y), wx, wy)
    return val
