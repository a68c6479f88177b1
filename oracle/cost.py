"""Squared-Euclidean ground cost (oracle; test infrastructure only).

Section 2 defines c(x_i, x_j) = ||x_i - x_j||_p^p with p = 2 for D2-clustering,
and the notation list defines C(x, x^(k)) = (||x_i - x_j^(k)||^2)_{i,j} in
R^{m x m_k}.
"""
import numpy as np


def cost_matrix(x, y):
    """C[i, j] = sum_d (x[i, d] - y[j, d])^2, by direct differences in FP64
    (Section 2: the ground cost with p = 2, C(x, x^(k)) of the notation list).

    x: (m, d) barycenter support, y: (m_k, d) member support -> (m, m_k).
    """
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    diff = x[:, None, :] - y[None, :, :]
    return np.sum(diff * diff, axis=2)
