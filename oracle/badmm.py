"""Modified Bregman-ADMM Wasserstein barycenter (oracle; test infrastructure only).

Follows "Centroid Update with B-ADMM" (Algorithm badmm, Section 3.3) step by
step in FP64, one cluster at a time, with the plan of member k held as an
m x m_k matrix (rows i = barycenter support points, columns j = the member's
support points), exactly the paper's Pi^(k).

Readings where the paper is silent or ambiguous (each listed in the design
notes):
  * rho (Eq. rho): rho0 times the MEAN entry of all cost matrices of the
    cluster, computed once per call from the initial support, not recomputed
    after the support moves; if every cost is zero, rho = 1 (with C = 0 the
    plans depend on Lambda / rho only, which does not depend on rho).
  * "Update x per tau loops": the support update (Eq. updatex) runs at the top
    of iterations n > 0 with n mod tau == 0 and uses the current Pi^(k,2) and
    w, whose row sums equal w_i, so N*w_i is the transported mass; a point
    whose mass N*w_i is below 1e-300 keeps its position.
  * eps is added after the exponential scaling, literally as printed
    (Eqs. badmmc0b and badmmc1b).
  * The returned objective is (1/N) sum_k <C_k, Pi^(k,1)> with the final
    plans and the cost of the final support.
"""
import numpy as np

from .cost import cost_matrix


def update_support(x, w, P2, Y):
    """Eq. (updatex): x_i := (1 / (N w_i)) sum_k sum_j pi_ij^(k) x_j^(k)  (with Pi^(k,2))."""
    N = len(Y)
    num = np.zeros_like(x)
    for k in range(N):
        num += P2[k] @ Y[k]
    mass = N * w
    keep = mass < 1e-300
    return np.where(keep[:, None], x, num / np.where(keep, 1.0, mass)[:, None])


def consensus_weights(wtil, rule):
    """Eq. (badmmw) for R1 and Eq. (badmmw2) for R2, normalised to the simplex."""
    N = len(wtil)
    if rule == "R1":
        s = np.sum(wtil, axis=0) / N
        return s / s.sum()
    if rule == "R2":
        s = np.sum([np.sqrt(v) for v in wtil], axis=0) / N
        return s * s / np.sum(s * s)
    raise ValueError(rule)


def badmm_barycenter(members, x0, w0, *, rho0=2.0, T=100, tau=10, eps=1e-16, rule="R1",
                     plan0=None, warm=None, fix_w=False, fix_x=False, rho=None, costs=None):
    """Run T iterations of Algorithm badmm on one cluster.

    members : list of (y_k (m_k, d), w_k (m_k,)) -- the cluster's distributions P^(k)
    x0, w0  : initial barycenter support (m, d) and weights (m,)
    plan0   : optional list of cached Pi^(k,2) (m, m_k) for a warm start
    warm    : optional list of bools; member k starts from plan0[k] when True,
              else from pi_ij = w_i w_j^(k) (Section 5, warm start paragraph)
    fix_w   : keep w = w0 (then every member solves the OT problem between w0
              and w^(k); used as a test mode)
    fix_x   : never move the support (pre-fixed support track of Section 4)
    rho     : override rho (else Eq. rho with the reading above)
    costs   : optional list of the members' cost matrices C_k (m x m_k), given
              instead of computed from coordinates: symbolic supports with a
              given symbol-to-symbol dissimilarity (Section 5), whose support
              is fixed; members' y and x0 are then unused (x0 may be None)
    Returns dict(x, w, P1, P2, Lam, obj, rho).
    """
    N = len(members)
    w = np.array(w0, dtype=np.float64, copy=True)
    m = w.shape[0]
    Wk = [np.asarray(wk, dtype=np.float64) for _, wk in members]
    if costs is not None:
        fix_x = True
        x = None if x0 is None else np.array(x0, dtype=np.float64, copy=True)
        C = [np.asarray(Ck, dtype=np.float64) for Ck in costs]
        Y = [np.zeros((Ck.shape[1], 0)) for Ck in C]
    else:
        x = np.array(x0, dtype=np.float64, copy=True)
        Y = [np.asarray(y, dtype=np.float64) for y, _ in members]
        C = [cost_matrix(x, Y[k]) for k in range(N)]
    if rho is None:
        # Eq. rho: rho0 times the average transport cost over all m*m_k entries
        total = sum(float(Ck.sum()) for Ck in C)
        count = m * sum(y.shape[0] for y in Y)
        rho = rho0 * total / count
        if not rho > 0.0:
            rho = 1.0  # all costs zero: every rho > 0 gives the same plans
    rho = float(rho)

    # Algorithm badmm, first line: Lambda := 0; Pi^(2),0 := Pi
    Lam = [np.zeros((m, Y[k].shape[0])) for k in range(N)]
    P2 = []
    for k in range(N):
        if plan0 is not None and warm is not None and warm[k]:
            P2.append(np.array(plan0[k], dtype=np.float64, copy=True))
        else:
            P2.append(np.outer(w, Wk[k]))
    P1 = [None] * N

    for n in range(T):
        # Support update (Eq. updatex) every tau loops
        if (not fix_x) and n > 0 and n % tau == 0:
            x = update_support(x, w, P2, Y)
            C = [cost_matrix(x, Y[k]) for k in range(N)]

        Ptil = [None] * N
        r = [None] * N
        wtil = [None] * N
        for k in range(N):
            # Eq. badmmc0b
            T1 = P2[k] * np.exp((C[k] + Lam[k]) / (-rho)) + eps
            # Eq. badmmc0: normalise each column j over i, scale to w_j^(k)
            P1[k] = T1 / T1.sum(axis=0, keepdims=True) * Wk[k][None, :]
            # Eq. badmmc1b
            Ptil[k] = P1[k] * np.exp(Lam[k] / rho) + eps
            # row sums and their normalisation (the w-tilde^(k) of Section 3.3)
            r[k] = Ptil[k].sum(axis=1)
            wtil[k] = r[k] / r[k].sum()

        if not fix_w:
            w = consensus_weights(wtil, rule)

        for k in range(N):
            # Eq. badmmc1: normalise each row i over j, scale to w_i
            P2[k] = Ptil[k] / r[k][:, None] * w[:, None]
            # Eq. badmm2
            Lam[k] = Lam[k] + rho * (P1[k] - P2[k])

    obj = sum(float(np.sum(C[k] * P1[k])) for k in range(N)) / N if T > 0 else float("nan")
    return dict(x=x, w=w, P1=P1, P2=P2, Lam=Lam, obj=obj, rho=rho, C=C)
