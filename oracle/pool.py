"""Process-pool job for timing the oracle on every host core (test and
baseline infrastructure only, like the rest of this package)."""


def barycenter_job(args):
    """One whole cluster through badmm_barycenter (Algorithm badmm):
    (members, x0, w0, T, tau)."""
    from .badmm import badmm_barycenter
    members, x0, w0, T, tau = args
    badmm_barycenter(members, x0, w0, T=T, tau=tau)
    return 0
