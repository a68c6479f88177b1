"""Shared test helpers: run the GPU path through the binding and the oracle on
the same seeded inputs, and slice per-member plans out of the j-major layout."""
import numpy as np
import torch

import synth


def cluster_members(bags, cluster_offsets, members, c):
    co = cluster_offsets.cpu()
    ids = members.cpu()[int(co[c]):int(co[c + 1])].tolist()
    return ids, [bags.bag(k) for k in ids]


def member_plan(plan, offsets, k):
    """Pi^(k) (m x m_k) from the n x m j-major plan array."""
    a, b = int(offsets[k]), int(offsets[k + 1])
    return plan[a:b].double().cpu().numpy().T


def split_clusters(labels, K):
    """cluster_offsets / members (sorted by cluster, stable by id) for labels."""
    labels = torch.as_tensor(labels, dtype=torch.int64)
    order = torch.sort(labels, stable=True).indices
    counts = torch.bincount(labels, minlength=K)
    co = torch.zeros(K + 1, dtype=torch.int64)
    co[1:] = torch.cumsum(counts, 0)
    return co, order


def run_gpu_badmm(d2, ctx, bags, cluster_offsets, members, x0, w0, plan0=None, warm=None, nopipe=False, **kw):
    db = d2.DeviceBags.from_synth(bags)
    x = x0.clone().cuda().contiguous()
    w = w0.clone().cuda().contiguous()
    plan = (plan0.clone().cuda() if plan0 is not None
            else torch.zeros(bags.n, x.shape[1], dtype=torch.float32, device="cuda"))
    wm = None if warm is None else warm.to(torch.uint8).cuda()
    opts = d2.badmm_opts(**kw)
    if nopipe:
        opts.flags |= d2.D2_NO_PIPE
    x, w, plan, obj = d2.badmm_barycenter(ctx, db, cluster_offsets.cuda(), members.cuda(), x, w, plan,
                                          wm, opts)
    torch.cuda.synchronize()
    return x.cpu(), w.cpu(), plan.cpu(), obj.cpu()


def compare_cluster(bags, cluster_offsets, members, c, gx, gw, gplan, gobj, ref,
                    plan_tol=1e-5, w_tol=1e-5, obj_rtol=1e-4, x_tol=None):
    ids, _ = cluster_members(bags, cluster_offsets, members, c)
    np.testing.assert_allclose(gw[c].double().numpy(), ref["w"], rtol=0, atol=w_tol)
    for t, k in enumerate(ids):
        np.testing.assert_allclose(member_plan(gplan, bags.offsets, k), ref["P2"][t], rtol=0,
                                   atol=plan_tol, err_msg="cluster %d member %d" % (c, k))
    assert abs(float(gobj[c]) - ref["obj"]) <= obj_rtol * abs(ref["obj"]), (float(gobj[c]), ref["obj"])
    if x_tol is not None:
        np.testing.assert_allclose(gx[c].double().numpy(), ref["x"], rtol=0, atol=x_tol)


def oracle_cluster_job(args):
    """One oracle barycenter (a process-pool job): (members, x0, w0, T, tau)."""
    from oracle import badmm_barycenter
    members, x0, w0, T, tau = args
    return badmm_barycenter(members, x0, w0, T=T, tau=tau)


def oracle_clusters(jobs, procs=8):
    """Oracle barycenters of several clusters in spawned worker processes
    (spawn: the parent has already initialised CUDA)."""
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(min(procs, max(1, len(jobs)))) as pool:
        return pool.map(oracle_cluster_job, jobs, chunksize=1)
