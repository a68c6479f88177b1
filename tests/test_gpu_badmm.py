"""GPU parity of d2_cost and badmm_barycenter (through the C ABI) against the
FP64 oracle on the same seeded inputs.

Tolerances (stated by the target): plan entries and barycenter weights within
1e-5 absolute, the objective within 1e-4 relative.  Supports are compared
within 2e-4 x (1 + max |x|): they are plan-weighted means of FP32 data.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import badmm_barycenter as oracle_badmm, cost_matrix
from tests.helpers import (cluster_members, compare_cluster, member_plan, oracle_clusters, run_gpu_badmm,
                           split_clusters)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def d2():
    import paper_1510_00012_gb300 as d2mod
    from paper_1510_00012_gb300 import build
    build.build()
    return d2mod


@pytest.fixture(scope="module")
def ctx(d2):
    return d2.Context(0)


def x_tol(ref):
    return 2e-4 * (1.0 + float(np.abs(ref["x"]).max()))


def test_single_barycenter_circle_mixture(d2, ctx):
    """N=64 distributions in d=2, m_k ~ U{4..16}, m=8, 200 iterations."""
    bags = synth.circle_mixture_bags(0)
    co = torch.tensor([0, bags.N], dtype=torch.int64)
    mem = torch.arange(bags.N, dtype=torch.int64)
    x0, w0 = synth.sample_initial_barycenters(1, bags, co, mem, 8)
    gx, gw, gplan, gobj = run_gpu_badmm(d2, ctx, bags, co, mem, x0, w0, iters=200, tau=10)
    _, members = cluster_members(bags, co, mem, 0)
    ref = oracle_badmm(members, x0[0].double().numpy(), w0[0].double().numpy(), T=200, tau=10)
    compare_cluster(bags, co, mem, 0, gx, gw, gplan, gobj, ref, x_tol=x_tol(ref))


def ragged_case(seed, K, m, d=16, N=150, mk=(1, 24)):
    bags = synth.gaussian_class_bags(seed, N, d, K - 2, mk=mk)
    lab = bags.labels.clone()
    lab[0] = K - 2                      # a single-member cluster
    # cluster K-1 stays empty
    co, mem = split_clusters(lab, K)
    x0, w0 = synth.sample_initial_barycenters(seed + 1, bags, co, mem, m)
    return bags, co, mem, x0, w0


@pytest.mark.parametrize("m,nopipe", [(16, False), (16, True), (12, False), (5, False), (32, False),
                                      (32, True), (1, False), (64, False), (128, False)])
def test_batched_ragged_clusters(d2, ctx, m, nopipe):
    K = 7
    bags, co, mem, x0, w0 = ragged_case(3, K, m)
    gx, gw, gplan, gobj = run_gpu_badmm(d2, ctx, bags, co, mem, x0, w0, iters=31, tau=10, nopipe=nopipe)
    for c in range(K):
        ids, members = cluster_members(bags, co, mem, c)
        if not ids:
            assert torch.equal(gx[c], x0[c]) and torch.equal(gw[c], w0[c])
            assert float(gobj[c]) == 0.0
            continue
        ref = oracle_badmm(members, x0[c].double().numpy(), w0[c].double().numpy(), T=31, tau=10)
        compare_cluster(bags, co, mem, c, gx, gw, gplan, gobj, ref, x_tol=x_tol(ref))


@pytest.mark.parametrize("variant", ["R2", "fix_x", "fix_w", "tau1", "T1"])
def test_rules_and_modes(d2, ctx, variant):
    K, m = 4, 8
    bags, co, mem, x0, w0 = ragged_case(11, K, m, d=5, N=60, mk=(2, 12))
    kw = dict(iters=25, tau=10)
    okw = dict(T=25, tau=10)
    if variant == "R2":
        kw["rule"] = okw["rule"] = "R2"
    elif variant == "fix_x":
        kw["fix_x"] = okw["fix_x"] = True
    elif variant == "fix_w":
        kw["fix_w"] = okw["fix_w"] = True
    elif variant == "tau1":
        kw["tau"] = okw["tau"] = 1
    elif variant == "T1":
        kw["iters"] = okw["T"] = 1
    gx, gw, gplan, gobj = run_gpu_badmm(d2, ctx, bags, co, mem, x0, w0, **kw)
    for c in range(K):
        ids, members = cluster_members(bags, co, mem, c)
        if not ids:
            continue
        ref = oracle_badmm(members, x0[c].double().numpy(), w0[c].double().numpy(), **okw)
        compare_cluster(bags, co, mem, c, gx, gw, gplan, gobj, ref, x_tol=x_tol(ref))


def test_fixed_rho_override(d2, ctx):
    K, m = 3, 8
    bags, co, mem, x0, w0 = ragged_case(12, K, m, d=4, N=40, mk=(2, 10))
    gx, gw, gplan, gobj = run_gpu_badmm(d2, ctx, bags, co, mem, x0, w0, iters=12, tau=5, rho=3.5)
    for c in range(K):
        ids, members = cluster_members(bags, co, mem, c)
        if ids:
            ref = oracle_badmm(members, x0[c].double().numpy(), w0[c].double().numpy(), T=12, tau=5,
                               rho=3.5)
            compare_cluster(bags, co, mem, c, gx, gw, gplan, gobj, ref, x_tol=x_tol(ref))


def test_warm_start_chain(d2, ctx):
    """Second call warm-starts half the members from each side's own first call."""
    K, m = 3, 8
    bags, co, mem, x0, w0 = ragged_case(13, K, m, d=6, N=50, mk=(2, 10))
    gx, gw, gplan, gobj = run_gpu_badmm(d2, ctx, bags, co, mem, x0, w0, iters=20, tau=10)
    warm = torch.zeros(bags.N, dtype=torch.bool)
    warm[::2] = True
    gx2, gw2, gplan2, gobj2 = run_gpu_badmm(d2, ctx, bags, co, mem, gx, gw, plan0=gplan, warm=warm,
                                            iters=15, tau=10)
    for c in range(K):
        ids, members = cluster_members(bags, co, mem, c)
        if not ids:
            continue
        r1 = oracle_badmm(members, x0[c].double().numpy(), w0[c].double().numpy(), T=20, tau=10)
        r2 = oracle_badmm(members, r1["x"], r1["w"], T=15, tau=10, plan0=r1["P2"],
                          warm=[bool(warm[k]) for k in ids])
        compare_cluster(bags, co, mem, c, gx2, gw2, gplan2, gobj2, r2, x_tol=x_tol(r2))


@pytest.mark.parametrize("d,m,mk", [(48, 8, (3, 20)), (300, 64, (10, 60))])
def test_vocabulary_bags(d2, ctx, d, m, mk):
    """Supports stored as indices into a word table (document-like bags)."""
    bags = synth.document_bags(5, 80, V=400, d=d, mk=mk)
    K = 3
    lab = torch.arange(bags.N) % K
    co, mem = split_clusters(lab, K)
    x0, w0 = synth.sample_initial_barycenters(6, bags, co, mem, m)
    gx, gw, gplan, gobj = run_gpu_badmm(d2, ctx, bags, co, mem, x0, w0, iters=25, tau=10)
    for c in range(K):
        ids, members = cluster_members(bags, co, mem, c)
        ref = oracle_badmm(members, x0[c].double().numpy(), w0[c].double().numpy(), T=25, tau=10)
        compare_cluster(bags, co, mem, c, gx, gw, gplan, gobj, ref, x_tol=x_tol(ref))


def test_deterministic(d2, ctx):
    K, m = 5, 16
    bags, co, mem, x0, w0 = ragged_case(14, K, m)
    a = run_gpu_badmm(d2, ctx, bags, co, mem, x0, w0, iters=21, tau=10)
    b = run_gpu_badmm(d2, ctx, bags, co, mem, x0, w0, iters=21, tau=10)
    for u, v in zip(a, b):
        assert torch.equal(u, v)


@pytest.mark.parametrize("m,d", [(8, 2), (16, 16), (12, 7), (64, 300), (100, 3), (100, 8), (32, 64)])
def test_cost_matches_definition(d2, ctx, m, d):
    K = 3
    bags = synth.gaussian_class_bags(20 + m, 40, d, K, mk=(1, 30), mu_sigma=4.0)
    co, mem = split_clusters(bags.labels, K)
    x0, _ = synth.sample_initial_barycenters(21, bags, co, mem, m)
    x0 = x0 + 3.0  # off-centre barycenters
    db = d2.DeviceBags.from_synth(bags)
    C = d2.d2_cost(ctx, db, co.cuda(), mem.cuda(), x0.cuda()).cpu()
    for c in range(K):
        ids, members = cluster_members(bags, co, mem, c)
        for k, (y, _) in zip(ids, members):
            ref = cost_matrix(x0[c].double().numpy(), y)
            got = member_plan(C, bags.offsets, k)
            np.testing.assert_allclose(got, ref, rtol=2e-5, atol=2e-5 * (1 + ref.max()))


def test_invalid_arguments(d2, ctx):
    bags = synth.circle_mixture_bags(1, N=4)
    db = d2.DeviceBags.from_synth(bags)
    co = torch.tensor([0, 4], dtype=torch.int64, device="cuda")
    mem = torch.arange(4, dtype=torch.int64, device="cuda")
    x = torch.zeros(1, 300, 2, device="cuda")
    w = torch.full((1, 300), 1 / 300, device="cuda")
    with pytest.raises(d2.D2Error) as e:
        d2.badmm_barycenter(ctx, db, co, mem, x, w)
    assert e.value.code == d2.D2_EINVAL
    bad = bags.wt.clone()
    bad[0] += 0.5
    db2 = d2.DeviceBags(db.offsets, bad.cuda(), db.d, supp=db.supp)
    with pytest.raises(d2.D2Error) as e:
        d2.d2_check_bags(ctx, db2)
    assert e.value.code == d2.D2_EINVAL
    d2.d2_check_bags(ctx, db)


@pytest.fixture(scope="module")
def full_size():
    """The benchmark's workload: 4,096 clusters with log-uniform member counts
    in [16, 4096] (~3M distributions), d=64, m_k ~ U{16..64}, m=32, T=100, and
    the FP64 oracle on a 34-cluster subset: clusters at 32 evenly spaced ranks
    of size up to the 75th percentile, the cluster at the 97th percentile and
    the largest one (thousands of members: the cross-member weight sums then
    add the most terms)."""
    bags, co, mem = synth.ragged_cluster_bags(7, 4096, device="cuda")
    m = 32
    x0, w0 = synth.sample_initial_barycenters(8, bags, co, mem, m)
    sizes = (co[1:] - co[:-1]).cpu()
    order = torch.argsort(sizes)
    # the two large clusters first, so that the process pool starts them first
    picks = [int(order[-1]), int(order[3973])]
    picks += [int(order[i]) for i in np.linspace(0, 3072, 32).astype(int)]
    host = bags.to("cpu")
    jobs = []
    for c in picks:
        _, members = cluster_members(host, co, mem, c)
        jobs.append((members, x0[c].double().cpu().numpy(), w0[c].double().cpu().numpy(), 100, 10))
    refs = oracle_clusters(jobs)
    return bags, host, co, mem, x0, w0, picks, refs


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_full_size_ragged_clusters(d2, ctx, full_size, precision):
    """The launch configuration the benchmark times (FP32 cost build, and the
    split-BF16 tensor-core build the benchmark uses).  Checks plan marginals on
    every cluster and full parity against the oracle on the 34-cluster subset."""
    bags, host, co, mem, x0, w0, picks, refs = full_size
    m = 32
    db = d2.DeviceBags.from_synth(bags)
    x, w = x0.clone(), w0.clone()
    plan = torch.empty(bags.n, m, dtype=torch.float32, device="cuda")
    obj = torch.empty(4096, dtype=torch.float64, device="cuda")
    d2.badmm_barycenter(ctx, db, co, mem, x, w, plan, None, d2.badmm_opts(iters=100, tau=10, cost=precision),
                        obj)
    torch.cuda.synchronize()
    assert ctx.device_errors() == 0
    # Pi^(k,2) row sums equal w_i for every member (Eq. badmmc1), w in the simplex
    owner = torch.repeat_interleave(torch.arange(bags.N, device="cuda"), bags.offsets[1:] - bags.offsets[:-1])
    rows = torch.zeros(bags.N, m, dtype=torch.float64, device="cuda").index_add_(0, owner, plan.double())
    clus = torch.repeat_interleave(torch.arange(4096, device="cuda"), co[1:] - co[:-1])
    assert torch.allclose(rows, w[clus].double(), atol=1e-6, rtol=0)
    assert torch.allclose(w.double().sum(1), torch.ones(4096, dtype=torch.float64, device="cuda"), atol=1e-6)
    assert torch.isfinite(obj).all() and (obj > 0).all()
    gw, gobj, gx = w.cpu(), obj.cpu(), x.cpu()
    worst = np.zeros(4)
    for c, ref in zip(picks, refs):
        ids, _ = cluster_members(host, co, mem, c)
        ew = float(np.abs(gw[c].double().numpy() - ref["w"]).max())
        eo = abs(float(gobj[c]) - ref["obj"]) / ref["obj"]
        ex = float(np.abs(gx[c].double().numpy() - ref["x"]).max())
        ep = 0.0
        for t, k in enumerate(ids):
            a, b = int(host.offsets[k]), int(host.offsets[k + 1])
            ep = max(ep, float(np.abs(plan[a:b].double().cpu().numpy().T - ref["P2"][t]).max()))
        worst = np.maximum(worst, [ew, ep, eo, ex / (1 + float(np.abs(ref["x"]).max()))])
    print("full size, %s cost, 34 clusters (largest %d members): max |w| err %.2e, max |plan| err %.2e, max rel obj err %.2e, "
          "max x err / (1 + max|x|) %.2e" % (precision, int(co[picks[0] + 1] - co[picks[0]]), *worst))
    assert worst[0] <= 1e-5 and worst[1] <= 1e-5 and worst[2] <= 1e-4 and worst[3] <= 2e-4


def test_graph_replay_matches_direct_launches(d2, ctx):
    """On a non-default stream the launch sequence is captured once and
    replayed; new data in the same buffers must give the direct results."""
    K, m = 5, 16
    bags, co, mem, x0, w0 = ragged_case(15, K, m)
    db = d2.DeviceBags.from_synth(bags)
    co_d, mem_d = co.cuda(), mem.cuda()
    s = torch.cuda.Stream()
    x = torch.empty(K, m, bags.d, device="cuda")
    w = torch.empty(K, m, device="cuda")
    plan = torch.zeros(bags.n, m, device="cuda")
    obj = torch.empty(K, dtype=torch.float64, device="cuda")
    results = []
    for shift in (0.0, 0.5, 0.5):
        for graph in (True, False):
            with torch.cuda.stream(s):
                x.copy_(x0.cuda() + shift)
                w.copy_(w0.cuda())
                d2.badmm_barycenter(ctx, db, co_d, mem_d, x, w, plan, None,
                                    d2.badmm_opts(iters=23, tau=10, graph=graph), obj)
            s.synchronize()
            results.append((x.clone(), w.clone(), plan.clone(), obj.clone()))
    for i in range(0, len(results), 2):
        for a, b in zip(results[i], results[i + 1]):
            assert torch.equal(a, b)
    assert not torch.equal(results[0][0], results[2][0])


def test_autotuned_sweep(d2):
    """The autotuning call cycles its fused passes through every candidate
    launch shape (all compute the same iteration) and keeps the fastest; that
    call and a later one using the kept shape both match the oracle."""
    ctx = d2.Context(0)
    K, m = 5, 32
    bags, co, mem, x0, w0 = ragged_case(16, K, m, d=8, N=200, mk=(4, 40))
    assert ctx.sweep_tuning(m) is None
    for call in range(2):
        gx, gw, gplan, gobj = run_gpu_badmm(d2, ctx, bags, co, mem, x0, w0, iters=41, tau=10,
                                            autotune=(call == 0))
        rec = ctx.sweep_tuning(m)
        assert rec is not None and 0 <= rec["chosen"] < len(rec["candidates"])
        assert len(rec["candidates"]) >= 3 and all(c["ms"] > 0 for c in rec["candidates"])
        for c in range(K):
            ids, members = cluster_members(bags, co, mem, c)
            if not ids:
                continue
            ref = oracle_badmm(members, x0[c].double().numpy(), w0[c].double().numpy(), T=41, tau=10)
            compare_cluster(bags, co, mem, c, gx, gw, gplan, gobj, ref, x_tol=x_tol(ref))
    print("autotune m=32:", rec)


@pytest.mark.parametrize("side_stream", [False, True])
def test_split_streams_equal_single_call(d2, side_stream):
    """D2_SPLIT_STREAMS runs two halves of the clusters concurrently in child
    contexts; clusters are independent in the update, so every output is
    bitwise the single call's (also on a side stream, where the children
    replay CUDA graphs, and on a second call with new data)."""
    ctx = d2.Context(0)
    K, m = 9, 16
    bags, co, mem, x0, w0 = ragged_case(17, K, m, d=8, N=240, mk=(2, 30))
    db = d2.DeviceBags.from_synth(bags)
    s = torch.cuda.Stream() if side_stream else torch.cuda.current_stream()
    outs = []
    for split in (False, True):
        for shift in (0.0, 0.25):
            with torch.cuda.stream(s):
                x, w = (x0 + shift).cuda(), w0.clone().cuda()
                plan = torch.zeros(bags.n, m, device="cuda")
                obj = torch.empty(K, dtype=torch.float64, device="cuda")
                d2.badmm_barycenter(ctx, db, co.cuda(), mem.cuda(), x, w, plan, None,
                                    d2.badmm_opts(iters=23, tau=10, split_streams=split), obj)
            s.synchronize()
            outs.append((x.cpu(), w.cpu(), plan.cpu(), obj.cpu()))
    for a, b in zip(outs[:2], outs[2:]):
        for u, v in zip(a, b):
            assert torch.equal(u, v)
    ref = oracle_badmm(cluster_members(bags, co, mem, 1)[1], x0[1].double().numpy(), w0[1].double().numpy(),
                       T=23, tau=10)
    compare_cluster(bags, co, mem, 1, *outs[2], ref, x_tol=x_tol(ref))
