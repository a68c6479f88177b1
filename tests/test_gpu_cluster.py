"""GPU parity of the exact assignment (Eq. primal + argmin of Algorithm 1),
the merge initialisation (Eq. merge) and the D2-clustering loop against the
FP64 oracle.  W^2 values within 1e-4 relative; labels bit-exact wherever the
gap between the two smallest W^2 exceeds 1e-4 of the smallest."""
import numpy as np
import pytest
import torch

import synth
from oracle import w2_exact, merge_reduce, d2_cluster as oracle_cluster, init_pick
from tests.test_oracle_cluster_mlp import lloyd_on_means

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


def centroids(seed, K, m, d, scale=2.0):
    g = torch.Generator().manual_seed(seed)
    x = torch.randn(K, m, d, generator=g) * scale
    w = torch.rand(K, m, generator=g) + 0.05
    w = (w / w.sum(1, keepdim=True)).float()
    return x.float(), w


def gpu_w2_matrix(d2, ctx, db, x, w):
    cols = []
    for c in range(x.shape[0]):
        _, dist = d2.d2_assign(ctx, db, x[c:c + 1].cuda().contiguous(), w[c:c + 1].cuda().contiguous())
        cols.append(dist.cpu().double())
    return torch.stack(cols, 1).numpy()


@pytest.mark.parametrize("case", ["d5_m6", "d2_m1", "d16_m16", "d1_m4", "d32_m32"])
def test_w2_values_match_exact_lp(d2, ctx, case):
    d, m = {"d5_m6": (5, 6), "d2_m1": (2, 1), "d16_m16": (16, 16), "d1_m4": (1, 4), "d32_m32": (32, 32)}[case]
    bags = synth.gaussian_class_bags(40 + m, 24, d, 3, mk=(1, 40), mu_sigma=2.0)
    db = d2.DeviceBags.from_synth(bags)
    x, w = centroids(m + d, 3, m, d)
    G = gpu_w2_matrix(d2, ctx, db, x, w)
    for k in range(bags.N):
        y, wy = bags.bag(k)
        for c in range(3):
            ref = w2_exact(x[c].double().numpy(), w[c].double().numpy(), y, wy)
            assert abs(G[k, c] - ref) <= 1e-4 * ref + 1e-6, (k, c, G[k, c], ref)


def test_w2_zero_for_identical_distribution(d2, ctx):
    bags = synth.gaussian_class_bags(3, 5, 3, 1, mk=(4, 4))
    db = d2.DeviceBags.from_synth(bags)
    y, wy = bags.bag(2)
    x = torch.tensor(y, dtype=torch.float32)[None]
    w = torch.tensor(wy, dtype=torch.float32)[None]
    _, dist = d2.d2_assign(ctx, db, x.cuda(), w.cuda())
    assert abs(float(dist[2])) < 1e-6


def test_labels_match_oracle_where_margin_is_clear(d2, ctx):
    bags = synth.gaussian_class_bags(9, 60, 4, 4, mk=(2, 12), mu_sigma=2.5)
    db = d2.DeviceBags.from_synth(bags)
    x, w = centroids(10, 4, 5, 4, scale=2.5)
    labels, dist, st = d2.d2_assign(ctx, db, x.cuda(), w.cuda(), want_stats=True)
    labels, dist = labels.cpu().numpy(), dist.cpu().double().numpy()
    assert st["exact_solves"] == 60 * 4 and st["limit_hits"] == 0
    for k in range(bags.N):
        y, wy = bags.bag(k)
        D = np.array([w2_exact(x[c].double().numpy(), w[c].double().numpy(), y, wy) for c in range(4)])
        order = np.argsort(D, kind="stable")
        best = D[order[0]]
        assert abs(dist[k] - best) <= 1e-4 * best + 1e-6
        if D[order[1]] - best > 1e-4 * best:
            assert labels[k] == order[0]


def test_merge_init_matches_oracle(d2, ctx):
    bags = synth.gaussian_class_bags(12, 30, 3, 2, mk=(1, 20))
    db = d2.DeviceBags.from_synth(bags)
    ids = torch.arange(0, 30, 3, dtype=torch.int64)
    for m in (1, 4, 9):
        x, w = d2.d2_merge_init(ctx, db, ids.cuda(), m)
        x, w = x.cpu().double().numpy(), w.cpu().double().numpy()
        for t, k in enumerate(ids.tolist()):
            y, wy = bags.bag(k)
            rx, rw = merge_reduce(y, wy, m)
            q = rx.shape[0]
            np.testing.assert_allclose(x[t, :q], rx, atol=1e-5, rtol=0)
            np.testing.assert_allclose(w[t, :q], rw, atol=1e-6, rtol=0)
            if q < m:  # padding: zero-weight copies of the last point
                assert np.all(w[t, q:] == 0)


def test_d2_cluster_matches_oracle(d2, ctx):
    bags = synth.gaussian_class_bags(31, 90, 4, 3, mk=(4, 10), mu_sigma=4.0, alpha=1.0)
    db = d2.DeviceBags.from_synth(bags)
    K, m, rounds, T = 3, 4, 3, 20
    x, w, labels, objs = d2.d2_cluster(ctx, db, K, m, seed=77, rounds=rounds,
                                       opts=d2.badmm_opts(iters=T, tau=10))
    members = [bags.bag(k) for k in range(bags.N)]
    ref = oracle_cluster(members, K, m, seed=77, rounds=rounds, T=T, tau=10)
    np.testing.assert_array_equal(labels.cpu().numpy(), ref["labels"])
    for r in range(rounds):
        assert abs(objs[r] - ref["obj_per_round"][r]) <= 1e-4 * ref["obj_per_round"][r]
    np.testing.assert_allclose(w.cpu().double().numpy(), ref["w"], atol=1e-5, rtol=0)
    np.testing.assert_allclose(x.cpu().double().numpy(), ref["x"], atol=2e-4 * (1 + np.abs(ref["x"]).max()))


def test_d2_cluster_with_m_above_every_bag(d2, ctx):
    """m larger than every m_k (the document workload has m = 64 > 60): the
    largest bags seed the centroids, padded with zero-weight copies."""
    bags = synth.gaussian_class_bags(33, 60, 3, 3, mk=(2, 7), mu_sigma=4.0, alpha=1.0)
    db = d2.DeviceBags.from_synth(bags)
    K, m, rounds, T = 3, 9, 2, 15
    x, w, labels, objs = d2.d2_cluster(ctx, db, K, m, seed=78, rounds=rounds,
                                       opts=d2.badmm_opts(iters=T, tau=10))
    members = [bags.bag(k) for k in range(bags.N)]
    ref = oracle_cluster(members, K, m, seed=78, rounds=rounds, T=T, tau=10)
    np.testing.assert_array_equal(labels.cpu().numpy(), ref["labels"])
    for r in range(rounds):
        assert abs(objs[r] - ref["obj_per_round"][r]) <= 1e-4 * ref["obj_per_round"][r]
    np.testing.assert_allclose(w.cpu().double().numpy(), ref["w"], atol=1e-5, rtol=0)


def test_d2_cluster_m1_is_kmeans_on_means(d2, ctx):
    bags = synth.gaussian_class_bags(32, 120, 3, 4, mk=(1, 8), mu_sigma=3.0)
    db = d2.DeviceBags.from_synth(bags)
    K, rounds = 4, 4
    x, w, labels, objs = d2.d2_cluster(ctx, db, K, 1, seed=5, rounds=rounds, opts=d2.badmm_opts(iters=12, tau=10))
    means = np.array([wy @ y for y, wy in (bags.bag(k) for k in range(bags.N))])
    picks = init_pick(bags.sizes().tolist(), K, 1, 5)
    labels_ref, cent = lloyd_on_means(means, means[picks], rounds)
    np.testing.assert_array_equal(labels.cpu().numpy(), labels_ref[-1])
    np.testing.assert_allclose(x.cpu().double().numpy()[:, 0, :], cent, atol=1e-4)
    assert np.allclose(w.cpu().numpy(), 1.0)


def test_elkan_skipping_matches_exact_clustering(d2, ctx):
    """Triangle-inequality skipping (Section 5) changes which pairs are solved,
    never the labels or the per-round objective."""
    bags = synth.gaussian_class_bags(41, 400, 4, 6, mk=(4, 16), mu_sigma=3.0, alpha=1.0)
    db = d2.DeviceBags.from_synth(bags)
    K, m, rounds = 6, 5, 5
    x1, w1, l1, o1 = d2.d2_cluster(ctx, db, K, m, seed=3, rounds=rounds, opts=d2.badmm_opts(iters=30))
    full = ctx.cluster_stats()
    x2, w2, l2, o2 = d2.d2_cluster(ctx, db, K, m, seed=3, rounds=rounds, opts=d2.badmm_opts(iters=30, elkan=True))
    skip = ctx.cluster_stats()
    np.testing.assert_array_equal(l1.cpu().numpy(), l2.cpu().numpy())
    np.testing.assert_allclose(o2, o1, rtol=1e-6)
    assert torch.equal(x1, x2) and torch.equal(w1, w2)
    assert full["exact_solves"] == bags.N * K * rounds
    assert skip["exact_solves"] < full["exact_solves"]


@pytest.mark.parametrize("case", ["dense", "vocab", "m_above"])
def test_bounded_assignment_equals_full_exact(d2, ctx, case):
    """d2_assign_bounded skips every LP whose certified lower bound exceeds the
    best value found; its labels and distances equal the full N x K solve."""
    if case == "dense":
        bags = synth.gaussian_class_bags(61, 300, 16, 6, mk=(4, 40), mu_sigma=2.0)
        K, m = 12, 16
    elif case == "vocab":
        bags = synth.document_bags(62, 200, V=300, d=48, mk=(8, 60))
        K, m = 10, 24
    else:
        bags = synth.gaussian_class_bags(63, 150, 8, 4, mk=(2, 9), mu_sigma=3.0)
        K, m = 7, 12
    db = d2.DeviceBags.from_synth(bags)
    g = torch.Generator().manual_seed(5)
    ids = torch.randperm(bags.N, generator=g)[:K].cuda()
    x, w = d2.d2_merge_init(ctx, db, ids, m)
    lf, df_, sf = d2.d2_assign(ctx, db, x, w, want_stats=True)
    lb, db_, sb = d2.d2_assign(ctx, db, x, w, want_stats=True, bounded=True)
    assert torch.equal(lf, lb)
    assert torch.equal(df_, db_)
    assert sf["exact_solves"] == bags.N * K
    assert sb["exact_solves"] < sf["exact_solves"]
    print("%s: bounded solves %d of %d" % (case, sb["exact_solves"], sf["exact_solves"]))


@pytest.mark.parametrize("case", ["docs64", "docs32_long"])
def test_entropic_dual_bound_keeps_the_exact_argmin(d2, ctx, case):
    """The entropic dual bound (Sinkhorn potentials made feasible by a
    c-transform, a lower bound of the LP of Eq. primal) excludes more pairs
    than the cheap bounds and leaves the labels and distances of the full
    N x K solve unchanged; merge-initialised centroids carry zero-weight
    padding points, which the bound must handle."""
    if case == "docs64":
        bags = synth.document_bags(81, 400, V=3000, d=300, mk=(10, 60))
        K, m = 16, 64
    else:
        bags = synth.document_bags(82, 300, V=2000, d=64, mk=(40, 120))
        K, m = 12, 32
    db = d2.DeviceBags.from_synth(bags)
    g = torch.Generator().manual_seed(6)
    ids = torch.randperm(bags.N, generator=g)[:K].cuda()
    x, w = d2.d2_merge_init(ctx, db, ids, m)
    lf, df_, sf = d2.d2_assign(ctx, db, x, w, want_stats=True)
    ctx.set_dual_bound(0)
    l0, d0, s0 = d2.d2_assign(ctx, db, x, w, want_stats=True, bounded=True)
    ctx.set_dual_bound(-1)
    l1, d1, s1 = d2.d2_assign(ctx, db, x, w, want_stats=True, bounded=True)
    ctx.set_dual_bound(60, 0.02)
    l2, d2_, s2 = d2.d2_assign(ctx, db, x, w, want_stats=True, bounded=True)
    ctx.set_dual_bound(-1)
    for lab, dist in ((l0, d0), (l1, d1), (l2, d2_)):
        assert torch.equal(lf, lab)
        assert torch.equal(df_, dist)
    assert s1["exact_solves"] < s0["exact_solves"] < sf["exact_solves"]
    assert s2["exact_solves"] < s0["exact_solves"]
    print("%s: exact solves full %d, cheap bounds %d, dual bound %d (60 iterations, eps 0.02: %d)"
          % (case, sf["exact_solves"], s0["exact_solves"], s1["exact_solves"], s2["exact_solves"]))
    for bad in ((-2, 0.0), (10001, 0.0), (5, -1.0), (5, float("nan"))):
        with pytest.raises(d2.D2Error) as e:
            ctx.set_dual_bound(*bad)
        assert e.value.code == d2.D2_EINVAL


@pytest.mark.parametrize("case", ["docs300_m64", "gauss64_m32", "gauss96_m16"])
def test_tensor_core_bounds_keep_the_exact_argmin(d2, ctx, case):
    """The cheap bounds with their cost entries on the tensor cores (split
    BF16, each bound lowered by the products' error bound) exclude as many
    LPs as the CUDA-core bounds, up to that margin, and the labels and
    distances stay those of the full N x K solve."""
    if case == "docs300_m64":
        bags = synth.document_bags(91, 500, V=4000, d=300, mk=(10, 60))
        K, m = 20, 64
    elif case == "gauss64_m32":
        bags = synth.gaussian_class_bags(92, 600, 64, 12, mk=(4, 64), mu_sigma=1.0)
        K, m = 12, 32
    else:
        bags = synth.gaussian_class_bags(93, 400, 96, 9, mk=(2, 40), mu_sigma=0.7)
        K, m = 9, 16
    db = d2.DeviceBags.from_synth(bags)
    g = torch.Generator().manual_seed(7)
    ids = torch.randperm(bags.N, generator=g)[:K].cuda()
    x, w = d2.d2_merge_init(ctx, db, ids, m)
    lf, df_, sf = d2.d2_assign(ctx, db, x, w, want_stats=True)
    out = {}
    for path in ("cuda_cores", "auto"):
        ctx.set_bound_kernels(path)
        for dual in (0, -1):
            ctx.set_dual_bound(dual)
            lab, dist, st = d2.d2_assign(ctx, db, x, w, want_stats=True, bounded=True)
            assert torch.equal(lf, lab), (path, dual)
            assert torch.equal(df_, dist), (path, dual)
            out[path, dual] = st["exact_solves"]
    ctx.set_bound_kernels("auto")
    ctx.set_dual_bound(-1)
    assert ctx.device_errors() == 0
    for dual in (0, -1):
        assert out["auto", dual] <= 1.02 * out["cuda_cores", dual] + 2, out
        assert out["auto", dual] < sf["exact_solves"]
    print("%s: exact solves full %d; cheap bounds CUDA cores %d, tensor cores %d; with the dual bound %d, %d"
          % (case, sf["exact_solves"], out["cuda_cores", 0], out["auto", 0], out["cuda_cores", -1],
             out["auto", -1]))
    with pytest.raises(d2.D2Error) as e:
        ctx.check(d2.lib().d2_set_bound_kernels(ctx.h, 2))
    assert e.value.code == d2.D2_EINVAL


def test_bounded_assignment_with_pruner_candidates(d2, ctx):
    bags = synth.gaussian_class_bags(64, 400, 8, 5, mk=(4, 30), mu_sigma=2.5)
    db = d2.DeviceBags.from_synth(bags)
    K, m = 8, 8
    x, w = d2.d2_merge_init(ctx, db, torch.arange(K, device="cuda") * 7, m)
    pr = d2.Pruner(ctx, 8, hidden=32, embed=16, seed=1)
    pr.set_margin(3, 0.0)
    lf, df_ = d2.d2_assign(ctx, db, x, w)
    lb, db_, st = d2.d2_assign(ctx, db, x, w, prune=pr, want_stats=True, bounded=True)
    assert torch.equal(lf, lb) and torch.equal(df_, db_)
    assert st["exact_solves"] < bags.N * K


def test_d2_cluster_bounded_assignment_matches_exact(d2, ctx):
    bags = synth.gaussian_class_bags(65, 240, 6, 4, mk=(4, 20), mu_sigma=3.0)
    db = d2.DeviceBags.from_synth(bags)
    K, m, rounds = 4, 6, 3
    a = d2.d2_cluster(ctx, db, K, m, seed=9, rounds=rounds, opts=d2.badmm_opts(iters=20))
    b = d2.d2_cluster(ctx, db, K, m, seed=9, rounds=rounds, opts=d2.badmm_opts(iters=20, assign_bounded=True))
    assert torch.equal(a[2], b[2])
    assert a[3] == b[3]
    assert ctx.cluster_stats()["exact_solves"] < bags.N * K * rounds


def test_d2_cluster_with_split_streams_and_tensor_core_cost(d2, ctx):
    """The clustering loop with every update as a split call on the
    split-BF16 tensor-core cost build: labels and objectives per round equal
    those of one-stream updates (clusters are independent in the update)."""
    bags = synth.gaussian_class_bags(66, 300, 32, 5, mk=(8, 30), mu_sigma=2.0)
    db = d2.DeviceBags.from_synth(bags)
    K, m, rounds = 5, 8, 3
    a = d2.d2_cluster(ctx, db, K, m, seed=12, rounds=rounds, opts=d2.badmm_opts(iters=20, cost="bf16x3"))
    b = d2.d2_cluster(ctx, db, K, m, seed=12, rounds=rounds,
                      opts=d2.badmm_opts(iters=20, cost="bf16x3", split_streams=True))
    assert torch.equal(a[2], b[2])
    assert a[3] == b[3]
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


@pytest.fixture(scope="module")
def doc_shape_case():
    """Bags of the document workload's shape (d = 300 unit word vectors from a
    50,000-word vocabulary, m_k ~ U{10..60} distinct Zipf words) against
    m = 64 centroids: the solver then collects 8 deficit sinks per
    shortest-path pass (m >= 64 and m + m_k > 64).  Two centroid sets, both
    computed by the oracle: padded seeds (Eq. merge; m_k < 64, so zero-weight
    copies) and the barycenters after one B-ADMM update of 12-bag clusters."""
    from oracle import badmm_barycenter
    from oracle.cluster import pad_support
    bags = synth.document_bags(71, 48, V=50_000, d=300, mk=(10, 60))
    K, m = 4, 64
    seeds = [pad_support(*merge_reduce(*bags.bag(k), m), m) for k in (3, 17, 29, 41)]
    upd = []
    for c in range(K):
        members = [bags.bag(k) for k in range(c * 12, (c + 1) * 12)]
        r = badmm_barycenter(members, seeds[c][0], seeds[c][1], T=50, tau=10)
        upd.append((r["x"], r["w"]))
    sets = {}
    for name, cents in (("merge", seeds), ("updated", upd)):
        x = torch.tensor(np.array([c[0] for c in cents]), dtype=torch.float32)
        w = torch.tensor(np.array([c[1] for c in cents]), dtype=torch.float32)
        w = w / w.sum(1, keepdim=True)
        ref = np.array([[w2_exact(x[c].double().numpy(), w[c].double().numpy(), *bags.bag(k))
                         for c in range(K)] for k in range(bags.N)])
        sets[name] = (x, w, ref)
    return bags, sets


@pytest.mark.parametrize("centroids", ["merge", "updated"])
def test_w2_document_shape_eight_sinks(d2, ctx, doc_shape_case, centroids):
    bags, sets = doc_shape_case
    x, w, ref = sets[centroids]
    db = d2.DeviceBags.from_synth(bags)
    K = x.shape[0]
    pb = torch.arange(bags.N, dtype=torch.int64).repeat_interleave(K).cuda()
    pc = torch.arange(K, dtype=torch.int32).repeat(bags.N).cuda()
    vals = d2.d2_w2_pairs(ctx, db, x.cuda(), w.cuda(), pb, pc).cpu().double().numpy().reshape(bags.N, K)
    np.testing.assert_array_less(np.abs(vals - ref), 1e-4 * ref + 1e-6)
    labels, dist, st = d2.d2_assign(ctx, db, x.cuda(), w.cuda(), want_stats=True)
    assert st["limit_hits"] == 0
    labels, dist = labels.cpu().numpy(), dist.cpu().double().numpy()
    clear = 0
    for k in range(bags.N):
        order = np.argsort(ref[k], kind="stable")
        best = ref[k, order[0]]
        assert abs(dist[k] - best) <= 1e-4 * best + 1e-6
        if ref[k, order[1]] - best > 1e-4 * best:
            assert labels[k] == order[0]
            clear += 1
    assert clear >= bags.N // 2
    print("document shape (%s centroids): max rel W^2 err %.2e, %d of %d labels with a clear margin"
          % (centroids, float(np.max(np.abs(vals - ref) / np.maximum(ref, 1e-6))), clear, bags.N))


def test_elkan_clustering_matches_oracle(d2, ctx):
    """Triangle-inequality skipping (Section 5) inside the clustering loop:
    labels and per-round objectives against the FP64 oracle's Algorithm 1 (which
    solves every pair), and fewer exact solves than the full loop."""
    bags = synth.gaussian_class_bags(42, 160, 4, 5, mk=(4, 12), mu_sigma=3.0, alpha=1.0)
    db = d2.DeviceBags.from_synth(bags)
    K, m, rounds, T = 5, 5, 4, 20
    x, w, labels, objs = d2.d2_cluster(ctx, db, K, m, seed=21, rounds=rounds,
                                       opts=d2.badmm_opts(iters=T, tau=10, elkan=True))
    solves = ctx.cluster_stats()["exact_solves"]
    members = [bags.bag(k) for k in range(bags.N)]
    ref = oracle_cluster(members, K, m, seed=21, rounds=rounds, T=T, tau=10)
    np.testing.assert_array_equal(labels.cpu().numpy(), ref["labels"])
    for r in range(rounds):
        assert abs(objs[r] - ref["obj_per_round"][r]) <= 1e-4 * ref["obj_per_round"][r]
    np.testing.assert_allclose(w.cpu().double().numpy(), ref["w"], atol=1e-5, rtol=0)
    np.testing.assert_allclose(x.cpu().double().numpy(), ref["x"], atol=2e-4 * (1 + np.abs(ref["x"]).max()))
    assert solves < bags.N * K * rounds
    print("Elkan: %d exact solves of %d" % (solves, bags.N * K * rounds))


def test_phase_cap_is_reported_as_enoconv(d2):
    """A solve that reaches its phase cap returns the cost of an unfinished
    flow; every path that runs the exact solver must say so (D2_ENOCONV)
    rather than hand back a silently wrong W^2 or label.  The cap is lowered
    on a context of its own so that solves stop early, without any fault."""
    bags = synth.gaussian_class_bags(81, 120, 4, 3, mk=(8, 20), mu_sigma=2.0)
    db = d2.DeviceBags.from_synth(bags)
    x, w = centroids(82, 3, 8, 4)
    x, w = x.cuda(), w.cuda()
    c = d2.Context(0)
    ref_lab, ref_dist = d2.d2_assign(c, db, x, w)
    assert c.device_errors() == 0
    c.set_phase_limit(1)
    with pytest.raises(d2.D2Error) as e:
        d2.d2_assign(c, db, x, w, want_stats=True)
    assert e.value.code == d2.D2_ENOCONV
    with pytest.raises(d2.D2Error) as e:
        d2.d2_assign(c, db, x, w, want_stats=True, bounded=True)
    assert e.value.code == d2.D2_ENOCONV
    with pytest.raises(d2.D2Error) as e:
        c.device_errors()
    assert e.value.code == d2.D2_ENOCONV
    # asynchronous calls leave the sticky bit for d2_device_errors
    d2.d2_assign(c, db, x, w)
    pb = torch.arange(bags.N, dtype=torch.int64, device="cuda")
    d2.d2_w2_pairs(c, db, x, w, pb, torch.zeros(bags.N, dtype=torch.int32, device="cuda"))
    with pytest.raises(d2.D2Error) as e:
        c.device_errors()
    assert e.value.code == d2.D2_ENOCONV
    assert c.device_errors() == 0                      # read and cleared
    with pytest.raises(d2.D2Error) as e:
        d2.d2_cluster(c, db, 3, 8, seed=1, rounds=2, opts=d2.badmm_opts(iters=5))
    assert e.value.code == d2.D2_ENOCONV
    with pytest.raises(d2.D2Error):
        c.device_errors()
    # the default cap again: the same context gives the reference result
    c.set_phase_limit(0)
    lab, dist, st = d2.d2_assign(c, db, x, w, want_stats=True)
    assert st["limit_hits"] == 0 and c.device_errors() == 0
    assert torch.equal(lab, ref_lab) and torch.equal(dist, ref_dist)


@pytest.mark.parametrize("case", ["d16_m16", "d300_m64_vocab", "d32_m32", "d4_m5"])
def test_sparse_and_dense_flow_stores_agree(d2, case):
    """The exact solver's two flow stores run the same arithmetic: W^2 of every
    pair equal up to the order of the final FP64 sum; a sparse pool capped so
    that most pairs overflow hands them to the dense re-solve with the same
    result; and against the exact LP on a sample."""
    if case == "d300_m64_vocab":
        bags = synth.document_bags(91, 60, V=4000, d=300, mk=(10, 60))
        x, w = centroids(92, 3, 64, 300, scale=0.08)
    else:
        d, m = {"d16_m16": (16, 16), "d32_m32": (32, 32), "d4_m5": (4, 5)}[case]
        bags = synth.gaussian_class_bags(93 + m, 120, d, 4, mk=(1, 60), mu_sigma=2.0)
        x, w = centroids(94 + m, 4, m, d)
    db = d2.DeviceBags.from_synth(bags)
    x, w = x.cuda(), w.cuda()
    K = x.shape[0]
    pb = torch.arange(bags.N, dtype=torch.int64).repeat_interleave(K).cuda()
    pc = torch.arange(K, dtype=torch.int32).repeat(bags.N).cuda()
    c = d2.Context(0)
    vals = {}
    for store, cap in (("dense", 0), ("sparse", 0), ("sparse", 4), ("auto", 0)):
        c.set_flow_store(store, cap)
        vals[(store, cap)] = d2.d2_w2_pairs(c, db, x, w, pb, pc).cpu().double().numpy()
        assert c.device_errors() == 0
    ref = vals[("dense", 0)]
    for key, v in vals.items():
        np.testing.assert_allclose(v, ref, rtol=2e-7, atol=1e-12, err_msg=str(key))
    for t in range(0, bags.N * K, max(1, bags.N * K // 24)):
        k, ci = t // K, t % K
        e = w2_exact(x[ci].double().cpu().numpy(), w[ci].double().cpu().numpy(), *bags.bag(k))
        assert abs(ref[t] - e) <= 1e-4 * e + 1e-6, (t, ref[t], e)
    # the assignment through both stores gives the same labels
    c.set_flow_store("dense")
    ld, dd = d2.d2_assign(c, db, x, w)
    c.set_flow_store("sparse")
    ls, ds = d2.d2_assign(c, db, x, w)
    assert torch.equal(ld, ls)
    np.testing.assert_allclose(ds.cpu().numpy(), dd.cpu().numpy(), rtol=2e-7)


def test_overflow_list_beyond_capacity_reports_enoconv(d2):
    """More overflowed pairs than the re-solve list holds (65,536): the ones
    beyond it are reported (D2_ENOCONV), never returned silently."""
    bags = synth.gaussian_class_bags(95, 2400, 3, 4, mk=(4, 12), mu_sigma=2.0)
    db = d2.DeviceBags.from_synth(bags)
    x, w = centroids(96, 32, 4, 3)
    c = d2.Context(0)
    c.set_flow_store("sparse", 1)   # one pool entry: every pair with more than one flow overflows
    with pytest.raises(d2.D2Error) as e:
        d2.d2_assign(c, db, x.cuda(), w.cuda(), want_stats=True)
    assert e.value.code == d2.D2_ENOCONV
    with pytest.raises(d2.D2Error) as e:     # the sticky bit, read and cleared
        c.device_errors()
    assert e.value.code == d2.D2_ENOCONV
    c.set_flow_store("auto")
    _, _, st = d2.d2_assign(c, db, x.cuda(), w.cuda(), want_stats=True)
    assert st["limit_hits"] == 0 and c.device_errors() == 0
