"""GPU checks of the learned pruner against the FP64 oracle (oracle/mlp.py)
and against the exact assignment.

Forward/backward take FP16-rounded inputs with FP32 accumulation, so the
embedding and the gradient blocks are compared in relative norm (2% / 5%).
With a certified-only margin (delta = inf) or r = K the pruned assignment
must equal the exact one label for label."""
import numpy as np
import pytest
import torch

import synth
from oracle import mlp, w2_exact

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


def small_problem(seed, N=40, d=6, K=5, m=4):
    bags = synth.gaussian_class_bags(seed, N, d, K, mk=(2, 12), mu_sigma=2.0, alpha=1.0)
    g = torch.Generator().manual_seed(seed + 1)
    x = (torch.randn(K, m, d, generator=g) * 2.0).float()
    w = torch.rand(K, m, generator=g) + 0.1
    w = (w / w.sum(1, keepdim=True)).float()
    return bags, x, w


def relnorm(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-12))


def test_embedding_matches_oracle(d2, ctx):
    bags, x, w = small_problem(1)
    db = d2.DeviceBags.from_synth(bags)
    p = d2.Pruner(ctx, bags.d, hidden=32, embed=16, seed=3)
    params = {k: v.double().numpy() for k, v in p.unpack(p.params()).items()}
    ids = torch.arange(bags.N, dtype=torch.int64, device="cuda")
    emb, mu = p.embed(db, ids)
    emb, mu = emb.cpu().double().numpy(), mu.cpu().double().numpy()
    for k in range(bags.N):
        y, wy = bags.bag(k)
        ref = mlp.embed(params, y, wy)
        assert relnorm(emb[k], ref) < 2e-2, k
        np.testing.assert_allclose(mu[k], wy @ y, atol=1e-5)


def test_loss_and_gradient_match_oracle(d2, ctx):
    bags, x, w = small_problem(2)
    db = d2.DeviceBags.from_synth(bags)
    p = d2.Pruner(ctx, bags.d, hidden=32, embed=16, seed=4)
    params = {k: v.double().numpy() for k, v in p.unpack(p.params()).items()}
    K = x.shape[0]
    pairs = [(a, (a * 7 + 3) % K) for a in range(0, bags.N, 2)]
    members = [bags.bag(k) for k in range(bags.N)]
    cents = [(x[q].double().numpy(), w[q].double().numpy()) for q in range(K)]
    targets = [w2_exact(cents[q][0], cents[q][1], *members[a]) for a, q in pairs]
    L, g = mlp.pair_loss_and_grad(params, members, cents, pairs, targets)
    pb = torch.tensor([a for a, _ in pairs], dtype=torch.int64, device="cuda")
    pc = torch.tensor([q for _, q in pairs], dtype=torch.int32, device="cuda")
    tg = torch.tensor(targets, dtype=torch.float32, device="cuda")
    loss, grad = p.loss_grad(db, x.cuda(), w.cuda(), pb, pc, tg)
    assert abs(float(loss) - L) <= 2e-2 * L
    gg = {k: v.double().numpy() for k, v in p.unpack(grad.cpu()).items()}
    for name in mlp.PARAM_NAMES:
        assert relnorm(gg[name], g[name]) < 5e-2, (name, relnorm(gg[name], g[name]))


def exact_labels(d2, ctx, db, x, w):
    lab, dist = d2.d2_assign(ctx, db, x.cuda(), w.cuda())
    return lab.cpu().numpy(), dist.cpu().numpy()


def test_certified_margin_and_r_equal_K_are_exact(d2, ctx):
    bags, x, w = small_problem(3, N=60, K=6)
    db = d2.DeviceBags.from_synth(bags)
    p = d2.Pruner(ctx, bags.d, hidden=32, embed=16, seed=5)
    ref_lab, ref_dist = exact_labels(d2, ctx, db, x, w)
    p.set_margin(2, 1e30)                 # only the exact mean-term bound prunes
    lab, dist, st = d2.d2_assign(ctx, db, x.cuda(), w.cuda(), prune=p, want_stats=True)
    np.testing.assert_array_equal(lab.cpu().numpy(), ref_lab)
    np.testing.assert_allclose(dist.cpu().numpy(), ref_dist, rtol=1e-6)
    assert st["exact_solves"] <= bags.N * 6 + bags.N * 2
    p.set_margin(6, 0.0)                  # r = K: every centroid is a candidate
    lab, dist, st = d2.d2_assign(ctx, db, x.cuda(), w.cuda(), prune=p, want_stats=True)
    np.testing.assert_array_equal(lab.cpu().numpy(), ref_lab)
    assert st["fallbacks"] == 0


def test_train_then_prune(d2, ctx):
    """Train on exact W^2 of every (bag, centroid) pair of a 16-class mixture,
    then assign with r = 4: the loss must fall, the misassignment rate against
    the exact assignment must stay small and fewer exact solves are needed."""
    K, m, d = 16, 8, 8
    bags = synth.gaussian_class_bags(7, 600, d, K, mk=(8, 24), mu_sigma=2.0, alpha=1.0)
    db = d2.DeviceBags.from_synth(bags)
    co = torch.zeros(K + 1, dtype=torch.int64)
    lab = bags.labels
    order = torch.sort(lab, stable=True).indices
    co[1:] = torch.cumsum(torch.bincount(lab, minlength=K), 0)
    x, w = synth.sample_initial_barycenters(8, bags, co, order, m)
    x, w = x.cuda(), w.cuda()
    N = bags.N
    pb = torch.arange(N, device="cuda").repeat_interleave(K)
    pc = torch.arange(K, device="cuda", dtype=torch.int32).repeat(N)
    perm = torch.randperm(N * K, generator=torch.Generator().manual_seed(0)).cuda()
    pb, pc = pb[perm].contiguous(), pc[perm].contiguous()
    tg = d2.d2_w2_pairs(ctx, db, x, w, pb, pc)
    p = d2.Pruner(ctx, d, hidden=64, embed=32, seed=9)
    losses = p.train(db, x, w, pb, pc, tg, steps=400, batch=256, lr=2e-3, seed=1)
    assert np.mean(losses[-20:]) < 0.3 * np.mean(losses[:20]), (losses[:5], losses[-5:])
    r_default, delta = p.margin()
    assert delta > 0
    p.set_margin(4, delta)
    ref_lab, _ = exact_labels(d2, ctx, db, x, w)
    lab, _, st = d2.d2_assign(ctx, db, x, w, prune=p, want_stats=True)
    mis = float(np.mean(lab.cpu().numpy() != ref_lab))
    assert mis <= 0.02, mis
    assert st["exact_solves"] < N * K


def test_calibrated_margin_follows_moved_centroids(d2, ctx):
    """A margin measured on the training centroids need not hold once the
    centroids move (as they do between rounds of Algorithm 1); recalibrating
    delta on exact W^2 against the moved centroids restores a small
    misassignment rate, and d2_cluster can recalibrate every round."""
    K, m, d = 12, 8, 8
    bags = synth.gaussian_class_bags(17, 800, d, K, mk=(8, 24), mu_sigma=1.5, alpha=1.0)
    db = d2.DeviceBags.from_synth(bags)
    co = torch.zeros(K + 1, dtype=torch.int64)
    lab = bags.labels
    order = torch.sort(lab, stable=True).indices
    co[1:] = torch.cumsum(torch.bincount(lab, minlength=K), 0)
    x, w = synth.sample_initial_barycenters(18, bags, co, order, m)
    x, w = x.cuda(), w.cuda()
    N = bags.N
    pb = torch.arange(N, device="cuda").repeat_interleave(K)
    pc = torch.arange(K, device="cuda", dtype=torch.int32).repeat(N)
    tg = d2.d2_w2_pairs(ctx, db, x, w, pb, pc)
    p = d2.Pruner(ctx, d, hidden=64, embed=32, seed=19)
    p.train(db, x, w, pb, pc, tg, steps=300, batch=256, lr=2e-3, seed=2)
    # move the centroids: one B-ADMM update on a perturbed clustering
    g = torch.Generator().manual_seed(3)
    lab2 = torch.where(torch.rand(N, generator=g) < 0.3, torch.randint(0, K, (N,), generator=g), lab)
    o2 = torch.sort(lab2, stable=True).indices
    co2 = torch.zeros(K + 1, dtype=torch.int64)
    co2[1:] = torch.cumsum(torch.bincount(lab2, minlength=K), 0)
    x2, w2 = x.clone(), w.clone()
    d2.badmm_barycenter(ctx, db, co2.cuda(), o2.cuda(), x2, w2, None, None, d2.badmm_opts(iters=40))
    ids = torch.arange(0, N, 4, device="cuda")
    delta = p.calibrate(db, x2, w2, ids)
    assert delta > 0
    p.set_margin(3, delta)
    ref, _ = d2.d2_assign(ctx, db, x2, w2)
    got, _, st = d2.d2_assign(ctx, db, x2, w2, prune=p, want_stats=True)
    mis = float((got != ref).float().mean())
    assert mis <= 0.01, mis
    assert st["exact_solves"] < N * K
    xc, wc, lc, oc = d2.d2_cluster(ctx, db, K, m, seed=4, rounds=3,
                                   opts=d2.badmm_opts(iters=20, recalibrate=True), prune=p)
    assert all(np.isfinite(oc))


def test_calibration_fallback_estimate_and_round_bypass(d2, ctx):
    """The calibration replays the margin test on its sample: its fall-back
    fraction matches the pruned assignment of the same bags.  On near-tie
    document bags an untrained pruner (random weights, wide delta) would send
    almost every bag to all K, so every recalibrated round of d2_cluster skips
    it: the labels are those of the exact loop and every bag of every round
    counts as a fall-back."""
    K, m, d = 10, 8, 8
    bags = synth.gaussian_class_bags(23, 600, d, K, mk=(8, 24), mu_sigma=1.5, alpha=1.0)
    db = d2.DeviceBags.from_synth(bags)
    lab = bags.labels
    order = torch.sort(lab, stable=True).indices
    co = torch.zeros(K + 1, dtype=torch.int64)
    co[1:] = torch.cumsum(torch.bincount(lab, minlength=K), 0)
    x, w = synth.sample_initial_barycenters(24, bags, co, order, m)
    x, w = x.cuda(), w.cuda()
    N = bags.N
    pb = torch.arange(N, device="cuda").repeat_interleave(K)
    pc = torch.arange(K, device="cuda", dtype=torch.int32).repeat(N)
    tg = d2.d2_w2_pairs(ctx, db, x, w, pb, pc)
    p = d2.Pruner(ctx, d, hidden=64, embed=32, seed=25)
    assert p.calibration_fallbacks() == -1.0
    p.train(db, x, w, pb, pc, tg, steps=300, batch=256, lr=2e-3, seed=2)
    p.set_margin(3, p.margin()[1])
    p.calibrate(db, x, w, torch.arange(N, device="cuda"))
    est = p.calibration_fallbacks()
    _, _, st = d2.d2_assign(ctx, db, x, w, prune=p, want_stats=True)
    assert 0.0 <= est <= 1.0
    assert abs(est - st["fallbacks"] / N) <= 0.02, (est, st["fallbacks"] / N)

    # near-tie document bags (random unit word vectors: every W^2 close to the
    # others, bag means near 0 so the mean term separates nothing)
    K, m, d = 8, 8, 16
    bags = synth.document_bags(27, 300, V=200, d=d, mk=(5, 20))
    db = d2.DeviceBags.from_synth(bags)
    N = bags.N
    rounds = 3
    xe, we, le, oe = d2.d2_cluster(ctx, db, K, m, seed=4, rounds=rounds, opts=d2.badmm_opts(iters=20))
    raw = d2.Pruner(ctx, d, hidden=64, embed=32, seed=26)
    raw.set_margin(1, 0.0)
    xr, wr, lr_, orr = d2.d2_cluster(ctx, db, K, m, seed=4, rounds=rounds,
                                     opts=d2.badmm_opts(iters=20, recalibrate=True), prune=raw)
    cs = ctx.cluster_stats()
    assert raw.calibration_fallbacks() >= 0.8 - 1.0 / K
    assert torch.equal(le, lr_)
    assert cs["fallbacks"] == N * rounds
    assert cs["exact_solves"] == N * K * rounds


def test_full_size_learned_pruning(d2, ctx):
    """The learned-pruning workload at full size: K = 256 centroids (m = 32,
    d = 32) from one B-ADMM update on 256 Gaussian classes, N = 500,000 bags of
    16..64 points; the MLP (128 hidden, 64-wide embedding) trained on 100k
    exact W^2 pairs (half the 8 nearest centroids by mean distance, half
    random); r = 8.  On 20,000 bags the pruned assignment agrees with the
    exact full-K one (misassignment <= 0.1 %) with far fewer exact solves; all
    500,000 bags are then assigned through the pruner."""
    K, m, d, r = 256, 32, 32, 8
    bags = synth.gaussian_class_bags(5, 500_000, d, K, mk=(16, 64), mu_sigma=2.0, alpha=1.0, device="cuda")
    db = d2.DeviceBags(bags.offsets, bags.wt, bags.d, supp=bags.supp)
    lab = bags.labels
    order = torch.sort(lab, stable=True).indices
    co = torch.zeros(K + 1, dtype=torch.int64, device="cuda")
    co[1:] = torch.cumsum(torch.bincount(lab, minlength=K), 0)
    x, w = synth.sample_initial_barycenters(6, bags, co, order, m)
    d2.badmm_barycenter(ctx, db, co, order.contiguous(), x, w, None, None, d2.badmm_opts(iters=100, tau=10))
    g = torch.Generator(device="cuda").manual_seed(7)
    npairs, half = 100_000, 50_000
    tb = torch.randint(0, bags.N, (npairs,), generator=g, device="cuda")
    owner = torch.repeat_interleave(torch.arange(bags.N, device="cuda"), bags.offsets[1:] - bags.offsets[:-1])
    mu_b = torch.zeros(bags.N, d, device="cuda").index_add_(0, owner, bags.supp * bags.wt[:, None])
    mu_c = (w[:, :, None] * x).sum(1)
    near = torch.cdist(mu_b[tb[:half]], mu_c).topk(8, largest=False).indices
    pick = torch.randint(0, 8, (half,), generator=g, device="cuda")
    pc = torch.empty(npairs, dtype=torch.int32, device="cuda")
    pc[:half] = near.gather(1, pick[:, None]).squeeze(1).to(torch.int32)
    pc[half:] = torch.randint(0, K, (npairs - half,), generator=g, device="cuda", dtype=torch.int32)
    tg = d2.d2_w2_pairs(ctx, db, x, w, tb.contiguous(), pc.contiguous())
    pr = d2.Pruner(ctx, d, hidden=128, embed=64, seed=8)
    pr.train(db, x, w, tb.contiguous(), pc.contiguous(), tg, steps=1500, batch=1024, lr=1e-3, seed=9)
    pr.set_margin(r, pr.margin()[1])
    ev = 20_000
    sub = synth.subset_bags(bags, torch.arange(ev, device="cuda"))
    dsub = d2.DeviceBags(sub.offsets, sub.wt, sub.d, supp=sub.supp)
    le, de = d2.d2_assign(ctx, dsub, x, w)
    lp, dp, st = d2.d2_assign(ctx, dsub, x, w, prune=pr, want_stats=True)
    assert ctx.device_errors() == 0
    mis = float((lp != le).float().mean())
    print("full-size pruning: misassignment %.2e, exact solves %d of %d, fall-backs %d"
          % (mis, st["exact_solves"], ev * K, st["fallbacks"]))
    assert mis <= 1e-3
    assert st["exact_solves"] <= ev * K // 10
    la, da, sa = d2.d2_assign(ctx, db, x, w, prune=pr, want_stats=True)
    assert torch.equal(la[:ev], lp)
    assert sa["exact_solves"] <= bags.N * K // 10


def test_loss_and_gradient_elementwise(d2, ctx):
    """Element-wise check of the embedding, the loss and every gradient entry.
    Parameters and support points are made FP16-representable first, so the
    only differences from the FP64 oracle are the kernels' FP16 roundings of
    intermediate values (centred points, first hidden layer, pooled vector;
    each 2^-11 relative) and FP32 accumulation: every entry must lie within
    3e-3 of its block's largest entry.  The same check must reject an oracle
    gradient that leaves out one pair's centroid-side contribution."""
    bags, x, w = small_problem(12, N=48, d=8, K=6, m=5)
    bags.supp = bags.supp.half().float()
    x = x.half().float()
    db = d2.DeviceBags.from_synth(bags)
    p = d2.Pruner(ctx, bags.d, hidden=32, embed=16, seed=13)
    p.set_params(p.params().half().float())
    params = {k: v.double().numpy() for k, v in p.unpack(p.params()).items()}
    members = [bags.bag(k) for k in range(bags.N)]
    K = x.shape[0]
    cents = [(x[q].double().numpy(), w[q].double().numpy()) for q in range(K)]
    # embeddings
    ids = torch.arange(bags.N, dtype=torch.int64, device="cuda")
    emb, _ = p.embed(db, ids)
    emb = emb.cpu().double().numpy()
    ref_emb = np.array([mlp.embed(params, *members[k]) for k in range(bags.N)])
    scale = np.abs(ref_emb).max()
    emb_err = float(np.abs(emb - ref_emb).max() / scale)
    assert emb_err <= 3e-3, emb_err
    # loss and gradient over 24 pairs
    pairs = [(a, (a * 5 + 1) % K) for a in range(0, bags.N, 2)]
    targets = [w2_exact(cents[q][0], cents[q][1], *members[a]) for a, q in pairs]
    L, g = mlp.pair_loss_and_grad(params, members, cents, pairs, targets)
    pb = torch.tensor([a for a, _ in pairs], dtype=torch.int64, device="cuda")
    pc = torch.tensor([q for _, q in pairs], dtype=torch.int32, device="cuda")
    tg = torch.tensor(targets, dtype=torch.float32, device="cuda")
    loss, grad = p.loss_grad(db, x.cuda(), w.cuda(), pb, pc, tg)
    assert abs(float(loss) - L) <= 3e-3 * L, (float(loss), L)
    gg = {k: v.double().numpy() for k, v in p.unpack(grad.cpu()).items()}
    worst = {}
    for name in mlp.PARAM_NAMES:
        tol = 3e-3 * np.abs(g[name]).max()
        err = np.abs(gg[name] - g[name])
        worst[name] = float(err.max() / np.abs(g[name]).max())
        assert (err <= tol).all(), (name, worst[name])
    # power: drop the centroid-side term of the first pair from the oracle
    a0, q0 = pairs[0]
    fa = mlp.embed(params, *members[a0])
    fq, cache = mlp.embed(params, *cents[q0], want_cache=True)
    mu2 = float(np.sum((mlp.mean_of(*members[a0]) - mlp.mean_of(*cents[q0])) ** 2))
    res = float((fa - fq) @ (fa - fq)) - (targets[0] - mu2)
    gq = mlp.embed_backward(params, cache, -(2.0 * res / len(pairs)) * 2.0 * (fa - fq))
    caught = [name for name in mlp.PARAM_NAMES
              if (np.abs((g[name] - gq[name]) - g[name]) > 3e-3 * np.abs(g[name]).max()).any()]
    assert caught, "the element-wise check cannot see a missing pair term"
    print("MLP element-wise: embedding %.2e, gradient blocks %s (relative to the block max)"
          % (emb_err, {k: "%.1e" % v for k, v in worst.items()}))


@pytest.mark.parametrize("d,H,E", [(8, 32, 16), (64, 128, 64), (100, 64, 32)])
def test_tensor_core_forward_matches_cuda_core_forward(d2, ctx, d, H, E):
    """Layers 1 and 2 as tcgen05 GEMMs (FP16 operands, FP32 accumulation in
    tensor memory, points of many slots packed into 128-row tiles and pooled
    per slot) and the weight-gradient contractions as tcgen05 GEMMs on
    MN-major split-BF16 operands, against the CUDA-core forward and backward:
    the same products up to the split's 2^-16, other addition orders, so the
    means are bitwise equal and the embeddings, loss and gradients agree to
    FP16 rounding of the first hidden layer."""
    bags = synth.gaussian_class_bags(70 + d, 300, d, 5, mk=(2, 60), mu_sigma=2.0, alpha=1.0)
    db = d2.DeviceBags.from_synth(bags)
    g = torch.Generator().manual_seed(d)
    K, m = 7, 12
    x = (torch.randn(K, m, d, generator=g) * 2.0).float().cuda()
    w = torch.rand(K, m, generator=g) + 0.1
    w = (w / w.sum(1, keepdim=True)).float().cuda()
    p = d2.Pruner(ctx, d, hidden=H, embed=E, seed=d + H)
    ids = torch.arange(bags.N, dtype=torch.int64, device="cuda")
    pb = torch.arange(0, bags.N, 3, dtype=torch.int64, device="cuda")
    pc = (pb % K).to(torch.int32)
    tg = torch.rand(pb.numel(), generator=g).float().cuda() * 10.0
    out = {}
    for path in ("auto", "cuda_cores"):
        ctx.set_prune_forward(path)
        emb, mu = p.embed(db, ids)
        loss, grad = p.loss_grad(db, x, w, pb, pc, tg)
        torch.cuda.synchronize()
        out[path] = (emb.cpu().double(), mu.cpu(), float(loss), grad.cpu().double())
    ctx.set_prune_forward("auto")
    (e1, m1, l1, g1), (e2, m2, l2, g2) = out["auto"], out["cuda_cores"]
    assert torch.equal(m1, m2)
    emb_err = float((e1 - e2).abs().max() / e2.abs().max())
    assert emb_err <= 3e-3, emb_err
    assert abs(l1 - l2) <= 3e-3 * abs(l2), (l1, l2)
    gerr = float((g1 - g2).abs().max() / g2.abs().max())
    assert gerr <= 1e-2, gerr
    assert ctx.device_errors() == 0
    print("tensor-core forward d=%d H=%d: embedding %.1e, loss %.1e, gradient %.1e (of the max)"
          % (d, H, emb_err, abs(l1 - l2) / abs(l2), gerr))
    with pytest.raises(d2.D2Error) as e:
        ctx.check(d2.lib().d2_set_prune_forward(ctx.h, 2))
    assert e.value.code == d2.D2_EINVAL
