"""GPU parity of the symbolic-support path (Sections 2 and 5: a given
symbol-to-symbol dissimilarity, fixed centroid symbols) against the FP64
oracle: cost rows bit for bit (a gather of the table), B-ADMM plans and w
within 1e-5 and the objective within 1e-4 relative, exact W^2 within 1e-4
relative with labels bit-exact where the margin is clear, and the clustering
loop round by round."""
import numpy as np
import pytest
import torch

import synth
from oracle.symbolic import badmm_sym, d2_cluster_sym as oracle_cluster_sym, sym_cost, w2_sym
from tests.helpers import split_clusters

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


def csym_for(K, m, V, seed):
    g = torch.Generator().manual_seed(seed)
    return torch.stack([torch.randperm(V, generator=g)[:m] for _ in range(K)]).to(torch.int32)


def test_sym_cost_is_the_table(d2, ctx):
    bags = synth.symbolic_bags(1, 90, V=30, mk=(3, 20))
    db = d2.DeviceBags.from_synth(bags)
    K, m = 4, 9
    co, mem = split_clusters(bags.labels, K)
    cs = csym_for(K, m, 30, 2)
    C = d2.d2_sym_cost(ctx, db, co.cuda(), mem.cuda(), cs.cuda()).cpu().numpy()
    D = bags.symcost.numpy()
    lab = bags.labels.numpy()
    for k in range(bags.N):
        t, _ = bags.symbols(k)
        a, b = int(bags.offsets[k]), int(bags.offsets[k + 1])
        np.testing.assert_array_equal(C[a:b].T, sym_cost(D, cs[lab[k]].numpy(), t).astype(np.float32))


@pytest.mark.parametrize("rule", ["R1", "R2"])
def test_badmm_sym_matches_oracle(d2, ctx, rule):
    bags = synth.symbolic_bags(3, 160, V=20, n_classes=4, mk=(2, 16))
    db = d2.DeviceBags.from_synth(bags)
    K, m = 5, 12
    lab = bags.labels.clone()
    lab[0] = K - 1   # a single-member cluster (class ids are 0..3)
    co, mem = split_clusters(lab, K)
    cs = csym_for(K, m, 20, 4)
    w0 = torch.full((K, m), 1.0 / m)
    w, plan, obj = d2.badmm_barycenter_sym(ctx, db, co.cuda(), mem.cuda(), cs.cuda(), w0.clone().cuda(),
                                           opts=d2.badmm_opts(iters=60, tau=10, rule=rule))
    torch.cuda.synchronize()
    w, plan, obj = w.cpu(), plan.cpu(), obj.cpu()
    D = bags.symcost.numpy()
    memc = mem.tolist()
    worst = np.zeros(3)
    for c in range(K):
        ids = memc[int(co[c]):int(co[c + 1])]
        ref = badmm_sym(D, [bags.symbols(k) for k in ids], cs[c].numpy(), w0[c].double().numpy(), T=60, tau=10,
                        rule=rule)
        ew = float(np.abs(w[c].double().numpy() - ref["w"]).max())
        ep = 0.0
        for t, k in enumerate(ids):
            a, b = int(bags.offsets[k]), int(bags.offsets[k + 1])
            ep = max(ep, float(np.abs(plan[a:b].double().numpy().T - ref["P2"][t]).max()))
        eo = abs(float(obj[c]) - ref["obj"]) / ref["obj"]
        worst = np.maximum(worst, [ew, ep, eo])
    print("symbolic B-ADMM %s: max |w| err %.2e, |plan| err %.2e, rel obj err %.2e" % (rule, *worst))
    assert worst[0] <= 1e-5 and worst[1] <= 1e-5 and worst[2] <= 1e-4


def test_assign_sym_matches_exact_lp(d2, ctx):
    bags = synth.symbolic_bags(5, 70, V=25, mk=(2, 20))
    db = d2.DeviceBags.from_synth(bags)
    K, m = 4, 10
    cs = csym_for(K, m, 25, 6)
    g = torch.Generator().manual_seed(7)
    w = torch.rand(K, m, generator=g) + 0.05
    w = (w / w.sum(1, keepdim=True)).float()
    labels, dist, st = d2.d2_assign_sym(ctx, db, cs.cuda(), w.cuda(), want_stats=True)
    assert st["limit_hits"] == 0 and st["exact_solves"] == bags.N * K
    labels, dist = labels.cpu().numpy(), dist.cpu().double().numpy()
    D = bags.symcost.numpy()
    for k in range(bags.N):
        vals = np.array([w2_sym(D, cs[c].numpy(), w[c].double().numpy(), *bags.symbols(k)) for c in range(K)])
        order = np.argsort(vals, kind="stable")
        assert abs(dist[k] - vals[order[0]]) <= 1e-4 * vals[order[0]] + 1e-6
        if vals[order[1]] - vals[order[0]] > 1e-4 * vals[order[0]]:
            assert labels[k] == order[0]


def test_cluster_sym_matches_oracle(d2, ctx):
    bags = synth.symbolic_bags(8, 120, V=20, n_classes=3, mk=(3, 14))
    db = d2.DeviceBags.from_synth(bags)
    K, rounds, T = 3, 3, 25
    sym = torch.arange(0, 20, 2, dtype=torch.int32)
    w, labels, objs = d2.d2_cluster_sym(ctx, db, K, sym.cuda(), seed=11, rounds=rounds,
                                        opts=d2.badmm_opts(iters=T, tau=10))
    ref = oracle_cluster_sym(bags.symcost.numpy(), [bags.symbols(k) for k in range(bags.N)], K, sym.numpy(),
                             seed=11, rounds=rounds, T=T, tau=10)
    np.testing.assert_array_equal(labels.cpu().numpy(), ref["labels"])
    for r in range(rounds):
        assert abs(objs[r] - ref["obj_per_round"][r]) <= 1e-4 * ref["obj_per_round"][r]
    np.testing.assert_allclose(w.cpu().double().numpy(), ref["w"], atol=1e-5, rtol=0)
    print("symbolic clustering: objective per round", objs)


def test_symbolic_and_coordinate_entry_points_reject_each_other(d2, ctx):
    sb = synth.symbolic_bags(9, 20, V=10, mk=(2, 6))
    dsb = d2.DeviceBags.from_synth(sb)
    cb = synth.gaussian_class_bags(9, 20, 3, 2, mk=(2, 6))
    dcb = d2.DeviceBags.from_synth(cb)
    x = torch.zeros(2, 4, 3, device="cuda")
    w = torch.full((2, 4), 0.25, device="cuda")
    cs = torch.zeros(2, 4, dtype=torch.int32, device="cuda")
    with pytest.raises(d2.D2Error) as e:
        d2.d2_assign(ctx, dsb, x, w)
    assert e.value.code == d2.D2_EINVAL
    with pytest.raises(d2.D2Error) as e:
        d2.d2_assign_sym(ctx, dcb, cs, w)
    assert e.value.code == d2.D2_EINVAL
    with pytest.raises(d2.D2Error) as e:
        d2.d2_assign_noalloc(dsb, x, w)
    assert e.value.code == d2.D2_EINVAL
