"""GPU tests of the vocabulary cost table (bags stored as word indices, the
symbolic supports of Section 5), through the C ABI.

The table path builds each cluster's cost row once per distinct word and
gathers it into the j-major rows; each table row goes through the same kernel
and arithmetic as the direct build of a row with that word, and the chunk sums
for Eq. (rho) are taken in the direct build's order.  So the check here is
bitwise equality with D2_COST_ROWS (every row built directly), for the cost
matrices and for whole B-ADMM calls; the direct build itself is held to the
oracle by test_gpu_cost_tc.py, and the B-ADMM vocabulary case there now runs
through the table.
"""
import numpy as np
import pytest
import torch

import synth
from tests.helpers import run_gpu_badmm, split_clusters

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


def _case(seed, N, V, d, m, K):
    """Document bags; K clusters of which the last is empty; every fifth bag
    left out of the member list (its rows must stay untouched)."""
    bags = synth.document_bags(seed, N, V=V, d=d, mk=(1, 60))
    ids = torch.tensor([k for k in range(N) if k % 5 != 0])
    lab = ids % (K - 1)
    co, order = split_clusters(lab, K)
    mem = ids[order]
    g = torch.Generator().manual_seed(seed + 1)
    x0 = 0.2 * torch.randn(K, m, d, generator=g)
    return bags, co, mem, x0


@pytest.mark.parametrize("precision", ["bf16x3", "bf16", "bf16x6"])
@pytest.mark.parametrize("m,d,V", [(64, 300, 300), (64, 300, 5000), (32, 64, 200), (8, 48, 50), (36, 128, 1000)])
def test_vocab_table_cost_is_bitwise_the_direct_build(d2, ctx, precision, m, d, V):
    """Heavy word reuse (V = 50, 200, 300), little reuse (V = 5000), several
    K blocks (d = 128, 300), N padded to 16 (m = 36), an empty cluster and
    unlisted bags."""
    bags, co, mem, x0 = _case(60 + m + d + V, 90, V, d, m, K=4)
    db = d2.DeviceBags.from_synth(bags)
    args = (ctx, db, co.cuda(), mem.cuda(), x0.cuda())
    l0 = ctx.launch_count()
    a = d2.d2_cost(*args, C_out=torch.full((bags.n, m), -1.0, device="cuda"), precision=precision)
    l1 = ctx.launch_count()
    b = d2.d2_cost(*args, C_out=torch.full((bags.n, m), -1.0, device="cuda"), precision=precision,
                   extra_flags=d2.D2_COST_ROWS)
    l2 = ctx.launch_count()
    assert ctx.device_errors() == 0
    # the table path ran (its word-list kernels, table build and gather), except
    # where the tensor-core build does not apply: six-product pieces of d = 300
    # exceed its shared memory, the FP32 build runs and builds every row
    tc = not (precision == "bf16x6" and d == 300)
    assert (l1 - l0 > l2 - l1) if tc else (l1 - l0 == l2 - l1)
    assert torch.equal(a, b)
    listed = torch.zeros(bags.n, dtype=torch.bool)
    for k in mem.tolist():
        listed[bags.offsets[k]:bags.offsets[k + 1]] = True
    assert (a.cpu()[~listed] == -1.0).all()
    assert (a.cpu()[listed] >= 0).all()


@pytest.mark.parametrize("split", [False, True])
def test_badmm_vocab_table_is_bitwise_the_direct_build(d2, ctx, split):
    """Whole B-ADMM calls (two support updates, so the word lists of the first
    build are reused by the later ones): x, w, plans and objectives equal to
    the call that builds every row directly; also when the call is split over
    two streams (each half builds its own table)."""
    bags = synth.document_bags(61, 120, V=400, d=300, mk=(10, 60))
    K, m = 4, 64
    co, mem = split_clusters(torch.arange(bags.N) % K, K)
    x0, w0 = synth.sample_initial_barycenters(62, bags, co, mem, m)
    kw = dict(iters=25, tau=10, cost="bf16x3", split_streams=split)
    ra = run_gpu_badmm(d2, ctx, bags, co, mem, x0, w0, **kw)
    rb = run_gpu_badmm(d2, ctx, bags, co, mem, x0, w0, cost_rows=True, **kw)
    assert ctx.device_errors() == 0
    for u, v in zip(ra, rb):
        assert torch.equal(u, v)


def test_full_size_documents_update(d2, ctx):
    """The document workload at full size (200,000 bags of 10..60 words from a
    50,000-word vocabulary, d = 300, K = 64, m = 64, T = 100, tau = 10) in the
    configuration the benchmark times (split-BF16 tensor-core cost through the
    vocabulary table).  Clusters 0..3 hold 20 bags each, the other 60 share the
    rest, all in one call.  Plan marginals on every cluster (Eq. badmmc1: the
    row sums of each member's Pi2 are w), w in the simplex, and full parity
    against the FP64 oracle on the four small clusters."""
    from tests.helpers import cluster_members, oracle_clusters
    N, K, m = 200_000, 64, 64
    bags = synth.document_bags(71, N, V=50_000, d=300, mk=(10, 60), device="cuda")
    lab = torch.empty(N, dtype=torch.int64)
    small = torch.arange(80) * (N // 80)
    rest = torch.ones(N, dtype=torch.bool)
    rest[small] = False
    lab[small] = torch.arange(80) // 20
    lab[rest] = 4 + torch.arange(int(rest.sum())) % (K - 4)
    co, mem = split_clusters(lab, K)
    x0, w0 = synth.sample_initial_barycenters(72, bags, co.cuda(), mem.cuda(), m)
    db = d2.DeviceBags.from_synth(bags)
    x, w = x0.clone().cuda(), w0.clone().cuda()
    plan = torch.empty(bags.n, m, dtype=torch.float32, device="cuda")
    obj = torch.empty(K, dtype=torch.float64, device="cuda")
    d2.badmm_barycenter(ctx, db, co.cuda(), mem.cuda(), x, w, plan, None,
                        d2.badmm_opts(iters=100, tau=10, cost="bf16x3"), obj)
    torch.cuda.synchronize()
    assert ctx.device_errors() == 0
    owner = torch.repeat_interleave(torch.arange(N, device="cuda"), bags.offsets[1:] - bags.offsets[:-1])
    rows = torch.zeros(N, m, dtype=torch.float64, device="cuda").index_add_(0, owner, plan.double())
    assert torch.allclose(rows, w[lab.cuda()].double(), atol=1e-6, rtol=0)
    assert torch.allclose(w.double().sum(1), torch.ones(K, dtype=torch.float64, device="cuda"), atol=1e-6)
    assert torch.isfinite(obj).all() and (obj > 0).all()
    host = bags.to("cpu")
    jobs = []
    for c in range(4):
        _, members = cluster_members(host, co, mem, c)
        jobs.append((members, x0[c].double().cpu().numpy(), w0[c].double().cpu().numpy(), 100, 10))
    refs = oracle_clusters(jobs)
    gw, gobj, gx, gplan = w.cpu(), obj.cpu(), x.cpu(), plan
    for c, ref in enumerate(refs):
        ids, _ = cluster_members(host, co, mem, c)
        assert float(np.abs(gw[c].double().numpy() - ref["w"]).max()) <= 1e-5
        assert abs(float(gobj[c]) - ref["obj"]) <= 1e-4 * abs(ref["obj"])
        assert float(np.abs(gx[c].double().numpy() - ref["x"]).max()) <= 2e-4 * (1 + float(np.abs(ref["x"]).max()))
        for t, k in enumerate(ids):
            a, b = int(host.offsets[k]), int(host.offsets[k + 1])
            assert float(np.abs(gplan[a:b].double().cpu().numpy().T - ref["P2"][t]).max()) <= 1e-5
