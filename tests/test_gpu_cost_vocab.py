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
