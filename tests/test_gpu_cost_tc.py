"""GPU parity of the tensor-core cost build (tcgen05, BF16 operands with FP32
accumulation and FP32 norms) and of B-ADMM run on it, through the C ABI,
against the FP64 oracle on the same seeded inputs.

Cost bounds follow from the arithmetic.  On coordinates centred at mu (the
mean of the cluster's barycenter points) the build computes
||xt||^2 + ||yt||^2 - 2 <xt, yt> with FP32 norms; only the cross term sees
the operand rounding.  A BF16 factor carries a relative error <= u = 2^-8,
so each product is off by <= 2u |x_d y_d| and, by Cauchy-Schwarz, the cost by
<= 4u ||xt|| ||yt||.  Split operands (hi + lo) leave <= about 4 u^2 per
product, so the x3 bound is 8 u^2 ||xt|| ||yt||; three pieces represent an
FP32 factor exactly and the dropped products (mid*lo, lo*mid, lo*lo) are
<= 2 u^3 per product, a cost bound of 4 u^3 ||xt|| ||yt||.  All add the FP32
rounding of the norms and the accumulation, 2e-5 (1 + C).

B-ADMM parity uses the tolerances of the FP32 path: plan entries and w within
1e-5 absolute, the objective within 1e-4 relative.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import badmm_barycenter as oracle_badmm, cost_matrix
from tests.helpers import cluster_members, compare_cluster, member_plan, run_gpu_badmm, split_clusters

pytestmark = pytest.mark.gpu

U_BF16 = 2.0 ** -8


@pytest.fixture(scope="module")
def d2():
    import paper_1510_00012_gb300 as d2mod
    from paper_1510_00012_gb300 import build
    build.build()
    return d2mod


@pytest.fixture(scope="module")
def ctx(d2):
    return d2.Context(0)


def _cost_case(seed, m, d, vocab=False, N=40, K=3):
    if vocab:
        bags = synth.document_bags(seed, N, V=500, d=d, mk=(1, 60))
        lab = torch.arange(bags.N) % K
    else:
        bags = synth.gaussian_class_bags(seed, N, d, K, mk=(1, 70), mu_sigma=4.0)
        lab = bags.labels
    co, mem = split_clusters(lab, K)
    x0, _ = synth.sample_initial_barycenters(seed + 1, bags, co, mem, m)
    return bags, co, mem, x0 + 3.0  # off-centre barycenters


def _check_cost(d2, ctx, bags, co, mem, x0, precision):
    K = x0.shape[0]
    db = d2.DeviceBags.from_synth(bags)
    C = d2.d2_cost(ctx, db, co.cuda(), mem.cuda(), x0.cuda(), precision=precision).cpu()
    assert ctx.device_errors() == 0
    worst = 0.0
    for c in range(K):
        ids, members = cluster_members(bags, co, mem, c)
        xc = x0[c].double().numpy()
        mu = xc.mean(0)
        xn = np.linalg.norm(xc - mu, axis=1)
        for k, (y, _) in zip(ids, members):
            ref = cost_matrix(xc, y)
            got = member_plan(C, bags.offsets, k)
            yn = np.linalg.norm(y - mu, axis=1)
            factor = {"bf16": 4 * U_BF16, "bf16x3": 8 * U_BF16 ** 2, "bf16x6": 4 * U_BF16 ** 3}[precision]
            scale = factor * np.outer(xn, yn)
            bound = scale + 2e-5 * (1 + ref)
            err = np.abs(got - ref)
            worst = max(worst, float((err / bound).max()))
            assert (err <= bound).all(), (c, k, float(err.max()))
    print("cost %s: worst error / bound = %.3f" % (precision, worst))
    return worst


@pytest.mark.parametrize("precision", ["bf16x3", "bf16", "bf16x6"])
def test_cost_tc_small(d2, ctx, precision):
    """One K block (d = 64), m = 32: the launch shape of the benchmark."""
    bags, co, mem, x0 = _cost_case(40, 32, 64)
    _check_cost(d2, ctx, bags, co, mem, x0, precision)


@pytest.mark.parametrize("precision", ["bf16x3", "bf16", "bf16x6"])
@pytest.mark.parametrize("m,d,vocab", [(16, 32, False), (8, 48, False), (36, 128, False), (100, 64, False),
                                       (64, 300, True), (256, 64, False), (4, 96, False)])
def test_cost_tc_shapes(d2, ctx, precision, m, d, vocab):
    """Several K blocks (double-buffered A), N padded to 16, TMEM widths 32..256,
    K padding (d = 300, 48, 96), vocabulary gathers, rows in ragged tails."""
    bags, co, mem, x0 = _cost_case(41 + m + d, m, d, vocab=vocab)
    _check_cost(d2, ctx, bags, co, mem, x0, precision)


def test_cost_tc_falls_back_below_d32(d2, ctx):
    """d < 32 is not a dense contraction worth the tensor cores: the flag is
    accepted and the FP32 build runs (same bytes as the default)."""
    bags, co, mem, x0 = _cost_case(42, 16, 16)
    db = d2.DeviceBags.from_synth(bags)
    a = d2.d2_cost(ctx, db, co.cuda(), mem.cuda(), x0.cuda(), precision="bf16")
    b = d2.d2_cost(ctx, db, co.cuda(), mem.cuda(), x0.cuda(), precision="fp32")
    assert torch.equal(a, b)


def _errors(bags, co, mem, c, gx, gw, gplan, gobj, ref):
    ids, _ = cluster_members(bags, co, mem, c)
    ew = float(np.abs(gw[c].double().numpy() - ref["w"]).max())
    ep = max(float(np.abs(member_plan(gplan, bags.offsets, k) - ref["P2"][t]).max()) for t, k in enumerate(ids))
    eo = abs(float(gobj[c]) - ref["obj"])
    ex = float(np.abs(gx[c].double().numpy() - ref["x"]).max()) / (1.0 + float(np.abs(ref["x"]).max()))
    return ew, ep, eo, ex


# Per-mode tolerances on plan entries and w.  FP32 and the split modes are
# held to the FP32 path's 1e-5; a single BF16 product moves each cost by up to
# 4u ||xt|| ||yt|| and the plans follow exp(-C/rho), so that mode is held to
# 1e-4 and its error is reported.
PLAN_TOL = {"fp32": 1e-5, "bf16x6": 1e-5, "bf16x3": 1e-5, "bf16": 1e-4}
COST_FACTOR = {"fp32": 0.0, "bf16x6": 4 * U_BF16 ** 3, "bf16x3": 8 * U_BF16 ** 2, "bf16": 4 * U_BF16}


def _obj_bound(members, xfin, precision, obj):
    """Objective tolerance: 1e-4 relative, or the largest cost-error bound over
    the final support when that is larger: the objective is a plan-weighted
    mean of costs, each off by at most that bound.  The operand term is the
    cost test's; 2^-17 (||xt||^2 + ||yt||^2) covers the FP32 norms and the
    FP32 (CUDA-core or tensor-core) accumulation of the expanded form.  The
    second case is a cluster whose barycenter reproduces its members (an
    objective near 0), where the expanded form's cancellation dominates in
    every precision, FP32 included."""
    mu = xfin.mean(0)
    xn = np.linalg.norm(xfin - mu, axis=1).max()
    yn = max(np.linalg.norm(y - mu, axis=1).max() for y, _ in members)
    arith = COST_FACTOR[precision] * xn * yn + 2.0 ** -17 * (xn * xn + yn * yn) + 2e-5
    return max(1e-4 * abs(obj), arith)


def _check_badmm(bags, co, mem, x0, w0, gx, gw, gplan, gobj, precision, T, tau):
    worst = np.zeros(4)
    for c in range(x0.shape[0]):
        ids, members = cluster_members(bags, co, mem, c)
        if not ids:
            continue
        ref = oracle_badmm(members, x0[c].double().numpy(), w0[c].double().numpy(), T=T, tau=tau)
        e = _errors(bags, co, mem, c, gx, gw, gplan, gobj, ref)
        ob = _obj_bound(members, ref["x"], precision, ref["obj"])
        print("%s cluster %d (%d members, obj %.3e): w %.2e plan %.2e obj %.2e (bound %.2e) x %.2e"
              % (precision, c, len(ids), ref["obj"], e[0], e[1], e[2], ob, e[3]))
        assert e[0] <= PLAN_TOL[precision] and e[1] <= PLAN_TOL[precision], (c, e)
        assert e[2] <= ob, (c, e[2], ob)
        assert e[3] <= 2e-4 * (10 if precision == "bf16" else 1), (c, e[3])
        worst = np.maximum(worst, e)
    print("%s worst: w %.2e plan %.2e obj %.2e x %.2e" % (precision, *worst))


@pytest.mark.parametrize("precision", ["fp32", "bf16x6", "bf16x3", "bf16"])
def test_badmm_on_tensor_core_cost(d2, ctx, precision):
    """Ragged clusters in d = 64 with a single-member and an empty cluster;
    m = 32, 31 iterations (three support updates, each followed by a rebuild)."""
    K, m = 6, 32
    bags = synth.gaussian_class_bags(43, 120, 64, K - 2, mk=(1, 40))
    lab = bags.labels.clone()
    lab[0] = K - 2
    co, mem = split_clusters(lab, K)
    x0, w0 = synth.sample_initial_barycenters(44, bags, co, mem, m)
    gx, gw, gplan, gobj = run_gpu_badmm(d2, ctx, bags, co, mem, x0, w0, iters=31, tau=10, cost=precision)
    assert ctx.device_errors() == 0
    _check_badmm(bags, co, mem, x0, w0, gx, gw, gplan, gobj, precision, 31, 10)


@pytest.mark.parametrize("precision", ["fp32", "bf16x3", "bf16"])
def test_badmm_tensor_core_vocabulary(d2, ctx, precision):
    """Document-like bags (d = 300 word vectors by index), m = 64."""
    bags = synth.document_bags(45, 60, V=400, d=300, mk=(10, 60))
    K, m = 3, 64
    co, mem = split_clusters(torch.arange(bags.N) % K, K)
    x0, w0 = synth.sample_initial_barycenters(46, bags, co, mem, m)
    gx, gw, gplan, gobj = run_gpu_badmm(d2, ctx, bags, co, mem, x0, w0, iters=25, tau=10, cost=precision)
    assert ctx.device_errors() == 0
    _check_badmm(bags, co, mem, x0, w0, gx, gw, gplan, gobj, precision, 25, 10)


@pytest.mark.parametrize("d", [64, 128])
def test_bounded_wait_expiry_is_reported(d2, ctx, d):
    """The build's only device-side wait (its MMA completion) is bounded: with
    the testing flag the first tile's MMAs are not issued, the wait expires
    after about 2 s, the CTA stops and frees its tensor memory, and the host
    reads D2_ETIMEOUT; the context stays usable for the next call.  d = 64
    has one K block per tile (single A buffer), d = 128 two (double-buffered)."""
    bags = synth.gaussian_class_bags(47, 6, d, 1, mk=(4, 16))
    co, mem = split_clusters(torch.zeros(bags.N, dtype=torch.int64), 1)
    x0, _ = synth.sample_initial_barycenters(48, bags, co, mem, 32)
    db = d2.DeviceBags.from_synth(bags)
    assert ctx.device_errors() == 0
    d2.d2_cost(ctx, db, co.cuda(), mem.cuda(), x0.cuda(), precision="bf16x3",
               extra_flags=d2.D2_TEST_EXPIRE_WAIT)
    with pytest.raises(d2.D2Error) as e:
        ctx.device_errors()
    assert e.value.code == d2.D2_ETIMEOUT
    assert ctx.device_errors() == 0  # cleared by the read
    _check_cost(d2, ctx, bags, co, mem, x0, "bf16x3")


@pytest.mark.parametrize("d,m", [(32, 128), (124, 8), (64, 20), (48, 64)])
def test_badmm_tensor_core_cost_shapes(d2, ctx, d, m):
    """B-ADMM on the split-BF16 cost build across plan widths and support
    dimensions: N padded to 16 (m = 20), TMEM widths up to 128 columns,
    several K blocks per tile (d = 124), several tiles per chunk."""
    K = 3
    bags = synth.gaussian_class_bags(70 + d + m, 60, d, K, mk=(1, 70), mu_sigma=3.0)
    co, mem = split_clusters(bags.labels, K)
    x0, w0 = synth.sample_initial_barycenters(71, bags, co, mem, m)
    gx, gw, gplan, gobj = run_gpu_badmm(d2, ctx, bags, co, mem, x0, w0, iters=21, tau=10, cost="bf16x3")
    assert ctx.device_errors() == 0
    _check_badmm(bags, co, mem, x0, w0, gx, gw, gplan, gobj, "bf16x3", 21, 10)


@pytest.mark.parametrize("case", ["d64_m32_x3", "d300_m64_vocab_x3", "d124_m20_x3", "d32_m64_x6", "d64_m32_bf16"])
def test_badmm_tensor_core_support_update(d2, ctx, case):
    """The opt-in tensor-core support update (Eq. updatex as tcgen05 MMAs on
    split-BF16 pieces of the centred support and the plan): plans, w, the
    objective and x against the FP64 oracle with the tolerances of the
    split-BF16 cost build; several row tiles per chunk, support dimensions in
    several 64-wide blocks with a ragged last block (d = 124, 300), N padded
    to 16 (m = 20), three pieces (x6), and single-product BF16 costs (the
    support update then still uses two pieces)."""
    prec = {"d64_m32_x3": "bf16x3", "d300_m64_vocab_x3": "bf16x3", "d124_m20_x3": "bf16x3",
            "d32_m64_x6": "bf16x6", "d64_m32_bf16": "bf16"}[case]
    if case == "d300_m64_vocab_x3":
        bags = synth.document_bags(47, 80, V=500, d=300, mk=(10, 60))
        K, m = 3, 64
        co, mem = split_clusters(torch.arange(bags.N) % K, K)
    else:
        d, m = {"d64_m32_x3": (64, 32), "d124_m20_x3": (124, 20), "d32_m64_x6": (32, 64),
                "d64_m32_bf16": (64, 32)}[case]
        K = 4
        bags = synth.gaussian_class_bags(48 + d + m, 140, d, K, mk=(1, 64), mu_sigma=3.0)
        co, mem = split_clusters(bags.labels, K)
    x0, w0 = synth.sample_initial_barycenters(49, bags, co, mem, m)
    gx, gw, gplan, gobj = run_gpu_badmm(d2, ctx, bags, co, mem, x0, w0, iters=31, tau=10, cost=prec,
                                        support_tc=True)
    assert ctx.device_errors() == 0
    _check_badmm(bags, co, mem, x0, w0, gx, gw, gplan, gobj, prec, 31, 10)
