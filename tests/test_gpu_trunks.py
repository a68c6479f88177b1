"""Member-parallel trunks (the parallel implementation of Section 5) on one
GPU: the members of every cluster are split over two "processes" -- two host
threads, each with its own context and stream -- whose exact fixed-point
sums are combined by a host reducer between them.  The update must be bitwise
the update of one context holding every member: x, w and the objective of
every cluster, and the plan rows of every member.  The threads meet only on
the host (a barrier with a timeout); no kernel waits for another."""
import threading

import pytest
import torch

import synth
from paper_1510_00012_gb300.trunks import _CudaInt64View, trunk_split

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def d2():
    import paper_1510_00012_gb300 as d2mod
    from paper_1510_00012_gb300 import build
    build.build()
    return d2mod


class ThreadReducer:
    """Sums / maxima of the same int64 buffer of every thread, in place."""

    def __init__(self, n):
        self.n = n
        self.bar = threading.Barrier(n, timeout=120)
        self.bufs = [None] * n
        self.calls = [0] * n

    def for_rank(self, r):
        def fn(op, ptr, count, stream):
            torch.cuda.synchronize()  # the library's work so far, on every stream
            t = torch.as_tensor(_CudaInt64View(ptr, count), device="cuda")
            self.bufs[r] = t.clone()
            torch.cuda.synchronize()
            self.bar.wait()
            tot = self.bufs[0].clone()
            for b in self.bufs[1:]:
                tot = tot + b if op == 0 else torch.maximum(tot, b)
            t.copy_(tot)
            torch.cuda.synchronize()
            self.calls[r] += 1
            self.bar.wait()  # nobody replaces its buffer before every thread has read
            return 0
        return fn


@pytest.mark.parametrize("cost,rule", [("fp32", "R1"), ("bf16x3", "R2")])
def test_two_trunks_equal_one_process(d2, cost, rule):
    K, m, T = 12, 32, 31
    bags, co, mem = synth.ragged_cluster_bags(21, K, d=64, nc=(40, 400), mk=(16, 64), device="cpu")
    x0, w0 = synth.sample_initial_barycenters(22, bags, co, mem, m)
    db = d2.DeviceBags.from_synth(bags)
    opts = dict(iters=T, tau=10, cost=cost, rule=rule, graph=False)
    # one context, every member
    ctx = d2.Context(0)
    x1, w1 = x0.clone().cuda(), w0.clone().cuda()
    plan1 = torch.zeros(bags.n, m, device="cuda")
    obj1 = torch.empty(K, dtype=torch.float64, device="cuda")
    d2.badmm_barycenter(ctx, db, co.cuda(), mem.cuda(), x1, w1, plan1, None, d2.badmm_opts(**opts), obj1)
    torch.cuda.synchronize()
    # two trunks in two threads
    world = 2
    red = ThreadReducer(world)
    outs = [None] * world
    errs = []

    def run(r):
        try:
            c = d2.Context(0)
            c.set_reducer(red.for_rank(r))
            lco, lmem = trunk_split(co, mem, r, world)
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                x, w = x0.clone().cuda(), w0.clone().cuda()
                plan = torch.zeros(bags.n, m, device="cuda")
                obj = torch.empty(K, dtype=torch.float64, device="cuda")
                d2.badmm_barycenter(c, db, lco.cuda(), lmem.cuda(), x, w, plan, None, d2.badmm_opts(**opts), obj)
            s.synchronize()
            outs[r] = (x.cpu(), w.cpu(), plan.cpu(), obj.cpu(), lmem)
            c.close()
        except Exception as e:  # reported below; the barrier timeout frees the other thread
            errs.append(repr(e))
            red.bar.abort()

    th = [threading.Thread(target=run, args=(r,)) for r in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=300)
    assert not errs, errs
    assert red.calls[0] == red.calls[1] > T  # one consensus per iteration at least
    p1 = plan1.cpu()
    for r in range(world):
        x, w, plan, obj, lmem = outs[r]
        assert torch.equal(x, x1.cpu()), r
        assert torch.equal(w, w1.cpu()), r
        assert torch.equal(obj, obj1.cpu()), r
        rows = torch.cat([torch.arange(int(bags.offsets[k]), int(bags.offsets[k + 1])) for k in lmem.tolist()])
        assert torch.equal(plan[rows], p1[rows]), r
    print("two trunks (%s, %s): %d reducer calls per thread, bitwise equal to one context"
          % (cost, rule, red.calls[0]))
