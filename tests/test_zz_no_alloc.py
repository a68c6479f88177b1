"""The no-allocation assignment entry point (d2_assign_noalloc).

It exists for callers that may not allocate device memory (a process whose
device memory belongs to another framework's fixed pool, or a service that
must not allocate after start-up).  Its scratch is a fixed device array
shared by every call, so this checks two calls in a row, each against the
regular d2_assign on the same inputs, and the rejection of a problem larger
than the array.  Collected last on purpose; it creates its own state and
also passes when run alone in a fresh process."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def d2():
    import paper_1510_00012_gb300 as d2mod
    from paper_1510_00012_gb300 import build
    build.build()
    return d2mod


def problem(seed, N, K, m, d):
    bags = synth.gaussian_class_bags(seed, N, d, K, mk=(1, 24), mu_sigma=2.0, alpha=1.0)
    g = torch.Generator().manual_seed(seed + 1)
    x = (torch.randn(K, m, d, generator=g) * 2.0).float()
    w = torch.rand(K, m, generator=g) + 0.05
    w = (w / w.sum(1, keepdim=True)).float()
    return bags, x.cuda(), w.cuda()


def test_two_calls_match_the_regular_assignment(d2):
    ctx = d2.Context(0)
    for seed, N, K, m, d in ((1, 300, 7, 8, 5), (2, 150, 12, 16, 16)):
        bags, x, w = problem(seed, N, K, m, d)
        db = d2.DeviceBags.from_synth(bags)
        lab, dist = d2.d2_assign_noalloc(db, x, w)
        ref_lab, ref_dist = d2.d2_assign(ctx, db, x, w)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(lab.cpu().numpy(), ref_lab.cpu().numpy())
        np.testing.assert_allclose(dist.cpu().numpy(), ref_dist.cpu().numpy(), rtol=1e-4, atol=1e-6)


def test_rejects_problems_beyond_the_scratch(d2):
    bags, _, _ = problem(3, 1100, 2, 4, 3)
    db = d2.DeviceBags.from_synth(bags)
    K = d2.D2_NOALLOC_MAX_PAIRS // bags.N + 1
    x = torch.zeros(K, 4, 3, device="cuda")
    w = torch.full((K, 4), 0.25, device="cuda")
    with pytest.raises(d2.D2Error) as e:
        d2.d2_assign_noalloc(db, x, w)
    assert e.value.code == d2.D2_ESCRATCH


def test_rejects_unsupported_and_invalid_shapes(d2):
    """Both rejections happen on the host before any kernel runs: 32 ceil(m/32)
    + max_mk above the solver's 256 node slots (D2_ENOTSUP), and bags with neither a
    support matrix nor a vocabulary (D2_EINVAL)."""
    bags, _, _ = problem(4, 40, 1, 4, 3)
    db = d2.DeviceBags.from_synth(bags)
    m = 32 * ((257 - db.max_mk + 31) // 32)  # smallest multiple of 32 past the limit
    x = torch.zeros(1, m, 3, device="cuda")
    w = torch.full((1, m), 1.0 / m, device="cuda")
    with pytest.raises(d2.D2Error) as e:
        d2.d2_assign_noalloc(db, x, w)
    assert e.value.code == d2.D2_ENOTSUP
    bare = d2.DeviceBags(db.offsets, db.wt, db.d, supp=None, max_mk=db.max_mk)
    x = torch.zeros(1, 4, 3, device="cuda")
    w = torch.full((1, 4), 0.25, device="cuda")
    with pytest.raises(d2.D2Error) as e:
        d2.d2_assign_noalloc(bare, x, w)
    assert e.value.code == d2.D2_EINVAL
