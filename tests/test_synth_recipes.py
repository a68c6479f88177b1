"""The seeded input generators (synth/) follow the recipes the workloads are
stated with: determinism per seed, size ranges, weights on the simplex with
the Dirichlet moments, the Gamma sampler's moments, unit-norm vocabulary
vectors, distinct words per document with a Zipf-ordered frequency, log-uniform
member counts, and initial barycenters drawn from each cluster's own support.
CPU only."""
import math

import numpy as np
import torch

import synth


def _bag_sums(offsets, w):
    owner = torch.repeat_interleave(torch.arange(offsets.numel() - 1), offsets[1:] - offsets[:-1])
    return torch.zeros(offsets.numel() - 1, dtype=torch.float64).index_add_(0, owner, w.double())


def test_seeded_determinism():
    a = synth.gaussian_class_bags(3, 200, 4, 5)
    b = synth.gaussian_class_bags(3, 200, 4, 5)
    c = synth.gaussian_class_bags(4, 200, 4, 5)
    assert torch.equal(a.offsets, b.offsets) and torch.equal(a.supp, b.supp) and torch.equal(a.wt, b.wt)
    assert not torch.equal(a.supp[:50], c.supp[:50])


def test_circle_mixture_recipe():
    b = synth.circle_mixture_bags(1, N=400)
    sizes = b.offsets[1:] - b.offsets[:-1]
    assert int(sizes.min()) >= 4 and int(sizes.max()) <= 16
    assert torch.allclose(_bag_sums(b.offsets, b.wt), torch.ones(400, dtype=torch.float64), atol=1e-6)
    assert (b.wt > 0).all()
    ang = 2 * math.pi * torch.arange(3).double() / 3
    means = torch.stack([5 * torch.cos(ang), 5 * torch.sin(ang)], 1)
    dmin = torch.cdist(b.supp.double(), means).min(1).values
    assert float(dmin.max()) < 6.0            # every point within 6 sigma of a component mean
    assert 1.0 < float(dmin.mean()) < 1.5     # E|N(0, I_2)| = sqrt(pi / 2) ~ 1.25


def test_dirichlet_weights_and_gamma_moments():
    # two points per bag, Dirichlet(1): the first weight is Uniform(0, 1)
    b = synth.gaussian_class_bags(5, 20000, 1, 1, mk=(2, 2), alpha=1.0)
    w1 = b.wt.view(-1, 2)[:, 0].double()
    assert abs(float(w1.mean()) - 0.5) < 0.01 and abs(float(w1.var()) - 1 / 12) < 0.005
    g = torch.Generator().manual_seed(0)
    x = synth._gamma_ge1(g, torch.full((40000,), 2.5, dtype=torch.float64), "cpu")
    assert abs(float(x.mean()) - 2.5) < 0.05 and abs(float(x.var()) - 2.5) < 0.1


def test_gaussian_class_recipe():
    b = synth.gaussian_class_bags(7, 300, 8, 6, mk=(8, 32), mu_sigma=4.0)
    sizes = b.offsets[1:] - b.offsets[:-1]
    assert int(sizes.min()) >= 8 and int(sizes.max()) <= 32
    assert int(b.labels.min()) >= 0 and int(b.labels.max()) < 6
    mu = b.meta["class_means"]
    owner = torch.repeat_interleave(torch.arange(300), sizes)
    resid = b.supp.double() - mu[b.labels[owner]]
    assert abs(float(resid.std()) - 1.0) < 0.05 and float(resid.mean().abs()) < 0.05


def test_ragged_cluster_recipe():
    bags, co, mem = synth.ragged_cluster_bags(9, 3000, d=2, nc=(16, 4096), mk=(2, 4))
    ncs = (co[1:] - co[:-1]).double()
    assert int(ncs.min()) >= 16 and int(ncs.max()) <= 4096
    z = (torch.log(ncs) - math.log(16)) / (math.log(4096) - math.log(16))   # ~ U(0, 1)
    assert abs(float(z.mean()) - 0.5) < 0.03 and abs(float(z.var()) - 1 / 12) < 0.01
    assert torch.equal(mem, torch.arange(bags.N)) and torch.equal(bags.labels, torch.repeat_interleave(
        torch.arange(3000), co[1:] - co[:-1]))


def test_document_recipe():
    b = synth.document_bags(11, 500, V=2000, d=16, mk=(10, 60))
    assert torch.allclose(b.vocab.norm(dim=1), torch.ones(2000), atol=1e-5)
    sizes = b.offsets[1:] - b.offsets[:-1]
    assert int(sizes.min()) >= 10 and int(sizes.max()) <= 60
    for k in range(0, 500, 37):
        idx = b.vocab_idx[b.offsets[k]:b.offsets[k + 1]]
        assert idx.unique().numel() == idx.numel()           # distinct words
    assert torch.allclose(_bag_sums(b.offsets, b.wt), torch.ones(500, dtype=torch.float64), atol=1e-6)
    assert (b.wt > 0).all()
    freq = torch.bincount(b.vocab_idx.long(), minlength=2000)
    assert int(freq.argmax()) == 0 and freq[0] > freq[10] > freq[1000]   # Zipf ranks


def test_initial_barycenters_from_cluster_support():
    b = synth.gaussian_class_bags(13, 120, 3, 4, mk=(3, 9))
    lab = b.labels
    order = torch.sort(lab, stable=True).indices
    co = torch.zeros(5, dtype=torch.int64)
    co[1:] = torch.cumsum(torch.bincount(lab, minlength=4), 0)
    x0, w0 = synth.sample_initial_barycenters(14, b, co, order, 6)
    assert torch.allclose(w0, torch.full((4, 6), 1 / 6))
    for c in range(4):
        ids = order[int(co[c]):int(co[c + 1])]
        pts = torch.cat([b.supp[b.offsets[k]:b.offsets[k + 1]] for k in ids.tolist()])
        for i in range(6):
            assert bool((pts == x0[c, i]).all(1).any())


def test_symbolic_bags_recipe():
    """Symbolic histograms: the table is a squared-distance matrix (zero
    diagonal, symmetric, non-negative); every bag's symbols are distinct ids in
    [0, V) and its weights lie in the simplex."""
    b = synth.symbolic_bags(3, 200, V=20, n_classes=4, mk=(4, 16))
    D = b.symcost.double()
    assert D.shape == (20, 20)
    assert torch.allclose(D, D.T) and (D.diagonal() == 0).all() and (D >= 0).all()
    sizes = b.sizes()
    assert int(sizes.min()) >= 4 and int(sizes.max()) <= 16 and b.d == 1
    for k in range(b.N):
        t, w = b.symbols(k)
        assert len(set(t.tolist())) == len(t) and t.min() >= 0 and t.max() < 20
        assert abs(w.sum() - 1.0) < 1e-5 and (w >= 0).all()
