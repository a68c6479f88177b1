"""Seeded synthetic discrete distributions shaped like the paper's workloads.

This module is the ONE thing the CUDA path and the FP64 oracle share: it only
draws random inputs (support points, weights, ragged sizes, initial centroids)
and holds none of the method's arithmetic (no costs, plans, barycenters or
transport).  Every generator takes a seed and a torch device; the same seed on
the same device and torch build gives the same arrays.  Parity tests draw the
inputs once and hand the SAME arrays to both sides, so CPU/CUDA RNG streams
never need to agree with each other.

Layout of a set of distributions ("bags"), the paper's notation in Section 2:
  * bag k has m_k support points y_j^(k) in R^d and weights w^(k) in the
    simplex;  n = sum_k m_k;
  * ``offsets`` (int64, N+1): rows offsets[k] .. offsets[k+1]-1 belong to bag k;
  * ``supp`` (float32, n x d, row-major) the stacked support points X^T, or
    ``vocab_idx`` (int32, n) into a ``vocab`` table (float32, V x d) for
    symbolic / grid supports stored as indices (Section 5, last paragraph);
  * ``wt`` (float32, n) the stacked weights.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import torch


@dataclass
class Bags:
    offsets: torch.Tensor            # int64 (N+1)
    wt: torch.Tensor                 # float32 (n)
    d: int
    supp: Optional[torch.Tensor] = None       # float32 (n, d)
    vocab_idx: Optional[torch.Tensor] = None  # int32 (n)
    vocab: Optional[torch.Tensor] = None      # float32 (V, d)
    labels: Optional[torch.Tensor] = None     # int64 (N) ground-truth class
    meta: dict = field(default_factory=dict)
    symcost: Optional[torch.Tensor] = None    # float32 (V, V): symbolic bags (vocab_idx = symbols)

    @property
    def N(self) -> int:
        return int(self.offsets.numel() - 1)

    @property
    def n(self) -> int:
        return int(self.wt.numel())

    def sizes(self) -> torch.Tensor:
        return self.offsets[1:] - self.offsets[:-1]

    def to(self, device) -> "Bags":
        mv = lambda t: None if t is None else t.to(device)
        return Bags(mv(self.offsets), mv(self.wt), self.d, mv(self.supp),
                    mv(self.vocab_idx), mv(self.vocab), mv(self.labels), dict(self.meta), mv(self.symcost))

    def symbols(self, k: int):
        """(symbol ids (int64 numpy), weights (float64 numpy)) of symbolic bag k."""
        a, b = int(self.offsets[k]), int(self.offsets[k + 1])
        return (self.vocab_idx[a:b].detach().cpu().long().numpy(),
                self.wt[a:b].detach().cpu().double().numpy())

    def points(self) -> torch.Tensor:
        """(n, d) support points, gathering from the vocabulary if needed."""
        if self.supp is not None:
            return self.supp
        return self.vocab[self.vocab_idx.long()]

    def bag(self, k: int):
        """(y, w) of bag k as float64 numpy arrays (m_k x d, m_k)."""
        a, b = int(self.offsets[k]), int(self.offsets[k + 1])
        if self.supp is not None:
            y = self.supp[a:b]
        else:
            y = self.vocab[self.vocab_idx[a:b].long()]
        return (y.detach().cpu().double().numpy(),
                self.wt[a:b].detach().cpu().double().numpy())


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def _ragged(sizes: torch.Tensor) -> torch.Tensor:
    off = torch.zeros(sizes.numel() + 1, dtype=torch.int64, device=sizes.device)
    off[1:] = torch.cumsum(sizes.to(torch.int64), 0)
    return off


def _row_owner(offsets: torch.Tensor) -> torch.Tensor:
    sizes = offsets[1:] - offsets[:-1]
    return torch.repeat_interleave(torch.arange(sizes.numel(), device=offsets.device), sizes)


def _dirichlet_rows(g, offsets, alpha: float, device) -> torch.Tensor:
    """Per-bag Dirichlet(alpha) weights: Gamma(alpha) draws normalised per bag."""
    n = int(offsets[-1])
    conc = torch.full((n,), float(alpha), dtype=torch.float64, device=device)
    # torch._standard_gamma has no generator argument; draw through a
    # Dirichlet-free route that does: Gamma(a) = Gamma(a+1) * U^(1/a).
    gam1 = _gamma_ge1(g, conc + 1.0, device)
    u = torch.rand(n, generator=g, dtype=torch.float64, device=device).clamp_min(1e-300)
    gam = gam1 * u.pow(1.0 / conc)
    owner = _row_owner(offsets)
    tot = torch.zeros(offsets.numel() - 1, dtype=torch.float64, device=device)
    tot.index_add_(0, owner, gam)
    w = (gam / tot[owner]).to(torch.float32)
    return w


def _gamma_ge1(g, a: torch.Tensor, device) -> torch.Tensor:
    """Marsaglia-Tsang Gamma(a) sampler for a >= 1 (ACM TOMS 26(3), 2000)."""
    d = a - 1.0 / 3.0
    c = 1.0 / torch.sqrt(9.0 * d)
    out = torch.empty_like(a)
    todo = torch.arange(a.numel(), device=device)
    while todo.numel() > 0:
        dd, cc = d[todo], c[todo]
        z = torch.randn(todo.numel(), generator=g, dtype=torch.float64, device=device)
        u = torch.rand(todo.numel(), generator=g, dtype=torch.float64, device=device)
        v = (1.0 + cc * z) ** 3
        ok = (v > 0) & (torch.log(u.clamp_min(1e-300)) < 0.5 * z * z + dd - dd * v + dd * torch.log(v.clamp_min(1e-300)))
        out[todo[ok]] = (dd * v)[ok]
        todo = todo[~ok]
    return out


# ---------------------------------------------------------------------------
# Workload recipes (sizes and distributions of the paper's experiments)
# ---------------------------------------------------------------------------

def circle_mixture_bags(seed: int, N: int = 64, d: int = 2, mk=(4, 16), n_comp: int = 3,
                        radius: float = 5.0, sigma: float = 1.0, alpha: float = 1.0,
                        device="cpu") -> Bags:
    """Single-barycenter pilot workload (stand-in for the colour-histogram pilot
    of Section 4: ~6 support points per distribution in low dimension).

    Every support point picks a mixture component u ~ U{0..n_comp-1} whose mean
    sits on a circle of the given radius (first two coordinates), with
    isotropic Gaussian noise sigma; m_k ~ U{mk[0]..mk[1]}; weights Dirichlet(alpha).
    """
    g = _gen(seed, device)
    sizes = torch.randint(mk[0], mk[1] + 1, (N,), generator=g, device=device)
    offsets = _ragged(sizes)
    n = int(offsets[-1])
    comp = torch.randint(0, n_comp, (n,), generator=g, device=device)
    ang = 2.0 * math.pi * comp.double() / n_comp
    mean = torch.zeros(n, d, dtype=torch.float64, device=device)
    mean[:, 0] = radius * torch.cos(ang)
    if d > 1:
        mean[:, 1] = radius * torch.sin(ang)
    supp = (mean + sigma * torch.randn(n, d, generator=g, dtype=torch.float64, device=device)).float()
    wt = _dirichlet_rows(g, offsets, alpha, device)
    return Bags(offsets, wt, d, supp=supp, meta=dict(recipe="circle_mixture", seed=seed))


def gaussian_class_bags(seed: int, N: int, d: int, n_classes: int, mk=(8, 32),
                        mu_sigma: float = 2.0, sigma: float = 1.0, alpha: float = 0.5,
                        device="cpu") -> Bags:
    """Clustering workload: each distribution has a ground-truth class c ~
    U{0..n_classes-1}; class means mu_c ~ N(0, mu_sigma^2 I); its support points
    are N(mu_c, sigma^2 I); m_k ~ U{mk}; weights Dirichlet(alpha)."""
    g = _gen(seed, device)
    mu = mu_sigma * torch.randn(n_classes, d, generator=g, dtype=torch.float64, device=device)
    labels = torch.randint(0, n_classes, (N,), generator=g, device=device)
    sizes = torch.randint(mk[0], mk[1] + 1, (N,), generator=g, device=device)
    offsets = _ragged(sizes)
    owner = _row_owner(offsets)
    n = int(offsets[-1])
    supp = (mu[labels[owner]] + sigma * torch.randn(n, d, generator=g, dtype=torch.float64,
                                                    device=device)).float()
    wt = _dirichlet_rows(g, offsets, alpha, device)
    return Bags(offsets, wt, d, supp=supp, labels=labels,
                meta=dict(recipe="gaussian_class", seed=seed, class_means=mu))


def ragged_cluster_bags(seed: int, n_clusters: int, d: int = 64, nc=(16, 4096), mk=(16, 64),
                        mu_sigma: float = 3.0, sigma: float = 1.0, alpha: float = 1.0,
                        device="cpu"):
    """Batched-barycenter workload: ``n_clusters`` clusters whose member counts
    are log-uniform in [nc[0], nc[1]]; members of cluster c have support points
    N(mu_c, sigma^2 I) with mu_c ~ N(0, mu_sigma^2 I); m_k ~ U{mk}; weights
    Dirichlet(alpha).  Members are stored cluster by cluster, so the returned
    ``members`` list is the identity and ``cluster_offsets`` delimits it.

    Returns (bags, cluster_offsets int64 (K+1), members int64 (N)).
    """
    g = _gen(seed, device)
    lo, hi = math.log(nc[0]), math.log(nc[1])
    ncs = torch.round(torch.exp(lo + (hi - lo) * torch.rand(n_clusters, generator=g,
                                                              dtype=torch.float64, device=device))).long()
    cluster_offsets = _ragged(ncs)
    N = int(cluster_offsets[-1])
    mu = mu_sigma * torch.randn(n_clusters, d, generator=g, dtype=torch.float32, device=device)
    sizes = torch.randint(mk[0], mk[1] + 1, (N,), generator=g, device=device)
    offsets = _ragged(sizes)
    n = int(offsets[-1])
    member_cluster = _row_owner(cluster_offsets)
    supp = torch.randn(n, d, generator=g, dtype=torch.float32, device=device)
    if sigma != 1.0:
        supp.mul_(sigma)
    # add the cluster mean row by row in slabs to bound temporary memory
    row_owner = _row_owner(offsets)
    slab = 1 << 24
    for a in range(0, n, slab):
        b = min(n, a + slab)
        supp[a:b].add_(mu[member_cluster[row_owner[a:b]]])
    del row_owner
    wt = _dirichlet_rows(g, offsets, alpha, device)
    members = torch.arange(N, dtype=torch.int64, device=device)
    bags = Bags(offsets, wt, d, supp=supp, labels=member_cluster,
                meta=dict(recipe="ragged_cluster", seed=seed))
    return bags, cluster_offsets, members


def document_bags(seed: int, N: int, V: int = 50_000, d: int = 300, mk=(10, 60),
                  zipf_s: float = 1.1, draws: int = 512, device="cpu") -> Bags:
    """Document-like bags over a seeded word vocabulary (stand-in for the
    20newsgroups / word-embedding experiments of Section 7).

    vocab: V unit-norm Gaussian vectors in R^d.  A bag draws words i.i.d. from
    a Zipf(zipf_s) law over ranks 1..V (truncated, rank r -> word r-1) until
    m_k ~ U{mk} DISTINCT words have appeared (at most ``draws`` draws); its
    support is those words (stored as vocabulary indices) and its weights the
    normalised counts.
    """
    g = _gen(seed, device)
    vocab = torch.randn(V, d, generator=g, dtype=torch.float32, device=device)
    vocab = vocab / vocab.norm(dim=1, keepdim=True)
    target = torch.randint(mk[0], mk[1] + 1, (N,), generator=g, device=device)
    p = torch.arange(1, V + 1, dtype=torch.float64, device=device).pow(-zipf_s)
    cdf = torch.cumsum(p, 0)
    cdf = cdf / cdf[-1]
    sizes, idx_chunks, cnt_chunks = [], [], []
    chunk = max(1, (1 << 22) // draws)
    for a in range(0, N, chunk):
        b = min(N, a + chunk)
        B = b - a
        u = torch.rand(B, draws, generator=g, dtype=torch.float64, device=device)
        word = torch.searchsorted(cdf, u).clamp_max(V - 1)             # (B, draws)
        key = torch.arange(B, device=device)[:, None] * V + word
        flat = key.reshape(-1)
        order = torch.sort(flat, stable=True).indices
        sk = flat[order]
        first_sorted = torch.ones_like(sk, dtype=torch.bool)
        first_sorted[1:] = sk[1:] != sk[:-1]
        first = torch.zeros_like(first_sorted)
        first[order] = first_sorted
        first = first.view(B, draws)
        seen = torch.cumsum(first.long(), 1)
        tgt = target[a:b]
        reach = seen >= tgt[:, None]
        has = reach.any(1)
        cut = torch.where(has, reach.float().argmax(1), torch.full_like(tgt, draws - 1))
        keep = torch.arange(draws, device=device)[None, :] <= cut[:, None]
        kept_key = key[keep]                                            # row-major: bag-major
        uniq, counts = torch.unique(kept_key, return_counts=True)       # sorted: bag-major
        bag_of = uniq // V
        sizes.append(torch.bincount(bag_of, minlength=B))
        idx_chunks.append((uniq % V).to(torch.int32))
        cnt_chunks.append(counts)
    sizes = torch.cat(sizes)
    offsets = _ragged(sizes)
    vocab_idx = torch.cat(idx_chunks)
    counts = torch.cat(cnt_chunks).double()
    owner = _row_owner(offsets)
    tot = torch.zeros(N, dtype=torch.float64, device=device).index_add_(0, owner, counts)
    wt = (counts / tot[owner]).float()
    return Bags(offsets, wt, d, vocab_idx=vocab_idx, vocab=vocab,
                meta=dict(recipe="document", seed=seed, V=V))


def symbolic_bags(seed: int, N: int, V: int = 20, n_classes: int = 4, mk=(4, 16), q: int = 5,
                  alpha: float = 1.0, device="cpu") -> Bags:
    """Symbolic workload (stand-in for the paper's symbolic data, e.g. amino-acid
    histograms over V = 20 symbols): the symbol-to-symbol dissimilarity is the
    squared Euclidean distance between hidden embeddings of the symbols (N(0, I)
    in R^q); each class c has a symbol distribution pi_c ~ Dirichlet(1) over the
    V symbols; a bag of class c draws m_k ~ U{mk} distinct symbols from pi_c
    (sampling without replacement) with weights Dirichlet(alpha).  Supports are
    stored as symbol ids (vocab_idx) with the V x V table in symcost; d = 1."""
    g = _gen(seed, device)
    emb = torch.randn(V, q, generator=g, dtype=torch.float64, device=device)
    table = ((emb[:, None, :] - emb[None, :, :]) ** 2).sum(-1).float()
    pis = _gamma_ge1(g, torch.ones(n_classes * V, dtype=torch.float64, device=device), device).reshape(n_classes, V)
    pis = pis / pis.sum(1, keepdim=True)
    labels = torch.randint(0, n_classes, (N,), generator=g, device=device)
    sizes = torch.randint(mk[0], min(mk[1], V) + 1, (N,), generator=g, device=device)
    offsets = _ragged(sizes)
    n = int(offsets[-1])
    sym = torch.empty(n, dtype=torch.int32, device=device)
    # distinct symbols per bag: the first m_k of the class's weighted random order
    # (Efraimidis-Spirakis keys u^(1/pi))
    u = torch.rand(N, V, generator=g, dtype=torch.float64, device=device).clamp_min(1e-300)
    keys = u.log() / pis[labels]
    order = torch.argsort(keys, dim=1, descending=True)
    owner = _row_owner(offsets)
    pos = torch.arange(n, device=device) - offsets[:-1][owner]
    sym[:] = order[owner, pos].to(torch.int32)
    wt = _dirichlet_rows(g, offsets, alpha, device)
    return Bags(offsets, wt, 1, vocab_idx=sym, labels=labels, symcost=table,
                meta=dict(recipe="symbolic", seed=seed, V=V))


def sample_initial_barycenters(seed: int, bags: Bags, cluster_offsets: torch.Tensor,
                               members: torch.Tensor, m: int):
    """Synthetic starting centroids: for every cluster, m support points drawn
    uniformly (with replacement only if the cluster has fewer than m points)
    from the pooled support of its members, plus uniform weights 1/m.
    Empty clusters get zeros.  Returns x0 (K, m, d) float32, w0 (K, m) float32."""
    dev = bags.offsets.device
    g = _gen(seed, dev)
    K = cluster_offsets.numel() - 1
    pts = bags.points()
    x0 = torch.zeros(K, m, bags.d, dtype=torch.float32, device=dev)
    co = cluster_offsets.cpu()
    # first member of each cluster and a random member per support point
    ncl = (co[1:] - co[:-1]).to(dev)
    r = torch.rand(K, m, generator=g, dtype=torch.float64, device=dev)
    pick_pos = cluster_offsets[:-1, None].to(dev) + (r * ncl[:, None].clamp_min(1)).long().clamp_max(
        (ncl[:, None] - 1).clamp_min(0))
    pick_pos = pick_pos.clamp_max(max(members.numel() - 1, 0))
    mem = members.to(dev)[pick_pos] if members.numel() else torch.zeros_like(pick_pos)
    lo = bags.offsets[mem]
    sz = bags.offsets[mem + 1] - lo
    r2 = torch.rand(K, m, generator=g, dtype=torch.float64, device=dev)
    row = lo + (r2 * sz).long().clamp_max((sz - 1).clamp_min(0))
    x0 = pts[row.reshape(-1)].reshape(K, m, bags.d).float().clone()
    x0[ncl == 0] = 0
    w0 = torch.full((K, m), 1.0 / m, dtype=torch.float32, device=dev)
    return x0, w0


def subset_bags(bags: Bags, ids) -> Bags:
    """Bags restricted to the given bag ids (renumbered 0..len(ids)-1)."""
    dev = bags.offsets.device
    ids = torch.as_tensor(ids, dtype=torch.int64, device=dev)
    lo = bags.offsets[ids]
    sz = bags.offsets[ids + 1] - lo
    offsets = _ragged(sz)
    n = int(offsets[-1])
    owner = torch.repeat_interleave(torch.arange(ids.numel(), device=dev), sz)
    rows = lo[owner] + (torch.arange(n, device=dev) - offsets[:-1][owner])
    return Bags(offsets, bags.wt[rows].clone(), bags.d,
                supp=None if bags.supp is None else bags.supp[rows].clone(),
                vocab_idx=None if bags.vocab_idx is None else bags.vocab_idx[rows].clone(),
                vocab=bags.vocab,
                labels=None if bags.labels is None else bags.labels[ids].clone(),
                meta=dict(bags.meta))
