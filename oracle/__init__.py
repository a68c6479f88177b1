"""Plain, slow FP64 CPU oracle for the D2-clustering hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the ``libd2`` CUDA
library and its Python binding) imports, links or calls this package; only the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may.
It shares no code with the CUDA path; the only common module is ``synth``,
which draws random inputs and holds none of the method's arithmetic.

Every function follows a passage of Ye, Wu, Wang & Li, "Fast Discrete
Distribution Clustering Using Wasserstein Barycenter with Sparse Support"
(arXiv 1510.00012), cited in its docstring, in the paper's order and notation,
with numpy/scipy library primitives (sums, exp, an LP solver) as steps.

Parity status of each function (what pins it is listed in tests/test_oracle_*):
  cost.cost_matrix              pinned (brute force, norm identity)
  ot.w2_exact                   pinned (1-D closed form, permutation brute force,
                                translation identity, symmetry)
  badmm.badmm_barycenter        pinned by invariants (marginals, dual mass),
                                special cases (m=1 closed form, fixed-w -> OT,
                                N=1 identity, 1-D quantile barycenter bound,
                                full-batch LP band) and invariances; the exact
                                iterate values beyond those are parity unpinned
                                (the paper prints no worked example)
  merge.merge_reduce            pinned (brute-force criterion, moment invariants)
  cluster.d2_cluster            pinned (m=1 reduces exactly to Lloyd's K-means)
  mlp.*                         pinned (finite differences, hand-worked example)
"""
from .cost import cost_matrix
from .badmm import badmm_barycenter
from .ot import w2_exact
from .merge import merge_reduce
from .cluster import d2_assign, d2_cluster, splitmix64, init_pick
from . import mlp

__all__ = ["cost_matrix", "badmm_barycenter", "w2_exact", "merge_reduce",
           "d2_assign", "d2_cluster", "splitmix64", "init_pick", "mlp"]
