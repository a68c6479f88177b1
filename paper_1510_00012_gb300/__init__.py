"""Python binding of libd2, the GB300 (sm_103a) D2-clustering hot path.

Thin ctypes marshalling over the C ABI declared in include/d2.h: every
function below has the name of the C entry point it calls, takes torch CUDA
tensors, checks dtypes/shapes/contiguity, and passes raw device pointers and
the current CUDA stream.  All computation happens in the library's CUDA
kernels; there is no CPU fallback.  If libd2.so has not been built (see
``paper_1510_00012_gb300.build``) the first call raises ``D2Error``.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import c_double, c_float, c_int, c_int32, c_int64, c_size_t, c_uint64, c_void_p, c_char_p

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libd2.so")

D2_OK, D2_EINVAL, D2_ENOMEM, D2_ECUDA, D2_ETIMEOUT, D2_ENOTSUP, D2_ENOCONV, D2_ESCRATCH = 0, -1, -2, -3, -4, -5, -6, -7
D2_NOALLOC_MAX_PAIRS = 1 << 20
D2_RULE_R1, D2_RULE_R2 = 1, 2
D2_FIX_X, D2_FIX_W, D2_VALIDATE, D2_NO_GRAPH, D2_NO_PIPE, D2_ELKAN = 0x1, 0x2, 0x4, 0x8, 0x10, 0x20
D2_COST_BF16, D2_COST_BF16X3, D2_COST_BF16X6 = 0x40, 0x80, 0xC0
D2_AUTOTUNE = 0x100
D2_ASSIGN_BOUNDED = 0x200
D2_SPLIT_STREAMS = 0x400
D2_PRUNE_RECALIBRATE = 0x800
D2_COST_ROWS = 0x1000
D2_SUPPORT_TC = 0x2000
D2_TEST_EXPIRE_WAIT = 0x8000
D2_TUNE_MAX = 16
D2_REDUCE_SUM, D2_REDUCE_MAX = 0, 1
# int reducer(void* user, int32 op, int64* buf, int64 count, void* stream)
REDUCER_FN = ctypes.CFUNCTYPE(c_int, c_void_p, c_int32, c_void_p, c_int64, c_void_p)
COST_PRECISION = {"fp32": 0, "bf16": D2_COST_BF16, "bf16x3": D2_COST_BF16X3, "bf16x6": D2_COST_BF16X6}
KT_NAMES = ("sweep_fused", "sweep_half", "cost", "support", "assign", "prune", "other", "bound")
KT_COUNT = len(KT_NAMES)


class D2Error(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("libd2 error %d: %s" % (code, msg))
        self.code = code


class _Bags(ctypes.Structure):
    _fields_ = [("N", c_int64), ("n", c_int64), ("d", c_int32), ("max_mk", c_int32),
                ("offsets", c_void_p), ("supp", c_void_p), ("vocab_idx", c_void_p),
                ("vocab", c_void_p), ("V", c_int64), ("wt", c_void_p), ("symcost", c_void_p)]


class _Opts(ctypes.Structure):
    _fields_ = [("rho0", c_double), ("rho", c_double), ("eps", c_double), ("iters", c_int32),
                ("tau", c_int32), ("rule", c_int32), ("flags", c_int32)]


_SIGS = {
    "d2_create": (c_void_p, [c_int]),
    "d2_destroy": (None, [c_void_p]),
    "d2_last_error": (c_char_p, [c_void_p]),
    "d2_workspace_bytes": (c_size_t, [c_void_p]),
    "d2_badmm_opts_default": (None, [c_void_p]),
    "d2_check_bags": (c_int, [c_void_p, c_void_p, c_void_p]),
    "d2_timing_enable": (c_int, [c_void_p, c_int]),
    "d2_timing_read": (c_int, [c_void_p, c_void_p, c_void_p]),
    "d2_launch_count": (c_int64, [c_void_p]),
    "d2_device_errors": (c_int, [c_void_p, c_void_p]),
    "d2_set_phase_limit": (c_int, [c_void_p, c_int32]),
    "d2_set_flow_store": (c_int, [c_void_p, c_int32, c_int32]),
    "d2_set_dual_bound": (c_int, [c_void_p, c_int32, c_float]),
    "d2_set_prune_forward": (c_int, [c_void_p, c_int32]),
    "d2_set_bound_kernels": (c_int, [c_void_p, c_int32]),
    "d2_set_reducer": (c_int, [c_void_p, c_void_p, c_void_p]),
    "d2_sweep_tuning": (c_int, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_void_p]),
    "d2_cluster_stats": (c_int, [c_void_p, c_void_p]),
    "d2_cost": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_int32, c_int32,
                        c_void_p, c_void_p, c_int32, c_void_p]),
    "badmm_barycenter": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_int32, c_int32,
                                 c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "d2_assign": (c_int, [c_void_p, c_void_p, c_int32, c_int32, c_void_p, c_void_p, c_void_p,
                          c_void_p, c_void_p, c_void_p, c_void_p]),
    "d2_assign_bounded": (c_int, [c_void_p, c_void_p, c_int32, c_int32, c_void_p, c_void_p, c_void_p,
                                  c_void_p, c_void_p, c_void_p, c_void_p]),
    "d2_assign_noalloc": (c_int, [c_void_p, c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "d2_w2_pairs": (c_int, [c_void_p, c_void_p, c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_void_p,
                            c_int64, c_void_p, c_void_p]),
    "d2_sym_cost": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_int32, c_int32, c_void_p,
                            c_void_p, c_void_p]),
    "badmm_barycenter_sym": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_int32, c_int32,
                                     c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "d2_assign_sym": (c_int, [c_void_p, c_void_p, c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_void_p,
                              c_void_p, c_void_p]),
    "d2_cluster_sym": (c_int, [c_void_p, c_void_p, c_int32, c_int32, c_void_p, c_uint64, c_int32, c_void_p,
                               c_void_p, c_void_p, c_void_p, c_void_p]),
    "d2_merge_init": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_int32, c_void_p, c_void_p,
                              c_void_p]),
    "d2_cluster": (c_int, [c_void_p, c_void_p, c_int32, c_int32, c_uint64, c_int32, c_void_p,
                           c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "d2_prune_create": (c_void_p, [c_void_p, c_int32, c_int32, c_int32, c_void_p, c_uint64]),
    "d2_prune_destroy": (None, [c_void_p]),
    "d2_prune_param_count": (c_int64, [c_void_p]),
    "d2_prune_get_params": (c_int, [c_void_p, c_void_p, c_void_p]),
    "d2_prune_set_params": (c_int, [c_void_p, c_void_p, c_void_p]),
    "d2_prune_set_margin": (c_int, [c_void_p, c_int32, c_float]),
    "d2_prune_get_margin": (c_int, [c_void_p, c_void_p, c_void_p]),
    "d2_prune_calibrate": (c_int, [c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_void_p, c_void_p,
                                   c_void_p, c_int64, c_float, c_void_p]),
    "d2_prune_get_calibration": (c_int, [c_void_p, c_void_p]),
    "d2_prune_embed": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_void_p,
                               c_void_p]),
    "d2_prune_loss_grad": (c_int, [c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_void_p, c_void_p,
                                   c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_void_p, c_void_p]),
    "d2_prune_train": (c_int, [c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_void_p, c_void_p,
                               c_void_p, c_void_p, c_void_p, c_int64, c_int32, c_int32, c_float,
                               c_uint64, c_void_p]),
}

_lib = None


def lib():
    """The loaded libd2 (raises D2Error if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise D2Error(D2_ENOTSUP, "libd2.so is not built (%s); run paper_1510_00012_gb300.build.build()"
                          % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _need(t, dtype, name, device=None):
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return t


class Context:
    """Owns a d2_ctx (device workspaces, last error)."""

    def __init__(self, device=None):
        if device is None:
            device = torch.cuda.current_device()
        self.device = int(device)
        torch.cuda.init()
        self.h = lib().d2_create(self.device)
        if not self.h:
            raise D2Error(D2_ECUDA, "d2_create(%d) failed" % self.device)

    def close(self):
        if getattr(self, "h", None):
            lib().d2_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, rc):
        if rc != D2_OK:
            raise D2Error(rc, lib().d2_last_error(self.h).decode())
        return rc

    def workspace_bytes(self):
        return int(lib().d2_workspace_bytes(self.h))

    def timing(self, on=True):
        """Start (or stop) per-launch CUDA-event timing; totals restart."""
        self.check(lib().d2_timing_enable(self.h, 1 if on else 0))

    def timing_read(self):
        """{kind: (total_ms, launches)} since the last timing() call."""
        ms = (c_double * KT_COUNT)()
        n = (c_int64 * KT_COUNT)()
        self.check(lib().d2_timing_read(self.h, ms, n))
        return {KT_NAMES[k]: (ms[k], n[k]) for k in range(KT_COUNT)}

    def launch_count(self):
        return int(lib().d2_launch_count(self.h))

    def device_errors(self):
        """Sticky device-side error bits since the last call (cleared); raises
        D2Error(D2_ETIMEOUT) if a bounded device wait expired."""
        bits = c_int32(0)
        self.check(lib().d2_device_errors(self.h, ctypes.byref(bits)))
        return int(bits.value)

    def set_phase_limit(self, max_phases):
        """Cap the exact solver's shortest-path phases per pair (0 = default);
        a low cap makes solves stop early and report D2_ENOCONV."""
        self.check(lib().d2_set_phase_limit(self.h, int(max_phases)))

    def set_reducer(self, fn):
        """Install fn(op, ptr, count, stream) -> int as the cross-process reducer
        of badmm_barycenter's exact sums (D2_REDUCE_SUM / D2_REDUCE_MAX of an
        int64 buffer of `count` elements at device address `ptr`, in place,
        ordered on the CUDA stream `stream`); None removes it."""
        if fn is None:
            self._reducer = None
            self.check(lib().d2_set_reducer(self.h, None, None))
            return

        def tramp(user, op, ptr, count, stream):
            try:
                return int(fn(int(op), int(ptr), int(count), int(stream or 0)))
            except Exception:  # no exception may cross the C boundary
                return 1

        self._reducer = REDUCER_FN(tramp)
        self.check(lib().d2_set_reducer(self.h, ctypes.cast(self._reducer, c_void_p), None))

    def set_flow_store(self, store="auto", pool_cap=0):
        """Exact solver's flow store: "auto", "dense" or "sparse"; pool_cap > 0
        caps the sparse pool (overflowed pairs are solved again densely)."""
        code = {"auto": 0, "dense": 1, "sparse": 2}[store]
        self.check(lib().d2_set_flow_store(self.h, code, int(pool_cap)))

    def set_dual_bound(self, iters=-1, eps_rel=0.0):
        """Entropic dual bound of d2_assign_bounded: Sinkhorn iterations per
        pair (-1: automatic, 0: off) and eps as a fraction of the pair's mean
        cost (0: default)."""
        self.check(lib().d2_set_dual_bound(self.h, int(iters), float(eps_rel)))

    def set_bound_kernels(self, path="auto"):
        """Cheap bounds of the bounded assignment: "auto" (tensor cores where
        they apply) or "cuda_cores"."""
        self.check(lib().d2_set_bound_kernels(self.h, {"auto": 0, "cuda_cores": 1}[path]))

    def set_prune_forward(self, path="auto"):
        """Pruning network forward: "auto" (tensor cores where they apply) or
        "cuda_cores"."""
        self.check(lib().d2_set_prune_forward(self.h, {"auto": 0, "cuda_cores": 1}[path]))

    def sweep_tuning(self, m):
        """The plan-sweep autotuner's record for plan width m: None when untuned,
        else {"chosen": i, "candidates": [{"kind", "lanes_per_row",
        "float4_per_lane", "ctas_per_sm", "ms"}, ...]}."""
        n, ch = c_int32(0), c_int32(-1)
        ms = (c_float * D2_TUNE_MAX)()
        shape = (c_int32 * (4 * D2_TUNE_MAX))()
        self.check(lib().d2_sweep_tuning(self.h, int(m), ctypes.byref(n), ctypes.byref(ch), ms, shape))
        if n.value == 0:
            return None
        cands = [{"kind": ("pipelined", "prefetch")[shape[4 * i]], "lanes_per_row": shape[4 * i + 1],
                  "float4_per_lane": shape[4 * i + 2], "ctas_per_sm": shape[4 * i + 3], "ms": ms[i]}
                 for i in range(n.value)]
        return {"chosen": ch.value, "candidates": cands}

    def cluster_stats(self):
        """Exact W^2 solves and pruner fall-backs of the last d2_cluster call."""
        st = (c_int64 * 2)()
        self.check(lib().d2_cluster_stats(self.h, st))
        return dict(exact_solves=st[0], fallbacks=st[1])


class DeviceBags:
    """Device-resident bag set in the layout of d2_bags (see include/d2.h)."""

    def __init__(self, offsets, wt, d, supp=None, vocab_idx=None, vocab=None, max_mk=None, symcost=None):
        """Coordinates (supp, or vocab_idx into vocab) or symbols (vocab_idx
        into the V x V dissimilarity table symcost, d = 1)."""
        self.offsets = _need(offsets, torch.int64, "offsets")
        self.wt = _need(wt, torch.float32, "wt")
        self.supp = None if supp is None else _need(supp, torch.float32, "supp")
        self.vocab_idx = None if vocab_idx is None else _need(vocab_idx, torch.int32, "vocab_idx")
        self.vocab = None if vocab is None else _need(vocab, torch.float32, "vocab")
        self.symcost = None if symcost is None else _need(symcost, torch.float32, "symcost")
        self.d = int(d)
        self.N = offsets.numel() - 1
        self.n = wt.numel()
        if max_mk is None:
            max_mk = int((offsets[1:] - offsets[:-1]).max().item()) if self.N > 0 else 1
        self.max_mk = int(max_mk)
        self.V = vocab.shape[0] if vocab is not None else (symcost.shape[0] if symcost is not None else 0)
        self.c = _Bags(self.N, self.n, self.d, self.max_mk, _ptr(self.offsets), _ptr(self.supp),
                       _ptr(self.vocab_idx), _ptr(self.vocab), self.V, _ptr(self.wt), _ptr(self.symcost))

    @classmethod
    def from_synth(cls, b, device="cuda"):
        mv = lambda t, dt: None if t is None else t.to(device=device, dtype=dt).contiguous()
        return cls(mv(b.offsets, torch.int64), mv(b.wt, torch.float32), b.d,
                   supp=mv(b.supp, torch.float32), vocab_idx=mv(b.vocab_idx, torch.int32),
                   vocab=mv(b.vocab, torch.float32), symcost=mv(getattr(b, "symcost", None), torch.float32))

    def ref(self):
        return ctypes.byref(self.c)


def _cost_flag(precision):
    if precision not in COST_PRECISION:
        raise ValueError("cost precision must be one of %s" % sorted(COST_PRECISION))
    return COST_PRECISION[precision]


def badmm_opts(rho0=2.0, iters=100, tau=10, eps=1e-16, rule="R1", fix_x=False, fix_w=False,
               validate=False, rho=0.0, graph=True, elkan=False, cost="fp32", autotune=False,
               assign_bounded=False, split_streams=False, recalibrate=False, cost_rows=False, support_tc=False):
    """d2_badmm_opts; cost = "fp32" | "bf16" | "bf16x3" | "bf16x6" selects the cost build."""
    o = _Opts()
    lib().d2_badmm_opts_default(ctypes.byref(o))
    o.rho0, o.iters, o.tau, o.eps, o.rho = float(rho0), int(iters), int(tau), float(eps), float(rho)
    o.rule = D2_RULE_R2 if rule == "R2" else D2_RULE_R1
    o.flags = ((D2_FIX_X if fix_x else 0) | (D2_FIX_W if fix_w else 0) | (D2_VALIDATE if validate else 0)
               | (0 if graph else D2_NO_GRAPH) | (D2_ELKAN if elkan else 0) | _cost_flag(cost)
               | (D2_AUTOTUNE if autotune else 0) | (D2_ASSIGN_BOUNDED if assign_bounded else 0)
               | (D2_SPLIT_STREAMS if split_streams else 0) | (D2_PRUNE_RECALIBRATE if recalibrate else 0)
               | (D2_COST_ROWS if cost_rows else 0) | (D2_SUPPORT_TC if support_tc else 0))
    return o


def d2_check_bags(ctx, bags):
    return ctx.check(lib().d2_check_bags(ctx.h, bags.ref(), _stream()))


def d2_cost(ctx, bags, cluster_offsets, members, x, C_out=None, precision="fp32", extra_flags=0):
    """C (n x m, j-major rows) between each cluster's support x[c] and its members;
    precision = "fp32" | "bf16" | "bf16x3" | "bf16x6" (tensor cores where d >= 32)."""
    _need(cluster_offsets, torch.int64, "cluster_offsets")
    _need(members, torch.int64, "members")
    _need(x, torch.float32, "x")
    K, m = x.shape[0], x.shape[1]
    if C_out is None:
        C_out = torch.zeros(bags.n, m, dtype=torch.float32, device=x.device)
    _need(C_out, torch.float32, "C_out")
    ctx.check(lib().d2_cost(ctx.h, bags.ref(), _ptr(cluster_offsets), _ptr(members), members.numel(),
                            K, m, _ptr(x), _ptr(C_out), _cost_flag(precision) | int(extra_flags),
                            _stream()))
    return C_out


def badmm_barycenter(ctx, bags, cluster_offsets, members, x, w, plan=None, warm_mask=None,
                     opts=None, obj=None):
    """Algorithm badmm on every cluster; updates x (K,m,d), w (K,m), plan (n,m) in place.

    Returns (x, w, plan, obj) with obj (K,) float64 on the device."""
    _need(cluster_offsets, torch.int64, "cluster_offsets")
    _need(members, torch.int64, "members")
    _need(x, torch.float32, "x")
    _need(w, torch.float32, "w")
    K, m = x.shape[0], x.shape[1]
    if plan is None:
        plan = torch.empty(bags.n, m, dtype=torch.float32, device=x.device)
    _need(plan, torch.float32, "plan")
    if warm_mask is not None:
        _need(warm_mask, torch.uint8, "warm_mask")
    if obj is None:
        obj = torch.empty(K, dtype=torch.float64, device=x.device)
    _need(obj, torch.float64, "obj")
    if opts is None:
        opts = badmm_opts()
    ctx.check(lib().badmm_barycenter(ctx.h, bags.ref(), _ptr(cluster_offsets), _ptr(members),
                                     members.numel(), K, m, _ptr(x), _ptr(w), _ptr(plan),
                                     _ptr(warm_mask), ctypes.byref(opts), _ptr(obj), _stream()))
    return x, w, plan, obj


def d2_sym_cost(ctx, bags, cluster_offsets, members, csym, C_out=None):
    """Symbolic bags: C (n x m, j-major rows) from the table for each cluster's symbols csym (K, m) int32."""
    _need(cluster_offsets, torch.int64, "cluster_offsets")
    _need(members, torch.int64, "members")
    _need(csym, torch.int32, "csym")
    K, m = csym.shape[0], csym.shape[1]
    if C_out is None:
        C_out = torch.zeros(bags.n, m, dtype=torch.float32, device=csym.device)
    _need(C_out, torch.float32, "C_out")
    ctx.check(lib().d2_sym_cost(ctx.h, bags.ref(), _ptr(cluster_offsets), _ptr(members), members.numel(), K, m,
                                _ptr(csym), _ptr(C_out), _stream()))
    return C_out


def badmm_barycenter_sym(ctx, bags, cluster_offsets, members, csym, w, plan=None, warm_mask=None, opts=None,
                         obj=None):
    """Algorithm badmm with fixed symbolic supports csym (K, m) int32; updates w (K, m) and plan (n, m)."""
    _need(cluster_offsets, torch.int64, "cluster_offsets")
    _need(members, torch.int64, "members")
    _need(csym, torch.int32, "csym")
    _need(w, torch.float32, "w")
    K, m = csym.shape[0], csym.shape[1]
    if plan is None:
        plan = torch.empty(bags.n, m, dtype=torch.float32, device=w.device)
    _need(plan, torch.float32, "plan")
    if warm_mask is not None:
        _need(warm_mask, torch.uint8, "warm_mask")
    if obj is None:
        obj = torch.empty(K, dtype=torch.float64, device=w.device)
    if opts is None:
        opts = badmm_opts()
    ctx.check(lib().badmm_barycenter_sym(ctx.h, bags.ref(), _ptr(cluster_offsets), _ptr(members), members.numel(),
                                         K, m, _ptr(csym), _ptr(w), _ptr(plan), _ptr(warm_mask), ctypes.byref(opts),
                                         _ptr(obj), _stream()))
    return w, plan, obj


def d2_assign_sym(ctx, bags, csym, w, want_stats=False):
    """Exact assignment of symbolic bags to centroids (csym (K, m) int32, w (K, m))."""
    _need(csym, torch.int32, "csym")
    _need(w, torch.float32, "w")
    K, m = csym.shape[0], csym.shape[1]
    labels = torch.empty(bags.N, dtype=torch.int32, device=w.device)
    dist = torch.empty(bags.N, dtype=torch.float32, device=w.device)
    st = (c_int64 * 3)() if want_stats else None
    ctx.check(lib().d2_assign_sym(ctx.h, bags.ref(), K, m, _ptr(csym), _ptr(w), _ptr(labels), _ptr(dist), st,
                                  _stream()))
    if want_stats:
        return labels, dist, dict(exact_solves=st[0], fallbacks=st[1], limit_hits=st[2])
    return labels, dist


def d2_cluster_sym(ctx, bags, K, sym, seed, rounds, opts=None):
    """Algorithm 1 on symbolic bags, every centroid on the symbols sym (m,) int32
    -> (w (K, m), labels (N), obj_per_round list)."""
    _need(sym, torch.int32, "sym")
    m = sym.numel()
    dev = bags.offsets.device
    w = torch.empty(K, m, dtype=torch.float32, device=dev)
    labels = torch.empty(bags.N, dtype=torch.int32, device=dev)
    objs = (c_double * rounds)()
    if opts is None:
        opts = badmm_opts()
    ctx.check(lib().d2_cluster_sym(ctx.h, bags.ref(), K, m, _ptr(sym), c_uint64(seed), rounds, ctypes.byref(opts),
                                   _ptr(w), _ptr(labels), objs, _stream()))
    return w, labels, list(objs)


def d2_merge_init(ctx, bags, ids, m):
    """Eq. (merge) reduction of the bags `ids` to m points -> x (cnt, m, d), w (cnt, m)."""
    _need(ids, torch.int64, "ids")
    cnt = ids.numel()
    x = torch.empty(cnt, m, bags.d, dtype=torch.float32, device=ids.device)
    w = torch.empty(cnt, m, dtype=torch.float32, device=ids.device)
    ctx.check(lib().d2_merge_init(ctx.h, bags.ref(), _ptr(ids), cnt, m, _ptr(x), _ptr(w), _stream()))
    return x, w


def d2_assign(ctx, bags, x, w, prune=None, want_stats=False, bounded=False):
    """Exact (or pruned) assignment: labels (N int32), W^2 to the chosen centroid (N float32)[, stats].
    bounded=True calls d2_assign_bounded (same result, certified lower bounds skip most LPs)."""
    _need(x, torch.float32, "x")
    _need(w, torch.float32, "w")
    K, m = x.shape[0], x.shape[1]
    labels = torch.empty(bags.N, dtype=torch.int32, device=x.device)
    dist = torch.empty(bags.N, dtype=torch.float32, device=x.device)
    st = (c_int64 * 3)() if want_stats else None
    fn = lib().d2_assign_bounded if bounded else lib().d2_assign
    ctx.check(fn(ctx.h, bags.ref(), K, m, _ptr(x), _ptr(w),
                 None if prune is None else c_void_p(prune.h), _ptr(labels), _ptr(dist), st, _stream()))
    if want_stats:
        return labels, dist, dict(exact_solves=st[0], fallbacks=st[1], limit_hits=st[2])
    return labels, dist


def d2_cluster(ctx, bags, K, m, seed, rounds, opts=None, prune=None):
    """Algorithm 1 on the device -> (x (K,m,d), w (K,m), labels (N), obj_per_round list)."""
    dev = bags.offsets.device
    x = torch.empty(K, m, bags.d, dtype=torch.float32, device=dev)
    w = torch.empty(K, m, dtype=torch.float32, device=dev)
    labels = torch.empty(bags.N, dtype=torch.int32, device=dev)
    objs = (c_double * rounds)()
    if opts is None:
        opts = badmm_opts()
    ctx.check(lib().d2_cluster(ctx.h, bags.ref(), K, m, c_uint64(seed), rounds, ctypes.byref(opts),
                               None if prune is None else c_void_p(prune.h), _ptr(x), _ptr(w), _ptr(labels),
                               objs, _stream()))
    return x, w, labels, list(objs)


def d2_w2_pairs(ctx, bags, x, w, pair_bag, pair_cent):
    """Exact W^2 for explicit (bag, centroid) pairs -> (npairs,) float32."""
    _need(x, torch.float32, "x")
    _need(w, torch.float32, "w")
    _need(pair_bag, torch.int64, "pair_bag")
    _need(pair_cent, torch.int32, "pair_cent")
    out = torch.empty(pair_bag.numel(), dtype=torch.float32, device=x.device)
    ctx.check(lib().d2_w2_pairs(ctx.h, bags.ref(), x.shape[0], x.shape[1], _ptr(x), _ptr(w), _ptr(pair_bag),
                                _ptr(pair_cent), pair_bag.numel(), _ptr(out), _stream()))
    return out


class Pruner:
    """Learned candidate pruner (d2_prune): MLP embedding trained on exact W^2."""

    def __init__(self, ctx, d, hidden=128, embed=64, init=None, seed=0):
        self.ctx = ctx
        buf = None
        if init is not None:
            buf = torch.as_tensor(init, dtype=torch.float32).contiguous()
        self.h = lib().d2_prune_create(ctx.h, d, hidden, embed, None if buf is None else ctypes.c_void_p(buf.data_ptr()),
                                       c_uint64(seed))
        if not self.h:
            raise D2Error(D2_EINVAL, lib().d2_last_error(ctx.h).decode())
        self.d, self.H, self.E = d, hidden, embed

    def close(self):
        if getattr(self, "h", None):
            lib().d2_prune_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def nparam(self):
        return int(lib().d2_prune_param_count(self.h))

    def params(self):
        out = torch.empty(self.nparam(), dtype=torch.float32)
        self.ctx.check(lib().d2_prune_get_params(self.ctx.h, self.h, ctypes.c_void_p(out.data_ptr())))
        return out

    def unpack(self, flat):
        d, H, E = self.d, self.H, self.E
        o = 0
        out = {}
        for name, shape in (("W1", (H, d)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (E, H))):
            n = 1
            for s_ in shape:
                n *= s_
            out[name] = flat[o:o + n].reshape(shape)
            o += n
        return out

    def set_params(self, flat):
        flat = torch.as_tensor(flat, dtype=torch.float32).contiguous()
        self.ctx.check(lib().d2_prune_set_params(self.ctx.h, self.h, ctypes.c_void_p(flat.data_ptr())))

    def set_margin(self, r, delta):
        rc = lib().d2_prune_set_margin(self.h, int(r), float(delta))
        if rc != D2_OK:
            raise D2Error(rc, "d2_prune_set_margin: need 1 <= r <= 16 and delta >= 0")

    def margin(self):
        r, dl = c_int32(), c_float()
        lib().d2_prune_get_margin(self.h, ctypes.byref(r), ctypes.byref(dl))
        return int(r.value), float(dl.value)

    def calibrate(self, bags, x, w, ids, quantile=0.999):
        """delta := quantile of |What^2 - W^2| over every (ids[t], centroid) pair (exact W^2)."""
        _need(ids, torch.int64, "ids")
        K, m = x.shape[0], x.shape[1]
        self.ctx.check(lib().d2_prune_calibrate(self.ctx.h, self.h, bags.ref(), K, m, _ptr(x), _ptr(w),
                                                _ptr(ids), ids.numel(), float(quantile), _stream()))
        return self.margin()[1]

    def calibration_fallbacks(self):
        """Fraction of the last calibration sample whose margin test fails (-1 before any)."""
        f = c_float()
        self.ctx.check(lib().d2_prune_get_calibration(self.h, ctypes.byref(f)))
        return float(f.value)

    def embed(self, bags, ids):
        _need(ids, torch.int64, "ids")
        emb = torch.empty(ids.numel(), self.E, dtype=torch.float32, device=ids.device)
        mu = torch.empty(ids.numel(), bags.d, dtype=torch.float32, device=ids.device)
        self.ctx.check(lib().d2_prune_embed(self.ctx.h, self.h, bags.ref(), _ptr(ids), ids.numel(), _ptr(emb),
                                            _ptr(mu), _stream()))
        return emb, mu

    def loss_grad(self, bags, x, w, pair_bag, pair_cent, target):
        _need(pair_bag, torch.int64, "pair_bag")
        _need(pair_cent, torch.int32, "pair_cent")
        _need(target, torch.float32, "target")
        loss = torch.empty(1, dtype=torch.float64, device=x.device)
        grad = torch.empty(self.nparam(), dtype=torch.float32, device=x.device)
        self.ctx.check(lib().d2_prune_loss_grad(self.ctx.h, self.h, bags.ref(), x.shape[0], x.shape[1], _ptr(x),
                                                _ptr(w), _ptr(pair_bag), _ptr(pair_cent), _ptr(target),
                                                pair_bag.numel(), _ptr(loss), _ptr(grad), _stream()))
        return loss, grad

    def train(self, bags, x, w, pair_bag, pair_cent, target, steps, batch=1024, lr=1e-3, seed=0):
        _need(pair_bag, torch.int64, "pair_bag")
        _need(pair_cent, torch.int32, "pair_cent")
        _need(target, torch.float32, "target")
        losses = (c_float * steps)()
        torch.cuda.synchronize()
        self.ctx.check(lib().d2_prune_train(self.ctx.h, self.h, bags.ref(), x.shape[0], x.shape[1], _ptr(x), _ptr(w),
                                            _ptr(pair_bag), _ptr(pair_cent), _ptr(target), pair_bag.numel(),
                                            steps, batch, c_float(lr), c_uint64(seed), losses))
        return list(losses)


def d2_assign_noalloc(bags, x, w):
    """Exact assignment through the no-allocation entry point (no context):
    labels (N int32), W^2 to the chosen centroid (N float32).  The output
    tensors are allocated here by torch, not by the library."""
    _need(x, torch.float32, "x")
    _need(w, torch.float32, "w")
    labels = torch.empty(bags.N, dtype=torch.int32, device=x.device)
    dist = torch.empty(bags.N, dtype=torch.float32, device=x.device)
    rc = lib().d2_assign_noalloc(bags.ref(), x.shape[0], x.shape[1], _ptr(x), _ptr(w), _ptr(labels), _ptr(dist),
                                 _stream())
    if rc != D2_OK:
        why = {D2_ESCRATCH: ": N * K exceeds the fixed scratch", D2_ENOTSUP: ": 32 ceil(m/32) + max_mk above 256 or the tableaus too large",
               D2_EINVAL: ": invalid arguments", D2_ENOCONV: ": a solve reached the phase cap"}.get(rc, "")
        raise D2Error(rc, "d2_assign_noalloc failed" + why)
    return labels, dist
