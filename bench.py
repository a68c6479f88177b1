#!/usr/bin/env python
"""Benchmark of the B-ADMM barycenter hot path on one GB300 per rank.

Workload (default ``ragged4096``): 4,096 clusters whose member counts are
log-uniform in [16, 4096] (~3.0M distributions), d = 64, m_k ~ U{16..64},
supports N(mu_c, I) with mu_c ~ N(0, 9I), Dirichlet(1) weights, barycenters of
m = 32 points; one step = one badmm_barycenter call of T = 100 iterations
(tau = 10, rule R1) over every cluster, started from the same synthetic
barycenters.  Metric: plan-entry updates per second = sum_c m * n_c * T / step
time.  With N ranks (torchrun) every rank solves its own independent problem
of the same size (weak scaling; the clusters shard with no collective).

Prints ONE JSON line on rank 0.  ``--impl reference`` times the FP64 CPU
oracle on a bounded sample of the same workload instead.
"""
import os

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import hashlib
import json
import statistics
import subprocess
import sys
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "B-ADMM plan-entry updates/s; D2-clustering s/round vs plain form @1e-4 obj"
UNIT = "plan-entry updates/s"
BYTES_PER_ENTRY = 20  # fused sweep: read Pi, Lambda, C; write Pi, Lambda (FP32)

WORKLOADS = {
    "ragged4096": dict(clusters=4096, d=64, nc=(16, 4096), mk=(16, 64), m=32, iters=100, tau=10,
                       desc="batched ragged barycenters: 4096 clusters, member counts log-uniform "
                            "in [16,4096], d=64, m_k~U{16..64}, m=32, N(mu_c,I) with mu_c~N(0,9I), "
                            "Dirichlet(1) weights, T=100, tau=10, R1"),
    "ragged256": dict(clusters=256, d=64, nc=(16, 4096), mk=(16, 64), m=32, iters=100, tau=10,
                      desc="256 clusters of the ragged recipe (profiling size)"),
}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            j = json.load(open(p))
            return float(j["hbm_gbs"]), "measured"
        except Exception:
            pass
    return 6800.0, "fallback"


def sweep_traffic_per_entry():
    """DRAM bytes per plan entry of one fused-sweep launch from the committed
    ncu summary, valid only while the sweep source is unchanged."""
    src = os.path.join(ROOT, "paper_1510_00012_gb300", "csrc", "badmm.cu")
    digest = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    p = os.path.join(ROOT, "profiles", "k_sweep_traffic.txt")
    if not os.path.exists(p):
        return None
    for line in open(p):
        parts = dict(kv.split("=", 1) for kv in line.split() if "=" in kv)
        if parts.get("badmm_cu_sha256_16") == digest and "dram_bytes_per_entry" in parts:
            return float(parts["dram_bytes_per_entry"])
    return None


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.proc = None
        self.lines = []
        sel = []
        try:
            uuid = str(torch.cuda.get_device_properties(device).uuid)
            sel = ["-i", uuid if uuid.startswith("GPU-") else "GPU-" + uuid]
        except Exception:
            sel = []
        self.cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                    "-lms", "200"] + sel

    def start(self):
        try:
            self.proc = subprocess.Popen(self.cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def rank_seed(seed, rank):
    """Each rank solves its own independent problem of the same size."""
    return seed + 7919 * rank


def max_over_ranks(ms, dist=None, device="cpu"):
    """Slowest rank's time (the whole-job step time); identity on one rank."""
    if dist is None:
        return float(ms)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(entries_per_rank, iters, world, ms_per_step):
    """Whole-job plan-entry updates per second (weak scaling: every rank has
    entries_per_rank entries)."""
    return world * entries_per_rank * iters / (ms_per_step * 1e-3)


def make_workload(name, seed, device):
    W = WORKLOADS[name]
    bags, co, mem = synth.ragged_cluster_bags(seed, W["clusters"], d=W["d"], nc=W["nc"], mk=W["mk"],
                                              mu_sigma=3.0, device=device)
    x0, w0 = synth.sample_initial_barycenters(seed + 1, bags, co, mem, W["m"])
    return bags, co, mem, x0, w0


D2_WORKLOAD = dict(N=20000, d=16, K=10, mk=(8, 32), m=16, rounds=5, iters=100, tau=10,
                   desc="D2-clustering: K=10, N=20,000 distributions, d=16, m_k~U{8..32}, 10 Gaussian "
                        "classes (means N(0,4I), sigma=1), Dirichlet(0.5) weights, m=16, 5 rounds x 100 "
                        "B-ADMM iterations")


def d2_round_comparison(d2, ctx, dev, seed):
    """Runs _d2_round_comparison on a side stream, so that every variant's
    badmm_barycenter calls may replay their launch sequence as a CUDA graph."""
    side = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(side):
        return _d2_round_comparison(d2, ctx, dev, seed)


def _d2_round_comparison(d2, ctx, dev, seed):
    """Seconds per D2-clustering round: plain form vs batched vs batched + pruning.

    plain   : every round = exact full-K assignment, then one badmm_barycenter
              call per cluster with the register-prefetch sweep;
    batched : d2_cluster (all clusters in one call, pipelined sweep), exact;
    pruned  : d2_cluster with the learned pruner (trained on exact W^2 of
              100k (bag, centroid) pairs against the batched run's centroids;
              training time reported separately)."""
    W = D2_WORKLOAD
    bags = synth.gaussian_class_bags(seed, W["N"], W["d"], W["K"], mk=W["mk"], device=dev)
    db = d2.DeviceBags(bags.offsets, bags.wt, bags.d, supp=bags.supp)
    K, m, R = W["K"], W["m"], W["rounds"]
    # the warm-up call tunes the sweep's launch shape for this plan width
    # (kept in the context for every later batched call; the plain form's
    # register-prefetch sweep is not tuned)
    opts = d2.badmm_opts(iters=W["iters"], tau=W["tau"], autotune=True)
    out = {"workload": W["desc"]}

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return r, time.perf_counter() - t0

    # batched: warm-up once (which also tunes the sweep), then timed
    d2.d2_cluster(ctx, db, K, m, 11, 1, opts)
    tune = ctx.sweep_tuning(m)
    if tune:
        out["sweep_shape"] = tune["candidates"][tune["chosen"]]
    (xb, wb, lb, ob), tb = timed(lambda: d2.d2_cluster(ctx, db, K, m, 11, R, opts))
    # plain: the same rounds with one call per cluster
    nop = d2.badmm_opts(iters=W["iters"], tau=W["tau"])
    nop.flags |= d2.D2_NO_PIPE

    def plain():
        x, w = d2.d2_merge_init(ctx, db, torch.tensor(pick_ids(bags, K, m, 11), device=dev), m)
        plan = torch.empty(bags.n, m, dtype=torch.float32, device=dev)
        prev = None
        objs = []
        for _ in range(R):
            lab, dist = d2.d2_assign(ctx, db, x, w)
            objs.append(float(dist.double().mean()))
            warm = (lab == prev).to(torch.uint8) if prev is not None else torch.zeros_like(lab, dtype=torch.uint8)
            for c in range(K):
                ids = torch.nonzero(lab == c).flatten().to(torch.int64)
                if ids.numel() == 0:
                    continue
                co = torch.tensor([0, ids.numel()], dtype=torch.int64, device=dev)
                xc, wc = x[c:c + 1].clone(), w[c:c + 1].clone()
                d2.badmm_barycenter(ctx, db, co, ids, xc, wc, plan, warm, nop)
                x[c:c + 1], w[c:c + 1] = xc, wc
            prev = lab
        return x, w, prev, objs

    plain()
    (xp, wp, lp, op), tp = timed(plain)
    out["plain_s_per_round"] = tp / R
    out["batched_s_per_round"] = tb / R
    # the two halves of a batched round: the exact assignment and the update
    (la, _), t_as = timed(lambda: d2.d2_assign(ctx, db, xb, wb))
    co_a = torch.zeros(K + 1, dtype=torch.int64, device=dev)
    co_a[1:] = torch.cumsum(torch.bincount(la.long(), minlength=K), 0)
    mem_a = torch.sort(la.long(), stable=True).indices.contiguous()
    xu, wu = xb.clone(), wb.clone()
    _, t_up = timed(lambda: d2.badmm_barycenter(ctx, db, co_a, mem_a, xu, wu, None, None, opts))
    out["batched_round_split_s"] = {"exact_assignment": t_as, "badmm_update": t_up,
                                    "assignment_pairs_per_s": bags.N * K / t_as}
    out["obj_plain"] = op
    out["obj_batched"] = ob
    out["max_rel_obj_diff_batched_vs_plain"] = max(abs(a - b) / b for a, b in zip(ob, op))
    # learned pruning: train on exact W^2 against the batched centroids
    g = torch.Generator(device=dev).manual_seed(seed + 5)
    npairs = 100_000
    pb = torch.randint(0, bags.N, (npairs,), generator=g, device=dev)
    pc = torch.randint(0, K, (npairs,), generator=g, device=dev, dtype=torch.int32)
    (tg), tt = timed(lambda: d2.d2_w2_pairs(ctx, db, xb, wb, pb, pc))
    pr = d2.Pruner(ctx, bags.d, hidden=128, embed=64, seed=3)
    _, ttrain = timed(lambda: pr.train(db, xb, wb, pb, pc, tg, steps=300, batch=1024, lr=2e-3, seed=4))
    r, delta = pr.margin()
    pr.set_margin(3, delta)
    lab_exact, _ = d2.d2_assign(ctx, db, xb, wb)
    (lab_pr, _, st), _ = timed(lambda: d2.d2_assign(ctx, db, xb, wb, prune=pr, want_stats=True))
    d2.d2_cluster(ctx, db, K, m, 11, 1, opts, prune=pr)
    (xq, wq, lq, oq), tq = timed(lambda: d2.d2_cluster(ctx, db, K, m, 11, R, opts, prune=pr))
    out.update({"pruned_s_per_round": tq / R, "obj_pruned": oq,
                "max_rel_obj_diff_pruned_vs_plain": max(abs(a - b) / b for a, b in zip(oq, op)),
                "pruner": {"r": 3, "delta": delta, "train_pairs": npairs, "target_s": tt, "train_s": ttrain,
                           "misassignment_vs_exact": float((lab_pr != lab_exact).float().mean()),
                           "exact_solves": st["exact_solves"], "fallbacks": st["fallbacks"],
                           "exact_solves_full": bags.N * K}})
    # exact assignment by certified bounds (same labels as the full solve)
    bopts = d2.badmm_opts(iters=W["iters"], tau=W["tau"], assign_bounded=True)
    d2.d2_cluster(ctx, db, K, m, 11, 1, bopts)
    (xe, we, le, oe), te = timed(lambda: d2.d2_cluster(ctx, db, K, m, 11, R, bopts))
    out.update({"bounded_s_per_round": te / R, "obj_bounded": oe,
                "labels_equal_bounded_vs_batched": bool(torch.equal(le, lb)),
                "speedup_bounded_vs_plain": out["plain_s_per_round"] / (te / R)})
    # Elkan's triangle-inequality skipping (Section 5), exact
    eopts = d2.badmm_opts(iters=W["iters"], tau=W["tau"], elkan=True)
    d2.d2_cluster(ctx, db, K, m, 11, 1, eopts)
    (xk, wk, lk, ok), tk = timed(lambda: d2.d2_cluster(ctx, db, K, m, 11, R, eopts))
    out.update({"elkan_s_per_round": tk / R, "elkan_exact_solves": ctx.cluster_stats()["exact_solves"],
                "labels_equal_elkan_vs_batched": bool(torch.equal(lk, lb))})
    out["plain_form"] = ("this library one cluster per badmm_barycenter call with the register-prefetch "
                         "sweep (FP32, fused iterations) and the exact full-K assignment: a conservative "
                         "plain form")
    out["speedup_batched_vs_plain"] = out["plain_s_per_round"] / out["batched_s_per_round"]
    out["speedup_pruned_vs_plain"] = out["plain_s_per_round"] / out["pruned_s_per_round"]
    return out


PILOT_WORKLOAD = dict(N=64, d=2, mk=(4, 16), m=8, iters=200, tau=10,
                      desc="single barycenter: N=64 distributions in d=2, m_k~U{4..16} from a 3-component "
                           "Gaussian mixture (sigma=1, means on a radius-5 circle), Dirichlet(1) weights, "
                           "m=8, rho0=2, T=200, tau=10")
RHO0_SWEEP = (0.5, 1.0, 2.0, 4.0, 8.0, 16.0)


def pilot_and_rho_study(d2, ctx, dev, seed, reps=20):
    """The small single-barycenter workload (latency-bound: 5e3 plan entries):
    plan-entry updates/s of one badmm_barycenter call, and the objective after
    T iterations for rho0 in {0.5, ..., 16} under rules R1 and R2 (the
    robustness study of Section 7.1 and the R1/R2 comparison of Table 1), on
    this workload and on the K=10 Gaussian-class clusters at their true labels
    (one update of T=100 iterations of all ten clusters)."""
    W = PILOT_WORKLOAD
    bags = synth.circle_mixture_bags(seed, N=W["N"], d=W["d"], mk=W["mk"])
    co = torch.tensor([0, bags.N], dtype=torch.int64)
    mem = torch.arange(bags.N, dtype=torch.int64)
    x0, w0 = synth.sample_initial_barycenters(seed + 1, bags, co, mem, W["m"])
    bags = bags.to(dev)
    db = d2.DeviceBags(bags.offsets, bags.wt, bags.d, supp=bags.supp)
    co, mem, x0, w0 = co.to(dev), mem.to(dev), x0.to(dev), w0.to(dev)
    T, m = W["iters"], W["m"]
    x, w = x0.clone(), w0.clone()
    plan = torch.empty(bags.n, m, dtype=torch.float32, device=dev)
    obj = torch.empty(1, dtype=torch.float64, device=dev)
    side = torch.cuda.Stream(device=dev)   # graph replay needs a non-default stream
    out = {"workload": W["desc"], "plan_entries": m * bags.n}
    with torch.cuda.stream(side):
        opts = d2.badmm_opts(iters=T, tau=W["tau"])
        for _ in range(3):
            x.copy_(x0)
            w.copy_(w0)
            d2.badmm_barycenter(ctx, db, co, mem, x, w, plan, None, opts, obj)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(side)
        for _ in range(reps):
            x.copy_(x0)
            w.copy_(w0)
            d2.badmm_barycenter(ctx, db, co, mem, x, w, plan, None, opts, obj)
        e1.record(side)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out.update({"ms_per_call": ms, "value": m * bags.n * T / (ms * 1e-3), "unit": UNIT,
                    "note": "latency-bound (about 135 launches of a few microseconds, one CUDA graph)"})
        study = {}
        for rule in ("R1", "R2"):
            row = {}
            for r0 in RHO0_SWEEP:
                x.copy_(x0)
                w.copy_(w0)
                d2.badmm_barycenter(ctx, db, co, mem, x, w, plan, None,
                                    d2.badmm_opts(iters=T, tau=W["tau"], rho0=r0, rule=rule), obj)
                row[str(r0)] = float(obj.item())
            study[rule] = row
        out["objective_after_T"] = study
        # the K=10 Gaussian classes at their true labels
        D = D2_WORKLOAD
        gb = synth.gaussian_class_bags(seed + 2, D["N"], D["d"], D["K"], mk=D["mk"], device=dev)
        gdb = d2.DeviceBags(gb.offsets, gb.wt, gb.d, supp=gb.supp)
        order = torch.sort(gb.labels, stable=True).indices.contiguous()
        gco = torch.zeros(D["K"] + 1, dtype=torch.int64, device=dev)
        gco[1:] = torch.cumsum(torch.bincount(gb.labels, minlength=D["K"]), 0)
        gx0, gw0 = synth.sample_initial_barycenters(seed + 3, gb, gco, order, D["m"])
        nc = (gco[1:] - gco[:-1]).double()
        gobj = torch.empty(D["K"], dtype=torch.float64, device=dev)
        gstudy = {}
        for rule in ("R1", "R2"):
            row = {}
            for r0 in RHO0_SWEEP:
                gx, gw = gx0.clone(), gw0.clone()
                d2.badmm_barycenter(ctx, gdb, gco, order, gx, gw, None, None,
                                    d2.badmm_opts(iters=D["iters"], tau=D["tau"], rho0=r0, rule=rule), gobj)
                row[str(r0)] = float((gobj * nc).sum().item() / gb.N)
            gstudy[rule] = row
        torch.cuda.synchronize()
    out["gaussian_classes_objective_after_T"] = {
        "workload": "K=10 Gaussian classes of the D2-clustering workload at their true labels, one update "
                    "of T=%d iterations; objective = (1/N) sum_c N_c F_c" % D["iters"], **gstudy}
    allv = [v for r in study.values() for v in r.values()]
    out["objective_spread_rel"] = (max(allv) - min(allv)) / min(allv)
    return out


PRUNE_WORKLOAD = dict(N=500_000, d=32, K=256, mk=(16, 64), m=32, r=8, train_pairs=100_000, eval_bags=50_000,
                      desc="learned-pruning assignment: K=256 centroids (m=32, d=32) from one B-ADMM update "
                           "on 256 Gaussian classes (means N(0,4I), sigma=1), N=500,000 distributions, "
                           "m_k~U{16..64}, Dirichlet(1); MLP 32->128->128->64; r=8")


def pruning_at_scale(d2, ctx, dev, seed, steps=1500):
    """Misassignment rate and speedup of the learned pruner against the exact
    full-K assignment (both on the same evaluation bags), plus the pruned
    assignment time over all N bags."""
    W = PRUNE_WORKLOAD
    K, m, r = W["K"], W["m"], W["r"]
    bags = synth.gaussian_class_bags(seed, W["N"], W["d"], K, mk=W["mk"], mu_sigma=2.0, alpha=1.0, device=dev)
    db = d2.DeviceBags(bags.offsets, bags.wt, bags.d, supp=bags.supp)
    lab = bags.labels
    order = torch.sort(lab, stable=True).indices
    co = torch.zeros(K + 1, dtype=torch.int64, device=dev)
    co[1:] = torch.cumsum(torch.bincount(lab, minlength=K), 0)
    x, w = synth.sample_initial_barycenters(seed + 1, bags, co, order, m)
    d2.badmm_barycenter(ctx, db, co, order.contiguous(), x, w, None, None, d2.badmm_opts(iters=100, tau=10))
    out = {"workload": W["desc"]}

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = fn()
        torch.cuda.synchronize()
        return res, time.perf_counter() - t0

    # training pairs: half the 8 nearest centroids by mean distance, half random
    g = torch.Generator(device=dev).manual_seed(seed + 2)
    npairs = W["train_pairs"]
    half = npairs // 2
    tb = torch.randint(0, bags.N, (npairs,), generator=g, device=dev)
    owner = torch.repeat_interleave(torch.arange(bags.N, device=dev), bags.offsets[1:] - bags.offsets[:-1])
    mu_b = torch.zeros(bags.N, W["d"], device=dev).index_add_(0, owner, bags.supp * bags.wt[:, None])
    mu_c = (w[:, :, None] * x).sum(1)
    near = torch.cdist(mu_b[tb[:half]], mu_c).topk(8, largest=False).indices
    pick = torch.randint(0, 8, (half,), generator=g, device=dev)
    pc = torch.empty(npairs, dtype=torch.int32, device=dev)
    pc[:half] = near.gather(1, pick[:, None]).squeeze(1).to(torch.int32)
    pc[half:] = torch.randint(0, K, (npairs - half,), generator=g, device=dev, dtype=torch.int32)
    perm = torch.randperm(npairs, generator=g, device=dev)
    tb, pc = tb[perm].contiguous(), pc[perm].contiguous()
    tg, t_tg = timed(lambda: d2.d2_w2_pairs(ctx, db, x, w, tb, pc))
    pr = d2.Pruner(ctx, W["d"], hidden=128, embed=64, seed=seed + 3)
    losses, t_train = timed(lambda: pr.train(db, x, w, tb, pc, tg, steps=steps, batch=1024, lr=1e-3,
                                             seed=seed + 4))
    _, delta = pr.margin()
    pr.set_margin(r, delta)
    # evaluation bags: exact full K vs pruned on the same bags
    ev = min(W["eval_bags"], bags.N)
    sub = synth.subset_bags(bags, torch.arange(ev, device=dev))
    dsub = d2.DeviceBags(sub.offsets, sub.wt, sub.d, supp=sub.supp)
    d2.d2_assign(ctx, dsub, x, w)  # warm-up
    (le, _), t_exact = timed(lambda: d2.d2_assign(ctx, dsub, x, w))
    (lp, _, st), t_pruned = timed(lambda: d2.d2_assign(ctx, dsub, x, w, prune=pr, want_stats=True))
    (la, _, st_all), t_all = timed(lambda: d2.d2_assign(ctx, db, x, w, prune=pr, want_stats=True))
    mis = float((lp != le).float().mean())
    # the non-learned alternatives on the same evaluation bags: the exact mean
    # term alone as the margin (delta = infinity), the certified lower bounds
    # (Eq. primal relaxations and the mean term; exact), and the learned
    # candidates followed by the certified bounds (exact)
    pr.set_margin(r, 1e30)
    (lm, _, stm), t_mean = timed(lambda: d2.d2_assign(ctx, dsub, x, w, prune=pr, want_stats=True))
    # candidate counts: the exact solves per bag are what a pruned assignment costs
    r_sweep = {}
    for rr in (1, 2, 4, 8):
        pr.set_margin(rr, delta)
        d2.d2_assign(ctx, dsub, x, w, prune=pr)
        (lr_, _, str_), t_r = timed(lambda: d2.d2_assign(ctx, dsub, x, w, prune=pr, want_stats=True))
        (lrb, _, strb), t_rb = timed(lambda: d2.d2_assign(ctx, dsub, x, w, prune=pr, want_stats=True, bounded=True))
        r_sweep[str(rr)] = {"s": t_r, "exact_solves": str_["exact_solves"], "fallbacks": str_["fallbacks"],
                            "misassignment_vs_exact": float((lr_ != le).float().mean()),
                            "then_certified_bounds_s": t_rb, "then_certified_bounds_solves": strb["exact_solves"],
                            "then_certified_bounds_misassignment": float((lrb != le).float().mean())}
    pr.set_margin(r, delta)
    (lb, _, stb), t_bnd = timed(lambda: d2.d2_assign(ctx, dsub, x, w, want_stats=True, bounded=True))
    (lbp, _, stbp), t_bndp = timed(lambda: d2.d2_assign(ctx, dsub, x, w, prune=pr, want_stats=True, bounded=True))
    out["alternatives"] = {
        "mean_term_only": {"s": t_mean, "exact_solves": stm["exact_solves"], "fallbacks": stm["fallbacks"],
                           "misassignment_vs_exact": float((lm != le).float().mean())},
        "certified_bounds": {"s": t_bnd, "exact_solves": stb["exact_solves"],
                             "misassignment_vs_exact": float((lb != le).float().mean())},
        "learned_then_certified_bounds": {"s": t_bndp, "exact_solves": stbp["exact_solves"],
                                          "misassignment_vs_exact": float((lbp != le).float().mean())},
        "elkan": "applies across rounds only (its bounds come from the previous round's centroids); "
                 "compared in d2_round",
        "learned_speedup_vs_certified_bounds": t_bnd / t_pruned,
        "learned_speedup_vs_mean_term_only": t_mean / t_pruned,
        "learned_r_sweep": r_sweep,
        "best_learned_s": min(v["s"] for v in r_sweep.values()),
        "best_learned_speedup_vs_certified_bounds": t_bnd / min(v["s"] for v in r_sweep.values())}
    out.update({"train_pairs": npairs, "target_w2_s": t_tg, "train_steps": steps, "train_s": t_train,
                "loss_first": float(np.mean(losses[:20])), "loss_last": float(np.mean(losses[-20:])),
                "r": r, "delta": delta, "eval_bags": ev,
                "exact_full_K_s": t_exact, "exact_pairs_per_s": ev * K / t_exact,
                "pruned_s": t_pruned, "speedup_vs_full_K": t_exact / t_pruned,
                "misassignment_vs_exact": mis,
                "pruned_exact_solves": st["exact_solves"], "pruned_fallbacks": st["fallbacks"],
                "full_K_solves": ev * K,
                "all_bags_pruned_s": t_all, "all_bags": bags.N, "all_bags_fallbacks": st_all["fallbacks"]})
    return out


DOCS_WORKLOAD = dict(N=200_000, V=50_000, d=300, mk=(10, 60), K=64, m=64, rounds=5, iters=100, tau=10,
                     desc="document-like sparse bags: N=200,000 distributions in d=300 (unit-norm Gaussian "
                          "word vectors from a 50,000-entry seeded vocabulary, stored as indices), "
                          "m_k~U{10..60} distinct words sampled Zipf(1.1), weights = normalised counts; "
                          "K=64, m=64; D2-clustering, 5 rounds x 100 B-ADMM iterations; split-BF16 "
                          "tensor-core cost build")


def docs_clustering(d2, ctx, dev, seed, n_docs=None):
    """D2-clustering of the document-like workload with the tensor-core cost
    build: seconds per round with the learned pruner (trained on 100k exact
    W^2 pairs against the merge-initialised centroids) and the B-ADMM share of
    a round; the exact full-K assignment of the plain form is timed on a
    sample of bags and scaled to all N (its full run takes minutes)."""
    W = dict(DOCS_WORKLOAD)
    if n_docs:
        W["N"] = n_docs
    K, m, R = W["K"], W["m"], W["rounds"]

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = fn()
        torch.cuda.synchronize()
        return res, time.perf_counter() - t0

    bags, t_gen = timed(lambda: synth.document_bags(seed, W["N"], V=W["V"], d=W["d"], mk=W["mk"], device=dev))
    db = d2.DeviceBags(bags.offsets, bags.wt, bags.d, vocab_idx=bags.vocab_idx, vocab=bags.vocab)
    opts = d2.badmm_opts(iters=W["iters"], tau=W["tau"], cost="bf16x3")
    out = {"workload": W["desc"] if not n_docs else W["desc"] + " (N=%d)" % n_docs, "N": bags.N, "support_rows": bags.n, "generate_s": t_gen}
    # centroids of Algorithm 1's initialisation, for the pruner's training pairs
    x0, w0 = d2.d2_merge_init(ctx, db, torch.tensor(pick_ids(bags, K, m, 11), device=dev), m)
    g = torch.Generator(device=dev).manual_seed(seed + 5)
    npairs = 100_000
    pb = torch.randint(0, bags.N, (npairs,), generator=g, device=dev)
    pc = torch.randint(0, K, (npairs,), generator=g, device=dev, dtype=torch.int32)
    tg, t_tg = timed(lambda: d2.d2_w2_pairs(ctx, db, x0, w0, pb, pc))
    pr = d2.Pruner(ctx, bags.d, hidden=128, embed=64, seed=3)
    _, t_train = timed(lambda: pr.train(db, x0, w0, pb, pc, tg, steps=600, batch=1024, lr=2e-3, seed=4))
    _, delta = pr.margin()
    pr.set_margin(8, delta)
    # exact full-K rate on a sample (the plain form's assignment)
    ns = 2000
    sub = synth.subset_bags(bags, torch.arange(ns, device=dev))
    dsub = d2.DeviceBags(sub.offsets, sub.wt, sub.d, vocab_idx=sub.vocab_idx, vocab=sub.vocab)
    d2.d2_assign(ctx, dsub, x0, w0)
    (le, _), t_ex = timed(lambda: d2.d2_assign(ctx, dsub, x0, w0))
    (lp, _, st), t_pr = timed(lambda: d2.d2_assign(ctx, dsub, x0, w0, prune=pr, want_stats=True))
    (lbd, _, stb), t_bd = timed(lambda: d2.d2_assign(ctx, dsub, x0, w0, want_stats=True, bounded=True))
    # D2-clustering, all rounds, timed as one call: the learned pruner with its
    # margin test (fall-back to all K), and the pruner's candidates followed by
    # the certified-bound solves (exact by construction)
    popts = d2.badmm_opts(iters=W["iters"], tau=W["tau"], cost="bf16x3")
    (xq, wq, lq, oq), t_cl = timed(lambda: d2.d2_cluster(ctx, db, K, m, 11, R, popts, prune=pr))
    cs = ctx.cluster_stats()
    # the same with the margin recalibrated against each round's centroids
    ropts = d2.badmm_opts(iters=W["iters"], tau=W["tau"], cost="bf16x3", recalibrate=True)
    (xc, wc, lc, oc), t_rc = timed(lambda: d2.d2_cluster(ctx, db, K, m, 11, R, ropts, prune=pr))
    csr = ctx.cluster_stats()
    out.update({"recalibrated_pruned_s_per_round": t_rc / R, "recalibrated_exact_solves": csr["exact_solves"],
                "recalibrated_fallbacks": csr["fallbacks"], "obj_per_round_recalibrated": oc})
    # certified-bound assignment, the pruner's candidates as first upper
    # bounds in the rounds where its recalibrated margin can pay (exact either way)
    bopts = d2.badmm_opts(iters=W["iters"], tau=W["tau"], cost="bf16x3", assign_bounded=True, recalibrate=True)
    (xr, wr, lr_, orr), t_cp = timed(lambda: d2.d2_cluster(ctx, db, K, m, 11, R, bopts, prune=pr))
    csp = ctx.cluster_stats()
    out.update({"pruned_s_per_round": t_cl / R, "pruned_exact_solves": cs["exact_solves"],
                "pruned_fallbacks": cs["fallbacks"],
                "bounded_recalibrated_s_per_round": t_cp / R, "bounded_recalibrated_exact_solves": csp["exact_solves"],
                "bounded_recalibrated_fallbacks": csp["fallbacks"],
                "labels_equal_recalibrated_vs_bounded": bool(torch.equal(lc, lr_)),
                "obj_per_round": orr, "obj_per_round_pruned": oq})
    # one B-ADMM update of all clusters at the final labels (the update step of a round)
    order = torch.sort(lq.long(), stable=True).indices
    co = torch.zeros(K + 1, dtype=torch.int64, device=dev)
    co[1:] = torch.cumsum(torch.bincount(lq.long(), minlength=K), 0)
    xb, wb = xq.clone(), wq.clone()
    d2.badmm_barycenter(ctx, db, co, order.contiguous(), xb, wb, None, None, opts)
    xb, wb = xq.clone(), wq.clone()
    _, t_b = timed(lambda: d2.badmm_barycenter(ctx, db, co, order.contiguous(), xb, wb, None, None, opts))
    # the same update once more with per-launch CUDA events: the fused plan
    # sweep's HBM roofline on this workload and the kernel split
    xb, wb = xq.clone(), wq.clone()
    ctx.timing(True)
    d2.badmm_barycenter(ctx, db, co, order.contiguous(), xb, wb, None, None, opts)
    torch.cuda.synchronize()
    kt = ctx.timing_read()
    ctx.timing(False)
    f_ms, f_n = kt["sweep_fused"]
    if f_n:
        peak, peak_kind = load_peaks()
        sbytes = BYTES_PER_ENTRY * m * bags.n
        ach = sbytes / (f_ms / f_n * 1e-3) / 1e9
        out["sweep_roofline"] = {"bound": "hbm", "kernel": "k_sweep_pipe (fused B+A pass, default shape)",
                                 "achieved": ach, "peak": peak, "peak_source": peak_kind, "unit": "GB/s",
                                 "frac": ach / peak, "algorithmic_bytes_per_launch": sbytes,
                                 "avg_launch_ms": f_ms / f_n, "launches": f_n}
    out["badmm_kernel_breakdown_ms"] = {k: {"ms": v[0], "launches": v[1]} for k, v in kt.items() if v[1]}
    out.update({"badmm_update_s": t_b, "badmm_updates_per_s": m * bags.n * W["iters"] / t_b,
                "full_K_solves_per_round": bags.N * K,
                "pruner": {"r": 8, "delta": delta, "train_pairs": npairs, "target_s": t_tg, "train_s": t_train,
                           "sample_bags": ns, "misassignment_vs_exact_on_sample": float((lp != le).float().mean()),
                           "sample_exact_solves": st["exact_solves"], "sample_fallbacks": st["fallbacks"]},
                "exact_pairs_per_s": ns * K / t_ex,
                "sample_bounded": {"s": t_bd, "full_K_s": t_ex, "exact_solves": stb["exact_solves"],
                                   "labels_equal_full_K": bool(torch.equal(lbd, le))},
                # (against the merge-initialised centroids; later rounds' LPs take longer)
                "full_K_assign_s_initial_centroids_est": bags.N * K / (ns * K / t_ex)})
    return out


def docs_rounds(d2, ctx, dev, seed, rounds=2):
    """The document workload at full size, a short run: D2-clustering rounds
    (Algorithm 1) with the exact assignment by certified bounds and the
    split-BF16 tensor-core cost build, timed as one d2_cluster call with
    per-launch CUDA events: seconds per round, the exact solver's pair rate,
    the B-ADMM update's share and the fused plan sweep's HBM roofline."""
    W = DOCS_WORKLOAD
    K, m = W["K"], W["m"]
    t0 = time.perf_counter()
    bags = synth.document_bags(seed, W["N"], V=W["V"], d=W["d"], mk=W["mk"], device=dev)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    db = d2.DeviceBags(bags.offsets, bags.wt, bags.d, vocab_idx=bags.vocab_idx, vocab=bags.vocab)
    opts = d2.badmm_opts(iters=W["iters"], tau=W["tau"], cost="bf16x3", assign_bounded=True)
    ctx.timing(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    x, w, lab, objs = d2.d2_cluster(ctx, db, K, m, 11, rounds, opts)
    torch.cuda.synchronize()
    t_cl = time.perf_counter() - t0
    kt = ctx.timing_read()
    ctx.timing(False)
    cs = ctx.cluster_stats()
    out = {"workload": W["desc"].replace("5 rounds", "%d rounds" % rounds), "N": bags.N,
           "support_rows": bags.n, "generate_s": t_gen, "rounds": rounds,
           "s_per_round": t_cl / rounds, "obj_per_round": objs,
           "assignment": "exact (certified lower bounds -- the LP's one-sided relaxations, the means, and an "
                         "entropic dual made feasible by a c-transform -- skip LPs; labels equal to the full N x K "
                         "solve)",
           "exact_solves": cs["exact_solves"], "full_K_pairs": bags.N * K * rounds,
           "kernel_ms": {k: {"ms": v[0], "launches": v[1]} for k, v in kt.items() if v[1]}}
    a_ms, a_n = kt["assign"]
    if a_n:
        out["exact_pairs_per_s"] = cs["exact_solves"] / (a_ms * 1e-3)
    out["bound_s_per_round"] = kt["bound"][0] * 1e-3 / rounds
    out["exact_solve_s_per_round"] = a_ms * 1e-3 / rounds
    f_ms, f_n = kt["sweep_fused"]
    if f_n:
        peak, peak_kind = load_peaks()
        sbytes = BYTES_PER_ENTRY * m * bags.n
        ach = sbytes / (f_ms / f_n * 1e-3) / 1e9
        out["sweep_roofline"] = {"bound": "hbm", "kernel": "k_sweep_pipe (fused B+A pass)", "achieved": ach,
                                 "peak": peak, "peak_source": peak_kind, "unit": "GB/s", "frac": ach / peak,
                                 "algorithmic_bytes_per_launch": sbytes, "avg_launch_ms": f_ms / f_n,
                                 "launches": f_n}
    upd = sum(kt[k][0] for k in ("sweep_fused", "sweep_half", "cost", "support"))
    out["badmm_update_ms_per_round"] = upd / rounds
    out["badmm_updates_per_s"] = m * bags.n * W["iters"] * rounds / max(upd * 1e-3, 1e-12)
    del bags, db
    torch.cuda.empty_cache()
    return out


def grouped_resident(d2, dev, bags, co, x0, w0, W, T, entries, steps, groups, cost, dist, world):
    """The same step with inputs resident in HBM, issued as `groups` cluster
    groups of about equal support rows round-robin on two streams (one
    context each): independent clusters, so the groups' launches overlap each
    other's tails and the HBM-bound sweeps overlap the cost builds."""
    K, m, d = W["clusters"], W["m"], W["d"]
    off = bags.offsets
    n = bags.n
    rows_at = off[co].cpu()
    cuts = [0] + [int(torch.searchsorted(rows_at, torch.tensor(n * g // groups))) for g in range(1, groups)] + [K]
    cuts = sorted(set(cuts))
    co_h = co.cpu()
    off_h = off.cpu()
    x = torch.empty_like(x0)
    w = torch.empty_like(w0)
    obj = torch.empty(K, dtype=torch.float64, device=dev)
    plan = torch.empty(n, m, dtype=torch.float32, device=dev)
    parts = []
    for c0, c1 in zip(cuts[:-1], cuts[1:]):
        b0, b1 = int(co_h[c0]), int(co_h[c1])
        r0, r1 = int(off_h[b0]), int(off_h[b1])
        gb = d2.DeviceBags((off[b0:b1 + 1] - r0).contiguous(), bags.wt[r0:r1], d, supp=bags.supp[r0:r1],
                           max_mk=W["mk"][1])
        parts.append(dict(c0=c0, c1=c1, r0=r0, r1=r1, bags=gb, co=(co[c0:c1 + 1] - b0).contiguous(),
                          mem=torch.arange(b1 - b0, dtype=torch.int64, device=dev)))
    slots = [dict(stream=torch.cuda.Stream(device=dev), ctx=d2.Context(dev.index)) for _ in range(2)]
    opts = d2.badmm_opts(iters=T, tau=W["tau"], cost=cost, graph=False)

    def one_step():
        for gi, p in enumerate(parts):
            sl = slots[gi % 2]
            with torch.cuda.stream(sl["stream"]):
                xg, wg = x[p["c0"]:p["c1"]], w[p["c0"]:p["c1"]]
                xg.copy_(x0[p["c0"]:p["c1"]])
                wg.copy_(w0[p["c0"]:p["c1"]])
                d2.badmm_barycenter(sl["ctx"], p["bags"], p["co"], p["mem"], xg, wg, plan[p["r0"]:p["r1"]], None,
                                    opts, obj[p["c0"]:p["c1"]])

    main = torch.cuda.current_stream(dev)
    for sl in slots:
        sl["stream"].wait_stream(main)
    one_step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(main)
    for sl in slots:
        sl["stream"].wait_event(e0)
    for _ in range(steps):
        one_step()
    for sl in slots:
        ev = torch.cuda.Event()
        ev.record(sl["stream"])
        main.wait_event(ev)
    e1.record(main)
    torch.cuda.synchronize()
    assert torch.isfinite(obj).all()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, dev) / steps
    for sl in slots:
        sl["ctx"].close()
    del plan
    return {"value": job_rate(entries, T, world, ms), "ms_per_step": ms, "groups": len(parts), "steps": steps}


def e2e_pipelined(d2, dev, h, W, T, entries, steps, groups, cost, dist, world):
    """End to end through the public API from pinned host buffers: every step
    copies its inputs host -> device (offsets, weights, supports, clustering,
    initial barycenters), runs badmm_barycenter and copies x, w and the
    objectives back.  The clusters are split into `groups` groups of about
    equal support rows, issued round-robin on two streams, each with its own
    context and device buffers, so the copies of group g+1 overlap the B-ADMM
    update of group g (clusters are independent in the update step)."""
    co_h, off_h = h["co"], h["offsets"]
    K, m, d = W["clusters"], W["m"], W["d"]
    n = int(off_h[-1])
    rows_at = off_h[co_h]                       # first support row of each cluster (K+1)
    cuts = [0]
    for g in range(1, groups):
        cuts.append(int(torch.searchsorted(rows_at, torch.tensor(n * g // groups))))
    cuts.append(K)
    cuts = sorted(set(cuts))
    parts = []
    for c0, c1 in zip(cuts[:-1], cuts[1:]):
        b0, b1 = int(co_h[c0]), int(co_h[c1])
        r0, r1 = int(off_h[b0]), int(off_h[b1])
        parts.append(dict(c0=c0, c1=c1, b0=b0, b1=b1, r0=r0, r1=r1,
                          off=(off_h[b0:b1 + 1] - r0).pin_memory(),
                          co=(co_h[c0:c1 + 1] - b0).pin_memory(),
                          mem=torch.arange(b1 - b0, dtype=torch.int64).pin_memory()))
    out_x = torch.empty_like(h["x0"]).pin_memory()
    out_w = torch.empty_like(h["w0"]).pin_memory()
    out_o = torch.empty(K, dtype=torch.float64).pin_memory()
    nb_max = max(p["b1"] - p["b0"] for p in parts)
    nr_max = max(p["r1"] - p["r0"] for p in parts)
    nc_max = max(p["c1"] - p["c0"] for p in parts)
    slots = []
    for _ in range(2):
        slots.append(dict(stream=torch.cuda.Stream(device=dev), ctx=d2.Context(dev.index),
                          off=torch.empty(nb_max + 1, dtype=torch.int64, device=dev),
                          wt=torch.empty(nr_max, dtype=torch.float32, device=dev),
                          supp=torch.empty(nr_max, d, dtype=torch.float32, device=dev),
                          co=torch.empty(nc_max + 1, dtype=torch.int64, device=dev),
                          mem=torch.empty(nb_max, dtype=torch.int64, device=dev),
                          x=torch.empty(nc_max, m, d, dtype=torch.float32, device=dev),
                          w=torch.empty(nc_max, m, dtype=torch.float32, device=dev),
                          plan=torch.empty(nr_max, m, dtype=torch.float32, device=dev),
                          obj=torch.empty(nc_max, dtype=torch.float64, device=dev)))
    opts = d2.badmm_opts(iters=T, tau=W["tau"], cost=cost, graph=False)
    bi = sum(t.numel() * t.element_size() for t in h.values())
    bo = sum(t.numel() * t.element_size() for t in (out_x, out_w, out_o))

    def one_step():
        for gi, p in enumerate(parts):
            sl = slots[gi % 2]
            nb, nr, nc = p["b1"] - p["b0"], p["r1"] - p["r0"], p["c1"] - p["c0"]
            with torch.cuda.stream(sl["stream"]):
                off, wt, supp = sl["off"][:nb + 1], sl["wt"][:nr], sl["supp"][:nr]
                cog, memg = sl["co"][:nc + 1], sl["mem"][:nb]
                x, w, obj = sl["x"][:nc], sl["w"][:nc], sl["obj"][:nc]
                off.copy_(p["off"], non_blocking=True)
                wt.copy_(h["wt"][p["r0"]:p["r1"]], non_blocking=True)
                supp.copy_(h["supp"][p["r0"]:p["r1"]], non_blocking=True)
                cog.copy_(p["co"], non_blocking=True)
                memg.copy_(p["mem"], non_blocking=True)
                x.copy_(h["x0"][p["c0"]:p["c1"]], non_blocking=True)
                w.copy_(h["w0"][p["c0"]:p["c1"]], non_blocking=True)
                eb = d2.DeviceBags(off, wt, d, supp=supp, max_mk=W["mk"][1])
                d2.badmm_barycenter(sl["ctx"], eb, cog, memg, x, w, sl["plan"][:nr], None, opts, obj)
                out_x[p["c0"]:p["c1"]].copy_(x, non_blocking=True)
                out_w[p["c0"]:p["c1"]].copy_(w, non_blocking=True)
                out_o[p["c0"]:p["c1"]].copy_(obj, non_blocking=True)

    one_step()  # untimed: workspaces grow to their sizes
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    main = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(main)
    for sl in slots:
        sl["stream"].wait_event(e0)
    for _ in range(steps):
        one_step()
    for sl in slots:
        ev = torch.cuda.Event()
        ev.record(sl["stream"])
        main.wait_event(ev)
    e1.record(main)
    torch.cuda.synchronize()
    assert torch.isfinite(out_o).all()
    e_ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    e_step = e_ms / steps
    for sl in slots:
        sl["ctx"].close()
    return {"value": job_rate(entries, T, world, e_step), "unit": UNIT, "ms_per_step": e_step, "steps": steps,
            "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo, "groups": len(parts),
            "pipeline": "%d cluster groups round-robin on 2 streams, one context each; the host->device "
                        "copies of a group overlap the B-ADMM update of the previous one" % len(parts)}


def pick_ids(bags, K, m, seed):
    """The K bags d2_cluster seeds its centroids from (SplitMix64 partial
    Fisher-Yates over the ids with m_k >= m), for the plain-form replay."""
    M = (1 << 64) - 1
    sizes = (bags.offsets[1:] - bags.offsets[:-1]).cpu().tolist()
    thr = min(m, sorted(sizes, reverse=True)[K - 1])
    elig = [k for k, s_ in enumerate(sizes) if s_ >= thr]
    st = seed & M
    for t in range(K):
        st = (st + 0x9E3779B97F4A7C15) & M
        z = st
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        z ^= z >> 31
        j = t + z % (len(elig) - t)
        elig[t], elig[j] = elig[j], elig[t]
    return elig[:K]


def oracle_sample(name, seed, budget_s):
    """Times the FP64 oracle on whole clusters of a CPU draw of the workload
    (smallest clusters first) for about budget_s seconds; returns
    (entry-updates/s, description)."""
    from oracle import badmm_barycenter as oracle_badmm
    W = WORKLOADS[name]
    n_cl = 64
    bags, co, mem = synth.ragged_cluster_bags(seed, n_cl, d=W["d"], nc=W["nc"], mk=W["mk"], mu_sigma=3.0,
                                              device="cpu")
    x0, w0 = synth.sample_initial_barycenters(seed + 1, bags, co, mem, W["m"])
    sizes = (co[1:] - co[:-1]).tolist()
    order = sorted(range(n_cl), key=lambda c: sizes[c])
    T, tau, m = W["iters"], W["tau"], W["m"]
    done_entries, spent, used = 0, 0.0, 0
    for c in order:
        ids = mem[int(co[c]):int(co[c + 1])].tolist()
        members = [bags.bag(k) for k in ids]
        t0 = time.perf_counter()
        oracle_badmm(members, x0[c].double().numpy(), w0[c].double().numpy(), T=T, tau=tau)
        spent += time.perf_counter() - t0
        done_entries += m * sum(y.shape[0] for y, _ in members) * T
        used += 1
        if spent >= budget_s:
            break
    desc = ("%d whole clusters (%d..%d members) of a CPU draw of the same recipe, T=%d, tau=%d, "
            "single-threaded numpy FP64" % (used, sizes[order[0]], sizes[order[used - 1]], T, tau))
    return done_entries / spent, desc, spent


def oracle_sample_all_cores(name, seed, budget_s):
    """The same oracle on every host core: whole clusters of the CPU draw in a
    spawned process pool (one single-threaded oracle per process), about
    budget_s seconds of wall time; returns (entry-updates/s, desc, cores)."""
    import multiprocessing as mp
    from oracle.pool import barycenter_job
    W = WORKLOADS[name]
    n_cl = 64
    bags, co, mem = synth.ragged_cluster_bags(seed, n_cl, d=W["d"], nc=W["nc"], mk=W["mk"], mu_sigma=3.0,
                                              device="cpu")
    x0, w0 = synth.sample_initial_barycenters(seed + 1, bags, co, mem, W["m"])
    sizes = (co[1:] - co[:-1]).tolist()
    order = sorted(range(n_cl), key=lambda c: sizes[c])
    T, tau, m = W["iters"], W["tau"], W["m"]
    cores = os.cpu_count() or 1
    # one pass of the single-threaded rate sizes the batch to the budget
    rate1, _, _ = oracle_sample(name, seed, min(3.0, budget_s / 4))
    want = rate1 * cores * budget_s
    jobs, entries, used = [], 0, 0
    for c in order:
        ids = mem[int(co[c]):int(co[c + 1])].tolist()
        members = [bags.bag(k) for k in ids]
        jobs.append((members, x0[c].double().numpy(), w0[c].double().numpy(), T, tau))
        entries += m * sum(y.shape[0] for y, _ in members) * T
        used += 1
        if entries >= want:
            break
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(barycenter_job, jobs[:cores])  # start-up and imports, untimed
        t0 = time.perf_counter()
        pool.map(barycenter_job, jobs, chunksize=1)
        spent = time.perf_counter() - t0
    desc = ("%d whole clusters (%d..%d members) of a CPU draw of the same recipe, T=%d, tau=%d, numpy FP64, "
            "one single-threaded oracle per process on %d processes" % (used, sizes[order[0]],
                                                                        sizes[order[used - 1]], T, tau, cores))
    return entries / spent, desc, cores


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    name = args.workload
    W = WORKLOADS[name]
    vals = []
    for s in range(args.warmup + args.steps):
        v, desc, spent = oracle_sample(name, 1234, args.ref_budget)
        if s >= args.warmup:
            vals.append((v, spent))
    value = statistics.median(v for v, _ in vals)
    ms = statistics.median(t for _, t in vals) * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": W["desc"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_probe(args):
    """Small single-kernel cases for profiling (ncu captures of one launch):
    assign_docs : exact W^2 of 4,000 document bags (d = 300, Zipf words from a
                  50,000-word vocabulary) against K = 64 merge-initialised
                  centroids of m = 64 points, solved once warm and once timed;
    bound_docs  : bounded exact assignment (certified and entropic dual
                  bounds) of 8,000 document bags against K = 64
                  merge-initialised centroids of m = 64 points;
    mlp_embed   : the pruning network's embedding (d = 32, H = 128, E = 64) of
                  50,000 Gaussian-class bags, tensor-core and CUDA-core forwards;
    support     : one badmm_barycenter call (T = 11, tau = 10: one support
                  update) on 256 clusters of the ragged recipe (m = 32,
                  d = 64) with the split-BF16 cost and the CUDA-core support
                  partials;
    support_tc  : the same with the tensor-core support update;
    support_docs: the same call on 100,000 document bags (d = 300, Zipf words
                  of a 50,000-word vocabulary) in 64 random clusters, m = 64.
    Prints one JSON line with the timing."""
    import paper_1510_00012_gb300 as d2
    from paper_1510_00012_gb300 import build
    build.build()
    dev = torch.device("cuda", 0)
    ctx = d2.Context(0)
    out = {"probe": args.probe}
    if args.probe == "assign_docs":
        N = args.probe_n or 4000
        bags = synth.document_bags(5, N, V=50000, d=300, mk=(10, 60), device=dev)
        db = d2.DeviceBags(bags.offsets, bags.wt, bags.d, vocab_idx=bags.vocab_idx, vocab=bags.vocab)
        ctx.set_flow_store(args.probe_store)
        ids = torch.arange(0, 64 * 37, 37, device=dev) % N
        x, w = d2.d2_merge_init(ctx, db, ids, 64)
        d2.d2_assign(ctx, db, x, w)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, _, st = d2.d2_assign(ctx, db, x, w, want_stats=True)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        out.update({"pairs": N * 64, "s": t, "pairs_per_s": N * 64 / t, "flow_store": args.probe_store,
                    "limit_hits": st["limit_hits"]})
    elif args.probe == "bound_docs":
        N = args.probe_n or 8000
        bags = synth.document_bags(5, N, V=50000, d=300, mk=(10, 60), device=dev)
        db = d2.DeviceBags(bags.offsets, bags.wt, bags.d, vocab_idx=bags.vocab_idx, vocab=bags.vocab)
        ids = torch.arange(0, 64 * 37, 37, device=dev) % N
        x, w = d2.d2_merge_init(ctx, db, ids, 64)
        d2.d2_assign(ctx, db, x, w, bounded=True)
        torch.cuda.synchronize()
        settings = [(-1, 0.0)]
        if args.probe_dual:
            settings = [tuple(float(v) for v in p.split(",")) for p in args.probe_dual.split(";")]
        runs = []
        for iters, eps in settings:
            ctx.set_dual_bound(int(iters), eps)
            ctx.timing(True)
            t0 = time.perf_counter()
            _, _, st = d2.d2_assign(ctx, db, x, w, want_stats=True, bounded=True)
            torch.cuda.synchronize()
            t = time.perf_counter() - t0
            kt = ctx.timing_read()
            runs.append({"dual_iters": int(iters), "dual_eps": eps, "s": t, "exact_solves": st["exact_solves"],
                         "bound_ms": kt["bound"][0], "assign_ms": kt["assign"][0]})
        ctx.set_dual_bound(-1, 0.0)
        out.update({"pairs": N * 64, "runs": runs})
    elif args.probe == "mlp_embed":
        N = args.probe_n or 50000
        bags = synth.gaussian_class_bags(3, N, 32, 64, mk=(16, 64), device=dev)
        db = d2.DeviceBags(bags.offsets, bags.wt, bags.d, supp=bags.supp)
        pr = d2.Pruner(ctx, 32, hidden=128, embed=64, seed=1)
        ids = torch.arange(N, dtype=torch.int64, device=dev)
        pr.embed(db, ids)
        runs = {}
        for path in ("auto", "cuda_cores"):
            ctx.set_prune_forward(path)
            pr.embed(db, ids)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            pr.embed(db, ids)
            torch.cuda.synchronize()
            runs[path] = time.perf_counter() - t0
        ctx.set_prune_forward("auto")
        out.update({"bags": N, "points": bags.n, "s": runs})
    elif args.probe in ("support", "support_tc", "support_docs"):
        if args.probe == "support_docs":
            N, K, m = args.probe_n or 100000, 64, 64
            bags = synth.document_bags(5, N, V=50000, d=300, mk=(10, 60), device=dev)
            db = d2.DeviceBags(bags.offsets, bags.wt, bags.d, vocab_idx=bags.vocab_idx, vocab=bags.vocab)
            lab = torch.randint(0, K, (N,), generator=torch.Generator().manual_seed(9))
            co = torch.zeros(K + 1, dtype=torch.int64)
            co[1:] = torch.cumsum(torch.bincount(lab, minlength=K), 0)
            co, mem = co.to(dev), torch.sort(lab, stable=True).indices.to(dev)
            row_bytes = 4 * (m + 300)
        else:
            m = 32
            bags, co, mem = synth.ragged_cluster_bags(7, args.probe_n or 256, device=dev)
            db = d2.DeviceBags(bags.offsets, bags.wt, bags.d, supp=bags.supp)
            row_bytes = 4 * (m + 64)
        x0, w0 = synth.sample_initial_barycenters(8, bags, co, mem, m)
        opts = d2.badmm_opts(iters=11, tau=10, cost="bf16x3", graph=False, support_tc=args.probe == "support_tc")
        x, w = x0.clone(), w0.clone()
        d2.badmm_barycenter(ctx, db, co, mem, x, w, None, None, opts)
        torch.cuda.synchronize()
        ctx.timing(True)
        x, w = x0.clone(), w0.clone()
        d2.badmm_barycenter(ctx, db, co, mem, x, w, None, None, opts)
        torch.cuda.synchronize()
        kt = ctx.timing_read()
        s_ms, s_n = kt["support"]
        out.update({"rows": bags.n, "support_ms": s_ms / s_n, "row_bytes": row_bytes,
                    "support_gbs": bags.n * row_bytes / (s_ms / s_n * 1e-3) / 1e9})
    assert ctx.device_errors() == 0
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="own", choices=["own", "reference"])
    ap.add_argument("--workload", default="ragged4096", choices=sorted(WORKLOADS))
    ap.add_argument("--seed", type=int, default=2024)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--e2e-groups", type=int, default=8, help="cluster groups pipelined in the e2e run")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--ref-budget", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-d2", action="store_true", help="skip the D2-clustering s/round comparison")
    ap.add_argument("--no-pruning", action="store_true", help="skip the learned-pruning assignment at scale")
    ap.add_argument("--no-pilot", action="store_true", help="skip the N=64 pilot and the rho0 / R1-R2 study")
    ap.add_argument("--no-docs-rounds", action="store_true", help="skip the two document-workload rounds")
    ap.add_argument("--dual-iters", type=int, default=None,
                    help="Sinkhorn iterations of the entropic dual bound in the bounded assignments of the "
                         "secondary workloads (default: the library's; a positive count also applies below m = 32)")
    ap.add_argument("--docs-n", type=int, default=None, help="document count of --docs (default 200,000)")
    ap.add_argument("--docs", action="store_true",
                    help="also run D2-clustering of the 200k document-like bags (d=300, K=64, m=64)")
    ap.add_argument("--cost", default="bf16x3", choices=["fp32", "bf16", "bf16x3", "bf16x6"],
                    help="cost-build precision (bf16*: tensor cores)")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default sweep launch shape")
    ap.add_argument("--no-grouped", action="store_true", help="skip the grouped two-stream measurement")
    ap.add_argument("--no-split", action="store_true",
                    help="one stream per call (no D2_SPLIT_STREAMS) for the timed steps")
    ap.add_argument("--no-cost-variants", action="store_true",
                    help="skip the timing of the other cost-build precisions")
    ap.add_argument("--probe", default=None, choices=["assign_docs", "bound_docs", "mlp_embed", "support", "support_tc", "support_docs"],
                    help="run one small profiling case instead of the benchmark")
    ap.add_argument("--probe-n", type=int, default=0)
    ap.add_argument("--probe-dual", default=None,
                    help="bound_docs: 'iters,eps;iters,eps;...' settings of the entropic dual bound")
    ap.add_argument("--probe-store", default="auto", choices=["auto", "dense", "sparse"])
    args = ap.parse_args()
    if args.probe:
        return run_probe(args)
    if args.impl == "reference":
        return run_reference(args)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    import paper_1510_00012_gb300 as d2
    from paper_1510_00012_gb300 import build
    build.build()
    W = WORKLOADS[args.workload]

    t0 = time.time()
    bags, co, mem, x0, w0 = make_workload(args.workload, rank_seed(args.seed, rank), dev)
    torch.cuda.synchronize()
    log("[bench] rank %d: generated %d distributions, %d support rows in %.1fs"
        % (rank, bags.N, bags.n, time.time() - t0))
    db = d2.DeviceBags(bags.offsets, bags.wt, bags.d, supp=bags.supp)
    K, m, T = W["clusters"], W["m"], W["iters"]
    entries = m * bags.n
    x = x0.clone()
    w = w0.clone()
    plan = torch.empty(bags.n, m, dtype=torch.float32, device=dev)
    obj = torch.empty(K, dtype=torch.float64, device=dev)
    opts = d2.badmm_opts(iters=T, tau=W["tau"], cost=args.cost, split_streams=not args.no_split)
    ctx = d2.Context(local)
    if args.dual_iters is not None:
        ctx.set_dual_bound(args.dual_iters)

    def step(o=opts):
        x.copy_(x0)
        w.copy_(w0)
        d2.badmm_barycenter(ctx, db, co, mem, x, w, plan, None, o, obj)

    # the first warm-up step (one call, no split) lets the autotuner pick the
    # sweep's launch shape; split calls hand it to their child contexts
    for i in range(args.warmup):
        step(d2.badmm_opts(iters=T, tau=W["tau"], cost=args.cost, autotune=not args.no_autotune)
             if i == 0 else opts)
    torch.cuda.synchronize()
    assert torch.isfinite(obj).all(), "non-finite objective"

    sampler = ClockSampler(dev)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = ctx.launch_count()
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = ctx.launch_count() - l0
    clocks = sampler.stop()
    ms_total = max_over_ranks(ev0.elapsed_time(ev1), dist, dev)
    ms_step = ms_total / args.steps
    value = job_rate(entries, T, world, ms_step)
    # one more step, as one call on one stream, with per-launch CUDA events for
    # the kernel split and the rooflines of isolated launches
    ctx.timing(True)
    step(d2.badmm_opts(iters=T, tau=W["tau"], cost=args.cost))
    torch.cuda.synchronize()
    kt = ctx.timing_read()
    ctx.timing(False)
    kt_steps = 1

    # roofline of the dominant kernel (the fused plan sweep)
    f_ms, f_n = kt["sweep_fused"]
    peak, peak_kind = load_peaks()
    roof = None
    if f_n:
        avg_s = f_ms / f_n * 1e-3
        achieved = BYTES_PER_ENTRY * entries / avg_s / 1e9
        tpe = sweep_traffic_per_entry()
        tun = ctx.sweep_tuning(m)
        kname = "k_sweep_pipe<4, 2, 4> (fused B+A pass)"
        if tun is not None:
            cd = tun["candidates"][tun["chosen"]]
            kname = "%s (fused B+A pass; %d lanes/row, %d float4/lane, %d CTAs/SM, autotuned)" % (
                "k_sweep_pipe" if cd["kind"] == "pipelined" else "k_sweep", cd["lanes_per_row"],
                cd["float4_per_lane"], cd["ctas_per_sm"])
        roof = {"bound": "hbm", "kernel": kname, "achieved": achieved,
                "peak": peak, "peak_source": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None if tpe is None else tpe * entries,
                "algorithmic_bytes_per_launch": BYTES_PER_ENTRY * entries,
                "avg_launch_ms": f_ms / f_n, "launches": f_n,
                "share_of_step": f_ms / kt_steps / max(ms_step, 1e-9)}
    breakdown = {k: {"ms": v[0] / kt_steps, "launches": v[1] // kt_steps} for k, v in kt.items() if v[1]}
    # the cost build (tensor cores for d >= 32): HBM roofline of its launches
    c_ms, c_n = kt["cost"]
    cost_roof = None
    if c_n:
        cbytes = bags.n * 4 * (W["d"] + m)  # read the support rows, write the cost rows (FP32)
        c_ach = cbytes / (c_ms / c_n * 1e-3) / 1e9
        cost_roof = {"bound": "hbm", "kernel": "k_cost_tc<%d>" % {"bf16": 1, "bf16x3": 2, "bf16x6": 3}[args.cost]
                     if args.cost != "fp32" else "k_cost_pipe<32>", "precision": args.cost,
                     "achieved": c_ach, "peak": peak, "unit": "GB/s", "frac": c_ach / peak,
                     "algorithmic_bytes_per_launch": cbytes, "avg_launch_ms": c_ms / c_n}

    grouped = None
    if not args.no_grouped:
        grouped = grouped_resident(d2, dev, bags, co, x0, w0, W, T, entries, max(2, args.steps // 2),
                                   args.e2e_groups, args.cost, dist, world)

    # the same step with the other cost-build precisions (fewer steps)
    variants = None
    if not args.no_cost_variants:
        variants = {}
        for prec in ("fp32", "bf16", "bf16x3", "bf16x6"):
            if prec == args.cost:
                continue
            vopts = d2.badmm_opts(iters=T, tau=W["tau"], cost=prec)
            for _ in range(1):
                x.copy_(x0)
                w.copy_(w0)
                d2.badmm_barycenter(ctx, db, co, mem, x, w, plan, None, vopts, obj)
            ctx.timing(True)
            torch.cuda.synchronize()
            v0, v1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            v0.record(stream)
            for _ in range(2):
                x.copy_(x0)
                w.copy_(w0)
                d2.badmm_barycenter(ctx, db, co, mem, x, w, plan, None, vopts, obj)
            v1.record(stream)
            torch.cuda.synchronize()
            vkt = ctx.timing_read()
            ctx.timing(False)
            vms = max_over_ranks(v0.elapsed_time(v1), dist, dev) / 2
            variants[prec] = {"value": job_rate(entries, T, world, vms), "ms_per_step": vms,
                              "cost_ms_per_launch": vkt["cost"][0] / max(vkt["cost"][1], 1)}
        ctx.device_errors()

    # end to end through the public API from pinned host buffers
    e2e = None
    if not args.no_e2e and args.e2e_steps > 0:
        h = {k: t.cpu().pin_memory() for k, t in (("offsets", bags.offsets), ("wt", bags.wt),
                                                  ("supp", bags.supp), ("co", co), ("mem", mem),
                                                  ("x0", x0), ("w0", w0))}
        del bags, db, plan
        torch.cuda.empty_cache()
        e2e = e2e_pipelined(d2, dev, h, W, T, entries, args.e2e_steps, args.e2e_groups, args.cost, dist, world)

    d2cmp = None
    if rank == 0 and not args.no_d2:
        try:
            d2cmp = d2_round_comparison(d2, ctx, dev, args.seed + 17)
        except Exception as exc:  # reported, never hides the main metric
            d2cmp = {"error": repr(exc)}

    pilot = None
    if rank == 0 and not args.no_pilot:
        try:
            pilot = pilot_and_rho_study(d2, ctx, dev, args.seed + 23)
        except Exception as exc:
            pilot = {"error": repr(exc)}

    docs_short = None
    if rank == 0 and not args.no_docs_rounds and not args.docs:
        try:
            docs_short = docs_rounds(d2, ctx, dev, args.seed + 41)
        except Exception as exc:
            docs_short = {"error": repr(exc)}

    prune_res = None
    if rank == 0 and not args.no_pruning:
        try:
            prune_res = pruning_at_scale(d2, ctx, dev, args.seed + 31)
        except Exception as exc:
            prune_res = {"error": repr(exc)}

    docs_res = None
    if rank == 0 and args.docs:
        try:
            docs_res = docs_clustering(d2, ctx, dev, args.seed + 41, args.docs_n)
        except Exception as exc:
            docs_res = {"error": repr(exc)}

    cpu = None
    cpu_all = None
    if rank == 0 and not args.no_cpu_baseline:
        v, desc, _ = oracle_sample(args.workload, args.seed, args.cpu_budget)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc}
        try:
            va, desca, cores = oracle_sample_all_cores(args.workload, args.seed, args.cpu_budget)
            cpu_all = {"value": va, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desca}
        except Exception as exc:
            cpu_all = {"error": repr(exc)}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": W["desc"], "clusters": K, "distributions_per_gpu": int(mem.numel()),
                           "support_rows_per_gpu": int(entries // m), "plan_entries_per_gpu": int(entries),
                           "iters": T, "cost_precision": args.cost,
                           "split_streams": not args.no_split, "l2": "inputs larger than L2 (Pi, Lambda, C: %.1f GB per GPU)"
                           % (12 * entries / 1e9),
                           "parallelism": "independent problem per GPU" if world > 1 else "single GPU"}
                          | ({"dual_bound_iters": args.dual_iters} if args.dual_iters is not None else {}),
                "roofline": roof, "cost_roofline": cost_roof, "cost_variants": variants,
                "sweep_autotune": ctx.sweep_tuning(m), "grouped_two_streams": grouped,
                "kernel_breakdown_ms_per_step": breakdown, "cpu_baseline": cpu,
                "e2e": e2e, "gpu_launches": launches, "clocks": clocks, "d2_round": d2cmp,
                "cpu_baseline_all_cores": cpu_all}
        if pilot is not None:
            line["pilot"] = pilot
        if docs_short is not None:
            line["docs_rounds"] = docs_short
        if prune_res is not None:
            line["pruning"] = prune_res
        if docs_res is not None:
            line["docs_clustering"] = docs_res
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
