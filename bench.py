#!/usr/bin/env python3
"""Throughput of the MAM iteration on one GB300 (plan-entry updates / s).

A step is one iteration of Algorithm 1: the fused column kernel (Step 2 for
every plan column of the index set, with the Step 3 row sums) and the
averaging kernel (Step 3 completion, Step 1 and t^k).  The default workload
is the largest one that fits one GPU: 100 seeded 100x100 Gaussian-mixture
images with unequal masses (the unbalanced problem, gamma = 0.01), R = 10000
grid points, 1.8e9 plan entries, FP32 plans and BF16 costs, 4 bundles of
Remark 2 (one bundle, about a quarter of the measures, per iteration),
rho = 100.  Every step streams about 4.4 GB, far more than L2, so no flush
is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Besides the headline it carries:
  nested_ellipses_f32   the same measurement on the 10-measure, R = 3600
                        nested-ellipse workload with FP32 costs;
  forms                 the mixed-precision, batched and differentiated forms
                        against the plain FP32 path on time to a 1e-4 gap;
  cpu_baseline          the FP64 oracle on the host cores (one thread and
                        all cores) on a bounded sample of the workload.
Under torchrun every rank solves its own seeded replica (independent
problems, weak scaling, no collective on the data path).  ``--impl
reference`` times the FP64 oracle on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MAM plan-entry updates/s"
UNIT = "plan-entry updates/s"
FALLBACK_HBM_GBS = 6800.0
NAMES = {1: "blobs16_M3_R256", 2: "nested_ellipses60_M10_R3600",
         3: "strokes28_256problems_R784", 4: "mixture40_M8_R1600",
         5: "mixture100_M100_R10000_unbalanced",
         6: "nested_ellipses60_M10_free_support_grid_R349281"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", type=int, default=5, choices=[1, 2, 3, 4, 5, 6],
                    help="1-5: the five synthetic workloads; 6: the nested ellipses on "
                         "their free-support grid (R = 349281, one cluster per column)")
    ap.add_argument("--measures", type=int, default=None,
                    help="keep only the first N measures of each problem (small cases "
                         "for profiling)")
    ap.add_argument("--cost-layout", default="per_column", choices=["per_column", "shared"],
                    help="shared: one cost matrix for measures on a common support")
    ap.add_argument("--cost-dtype", default=None, choices=["f32", "bf16", "f16"])
    ap.add_argument("--plan-layout", default="dense", choices=["dense", "sparse"],
                    help="sparse: plans stored as the (row, value) pairs of pihat "
                         "(mam_desc.plan_layout)")
    ap.add_argument("--sparse-slots", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the time-to-gap comparison of the three forms")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the nested-ellipse FP32 line")
    ap.add_argument("--autotune", action="store_true")
    ap.add_argument("--shard", action="store_true",
                    help="under torchrun: one problem, its measures split over the ranks "
                         "(mam_create_sharded, NCCL all-reduce of p's partial sums; strong "
                         "scaling) instead of one replica per rank")
    ap.add_argument("--eta", type=float, default=None,
                    help="capped columns (the full unbalanced extension: projection onto "
                         "Delta_<=(q_s), cost alpha_m (d - eta)) with this eta")
    ap.add_argument("--gap-ref-iters", type=int, default=50000)
    return ap.parse_args()


def workload(idx, rank=0):
    from workloads import generators as G
    if idx == 1:
        return [G.config1(rank)], "f32"
    if idx == 2:
        return [G.config2(rank)], "f32"
    if idx == 3:
        return G.config3(256, i0=256 * rank), "bf16"
    if idx == 4:
        return [G.config4(rank)], "f32"
    if idx == 6:
        return [G.config2_free_support(rank)], "f32"
    return [G.config5(rank)], "bf16"


def first_measures(probs, n):
    """The first n measures of each problem (the same images, sizes and
    costs; for profiling a smaller case of a workload)."""
    import copy
    out = []
    for p in probs:
        sub = copy.copy(p)
        k = min(n, p.M)
        sub.q = list(p.q[:k])
        sub.zeta = list(p.zeta[:k])
        sub.alpha = np.full(k, 1.0 / k)
        if p.n_bundles > k:
            sub.n_bundles = k
        out.append(sub)
    return out


def describe(idx, probs, cost_dtype, T, entries):
    p0 = probs[0]
    return {"workload": NAMES[idx], "problems": len(probs),
            "measures": int(sum(p.M for p in probs)), "R": p0.R,
            "kept_columns": int(T), "plan_entries": int(entries),
            "rho": p0.rho, "gamma": None if np.isinf(p0.gamma) else p0.gamma,
            "bundles": p0.n_bundles, "cost_dtype": cost_dtype, "theta_dtype": "f32",
            "parallelism": "replicas (one independent problem per rank)"}


def bytes_per_entry(cost_dtype):
    return 8 + (4 if cost_dtype == "f32" else 2)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# Sources of each column-step kernel: a recorded traffic figure holds only
# while the hash of its kernel's sources is unchanged.
KERNEL_SOURCES = {
    "column_kernel": ("mam_column.cuh", "mam_kernels.cu", "mam_device.cuh", "mam_internal.h"),
    "column_kernel_sparse": ("mam_column.cuh", "mam_sparse.cu", "mam_device.cuh",
                             "mam_internal.h"),
    "column_ring_kernel": ("mam_warp_kernel.cu", "mam_device.cuh", "mam_internal.h"),
}


def kernel_source_hash(kernel="column_kernel"):
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_2309_05315_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(workload_name, entries, kernel="column_kernel"):
    """DRAM bytes of one column-step launch from the committed ncu record
    (bytes per plan entry, times the entries of the launch); None if there is
    no record for this workload and kernel, or the kernel's sources changed
    since it was taken."""
    path = os.path.join(ROOT, "profiles", "column_kernel_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        return None
    rec = d.get(workload_name)
    if (not rec or rec.get("kernel", "column_kernel") != kernel
            or rec.get("kernel_sha") != kernel_source_hash(kernel)):
        return None
    return float(rec["dram_bytes_per_entry"]) * entries


class ClockSampler:
    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.proc = None
        self.uuid = None
        try:
            import torch
            u = getattr(torch.cuda.get_device_properties(device), "uuid", None)
            if u is not None:
                self.uuid = "GPU-" + str(u)
        except Exception:
            pass
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
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
        rows = [r.split(", ") for r in out.strip().splitlines() if r.count(",") >= 8]
        uu = {r[0] for r in rows}
        if self.uuid in uu:
            rows = [r for r in rows if r[0] == self.uuid]
        elif len(uu) > 1:
            rows = [r for r in rows if r[0] == sorted(uu)[0]]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4)
                          if r[5 + i].strip().lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


SHARD = None   # (rank, world) when the problem is measure-sharded over the ranks


def make(probs, **kw):
    from paper_2309_05315_gb300 import Mam
    if SHARD is not None:
        from paper_2309_05315_gb300.shard import sharded
        return sharded(probs[0], SHARD[0], SHARD[1], **kw)
    return Mam(problems=probs, **kw) if len(probs) > 1 else Mam(probs[0], **kw)


def measure(idx, probs, cost_dtype, steps, warmup, local, dist=None, ext=None,
            autotune=False):
    """The throughput line of one workload: CUDA events on the library's
    stream around `steps` graph-replayed iterations (inputs resident), clocks
    sampled meanwhile, and the column kernel's roofline from a window of
    individually timed launches after the timed region."""
    import torch
    ext = ext or {}
    # A dedicated (non-default) stream: the library orders its work on it and
    # the timing events below are recorded on the same stream.
    stream = torch.cuda.Stream()
    gpu = make(probs, cost_dtype=cost_dtype, diag="never", stream=stream, **ext)
    if autotune:
        gpu.autotune(5)
    gpu.step(warmup)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    w0 = gpu.work()["entries"]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    gpu.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    time.sleep(0.15)
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    entries = gpu.work()["entries"] - w0
    ms, value = aggregate_ranks(ms, entries / steps, steps, dist, "cuda")

    # Column-kernel duration for the roofline, over the timed region's steps:
    # a second handle of the same problem replays them (the iterates are
    # deterministic, so every launch does the same work as its counterpart
    # in the timed region), with CUDA events around every launch on the
    # library's stream (per-launch events keep the kernels from overlapping,
    # so this replay is not the throughput measurement).
    rep = make(probs, cost_dtype=cost_dtype, diag="never", stream=stream, **ext)
    if autotune:
        rep.set_config(**gpu.config())
    rep.step(warmup)
    rep.profile_enable(True)
    rep.profile_read()
    col_ms = avg_ms = 0.0
    n_timed = 0
    win_entries = 0
    left = steps
    while left > 0:
        n = min(500, left)
        w = rep.work()["entries"]
        rep.step(n)
        left -= n
        pr = rep.profile_read()
        win_entries += rep.work()["entries"] - w
        col_ms += pr["column_ms"]
        avg_ms += pr["average_ms"]
        n_timed += pr["iterations"]
    rep.profile_enable(False)
    rep.close()
    del rep
    # shared cost layout: the HBM traffic is theta (read and write); the one
    # cost matrix is read through L2
    bpe = 8 if ext.get("cost_layout") == "shared" else bytes_per_entry(cost_dtype)
    sparse_note = None
    if ext.get("plan_layout") == "sparse":
        # cost bytes, plus a pair (8 B) read and written per active entry:
        # the mean count of stored pairs after the window stands for the
        # window's mean
        cnt = np.frombuffer(gpu.get_state(), dtype=np.int32, count=gpu.T, offset=64)
        act = float(cnt[cnt >= 0].mean()) if (cnt >= 0).any() else 0.0
        bpe = (0 if ext.get("cost_layout") == "shared" else bpe - 8) + 16.0 * act / gpu.R
        sparse_note = f"sparse plans: {act:.1f} stored pairs per column after the window"
    peak, peak_kind = peaks()
    achieved = win_entries * bpe / (col_ms / 1e3) / 1e9
    alg_launch = win_entries * bpe / max(n_timed, 1)
    cfg = describe(idx, probs, cost_dtype, gpu.T, gpu.T * gpu.R)
    cfg.update(ext)
    cfg["l2"] = (f"inputs larger than L2: {alg_launch / 1e6:.0f} MB of plan/cost traffic per "
                 "step on average, no flush")
    cfg["kernel_config"] = gpu.config()
    kernel = "column_ring_kernel" if cfg["kernel_config"]["kind"] == 1 else "column_kernel"
    if sparse_note:
        kernel = "column_kernel_sparse"
        cfg["sparse_pairs"] = sparse_note
    traffic = ncu_traffic(cfg["workload"], win_entries / max(n_timed, 1), kernel)
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic,
            "kernel": kernel, "peak_kind": f"{peak_kind} copy bandwidth",
            "bytes_per_entry": bpe,
            "algorithmic_bytes_per_launch": alg_launch,
            "duration_window": f"the timed region's {n_timed} launches (steps {warmup + 1}-"
                               f"{warmup + steps} from creation), replayed on a second handle "
                               "of the same problem, one event pair each",
            "step_achieved_gbs": (entries / steps) * bpe / (ms / steps / 1e3) / 1e9,
            "avg_launch_ms": col_ms / max(n_timed, 1),
            "average_kernel_avg_ms": avg_ms / max(n_timed, 1)}
    gpu.close()
    del gpu
    return {"value": value, "ms_per_step": ms / steps, "entries_per_step": entries / steps,
            "config": cfg, "roofline": roof, "gpu_launches": 2 * steps, "clocks": clocks}


def time_to_gap(probs, cost_dtype, tol=1e-4, ref_iters=50000, ref_every=100,
                max_iters=50000, check_every=10, rho=None, ext=None):
    """Time to a 1e-4 objective gap.  The reference W* of each problem comes
    from a long run of its own: the largest dual lower bound seen (balanced)
    or the smallest F(pi-hat) seen (unbalanced).  Then, from theta^0, the
    iterations run until every problem has |F(pi-hat) - W*| / W* <= tol and,
    when balanced, dist_L(pi-hat) / mass <= tol, at two checks in a row; the
    checks (a diagnostic iteration and a host read every check_every
    iterations) are inside the timed wall clock."""
    import torch
    kw = dict(cost_dtype=cost_dtype, diag="last", rho=rho, **(ext or {}))
    balanced = [math.isinf(getattr(p, "gamma", math.inf)) for p in probs]
    qa = []
    for p in probs:
        S = np.array([int((np.asarray(q) > 0).sum()) for q in p.q], dtype=float)
        a = (1.0 / S) / (1.0 / S).sum()
        qa.append(float(sum(a[m] * float(np.sum(p.q[m])) for m in range(len(p.q)))))
    g = make(probs, **kw)
    wstar = [(-math.inf if b else math.inf) for b in balanced]
    for _ in range(ref_iters // ref_every):
        g.step(ref_every)
        for i, o in enumerate(g.objectives()):
            wstar[i] = max(wstar[i], o["lower_bound"]) if balanced[i] else min(wstar[i], o["f_unbal"])
    g.close()

    def gaps(objs):
        out = []
        for i, o in enumerate(objs):
            gp = abs(o["f_unbal"] - wstar[i]) / max(abs(wstar[i]), 1e-300)
            if balanced[i]:
                gp = max(gp, o["dist_pihat"] / qa[i])
            out.append(gp)
        return max(out)

    g = make(probs, **kw)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    it, gap, hits = 0, math.inf, 0
    while it < max_iters:
        g.step(check_every)
        it += check_every
        gap = gaps(g.objectives())
        hits = hits + 1 if gap <= tol else 0
        if hits >= 2:  # two checks in a row: an oscillating objective crossing W* does not count
            break
    dt = time.perf_counter() - t0
    g.close()
    return {"tol": tol, "reached": bool(hits >= 2), "iterations": int(it), "seconds": dt,
            "gap": gap, "check_every": check_every, "cost_dtype": cost_dtype,
            "rho": rho if rho is not None else probs[0].rho,
            "reference": f"W* = best dual lower bound (balanced) or best F(pi-hat) "
                         f"(unbalanced) over a {ref_iters}-iteration run, per problem",
            "w_star": wstar[0] if len(wstar) == 1 else None}


def forward_backward(prob, K=200, ckpt=20):
    """Wall time of mam_forward_record(K, ckpt) + mam_backward for
    L = ||p^K - target||^2 (host gradients), and of K plain iterations.
    ckpt > 0: checkpoints every ckpt iterations, segments recomputed in the
    backward sweep; ckpt = 0: the active sets of every step kept from the
    forward pass (when they fit), nothing recomputed."""
    import torch
    from paper_2309_05315_gb300 import Mam
    g = Mam(prob, cost_dtype="f32", diag="never")
    g.forward_record(K, ckpt)           # warm-up (allocations, graph capture)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g.forward_record(K, ckpt)
    p = g.barycenter()
    t1 = time.perf_counter()
    g.backward(2.0 * (p - prob.target))
    t2 = time.perf_counter()
    g.set_state(g.get_state())
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    g.step(K)
    g.barycenter()
    t4 = time.perf_counter()
    g.close()
    return {"K": K, "ckpt_every": ckpt, "forward_record_s": t1 - t0, "backward_s": t2 - t1,
            "fwd_bwd_s": t2 - t0, "plain_forward_s": t4 - t3,
            "loss": float(np.sum((p - prob.target) ** 2))}


def forms(args):
    """The three forms against the plain FP32 path on time to a 1e-4 gap
    (each against the W* of its own problem, so reduced-precision costs are
    judged on their rounded cost)."""
    from workloads import generators as G
    out = {}
    ell = [G.config2(0)]
    plain = time_to_gap(ell, "f32", ref_iters=args.gap_ref_iters,
                        max_iters=args.gap_ref_iters)
    out["mixed_precision"] = {
        "workload": NAMES[2] + ", rho = 100",
        "plain_f32": plain,
        "bf16_cost": time_to_gap(ell, "bf16", ref_iters=args.gap_ref_iters,
                                 max_iters=args.gap_ref_iters),
        "f16_cost": time_to_gap(ell, "f16", ref_iters=args.gap_ref_iters,
                                max_iters=args.gap_ref_iters)}
    batch = G.config3(256)
    rho_b = 10.0
    sample = batch[:8]
    single = [time_to_gap([p], "f32", rho=rho_b, ref_iters=args.gap_ref_iters,
                          max_iters=args.gap_ref_iters) for p in sample]
    one_s = float(np.mean([r["seconds"] for r in single]))
    out["batched"] = {
        "workload": NAMES[3] + f", rho = {rho_b:g}",
        "batched_bf16": time_to_gap(batch, "bf16", rho=rho_b, ref_iters=args.gap_ref_iters,
                                    max_iters=args.gap_ref_iters),
        "plain_f32_one_problem_at_a_time": {
            "seconds_extrapolated": one_s * len(batch),
            "sample": f"first {len(sample)} of {len(batch)} problems solved one by one "
                      "(FP32 cost, single-problem path), mean time to gap x 256",
            "mean_seconds_per_problem": one_s,
            "all_reached": all(r["reached"] for r in single),
            "mean_iterations": float(np.mean([r["iterations"] for r in single]))}}
    mix = G.config4(0)
    out["differentiation"] = {
        "workload": NAMES[4],
        "forward_backward": forward_backward(mix),
        "forward_backward_all_masks": forward_backward(mix, ckpt=0),
        "plain_f32_time_to_gap_rho300": time_to_gap([mix], "f32", rho=300.0,
                                                    ref_iters=args.gap_ref_iters,
                                                    max_iters=args.gap_ref_iters)}
    return out


def shared_cost_leg(args, local):
    """The shared cost layout (one cost matrix for measures on a common
    support; HBM traffic 8 B per entry, the matrix read through L2) against
    the per-column layout: the stroke batch (one 784 x 784 matrix for all 256
    problems) and the unbalanced mixtures (one 10000 x 10000 matrix)."""
    out = {}
    steps, warm = max(args.steps, 100), max(args.warmup, 10)
    for idx in (3, 5):
        probs, dt = workload(idx)
        sh = measure(idx, probs, dt, steps, warm, local, ext={"cost_layout": "shared"})
        rec = {"shared": {k: sh[k] for k in ("value", "ms_per_step")},
               "shared_roofline_frac": sh["roofline"]["frac"],
               "shared_kernel_config": sh["config"]["kernel_config"]}
        if idx == 3:
            pc = measure(idx, probs, dt, steps, warm, local)
            rec["per_column"] = {k: pc[k] for k in ("value", "ms_per_step")}
            rec["per_column_roofline_frac"] = pc["roofline"]["frac"]
        out[NAMES[idx]] = rec
    return out


def aggregate_ranks(ms, units_per_step, steps, dist=None, device="cpu"):
    """Whole-job throughput of independent replicas: the slowest rank's time
    (max over ranks) and the units every rank processed (sum over ranks);
    returns (ms, units per second).  Without a process group: this rank's."""
    if dist is None:
        return ms, steps * units_per_step / (ms / 1e3)
    import torch
    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    u = torch.tensor([float(units_per_step)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    ms = float(t.item())
    return ms, steps * float(u.item()) / (ms / 1e3)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def extension(args):
    """Keyword arguments of the capped-column extension, or none."""
    return {} if args.eta is None else {"capped": True, "eta": float(args.eta)}


def oracle_sample(prob, n_measures):
    """The first n measures of the workload, all their columns (a bounded
    sample of the same images, sizes and costs)."""
    import copy
    sub = copy.copy(prob)
    n = min(n_measures, prob.M)
    sub.q = list(prob.q[:n])
    sub.zeta = list(prob.zeta[:n])
    sub.alpha = np.asarray(prob.alpha[:n])
    if prob.cost is not None:
        sub.cost = list(prob.cost[:n])
    return sub


def time_oracle(prob, cost_dtype, ext, workers, seconds=None, iters=None, warmup=0):
    """Oracle iterations on `prob`: one thread (workers = 0, MamOracle) or
    worker processes (ParallelMamOracle).  Returns (entries/s, iterations,
    seconds, threads used)."""
    from oracle.mam_oracle import MamOracle, prepare
    from oracle.parallel import ParallelMamOracle
    eta, capped = ext.get("eta", 0.0), ext.get("capped", False)
    oc = "f64" if cost_dtype == "f32" else cost_dtype
    if workers:
        orc = ParallelMamOracle(prob, prob.rho, capped=capped, cost_dtype=oc, eta=eta,
                                workers=workers)
        used = orc.workers
    else:
        orc = MamOracle(prepare(prob, oc, eta=eta), prob.rho, capped=capped)
        used = 1
    entries = int(sum(int((np.asarray(q) > 0).sum()) for q in prob.q)) * prob.R
    for _ in range(warmup):
        orc.step(diagnostics=False)
    n = 0
    t0 = time.perf_counter()
    while True:
        orc.step(diagnostics=False)
        n += 1
        dt = time.perf_counter() - t0
        if (iters is not None and n >= iters) or (iters is None and dt >= seconds):
            break
    if workers:
        orc.close()
    return n * entries / dt, n, dt, used


def cpu_baseline(prob, cost_dtype, ext=None):
    """The FP64 oracle as it stands on the host cores, on a bounded sample of
    the workload: one thread, and one worker process per core."""
    ext = ext or {}
    cores = os.cpu_count() or 1
    one = oracle_sample(prob, 2)
    v1, n1, t1, _ = time_oracle(one, cost_dtype, ext, 0, seconds=10.0)
    allc = oracle_sample(prob, cores)
    va, na, ta, used = time_oracle(allc, cost_dtype, ext, cores, seconds=10.0, warmup=1)
    return {"value": va, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": f"the first {allc.M} of {prob.M} measures with all their columns, "
                      f"{na} iterations in {ta:.1f} s, one worker process per measure group "
                      f"(numpy FP64; host has {cores} cores)",
            "single_thread": {"value": v1, "unit": UNIT, "cores": 1,
                              "sample": f"the first {one.M} measures, {n1} iterations in "
                                        f"{t1:.1f} s, one thread"}}


def run_reference(args):
    """Reference arm: the FP64 oracle on the host cores (all of them), each
    step one oracle iteration over a bounded sample of the workload."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    probs, cost_dtype = workload(args.workload)
    if args.measures:
        probs = first_measures(probs, args.measures)
    if args.cost_dtype:
        cost_dtype = args.cost_dtype
    prob = probs[0]
    ext = extension(args)
    cores = os.cpu_count() or 1
    sample = oracle_sample(prob, cores)
    value, n, dt, used = time_oracle(sample, cost_dtype, ext, cores, iters=args.steps,
                                     warmup=args.warmup)
    T_full = int(sum(int((np.asarray(q) > 0).sum()) for p in probs for q in p.q))
    cfg = describe(args.workload, probs, cost_dtype, T_full, T_full * prob.R)
    cfg["theta_dtype"] = "f64"
    cfg.update(ext)
    desc = (f"the first {sample.M} of {prob.M} measures of problem 0 with all their columns "
            f"per step (numpy FP64 oracle, {used} worker processes)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / n, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded images shaped like the paper's workloads)", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    ws, rank, local = dist_env()
    import torch
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2309_05315_gb300.build import build
    if rank == 0:
        build()
    if dist:
        dist.barrier()
    global SHARD
    if args.shard:
        if len(workload(args.workload, 0)[0]) > 1:
            raise SystemExit("--shard needs a single-problem workload")
        SHARD = (rank, ws)
    # sharded: every rank holds part of problem 0; replicas: rank r solves problem r
    probs, cost_dtype = workload(args.workload, 0 if args.shard else rank)
    if args.measures:
        probs = first_measures(probs, args.measures)
    if args.cost_dtype:
        cost_dtype = args.cost_dtype
    ext = extension(args)
    if args.cost_layout != "per_column":
        ext["cost_layout"] = args.cost_layout
    if args.plan_layout != "dense":
        ext["plan_layout"] = args.plan_layout
        ext["sparse_slots"] = args.sparse_slots
    head = measure(args.workload, probs, cost_dtype, args.steps, args.warmup, local, dist,
                   ext, args.autotune)
    if args.shard:
        head["config"]["parallelism"] = (f"measure-sharded over {ws} rank(s): contiguous measure "
                                         "ranges of equal kept columns, one NCCL all-reduce of "
                                         "R int64 partial sums of p per iteration (plus 4 FP64 "
                                         "for t^k)")
    line = {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
            "higher_is_better": True, "scaling": "strong" if args.shard else "weak",
            "vs_baseline": None,
            "dtype": "f32", "data": "synthetic (seeded images standing in for the "
                                    "paper's datasets)",
            "config": head["config"], "roofline": head["roofline"],
            "gpu_launches": head["gpu_launches"], "clocks": head["clocks"],
            "entries_per_step": head["entries_per_step"]}

    if not args.no_e2e:
        # End to end through the public API from host buffers: create (h2d of
        # the problem data), the same number of steps, barycenter (d2h).
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g2 = make(probs, cost_dtype=cost_dtype, diag="never", **ext)
        t_created = time.perf_counter()
        nsteps = args.warmup + args.steps
        g2.step(nsteps)
        pbar = g2.barycenter()
        dt = time.perf_counter() - t0
        e2e_entries = g2.work()["entries"]
        g2.close()
        h2d = sum(8 * (sum(len(q) for q in p.q) * (1 + p.dim) + p.M + p.R * p.dim) + 4 * p.M
                  for p in probs)
        _, e2e_value = aggregate_ranks(dt * 1e3, e2e_entries / nsteps, nsteps, dist, "cuda")
        line["e2e"] = {"value": e2e_value, "unit": UNIT,
                       "h2d_bytes_per_step": h2d / nsteps,
                       "d2h_bytes_per_step": pbar.nbytes / nsteps,
                       "what": f"mam_create from host arrays + {nsteps} mam_step + "
                               "mam_get_barycenter to host, wall clock",
                       "create_ms": (t_created - t0) * 1e3,
                       "steps_and_read_ms": (t0 + dt - t_created) * 1e3}
    SHARD = None
    if rank == 0 and ws == 1:
        if not args.no_extra and args.workload != 2:
            ell, _ = workload(2)
            x = measure(2, ell, "f32", max(args.steps, 200), max(args.warmup, 10), local)
            line["nested_ellipses_f32"] = {k: x[k] for k in ("value", "ms_per_step", "config",
                                                             "roofline", "clocks")}
        if not args.no_extra and not ext:
            line["shared_cost"] = shared_cost_leg(args, local)
        if not args.no_forms:
            line["forms"] = forms(args)
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(probs[0], cost_dtype, ext)
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
