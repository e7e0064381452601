#!/usr/bin/env python3
"""Throughput of the MAM iteration on one GB300 (plan-entry updates / s).

A step is one iteration of Algorithm 1 over every measure of the workload:
the averaging kernel (Step 1, t^k, Step 3 reduction) and the fused column
kernel (Step 2 for every plan column).  Default workload: M = 10 seeded
60x60 nested-ellipse images, R = 3600 grid points, FP32 plans and costs,
rho = 100 (the paper's untuned value).  The working set (~276 MB per
iteration) is larger than L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun every rank solves its own
seeded replica (independent problems, weak scaling, no collective on the
data path).  ``--impl reference`` times the FP64 oracle on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
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


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", type=int, default=2, choices=[1, 2, 3, 4, 5])
    ap.add_argument("--cost-dtype", default=None, choices=["f32", "bf16", "f16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--autotune", action="store_true")
    ap.add_argument("--rho", type=float, default=None,
                    help="rho of the time-to-gap measurement (default: the workload's)")
    ap.add_argument("--gap-ref-iters", type=int, default=50000)
    ap.add_argument("--eta", type=float, default=None,
                    help="capped columns (the full unbalanced extension: projection onto "
                         "Delta_<=(q_s), cost alpha_m (d - eta)) with this eta")
    ap.add_argument("--no-gap", action="store_true", help="skip the time-to-gap measurement")
    ap.add_argument("--no-diff", action="store_true",
                    help="mixture workload: skip the forward+backward measurement")
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
    return [G.config5(rank)], "bf16"


def describe(idx, probs, cost_dtype, T, entries):
    names = {1: "blobs16_M3_R256", 2: "nested_ellipses60_M10_R3600",
             3: "strokes28_256problems_R784", 4: "mixture40_M8_R1600",
             5: "mixture100_M100_R10000_unbalanced"}
    p0 = probs[0]
    cfg = {"workload": names[idx], "problems": len(probs),
           "measures": int(sum(p.M for p in probs)), "R": p0.R,
           "kept_columns": int(T), "plan_entries": int(entries),
           "rho": p0.rho, "gamma": None if np.isinf(p0.gamma) else p0.gamma,
           "bundles": p0.n_bundles, "cost_dtype": cost_dtype, "theta_dtype": "f32",
           "parallelism": "replicas (one independent problem per rank)"}
    return cfg


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
    "column_kernel": ("mam_kernels.cu", "mam_device.cuh", "mam_internal.h"),
    "column_ring_kernel": ("mam_warp_kernel.cu", "mam_device.cuh", "mam_internal.h"),
}


def kernel_source_hash(kernel="column_kernel"):
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_2309_05315_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(workload_name, entries, kernel="column_kernel"):
    """DRAM bytes per column-step launch from the committed ncu summary,
    scaled to this launch by plan entries; None if there is no record for
    this workload and kernel, or the kernel's sources changed since."""
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
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
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


def time_to_gap(probs, cost_dtype, tol=1e-4, ref_iters=50000, ref_every=100,
                max_iters=50000, check_every=10, rho=None, ext=None):
    """Time to a 1e-4 objective gap.  The reference W* of each problem comes
    from a long run of its own: the largest dual lower bound seen (balanced)
    or the smallest F(pi-hat) seen (unbalanced).  Then, from theta^0, the
    iterations run until every problem has |F(pi-hat) - W*| / W* <= tol and,
    when balanced, dist_L(pi-hat) / mass <= tol, at two checks in a row; the
    checks (a diagnostic iteration and a host read every check_every
    iterations) are inside the timed wall clock."""
    import math
    import torch
    from paper_2309_05315_gb300 import Mam
    kw = dict(cost_dtype=cost_dtype, diag="last", rho=rho, **(ext or {}))
    make = (lambda: Mam(problems=probs, **kw)) if len(probs) > 1 else (lambda: Mam(probs[0], **kw))
    balanced = [math.isinf(getattr(p, "gamma", math.inf)) for p in probs]
    qa = []
    for p in probs:
        S = np.array([int((np.asarray(q) > 0).sum()) for q in p.q], dtype=float)
        a = (1.0 / S) / (1.0 / S).sum()
        qa.append(float(sum(a[m] * float(np.sum(p.q[m])) for m in range(len(p.q)))))
    g = make()
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

    g = make()
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
    L = ||p^K - target||^2 (host gradients), and of K plain iterations."""
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


def run_reference(args):
    """The FP64 oracle on the host cores (reference arm)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from oracle.mam_oracle import MamOracle, prepare
    probs, cost_dtype = workload(args.workload)
    prob = probs[0]
    ext = extension(args)
    eta, capped = ext.get("eta", 0.0), ext.get("capped", False)
    prep_full = prepare(prob, eta=eta)
    T = int(sum(prep_full.S))
    entries = T * prob.R
    # Each step is one oracle iteration over a bounded column sample of the
    # workload, sized so the whole run takes about two minutes.
    orc_full = MamOracle(prep_full, prob.rho, capped=capped)
    t0 = time.perf_counter()
    orc_full.step(diagnostics=False)
    per_entry = (time.perf_counter() - t0) / entries
    budget = 120.0
    n_steps = args.warmup + args.steps
    cols = int(max(1, min(T, budget / (n_steps * per_entry * prob.R))))
    import copy
    sub = copy.deepcopy(prob)
    keep_m = 0
    idx = np.nonzero(sub.q[keep_m] > 0)[0][:cols]
    mask = np.zeros_like(sub.q[keep_m])
    mask[idx] = sub.q[keep_m][idx]
    sub.q = [mask / mask.sum() * prob.q[keep_m].sum()]
    sub.zeta = [sub.zeta[keep_m]]
    sub.alpha = np.array([1.0])
    orc = MamOracle(prepare(sub, eta=eta), prob.rho, capped=capped)
    for _ in range(args.warmup):
        orc.step(diagnostics=False)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        orc.step(diagnostics=False)
    dt = time.perf_counter() - t0
    sample_entries = len(idx) * prob.R
    value = args.steps * sample_entries / dt
    cfg = describe(args.workload, probs, "f64", T, entries)
    cfg["theta_dtype"] = "f64"
    cfg.update(ext)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded images shaped like the paper's workloads)", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{len(idx)} columns x R={prob.R} of the workload per "
                                       f"step (numpy FP64 oracle, single thread)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def cpu_baseline(prob, entries, seconds=12.0, ext=None):
    from oracle.mam_oracle import MamOracle, prepare
    ext = ext or {}
    prep = prepare(prob, eta=ext.get("eta", 0.0))
    orc = MamOracle(prep, prob.rho, capped=ext.get("capped", False))
    n = 0
    t0 = time.perf_counter()
    while True:
        orc.step(diagnostics=False)
        n += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return {"value": n * entries / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n} full oracle iterations of the workload ({dt:.1f} s, numpy FP64, "
                      f"single thread; host has {os.cpu_count()} cores)"}


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
    from paper_2309_05315_gb300 import Mam
    from paper_2309_05315_gb300.build import build
    if rank == 0:
        build()
    if dist:
        dist.barrier()
    probs, cost_dtype = workload(args.workload, rank)
    if args.cost_dtype:
        cost_dtype = args.cost_dtype
    # A dedicated (non-default) stream: the library orders its work on it and
    # the timing events below are recorded on the same stream.
    stream = torch.cuda.Stream()
    ext = extension(args)
    kw = dict(cost_dtype=cost_dtype, diag="never", stream=stream, **ext)
    gpu = Mam(problems=probs, **kw) if len(probs) > 1 else Mam(probs[0], **kw)
    if args.autotune:
        gpu.autotune(5)
    entries_per_step = gpu.T * gpu.R
    if probs[0].n_bundles > 1:  # randomized: expected fraction of columns per step
        entries_per_step = entries_per_step / probs[0].n_bundles
    gpu.step(args.warmup)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    time.sleep(0.4)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    # Timed region: the production path (CUDA-graph replay, programmatic
    # dependent launch between the column and averaging kernels).
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    gpu.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    ms, value = aggregate_ranks(ms, entries_per_step, args.steps, dist, "cuda")

    # Column-kernel duration for the roofline: CUDA events around every
    # launch on the library's stream, over a window of the same workload run
    # right after the timed region (per-launch events keep the kernels from
    # overlapping, so this window is not the throughput measurement).
    gpu.profile_enable(True)
    gpu.profile_read()
    col_ms = avg_ms = 0.0
    n_timed = 0
    left = min(args.steps, 4000)
    while left > 0:
        n = min(500, left)
        gpu.step(n)
        left -= n
        pr = gpu.profile_read()
        col_ms += pr["column_ms"]
        avg_ms += pr["average_ms"]
        n_timed += pr["iterations"]
    gpu.profile_enable(False)

    # roofline of the column kernel
    bpe = bytes_per_entry(cost_dtype)
    col_avg_s = (col_ms / max(n_timed, 1)) / 1e3
    alg_bytes = entries_per_step * bpe
    peak, peak_kind = peaks()
    achieved = alg_bytes / col_avg_s / 1e9
    cfg = describe(args.workload, probs, cost_dtype, gpu.T, gpu.T * gpu.R)
    cfg.update(ext)
    cfg["l2"] = (f"inputs larger than L2: {alg_bytes / 1e6:.0f} MB of plan/cost traffic per "
                 "step, no flush")
    cfg["kernel_config"] = gpu.config()
    kernel = "column_ring_kernel" if cfg["kernel_config"]["kind"] == 1 else "column_kernel"
    traffic = ncu_traffic(cfg["workload"], entries_per_step, kernel)
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic,
            "kernel": kernel, "peak_kind": f"{peak_kind} copy bandwidth",
            "algorithmic_bytes_per_launch": alg_bytes,
            "duration_window": f"{n_timed} launches, one event pair each, after the timed region",
            "step_achieved_gbs": alg_bytes / (ms / args.steps / 1e3) / 1e9,
            "avg_launch_ms": col_avg_s * 1e3,
            "average_kernel_avg_ms": avg_ms / max(n_timed, 1)}
    gpu.close()

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic (seeded images standing in for the "
                                    "paper's datasets)",
            "config": cfg, "roofline": roof, "gpu_launches": 2 * args.steps,
            "clocks": clocks}

    if not args.no_gap:
        line["time_to_gap"] = time_to_gap(probs, cost_dtype, rho=args.rho,
                                          ref_iters=args.gap_ref_iters,
                                          max_iters=args.gap_ref_iters, ext=ext)
    if args.workload == 4 and not args.no_diff and not ext:
        line["differentiation"] = forward_backward(probs[0])

    if not args.no_e2e:
        # End to end through the public API from host buffers: create (h2d of
        # the problem data), the same number of steps, barycenter (d2h).
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g2 = Mam(problems=probs, cost_dtype=cost_dtype, diag="never", **ext) if len(probs) > 1 \
            else Mam(probs[0], cost_dtype=cost_dtype, diag="never", **ext)
        g2.step(args.warmup + args.steps)
        pbar = g2.barycenter()
        dt = time.perf_counter() - t0
        g2.close()
        nsteps = args.warmup + args.steps
        h2d = sum(8 * (sum(len(q) for q in p.q) * (1 + p.dim) + p.M + p.R * p.dim) + 4 * p.M
                  for p in probs)
        _, e2e_value = aggregate_ranks(dt * 1e3, entries_per_step, nsteps, dist, "cuda")
        line["e2e"] = {"value": e2e_value, "unit": UNIT,
                       "h2d_bytes_per_step": h2d / nsteps,
                       "d2h_bytes_per_step": pbar.nbytes / nsteps,
                       "what": f"mam_create from host arrays + {nsteps} mam_step + "
                               "mam_get_barycenter to host, wall clock"}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(probs[0], probs[0].R * int(
            sum(int((q > 0).sum()) for q in probs[0].q)), ext=ext)
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
