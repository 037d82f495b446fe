"""Benchmark: box fast Gauss transform throughput on one GB300 (or N replicas).

One step = one full transform (Algorithm 4: form, gather, evaluate, near field) of the
3D periodic density of the paper's periodic experiments (Section 6): a uniform level-5
tree (32768 leaves), p = 8 (16.8M target points), delta = 1e-3, sigma = 16 seeded
Gaussians plus uniform noise.

Printed value: target points/s of the plain FP64 form at tol 1e-10.  Beside it, on the same
GPU and input: the split-precision form at tol 1e-6 (3xTF32 contractions), the FP64 form at
tol 1e-6 and the FP64 tensor-core form, their ratios to the plain FP64 form, p50/p99 step
latency, every form's error against the oracle on a seeded sample of target leaves, the
dominant kernel's roofline fraction (FP64 pipe for the FP64 forms, the 3xTF32 tensor pipe
for the split form), an end-to-end number through the host-buffer entry point, and the CPU
oracle timed on a bounded sample of target leaves (extrapolated to the whole workload).
A second section runs the same forms on the 3D adaptive free-space workload (about 2.1M
points), then the delta sweep, the paper-shaped k = 16 runs, the batched and serving runs.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]

Multi-GPU: the transform does not shard across GPUs here; N ranks run N
independent replicas (weak scaling) and rank 0 reports the whole-job rate.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 / FP32 CUDA-core peaks of GB300 from unit counts and the maximum SM clock:
# 152 SMs x 2 FP64 FMA/clk (x2 flops) x 2.07 GHz, and 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# Double-float (FP32 pair) arithmetic of the FP64_TC gather and near field: one FP64-accurate
# fused multiply-add (2 flops) takes 15 FP32 instructions (exact product by FMA, two-sum, renormalise)
DF_INSTR_PER_FMA = 15
DF_PEAK_TFLOPS = FP32_PEAK_TFLOPS / DF_INSTR_PER_FMA
# TF32 runs at half the dense BF16 rate on this tensor core (nominal 1.1 against 2.25 PFLOP/s);
# 3xTF32 spends three TF32 products on each FP32-accurate product
TF32_PER_BF16 = 0.5
SPLIT_PRODUCTS = 3
SLICE_PRODUCTS = 21   # BF16 slice products per FP64 product in the sliced FP64 tensor-core stages
FALLBACK_BF16_TFLOPS = 1900.0
L2_FLUSH_BYTES = 256 << 20


WORKLOADS = {
    "periodic3d": lambda W: W.config_3d_periodic_uniform(seed=0),
    "adaptive3d": lambda W: W.config_3d_free_adaptive(seed=0, p=8, delta=1e-3),
    # the same tree and density at delta 1e-4 (a 16^3 cutoff grid, a third of its boxes anchors)
    "adaptive3d_d1e-4": lambda W: dataclasses.replace(W.config_3d_free_adaptive(seed=0, p=8, delta=1e-3), delta=1e-4),
    "uniform2d": lambda W: W.config_2d_free_uniform(seed=0),
}
FORMS = {"split": ("split_tol1e-6", 1e-6, 1), "fp64": ("fp64_tol1e-6", 1e-6, 0),
         "fp64_1e-10": ("fp64_tol1e-10", 1e-10, 0), "fp64tc": ("fp64tc_tol1e-6", 1e-6, 2),
         "fp64tc_1e-10": ("fp64tc_tol1e-10", 1e-10, 2)}
DEFAULT_FORMS = "fp64tc_1e-10,fp64_1e-10,split,fp64,fp64tc"


def workload(name="adaptive3d"):
    import workloads as W
    return WORKLOADS[name](W)


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 20 ms while active.  Entering waits (up to
    5 s) for nvidia-smi's first line, so that sampling is live before the caller's region starts;
    that line (taken before the region) is left out of the summary unless it is the only one."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")
    INTERVAL_MS = 20

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.first = None

    def __enter__(self):
        import select
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", str(self.INTERVAL_MS)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            ready, _, _ = select.select([self.proc.stdout], [], [], 5.0)
            if ready:
                self.first = self.proc.stdout.readline()
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.rows, self.pre = [], []
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                self.rows.append(f)
        if self.first:
            f = [x.strip() for x in self.first.split(",")]
            if len(f) >= 9:
                self.pre.append(f)

    def summary(self):
        rows = getattr(self, "rows", [])
        pre = getattr(self, "pre", [])
        note = None
        if not rows and pre:
            rows, note = pre, "only the sample taken before the timed region"
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        out = {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
               "reasons": reasons, "samples": len(rows), "interval_ms": self.INTERVAL_MS}
        if note:
            out["note"] = note
        return out


# DRAM bytes (read + write) per step of a phase's launches, measured by ncu on this workload
# (dram__bytes_read.sum + dram__bytes_write.sum of one capture), with the profile summary that
# holds the capture.  Keyed by (workload, form, phase); an entry is removed whenever the
# kernels of that phase change, and phases without a current capture report null.
NCU_TRAFFIC = {
    ("periodic3d", "fp64tc_tol1e-10", "evaluate"): {
        "bytes": 2087.4e6, "source": "profiles/sliced_fp64_kernels_periodic3d.md (oz_slice_kernel + oz_mma_kernel, stages 3-5)"},
    ("periodic3d", "fp64tc_tol1e-10", "form"): {
        "bytes": 1977.2e6, "source": "profiles/sliced_fp64_kernels_periodic3d.md (oz_slice_kernel + oz_mma_kernel, stages 0-2)"},
    ("periodic3d", "fp64_tol1e-10", "form"): {
        "bytes": 2150.2e6, "source": "profiles/fp64_kernels_periodic3d.md (form_kernel<3,double>, 1 launch a step)"},
    ("periodic3d", "fp64_tol1e-10", "evaluate"): {
        "bytes": 4447.0e6, "source": "profiles/fp64_kernels_periodic3d.md (eval5_kernel<double,1>, 1 launch a step)"},
    ("periodic3d", "split_tol1e-6", "form"): {
        "bytes": 251.9e6, "source": "profiles/tcgen05_kernels_periodic3d.md (sigma_pack_kernel + form7_kernel<32,16>)"},
    ("periodic3d", "split_tol1e-6", "evaluate"): {
        "bytes": 138.1e6, "source": "profiles/tcgen05_kernels_periodic3d.md (eval7_kernel<32,16>)"},
}


def peaks():
    """Measured peaks of the GB300s (MEASURED_PEAKS.json) or the recipe's fallbacks."""
    try:
        with open(PEAKS_FILE) as f:
            j = json.load(f)
        return {"bf16_tflops": float(j["bf16_tflops"]), "hbm_gbs": float(j["hbm_gbs"]), "source": "measured"}
    except Exception:
        return {"bf16_tflops": FALLBACK_BF16_TFLOPS, "hbm_gbs": 6800.0, "source": "fallback"}


def split_tensor_peak_tflops():
    """Roofline of the split form's contractions: the TF32 tensor pipe (measured BF16 burst rate x
    the TF32/BF16 ratio) divided by the three TF32 products of each 3xTF32 product."""
    pk = peaks()
    return pk["bf16_tflops"] * TF32_PER_BF16 / SPLIT_PRODUCTS, pk["source"]


def sliced_tensor_peak_tflops():
    """Roofline of the sliced FP64 tensor-core stages (precision FP64_TC, 3D): the BF16 tensor pipe
    (measured burst rate) divided by the 21 BF16 slice products of each FP64 product."""
    pk = peaks()
    return pk["bf16_tflops"] / SLICE_PRODUCTS, pk["source"]


def roofline_of(info, prof, nprof, prec, traffic_key=None):
    """Dominant phase of one form (per-phase CUDA events over the timed region) against the peak
    it is bound by: algorithmic flops of the phase / its average time per step.  FP64 forms: the
    FP64 pipe.  Split form: the plane-wave contractions (form, gather, evaluation) against the
    3xTF32 tensor-pipe roofline, with the fraction of the FP32 CUDA-core peak beside it; the near
    field stays FP64."""
    phase_flops = {"form": info["form_flops"], "evaluate": info["eval_flops"], "gather": info["gather_flops"],
                   "near": info["direct_flops"], "merge": 0, "push": 0}
    n = max(nprof, 1)
    tpk, tsrc = split_tensor_peak_tflops()
    spk, ssrc = sliced_tensor_peak_tflops()
    sliced = info.get("n_sliced_jobs", 0) > 0
    d3 = info.get("d", 3) == 3

    def on_tensor(ph):
        return (prec == 1 and ph in ("form", "evaluate", "gather")) or (sliced and ph in ("form", "evaluate"))

    def peak_of(ph):
        if prec == 1 and ph in ("form", "evaluate", "gather"):
            return tpk, (f"{tsrc}: BF16 burst x {TF32_PER_BF16} (TF32/BF16) / {SPLIT_PRODUCTS} (3xTF32)")
        if sliced and ph in ("form", "evaluate"):
            return spk, f"{ssrc}: BF16 burst / {SLICE_PRODUCTS} (BF16 slice products per FP64 product)"
        if sliced and d3 and ph in ("gather", "near"):
            return DF_PEAK_TFLOPS, (f"derived: FP32 CUDA-core peak / {DF_INSTR_PER_FMA} "
                                    "(FP32 instructions per double-float FMA)")
        return FP64_PEAK_TFLOPS, "derived: 152 SMs x 2 FP64 FMA/clk x 2 x 2.07 GHz"

    dom = max(prof, key=lambda k: prof[k])
    ms = prof[dom] / n
    achieved = phase_flops[dom] / (ms / 1e3) / 1e12 if ms > 0 else 0.0
    peak, src = peak_of(dom)
    traffic = NCU_TRAFFIC.get(traffic_key + (dom,)) if traffic_key else None
    phases = {}
    for ph, fl in phase_flops.items():
        t = prof.get(ph, 0.0) / n
        if fl > 0 and t > 0:
            pk, _ = peak_of(ph)
            a = fl / (t / 1e3) / 1e12
            phases[ph] = {"ms": t, "achieved_tflops": a, "peak_tflops": pk, "frac": a / pk}
            if prec == 1 and ph in ("form", "evaluate", "gather"):
                phases[ph]["frac_of_fp32_cuda_core"] = a / FP32_PEAK_TFLOPS
            if sliced and (ph in ("form", "evaluate") or (d3 and ph in ("gather", "near"))):
                phases[ph]["frac_of_fp64_alu"] = a / FP64_PEAK_TFLOPS
    out = {"bound": "tensor" if on_tensor(dom) else "alu",
           "kernel": dom, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
           "frac": achieved / peak, "traffic": traffic["bytes"] if traffic else None,
           "traffic_source": traffic["source"] if traffic else None, "phases": phases,
           "peak_source": src, "phase_ms_per_step": {k: v / n for k, v in prof.items()}}
    if out["bound"] == "tensor" and prec == 1:
        out["frac_of_fp32_cuda_core"] = achieved / FP32_PEAK_TFLOPS
    elif out["bound"] == "tensor":
        out["frac_of_fp64_alu"] = achieved / FP64_PEAK_TFLOPS
    return out


def max_over_ranks(x, world, device):
    """The slowest rank's value (replicas finish when the last one does)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(points_per_replica, steps, world, seconds):
    """Weak scaling: every rank transforms its own copy of the workload each step."""
    return world * points_per_replica * steps / seconds


def time_steps(plan, sigma, out, steps, warmup, flush):
    """Per-step device times (ms) with an L2 flush before every step (not timed).  The plan's
    per-phase profile, when on, is reset after the warm-up so that it covers the timed steps."""
    import torch
    st = torch.cuda.current_stream()
    for _ in range(warmup):
        flush.zero_()
        plan(sigma, out=out)
    torch.cuda.synchronize()
    plan.read_profile()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for e0, e1 in ev:
        flush.zero_()
        e0.record(st)
        plan(sigma, out=out)
        e1.record(st)
    torch.cuda.synchronize()
    return np.array([e0.elapsed_time(e1) for e0, e1 in ev])


def cpu_oracle_rate(w, budget_s=15.0, threads=0, min_leaves=1024):
    """Oracle points/s on a seeded sample of at least min_leaves target leaves (about budget_s of
    CPU work), extrapolated linearly to the whole workload (the oracle's cost is the same per
    target leaf of one level)."""
    import oracle
    rng = np.random.default_rng(123)
    n = w.tree.n_leaves
    probe = np.sort(rng.choice(n, size=min(n, 16), replace=False))
    t0 = time.perf_counter()
    oracle.box_fgt(w.d, w.p, w.delta, w.periodic, w.tree.level, w.tree.coord, w.sigma, targets=probe,
                   threads=threads)
    t_probe = max(time.perf_counter() - t0, 1e-3)
    m = int(np.clip(len(probe) * budget_s / t_probe, min(min_leaves, n), n))
    sample = np.sort(rng.choice(n, size=m, replace=False))
    t0 = time.perf_counter()
    u = oracle.box_fgt(w.d, w.p, w.delta, w.periodic, w.tree.level, w.tree.coord, w.sigma, targets=sample,
                       threads=threads)
    dt = time.perf_counter() - t0
    cores = threads if threads > 0 else oracle.default_threads()
    return m * w.p ** w.d / dt, cores, m, dt, sample, u


def oracle_sample(w, n, seed):
    """Seeded target leaves for an error check, plus the leaves nearest each Gaussian centre and a
    few on the faces of B, with the oracle's u there."""
    import oracle
    rng = np.random.default_rng(seed)
    tg = set(rng.choice(w.tree.n_leaves, min(n, w.tree.n_leaves), replace=False).tolist())
    lev = w.tree.level.astype(np.float64)
    centre = (w.tree.coord + 0.5) / (2.0 ** lev)[:, None] - 0.5
    for c in list(w.meta.get("centers", []))[:8]:
        tg.add(int(np.argmin(((centre - np.asarray(c)[: w.d]) ** 2).sum(axis=1))))
    face = np.where(np.any((w.tree.coord == 0) | (w.tree.coord == (2 ** w.tree.level)[:, None] - 1), axis=1))[0]
    if len(face):
        tg.update(rng.choice(face, min(4, len(face)), replace=False).tolist())
    sample = np.array(sorted(tg))
    u = oracle.box_fgt(w.d, w.p, w.delta, w.periodic, w.tree.level, w.tree.coord, w.sigma, targets=sample)
    return sample, u


def kernel_l1(d, delta, periodic):
    """max over x of the integral of G(x - y; delta) over y in B: sqrt(pi delta) per axis for the
    periodic kernel (one period), sqrt(pi delta) erf(1 / (2 sqrt(delta))) for the free one (x at the
    centre).  |u(x)| <= ||sigma||_inf times this for every density."""
    a = math.sqrt(math.pi * delta) * (1.0 if periodic else math.erf(0.5 / math.sqrt(delta)))
    return a ** d


def error_vs_oracle(u_all, sample, u_or, tol, w=None):
    """max |u - u_oracle| / max |u_oracle| on the sample (acceptance: 10 tol).

    Theorem 1 bounds the kernel's error in absolute terms, so the transform's error scales with
    ||sigma||_inf ||G||_1, not with |u|.  When the exact transform is itself below tol times that
    scale (the periodic trig density at large delta: u = (pi delta)^{d/2} exp(-d pi^2 delta n_p^2)
    sigma_p), max |u| holds only rounding and the row is judged against ||sigma||_inf ||G||_1
    instead ("degenerate")."""
    u = u_all.reshape(-1, u_or.shape[1])[sample]
    err = float(np.abs(u - u_or).max())
    umax = float(np.abs(u_or).max())
    e = err / umax if umax > 0 else math.inf
    out = {"max_abs_over_max_u": e, "bound": 10 * tol, "within_bound": bool(e <= 10 * tol),
           "sample_leaves": int(len(sample))}
    if w is not None:
        floor = float(np.abs(w.sigma).max()) * kernel_l1(w.d, w.delta, w.periodic)
        es = err / floor
        out["max_abs_over_sigma_g1"] = es
        if umax < tol * floor:
            out["degenerate"] = "max|u| below tol ||sigma||_inf ||G||_1; judged on that scale"
            out["within_bound"] = bool(es <= 10 * tol)
    return out


def run_batched_and_serving(args, F, torch, large=()):
    """256 independent free-space transforms (d 2/3, depth 2-7, p 8/12/16, delta 1e-5..1e-1):
    one after another on one stream vs one batched graph launch, split form at tol 1e-6 (FP64
    at 1e-6 too); then the serving runs."""
    import workloads as W
    ws = W.batched_configs(seed=0, n=256)
    npts = sum(w.n_points for w in ws)
    sig = [torch.from_numpy(w.sigma).cuda() for w in ws]
    out = [torch.empty_like(s) for s in sig]
    res = {"transforms": len(ws), "points": int(npts),
           "mix": "d 2/3, tree depth 2-7, p 8/12/16, delta log-U[1e-5,1e-1], 1-8 Gaussians, free space"}
    st = torch.cuda.current_stream()
    for name, prec in (("split_tol1e-6", F.PREC_SPLIT), ("fp64_tol1e-6", F.PREC_FP64)):
        plans = [F.Plan(w.d, w.p, w.delta, 1e-6, w.tree.level, w.tree.coord, prec=prec) for w in ws]
        # launch shapes picked per transform by the library's autotuner before the graph is built
        t0 = time.perf_counter()
        knobs = [p.autotune(s, o, reps=2) for p, s, o in zip(plans, sig, out)]
        tune_s = time.perf_counter() - t0
        batch = F.Batch(plans)
        reps = max(2, args.steps // 4)
        for _ in range(2):
            batch(sig, out)
            for p, s, o in zip(plans, sig, out):
                p(s, out=o)
        torch.cuda.synchronize()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(st)
        for _ in range(reps):
            for p, s, o in zip(plans, sig, out):
                p(s, out=o)
        e1.record(st)
        for _ in range(reps):
            batch(sig, out)
        e2.record(st)
        torch.cuda.synchronize()
        t_serial = e0.elapsed_time(e1) / reps
        t_graph = e1.elapsed_time(e2) / reps
        # the same transforms as one persistent kernel over a device work queue
        ref = [o.clone() for o in out]
        pb = F.Batch(plans, mode=F.BATCH_PERSISTENT)
        pout = [torch.empty_like(o) for o in out]
        for _ in range(2):
            pb(sig, pout)
        torch.cuda.synchronize()
        e3, e4 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e3.record(st)
        for _ in range(reps):
            pb(sig, pout)
        e4.record(st)
        torch.cuda.synchronize()
        t_pers = e3.elapsed_time(e4) / reps
        pdiff = max(float((a - r).abs().max() / r.abs().max()) for a, r in zip(pout, ref))
        pinfo, pstat = pb.info(), pb.status()
        pb.close()
        from collections import Counter
        res[name] = {"serial_ms": t_serial, "serial_points_per_s": npts / t_serial * 1e3,
                     "batched_ms": t_graph, "batched_points_per_s": npts / t_graph * 1e3,
                     "persistent_ms": t_pers, "persistent_points_per_s": npts / t_pers * 1e3,
                     "persistent": {"items": pinfo["items"], "grid": pinfo["grid"], "status": pstat,
                                    "max_rel_diff_vs_graph": pdiff},
                     "autotune_s": tune_s,
                     "autotuned": {k: dict(Counter(int(t[k]) for t in knobs))
                                   for k in ("form_group", "eval_rows16", "eval_rows_large", "near_phase")}}
        batch.close()
        for p in plans:
            p.close()
    return res, run_serving(F, torch, large)


def run_serving(F, torch, large=()):
    """Serving: requests on 24 request geometries (d 2/3, free/periodic, tol 1e-6/1e-10, about 4K
    to 16.8M points) with fresh densities, admitted by footprint, plans kept resident between
    requests (idle plans count against the same 16 GiB budget as the requests in flight).  One
    pass over the geometries warms the plan cache; a burst of 96 requests gives the saturation
    rate; then Poisson arrivals at 0.25, 0.5, 1 and 2 times that rate."""
    import workloads as W
    from paper_2305_07165_gb300 import serving as S
    ws = W.serving_mix(seed=0, n=24 - len(large), max_points=1 << 23) + list(large)
    rng = np.random.default_rng(5)
    srv = S.Server(hbm_budget_bytes=16 << 30, max_inflight=32, plan_cache_bytes=8 << 30).start()

    def req(w):
        return S.Request(d=w.d, k=w.p, delta=w.delta, tol=w.meta["tol"], level=w.tree.level, coord=w.tree.coord,
                         sigma=w.sigma * float(rng.uniform(0.5, 1.5)), bc=int(w.periodic))

    def run(n, rate):
        srv.completed = []
        hits0 = srv.cache_hits
        picks = rng.integers(len(ws), size=n)
        t0 = time.perf_counter()
        futs = []
        for i in picks:
            futs.append(srv.submit(req(ws[i])))
            if rate:
                time.sleep(rng.exponential(1.0 / rate))
        for f in futs:
            f.result(timeout=600)
        st = srv.stats(t0=t0)
        st["plan_cache_hits"] = srv.cache_hits - hits0
        return st

    for f in [srv.submit(req(w)) for w in ws]:   # warm: every geometry planned once
        f.result(timeout=600)
    burst = run(96, None)
    sat = burst["requests"] / (burst["points"] / burst["points_per_s"])
    out = {"geometries": len(ws), "mix": "d 2/3, 3 in 10 periodic, 1 in 4 at tol 1e-10, delta log-U[1e-4,1e-2], "
                                         f"{min(w.n_points for w in ws)}-{max(w.n_points for w in ws)} points",
           "admission_budget_bytes": 16 << 30, "plan_cache_cap_bytes": 8 << 30,
           "budget_counts": "requests in flight + idle cached plans",
           "saturation": dict(burst, requests_per_s=sat), "rate_sweep": {}}
    for frac in (0.25, 0.5, 1.0, 2.0):
        st = run(64, frac * sat)
        st["arrival_rate_per_s"] = frac * sat
        out["rate_sweep"][f"{frac:g}x"] = st
    srv.shutdown()
    return out


def run_sweeps(args, F, torch, w_adapt, flush):
    """The delta sweep of the 3D adaptive workload (delta 1e-4 and 1e-2 next to its 1e-3) in every
    form, and the paper-shaped k = 16 workloads over delta 1e-10 .. 1; every row with its error
    against the oracle on a seeded sample of target leaves.  Fewer steps than the headline (each
    row says how many)."""
    out = {"delta_sweep": {"workload": workload_text(w_adapt)}}
    steps, warm = max(3, args.steps // 4), 2

    def one(w, sig, outt, tol, prec, ref):
        plan = F.Plan(w.d, w.p, w.delta, tol, w.tree.level, w.tree.coord, bc=int(w.periodic), prec=prec)
        info = plan.info()
        t = time_steps(plan, sig, outt, steps, warm, flush)
        plan.close()
        ms = float(t.mean())
        row = {"ms_per_step": ms, "points_per_s": w.n_points / ms * 1e3, "steps": steps,
               "cutoff_level": info["cutoff_level"], "n_f": info["n_f"]}
        row["error_vs_oracle"] = error_vs_oracle(outt.cpu().numpy(), ref[0], ref[1], tol, w)
        return row

    import dataclasses
    import workloads as W_
    sig = torch.from_numpy(w_adapt.sigma).cuda()
    o = torch.empty_like(sig)
    for delta in (1e-4, 1e-2):
        wd = dataclasses.replace(w_adapt, delta=delta)
        ref = oracle_sample(wd, 24, 7)
        row = {}
        for key in args.forms.split(","):
            name, tol, prec = FORMS[key]
            row[name] = one(wd, sig, o, tol, prec, ref)
        out["delta_sweep"][f"{delta:g}"] = row
    del sig, o
    # the paper's experiment shapes (Section 6): sigma_f (five centres, alpha_i = 4e-3 / i) and the
    # periodic sigma_p (n_p = 4), k = 16, delta from 1e-10 to 1
    out["paper_shaped"] = {}
    wf = W_.paper_sigma_f(d=3, p=16, target_points=2_000_000)
    wpp = W_.paper_sigma_p(d=3, p=16, n_p=4, level=3)
    for wk, deltas in ((wf, (1e-10, 1e-8, 1e-6, 1e-4, 1e-3, 1e-2, 1e-1, 1.0)), (wpp, (1e-6, 1e-4, 1e-3, 1e-2, 1.0))):
        sig = torch.from_numpy(wk.sigma).cuda()
        o = torch.empty_like(sig)
        rows = {"workload": workload_text(wk)}
        for delta in deltas:
            wd = dataclasses.replace(wk, delta=delta)
            ref = oracle_sample(wd, 12, 8)
            rows[f"{delta:g}"] = {FORMS[f][0]: one(wd, sig, o, FORMS[f][1], FORMS[f][2], ref)
                                  for f in ("split", "fp64_1e-10")}
        out["paper_shaped"][wk.name] = rows
        del sig, o
    return out


def run_forms(args, F, torch, w, forms, flush, steps, warmup, world, local, clock_head=False):
    """Every form on workload w: launch shapes autotuned on the input, then `steps` timed steps
    (per-step CUDA events, per-phase profile), the roofline of its dominant phase, and its result
    kept for the error check.  With clock_head, the first form's timed region is bracketed by a
    barrier and sampled for clocks.  Returns (results, head, clocks, u per form)."""
    import torch.distributed as dist
    sigma = torch.from_numpy(w.sigma).cuda()
    out = torch.empty_like(sigma)
    results, u_forms, head, clocks = {}, {}, None, None
    for name, tol, prec in forms:
        plan = F.Plan(w.d, w.p, w.delta, tol, w.tree.level, w.tree.coord, bc=int(w.periodic), prec=prec)
        info = plan.info()
        tuned = None if args.no_autotune else plan.autotune(sigma, out, reps=3)
        is_head = head is None
        plan.set_profiling(True)
        if is_head and clock_head:
            with ClockSampler(local) as cs:
                if world > 1:
                    dist.barrier()
                torch.cuda.synchronize()
                times = time_steps(plan, sigma, out, steps, warmup, flush)
                torch.cuda.synchronize()
            clocks = cs.summary()
        else:
            times = time_steps(plan, sigma, out, steps, warmup, flush)
        prof, nprof = plan.read_profile()
        plan.set_profiling(False)
        rl = roofline_of(info, prof, nprof, prec, (args.workload if clock_head else "", name))
        if is_head:
            head = dict(name=name, plan=plan, info=info, prof=prof, nprof=nprof, times=times, tol=tol, prec=prec,
                        roofline=rl)
        else:
            plan.close()
        u_forms[name] = out.cpu().numpy()   # this form's result (last timed step), for its error
        tot = max_over_ranks(float(times.sum()), world, "cuda")
        results[name] = dict(points_per_s=whole_job_rate(w.n_points, steps, world, tot / 1e3),
                             ms_per_step=tot / steps, p50_ms=float(np.percentile(times, 50)),
                             p99_ms=float(np.percentile(times, 99)), steps=steps, cutoff_level=info["cutoff_level"],
                             n_f=info["n_f"], launches=info["launches"], tol=tol,
                             dtype="f32" if prec == 1 else "f64", roofline=rl, tuning=tuned,
                             arithmetic=arithmetic_of(prec, info))
    # the forms against the plain FP64 form at the same tolerance (the metric's comparison)
    for name, tol, prec in forms:
        base = "fp64_tol1e-10" if tol <= 1e-10 else "fp64_tol1e-6"
        if base in results and name != base:
            results[name]["vs_plain_fp64_same_tol"] = results[name]["points_per_s"] / results[base]["points_per_s"]
        if "fp64_tol1e-10" in results and name != "fp64_tol1e-10":
            results[name]["vs_plain_fp64_tol1e-10"] = (results[name]["points_per_s"] /
                                                      results["fp64_tol1e-10"]["points_per_s"])
    del sigma, out
    return results, head, clocks, u_forms


def hbm_peak_gbs():
    """Measured HBM copy bandwidth of the GB300s (MEASURED_PEAKS.json), else the fallback."""
    try:
        with open(PEAKS_FILE) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def run_hierarchical(F, torch, w, sigma, out, flush):
    """The literal order of Algorithm 4 (hierarchical mode): leaves form at their own level, the
    expansions are merged child -> parent level by level (T_c->p), gathered at the cutoff level
    and pushed parent -> child (T_p->c) before the leaves evaluate.  Reports the merge and push
    kernels against the HBM roofline: each merge item reads its 2^d children's slots and writes
    the parent's, each push item reads the parent's slot and writes its 2^d children's."""
    peak, src = hbm_peak_gbs()
    res = {"hbm_peak_gbs": peak, "peak_source": src}
    for name, tol, prec in (FORMS["split"], FORMS["fp64"]):
        plan = F.Plan(w.d, w.p, w.delta, tol, w.tree.level, w.tree.coord, bc=int(w.periodic), prec=prec,
                      mode=F.MODE_HIERARCHICAL)
        info = plan.info()
        plan.set_profiling(True)
        t = time_steps(plan, sigma, out, 5, 3, flush)
        prof, nprof = plan.read_profile()
        plan.close()
        slot_bytes = (8 if prec == F.PREC_SPLIT else 16) * info["modes_1d"] ** (w.d - 1) * info["modes_half"]
        row = {"ms_per_step": float(t.mean()), "merge_items": info["n_merge_items"], "push_items": info["n_push_items"],
               "slot_bytes": slot_bytes}
        for ph, n_items in (("merge", info["n_merge_items"]), ("push", info["n_push_items"])):
            ms = prof.get(ph, 0.0) / max(nprof, 1)
            nbytes = n_items * (2 ** w.d + 1) * slot_bytes
            gbs = nbytes / (ms / 1e3) / 1e9 if ms > 0 else None
            row[ph] = {"ms": ms, "bytes": nbytes, "bytes_kind": "algorithmic (2^d child slots + the parent's, "
                       "per item)", "achieved_gbs": gbs, "frac": gbs / peak if gbs else None}
        res[name] = row
    return res


def u_gauss_free(x, centers, alphas, delta):
    """u = int_B exp(-|x - y|^2 / delta) sum_i exp(-|y - c_i|^2 / alpha_i) dy (free space), per axis a
    Gaussian in y integrated over [-1/2, 1/2] by erf: the reference for the refinement errors."""
    from scipy.special import erf
    out = np.zeros(len(x))
    for c, a in zip(centers, alphas):
        s = np.sqrt(a * delta / (a + delta))
        term = np.ones(len(x))
        for ax in range(x.shape[1]):
            mu = (a * x[:, ax] + delta * c[ax]) / (a + delta)
            term *= (np.exp(-(x[:, ax] - c[ax]) ** 2 / (a + delta)) * s * np.sqrt(np.pi) / 2
                     * (erf((0.5 - mu) / s) - erf((-0.5 - mu) / s)))
        out += term
    return out


def run_refinement(F, torch):
    """Output-tree refinement and coarsening (Algorithms 5 and 6) in the setting of the paper's
    example (Section 4.3): two Gaussians with alpha = 1e-4 (seeded centres), delta = 4e-3, k = 8,
    eps = 1e-12, FP64, 2D, the source tree built on the GPU to resolve sigma (Algorithm 3).  As the
    paper does, the potential on each tree is interpolated to equispaced points (400 x 400 here)
    and compared with the exact u (relative l2 error), before refinement, after it, and after
    coarsening."""
    from paper_2305_07165_gb300 import refine as RF
    d, k, delta, eps = 2, 8, 4e-3, 1e-12
    rng = np.random.default_rng(11)
    centers, alphas = rng.uniform(-0.3, 0.3, size=(2, d)), np.array([1e-4, 1e-4])
    t0 = time.perf_counter()
    level, coord, sigma = F.build_gaussian_tree(d, k, centers, alphas, eps=eps, max_level=12)
    t_build = time.perf_counter() - t0
    plan = F.Plan(d, k, delta, 1e-12, level, coord)
    g = (np.arange(400) + 0.5) / 400 - 0.5
    pts = np.stack(np.meshgrid(g, g, indexing="ij"), axis=-1).reshape(-1, 2)
    ue = u_gauss_free(pts, centers, alphas, delta)

    def l2err(lev, crd, u):
        return float(np.linalg.norm(RF.interpolate(lev, crd, u, d, k, pts) - ue) / np.linalg.norm(ue))

    u0 = plan(sigma)
    err0, sq0 = RF.leaf_errors(u0, d, k)
    norm0 = RF._norm(sq0, level, d)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lev, crd, u, rounds = RF.refine(plan, sigma, eps)
    torch.cuda.synchronize()
    t_ref = time.perf_counter() - t0
    err1, sq1 = RF.leaf_errors(u, d, k)
    t0 = time.perf_counter()
    cl, cc, cu = RF.coarsen(lev, crd, u, d, k, eps)
    torch.cuda.synchronize()
    t_coa = time.perf_counter() - t0
    out = {"setting": "2D, two Gaussians alpha = 1e-4, delta = 4e-3, k = 8, eps = 1e-12, FP64; source tree by "
                      "Algorithm 3 on the GPU; errors: relative l2 at 400 x 400 equispaced points against the "
                      "exact u (erf closed form)",
           "source_leaves": int(len(level)), "source_tree_build_s": t_build,
           "source_tree": {"rel_l2_error": l2err(level, coord, u0),
                           "max_monitor_over_norm": float(err0.max().item() / norm0)},
           "refined_leaves": int(len(lev)), "rounds": rounds, "refine_s": t_ref,
           "refined_tree": {"rel_l2_error": l2err(lev, crd, u),
                            "max_monitor_over_norm": float(err1.max().item() / RF._norm(sq1, lev, d))},
           "coarsened_leaves": int(len(cl)), "coarsen_s": t_coa,
           "coarsened_tree": {"rel_l2_error": l2err(cl, cc, cu)},
           "paper": "input tree about 1e-7, after refinement about 1.3e-12 (4M points)"}
    o = torch.empty_like(u0)
    st = torch.cuda.current_stream()
    plan.set_output_tree(lev, crd)
    o = plan(sigma)
    for _ in range(2):
        plan(sigma, out=o)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(5):
        plan(sigma, out=o)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 5
    plan.close()
    out.update({"output_tree_transform_ms": ms, "output_points_per_s": len(lev) * k ** d / ms * 1e3})
    return out


def run_point_fgt(F, torch):
    """The discrete Gauss transform (Algorithm 2 with proxy grids): 1M sources and 1M targets
    (the same points) clustered around 8 centres in 3D and uniform in 2D, delta = 1e-3 (3D) /
    1e-4 (2D); FP64 at tol 1e-6 and 1e-10, split at tol 1e-6; n_s = 64; points/s = (sources +
    targets) / time."""
    rng = np.random.default_rng(17)
    out = {}
    c = rng.uniform(-0.4, 0.4, size=(8, 3))
    w = np.exp(rng.uniform(np.log(0.02), np.log(0.1), size=8))
    lab = rng.integers(0, 8, 1 << 20)
    sets = {"3d_clustered": (3, 1e-3, c[lab] + w[lab, None] * rng.standard_normal((1 << 20, 3))),
            "2d_uniform": (2, 1e-4, rng.uniform(-0.5, 0.5, size=(1 << 20, 2)))}
    for name, (d, delta, pts) in sets.items():
        q = torch.from_numpy(rng.uniform(0.5, 1.5, len(pts))).cuda()
        u = torch.empty_like(q)
        row = {"points": len(pts), "delta": delta}
        for tol, prec, key in ((1e-6, F.PREC_FP64, "tol1e-06"), (1e-6, F.PREC_SPLIT, "split_tol1e-06"),
                               (1e-10, F.PREC_FP64, "tol1e-10")):
            t0 = time.perf_counter()
            plan = F.PointPlan(d, delta, tol, pts, pts, n_s=64, prec=prec)
            t_plan = time.perf_counter() - t0
            st = torch.cuda.current_stream()
            for _ in range(2):
                plan(q, out=u)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(5):
                plan(q, out=u)
            e1.record(st)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / 5
            row[key] = dict(plan.info(), ms=ms, plan_s=t_plan, points_per_s=2 * len(pts) / ms * 1e3)
            plan.close()
        out[name] = row
    return out


def arithmetic_of(prec, info):
    """What the form's contractions compute in (the dtype key names the expansions' type)."""
    if prec == 1:
        return "split: FP32 expansions, contractions as 3xTF32 tensor-core products (FP32-accurate); near field FP64"
    if prec == 2 and info.get("n_sliced_jobs", 0) > 0:
        return ("FP64 expansions; form and evaluation contractions as exact sums of BF16 digit products on the "
                "tensor cores (operands rounded to 47 bits, six 8-bit digits each, FP32 accumulation exact, "
                "64-bit integer recombination); gather and near field in double-float arithmetic on the FP32 pipes "
                "(FP64 in, FP64 out)")
    if prec == 2:
        return "FP64 throughout, some contractions on the FP64 tensor cores (DMMA)"
    return "FP64 throughout (CUDA cores)"


def metric_name(w, form="fp64_tol1e-10"):
    name, tol = {"fp64_tol1e-10": ("FP64", 1e-10), "split_tol1e-6": ("split", 1e-6), "fp64_tol1e-6": ("FP64", 1e-6),
                 "fp64tc_tol1e-6": ("FP64 tensor-core", 1e-6),
                 "fp64tc_tol1e-10": ("FP64 tensor-core", 1e-10)}.get(form, (form, 0))
    return (f"target points/s (box FGT, {w.d}D {'periodic' if w.periodic else 'free space'}, "
            f"delta={w.delta:g}, tol {tol:g} {name} form)")


def workload_text(w):
    return (f"{w.name}: {w.d}D {'periodic' if w.periodic else 'free space'}, {w.tree.n_leaves} leaves (levels "
            f"{int(w.tree.level.min())}-{int(w.tree.level.max())}), p={w.p}, {w.n_points} points, delta={w.delta:g}")


def run_reference(args):
    """The CPU oracle as the reference arm: each step a bounded sample of target leaves."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    w = workload(args.workload)
    rng = np.random.default_rng(7)
    n = w.tree.n_leaves
    probe = np.sort(rng.choice(n, size=4, replace=False))
    t0 = time.perf_counter()
    oracle.box_fgt(w.d, w.p, w.delta, w.periodic, w.tree.level, w.tree.coord, w.sigma, targets=probe)
    t_leaf = max((time.perf_counter() - t0) / len(probe), 1e-4)
    per_step = 120.0 / max(args.steps + args.warmup, 1)
    m = int(np.clip(per_step / t_leaf, 1, n))
    samples = [np.sort(rng.choice(n, size=m, replace=False)) for _ in range(args.steps + args.warmup)]
    for s in samples[: args.warmup]:
        oracle.box_fgt(w.d, w.p, w.delta, w.periodic, w.tree.level, w.tree.coord, w.sigma, targets=s)
    t0 = time.perf_counter()
    for s in samples[args.warmup:]:
        oracle.box_fgt(w.d, w.p, w.delta, w.periodic, w.tree.level, w.tree.coord, w.sigma, targets=s)
    dt = time.perf_counter() - t0
    value = args.steps * m * w.p ** w.d / dt
    cores = oracle.default_threads()
    line = {
        "impl": "reference", "metric": metric_name(w, FORMS[args.forms.split(",")[0]][0]), "value": value,
        "unit": "points/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_text(w), "sample_leaves_per_step": m},
        "cpu_baseline": {"value": value, "unit": "points/s", "cores": cores, "kind": "oracle",
                         "sample": f"{m} seeded target leaves per step of {n}, rate extrapolated linearly to the "
                                   "whole workload"},
        "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="periodic3d", choices=sorted(WORKLOADS))
    ap.add_argument("--no-batch", action="store_true", help="skip the batched and serving sections")
    ap.add_argument("--no-sweep", action="store_true",
                    help="skip the adaptive-workload section, the delta sweep and the paper-shaped runs")
    ap.add_argument("--no-autotune", action="store_true", help="time the default launch shapes")
    ap.add_argument("--forms", default=DEFAULT_FORMS,
                    help="comma list of " + ", ".join(FORMS) + "; the first one is the headline")
    ap.add_argument("--point-fgt-only", action="store_true",
                    help="run only the point-FGT section and print its JSON (for profiling)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.point_fgt_only:
        import torch

        import paper_2305_07165_gb300 as F
        print(json.dumps({"point_fgt": run_point_fgt(F, torch)}))
        return 0

    import torch
    import torch.distributed as dist

    import paper_2305_07165_gb300 as F

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    w = workload(args.workload)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    forms = [FORMS[f] for f in args.forms.split(",")]
    results, head, clocks, u_forms = run_forms(args, F, torch, w, forms, flush, args.steps, args.warmup, world,
                                               local, clock_head=True)

    # second section: the same forms on the 3D adaptive free-space workload (config 2 shape)
    adaptive = batched = serving = sweeps = refinement = None
    if not args.no_sweep and rank == 0:
        w2 = workload("adaptive3d") if args.workload != "adaptive3d" else w
        r2, h2, _, u2 = run_forms(args, F, torch, w2, forms, flush, max(5, args.steps // 2), 2, 1, local)
        h2["plan"].close()
        ref2 = oracle_sample(w2, 48, 5)
        for fname, ftol, _ in forms:
            r2[fname]["error_vs_oracle"] = error_vs_oracle(u2[fname], ref2[0], ref2[1], ftol, w2)
        del u2
        adaptive = {"workload": workload_text(w2), "forms": r2}
    if not args.no_batch and rank == 0:
        import dataclasses
        # the serving mix reaches the largest single-GPU workload: the headline geometry (16.8M
        # points) at tol 1e-6 and the adaptive one (2.1M points) at tol 1e-10 join 22 drawn ones
        large = [dataclasses.replace(w, meta=dict(w.meta, tol=1e-6))]
        if not args.no_sweep:
            large.append(dataclasses.replace(w2, meta=dict(w2.meta, tol=1e-10)))
        batched, serving = run_batched_and_serving(args, F, torch, large)
    if not args.no_sweep and rank == 0:
        sweeps = run_sweeps(args, F, torch, w2, flush)
        refinement = run_refinement(F, torch)
        refinement["point_fgt"] = run_point_fgt(F, torch)
        s2 = torch.from_numpy(w2.sigma).cuda()
        refinement["hierarchical"] = run_hierarchical(F, torch, w2, s2, torch.empty_like(s2), flush)
        del s2

    # end to end through the host-buffer entry points (pinned host memory, every step's copy in and
    # copy out inside the timed region): pipelined calls (fgt_execute_host_async, two pairs of host
    # buffers in turn, one wait at the end) for the headline, one synchronous call per step beside it
    plan = head["plan"]
    sh = [torch.from_numpy(w.sigma).pin_memory() for _ in range(2)]
    uh = [torch.empty_like(sh[0]).pin_memory() for _ in range(2)]
    for i in range(args.warmup):
        plan.execute_host_async(sh[i % 2], uh[i % 2])
    plan.host_sync()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for i in range(args.steps):
        plan.execute_host_async(sh[i % 2], uh[i % 2])
    plan.host_sync()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, "cuda")
    for _ in range(args.warmup):
        plan.execute_host(sh[0], uh[0])
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        plan.execute_host(sh[0], uh[0])
    e2e_sync_s = max_over_ranks(time.perf_counter() - t0, world, "cuda")

    line = None
    if rank == 0:
        cpu = None
        err = None
        if not args.no_cpu_baseline and world == 1:
            rate, cores, m, dt, sample, u_or = cpu_oracle_rate(w)
            cpu = {"value": rate, "unit": "points/s", "cores": cores, "kind": "oracle",
                   "sample": f"{m} seeded target leaves of {w.tree.n_leaves} ({m * w.p ** w.d} points), {dt:.1f} s; "
                             "rate extrapolated linearly to the whole workload"}
            # every form's result on the same sample, against the oracle (acceptance: 10 tol)
            for fname, ftol, _ in forms:
                results[fname]["error_vs_oracle"] = error_vs_oracle(u_forms[fname], sample, u_or, ftol, w)
            err = dict(results[head["name"]]["error_vs_oracle"], sample=cpu["sample"])
        hr = results[head["name"]]
        line = {
            "metric": metric_name(w, head["name"]),
            "value": hr["points_per_s"], "unit": "points/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": hr["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": hr["dtype"], "data": "synthetic",
            "config": {"workload": workload_text(w), "tol": head["tol"], "form": head["name"],
                       "cache": "L2 flushed (256 MiB write) before every step, outside the timed events; "
                                "inputs (134 MB) and outputs (134 MB) larger than L2",
                       "parallelism": f"replicas x{world}"},
            "latency_ms": {"p50": hr["p50_ms"], "p99": hr["p99_ms"]},
            "forms": results,
            "split_vs_plain_fp64": {k: results["split_tol1e-6"].get(k) for k in
                                    ("vs_plain_fp64_same_tol", "vs_plain_fp64_tol1e-10")}
            if "split_tol1e-6" in results else None,
            "roofline": head["roofline"],
            "roofline_split": results.get("split_tol1e-6", {}).get("roofline"),
            "cpu_baseline": cpu,
            "error_vs_oracle": err,
            "e2e": {"value": world * w.n_points * args.steps / e2e_s, "unit": "points/s",
                    "h2d_bytes_per_step": int(w.n_points * 8), "d2h_bytes_per_step": int(w.n_points * 8),
                    "api": "fgt_execute_host_async per step (copy in / transform / copy out overlapped across "
                           "steps), fgt_host_sync once at the end",
                    "synchronous_value": world * w.n_points * args.steps / e2e_sync_s,
                    "synchronous_api": "fgt_execute_host per step (copy in, transform, copy out, wait)"},
            "gpu_launches": int(head["info"]["launches"] * args.steps),
            "clocks": clocks,
            "adaptive3d": adaptive,
            "batched": batched,
            "serving": serving,
            "sweeps": sweeps,
            "refinement": refinement,
        }
        print(json.dumps(line))
    plan.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
