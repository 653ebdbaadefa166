"""Benchmark: free-space stokeslet Spectral Ewald sum, N = 1e6 uniform points.

One step = one full evaluation (se_eval: binning, spreading, R2C FFT, scaling,
C2R FFT, gather + self term, real-space sum) of the FP32 path (relative error
2e-6, FFT grid capped at 256^3) on inputs already resident in HBM.  The FP64
path (relative error 1e-10) is timed on the same points and reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank evaluates its own copy of the workload
(replicas; weak scaling); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_POINTS = 1_000_000
BOX = (0.0, 0.0, 0.0, 1.0)
METRIC = "Mpoints/s, free-space stokeslet SE N=1e6: FP32 @2e-6 vs FP64 @1e-10; % HBM"
WORKLOAD = "stokeslet sum, N=1e6 uniform iid in [0,1)^3, f iid N(0,1)^3; FP32 path rel. err 2e-6 (P=12, FFT <= 256^3) beside FP64 path rel. err 1e-10"
# FP32 flops of one screened stokeslet pair (see the design notes): difference 3,
# |r|^2 5, rsqrt 1, r 1, xi r 1, -xi^2 r^2 1, exp 2, erfc 20, c e 1, A 2, B 3,
# r.f 5, B (r.f) 1, u += A f + B (r.f) r 12.
FLOP_PER_PAIR = 58
# the same split into the part shared by all right-hand sides (geometry and
# radial functions, 40) and the update per right-hand side (18)
FLOP_RADIAL, FLOP_UPDATE = 40, 18
# DRAM bytes (read + write) of one launch of the FP32 stokeslet real-space kernel on
# this workload, from one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum).
# Set to None whenever that kernel changes, until it is captured again.
REAL_TRAFFIC_BYTES = 58722355  # mean dram__bytes_read.sum + dram__bytes_write.sum over 5 launches
# The same kernel's executed work from that capture: the FP32 pipes' (FMA and
# ALU) busy fractions and the issue-slot utilisation (sm__inst_executed over
# 4 issue slots per SM cycle).  None whenever the kernel changes, until captured again.
REAL_EXECUTED = {"fma_pipe_cycles": 0.592, "alu_pipe": 0.349, "issue_active": 0.708,
                 "warp_inst_per_pair": 4.19e9 / 1.47e9,
                 "source": "ncu, one launch (profiles/k_real_symc_stokeslet_N1e6_fp32.md)"}


def pair_fraction_unit_cube(r: float) -> float:
    """P(|X - Y| <= r) for X, Y uniform in the unit cube (r <= 1): the integral of the
    distance density 4 pi r^2 - 6 pi r^3 + 8 r^4 - r^5."""
    return 4 * math.pi / 3 * r**3 - 1.5 * math.pi * r**4 + 1.6 * r**5 - r**6 / 6


def read_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix="se_clocks_", suffix=".csv")
        os.close(fd)

    def __enter__(self):
        try:
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            # the sampler is running before the timed region starts: wait (3 s at
            # most) for its first line
            t0 = time.perf_counter()
            while time.perf_counter() - t0 < 3.0 and os.path.getsize(self.path) == 0:
                time.sleep(0.01)
            self.skip = sum(1 for _ in open(self.path))
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc:
            return None
        try:
            lines = [ln for ln in open(self.path).read().strip().splitlines() if ln.strip()]
            # samples taken during the timed region (the lines present before it are
            # dropped unless nothing else came)
            rows = [ln.split(",") for ln in (lines[self.skip:] or lines)]
            os.unlink(self.path)
            sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
            mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            reasons = set()
            for r in rows:
                for k, nm in enumerate(names):
                    if len(r) > 5 + k and r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            return {"sm_mhz": float(np.median(sm)) if sm else None,
                    "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                    "samples": len(rows)}
        except Exception:
            return None


def rel_errors(got, ref, bar):
    """Relative L2 (rms) and relative max error of got against ref over all
    components (reading c10): |d|_2 / |ref|_2 and max|d| / max|ref|."""
    got, ref = np.asarray(got, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    d = got - ref
    l2 = float(np.linalg.norm(d) / np.linalg.norm(ref))
    mx = float(np.abs(d).max() / np.abs(ref).max())
    return {"rel_l2": l2, "rel_max": mx, "bar": bar, "ok": bool(l2 <= bar and mx <= bar)}


def cpu_baseline(x, f, budget_s=12.0):
    """The oracle's FP64 direct sum (all N sources) at a bounded random sample of
    targets, on the host cores; Mpoints/s = sampled targets / time.  Returns the
    line's object, the sampled targets and the oracle's values there (they also
    check the FP64 path's result)."""
    from oracle import direct
    rng = np.random.default_rng(123)
    t0 = time.perf_counter()
    # calibrate on enough targets to keep every host core busy
    ncal = 16 * (os.cpu_count() or 1)
    direct.direct("stokeslet", x, f, targets=rng.choice(len(x), ncal, replace=False))
    rate = ncal / max(time.perf_counter() - t0, 1e-6)
    nt = int(max(ncal, min(len(x), rate * budget_s)))
    idx = rng.choice(len(x), nt, replace=False)
    t0 = time.perf_counter()
    ref = direct.direct("stokeslet", x, f, targets=idx)
    dt = time.perf_counter() - t0
    return ({"value": nt / dt / 1e6, "unit": "Mpoints/s", "cores": os.cpu_count(), "kind": "oracle",
             "sample": f"FP64 direct sum over all {len(x)} sources at {nt} random targets "
                       f"({dt:.1f} s), scaled to targets per second"}, idx, ref)


def oracle_checks(chk):
    """Errors of the timed results against the FP64 direct sums of the oracle,
    at sampled targets, after every timed region (the oracle is the checker
    here, never on the timed path).  FP32 results are compared with the sums
    over the FP32-rounded inputs (reading c11).  `chk` holds, per result, the
    inputs and the GPU's output at the sampled targets."""
    from oracle import direct
    out = {}
    t0 = time.perf_counter()
    if "fp32" in chk:
        c = chk["fp32"]
        ref = direct.direct("stokeslet", c["x"], c["f"], targets=c["idx"])
        out["fp32"] = dict(rel_errors(c["u"], ref, 2e-6), targets=len(c["idx"]))
        if "deterministic" in chk:  # the same points and targets, deterministic mode
            out["stokeslet_deterministic"] = dict(rel_errors(chk["deterministic"]["u"], ref, 2e-6),
                                                  targets=len(c["idx"]))
    if "fp64" in chk:
        c = chk["fp64"]
        out["fp64"] = dict(rel_errors(c["u"], c["ref"], 1e-10), targets=len(c["idx"]))
    if "batched" in chk:
        c = chk["batched"]
        num = den = 0.0
        worst, worst_max, worst_s = 0.0, 0.0, -1
        for s, (x, f, idx, u) in enumerate(c["systems"]):
            d_s = n_s = 0.0
            dmax = rmax = 0.0
            for r in range(f.shape[1]):
                ref = direct.direct("stokeslet", x, f[:, r, :], targets=idx)
                d = u[:, r, :] - ref
                d_s += float(np.sum(d * d))
                n_s += float(np.sum(ref * ref))
                dmax, rmax = max(dmax, float(np.abs(d).max())), max(rmax, float(np.abs(ref).max()))
            num, den = num + d_s, den + n_s
            e = float(np.sqrt(d_s / n_s))
            if e > worst:
                worst, worst_s = e, c["ids"][s]
            worst_max = max(worst_max, dmax / rmax)
        out["batched"] = {"rel_l2_pooled": float(np.sqrt(num / den)), "rel_l2_worst_system": worst,
                          "worst_system": worst_s, "rel_max_worst_system": worst_max, "bar": 2e-6,
                          "ok": bool(worst <= 2e-6 and worst_max <= 2e-6),
                          "targets": c["targets_note"]}
    if "stresslet" in chk:
        c = chk["stresslet"]
        ref = direct.direct("stresslet", c["x"], c["f"], c["q"], targets=c["idx"])
        out["stresslet_clustered"] = dict(rel_errors(c["u"], ref, 2e-6), targets=len(c["idx"]))
    if "rotlet" in chk:
        c = chk["rotlet"]
        x, t, g, idx = c["x"], c["f"], c["g"], c["idx"]
        out["rotlet_backward"] = {
            "u": rel_errors(c["u"], direct.direct("rotlet", x, t, targets=idx), 2e-6),
            "grad_f": rel_errors(c["gf"], direct.grad_f("rotlet", x, g, targets=idx), 2e-6),
            "grad_x": rel_errors(c["gx"], direct.grad_x("rotlet", x, t, g, targets=idx), 2e-6),
            "targets": len(idx)}
    out["oracle_s"] = time.perf_counter() - t0
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return
    import workloads as W
    x, f = W.stokeslet_uniform(N_POINTS, 1)
    from oracle import direct
    rng = np.random.default_rng(7)
    t0 = time.perf_counter()
    ncal = 16 * (os.cpu_count() or 1)
    direct.direct("stokeslet", x, f, targets=rng.choice(N_POINTS, ncal, replace=False))
    rate = ncal / max(time.perf_counter() - t0, 1e-6)
    per_step = int(max(ncal, min(N_POINTS, rate * 8.0)))  # about 8 s of CPU work per step
    times = []
    for s in range(args.warmup + args.steps):
        idx = rng.choice(N_POINTS, per_step, replace=False)
        t0 = time.perf_counter()
        direct.direct("stokeslet", x, f, targets=idx)
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    ms = 1e3 * float(np.mean(times))
    val = per_step / (ms * 1e-3) / 1e6
    sample = (f"FP64 direct sum over all {N_POINTS} sources at {per_step} random targets per step")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": "Mpoints/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": N_POINTS, "reference": "CPU oracle (no reference code exists)"},
        "cpu_baseline": {"value": val, "unit": "Mpoints/s", "cores": os.cpu_count(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": val, "unit": "Mpoints/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def f32_in_box(x, L=1.0):
    """x as FP32, kept inside the half-open box [0, L)^3 after rounding."""
    return np.minimum(x.astype(np.float32), np.nextafter(np.float32(L), np.float32(0)))


def run_batched(args, rank, world, dist, dev, flush):
    """64 independent stokeslet systems (sizes lognormal(ln 1e4, 1) clipped to
    [1e3, 1e5], each in its own unit cube), 8 right-hand sides each, FP32 at
    2e-6; one se_batch_eval per step, replayed from its CUDA graph.  With N
    ranks the systems are split by estimated cost (no data-path collective);
    value = all systems' points / max-over-ranks step time."""
    import torch

    import paper_1607_04808_gb300 as se
    import workloads as W
    from paper_1607_04808_gb300 import shard

    R = 8
    systems = W.batched_systems(64, R, 5)
    sizes = [len(x) for x, _ in systems]
    mine = shard.partition(shard.system_costs("stokeslet", sizes, None, R), world)[rank]
    xs = torch.tensor(np.concatenate([f32_in_box(systems[s][0]) for s in mine]), device=dev)
    fs = torch.tensor(np.concatenate([systems[s][1] for s in mine]), dtype=torch.float32, device=dev)
    B = se.Batch("stokeslet", [sizes[s] for s in mine], None, R, tol=2e-6, prec="fp32")
    u = torch.empty_like(fs)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        B.eval(xs, fs, out=u)
    B.check()
    times = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for _ in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        B.eval(xs, fs, out=u)
        b.record(stream)
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    B.check()
    ms = float(np.mean(times))
    if dist:
        t = torch.tensor([ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    # per-stage times from 3 further evaluations with stage timing on (no graph)
    B.set_timing(True)
    st_acc = {}
    for _ in range(3):
        flush.zero_()
        B.eval(xs, fs, out=u)
        for k, v in B.stage_times().items():
            st_acc.setdefault(k, []).append(v)
    B.set_timing(False)
    stages = {k: float(np.mean(v)) for k, v in st_acc.items()}
    # the dominant kernel (real space: every ordered pair within each system's
    # rc, the radial functions once per pair, the update per right-hand side)
    pairs = sum(sizes[s] * (sizes[s] - 1) * pair_fraction_unit_cube(B.params(k)["rc"])
                for k, s in enumerate(mine))
    flop = pairs * (FLOP_RADIAL + FLOP_UPDATE * R)
    # this rank's systems at sampled targets (all targets of systems up to 2e3
    # points, 64 otherwise), for the error check after the timed regions
    uh = u.double().cpu().numpy()
    rng = np.random.default_rng(17)
    chk_sys = []
    for k, s in enumerate(mine):
        n = sizes[s]
        idx = np.arange(n) if n <= 2000 else np.sort(rng.choice(n, 64, replace=False))
        o = B.offsets[k]
        chk_sys.append((f32_in_box(systems[s][0]).astype(np.float64),
                        systems[s][1].astype(np.float32).astype(np.float64), idx, uh[o + idx]))
    check = {"systems": chk_sys, "ids": list(mine),
             "targets_note": "every target of systems up to 2e3 points, 64 random targets otherwise, "
                             f"all {R} right-hand sides, {len(mine)} systems of rank {rank}"}
    n_all = int(sum(sizes))
    out = {"value": n_all / (ms * 1e-3) / 1e6, "unit": "Mpoints/s", "rhs_per_point": R,
           "point_rhs_per_s": n_all * R / (ms * 1e-3), "ms_per_step": ms, "systems": 64, "points": n_all,
           "tol": 2e-6, "P": B.params(0)["P"], "launches_per_step": B.launch_count(),
           "graph": True, "workload": "64 stokeslet systems, N_s lognormal(ln 1e4, 1) clipped to [1e3, 1e5], "
                                      "each in [0,1)^3, 8 RHS ~ N(0,1)^3, FP32 rel. err 2e-6",
           "sharding": f"{len(mine)} of 64 systems on rank {rank} (cost-balanced), max over {world} ranks",
           "stages_ms": stages,
           "stages_note": "3 further evaluations with stage timing on (kernels launched without the graph); "
                          "spread includes the octant zeroing, real the cluster lists",
           "roofline": {"bound": "alu", "kernel": "k_real_cl (batched real-space sum, full candidate lists, "
                        f"{R} right-hand sides per pass)",
                        "achieved": flop / (stages["real"] * 1e-3) / 1e12 if stages.get("real") else None,
                        "unit": "TFLOP/s",
                        "work": f"algorithmic: ordered pairs within each system's rc (expected count for uniform "
                                f"points in its unit cube) x ({FLOP_RADIAL} + {FLOP_UPDATE} x {R}) flop (the "
                                "radial functions once per pair, the update per right-hand side)",
                        "pairs_per_launch": pairs}}
    B.close()
    return out, check


def run_other_configs(dev, flush, checks, x32=None, f32=None):
    """The clustered FP32 stresslet (N = 5e5: 16 Gaussian blobs, sigma 0.05,
    plus 20 % uniform background) and the FP32 rotlet with its backward
    (N = 2e5 uniform, du/df and du/dx, grid recomputed): median device times
    of 5 calls each after 2 warm-ups, stage times from one more timed call."""
    import torch

    import paper_1607_04808_gb300 as se
    import workloads as W

    def timed(fn, reps=5):
        fn()
        fn()
        ts = []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.median(ts))

    out = {}
    if x32 is not None:
        # the headline points without the FFT cap: parameters from the points
        prm = se.choose_params_points("stokeslet", x32.cpu().numpy(), BOX, tol=2e-6)
        plan = se.Plan("stokeslet", x32.shape[0], BOX, prec="fp32", tol=2e-6,
                       **{k: prm[k] for k in ("xi", "M", "P", "rc", "cell_width")})
        u = torch.empty_like(x32)
        ms = timed(lambda: plan.eval(x32, f32, out=u))
        plan.set_timing(True)
        plan.eval(x32, f32, out=u)
        torch.cuda.synchronize()
        st = plan.stage_times()
        plan.check()
        out["stokeslet_uncapped"] = {
            "workload": "the headline points and forces (N = 1e6 uniform, FP32 at 2e-6) without the 256^3 FFT cap, "
                        "parameters from se_choose_params_points",
            "value": x32.shape[0] / (ms * 1e-3) / 1e6, "unit": "Mpoints/s", "ms_per_step": ms,
            "params": {k: plan.params[k] for k in ("M", "P", "xi", "rc")}, "fft": plan.grid["Mf"][0],
            "stages_ms": st}
        plan.close()
        # the headline plan (FFT <= 256^3) in deterministic mode: stable bin
        # order, atomic-free spreading, full-list real-space sum, in sequence
        plan = se.Plan("stokeslet", x32.shape[0], BOX, prec="fp32", tol=2e-6, max_fft=256)
        plan.set_deterministic(True)
        u = torch.empty_like(x32)
        ms = timed(lambda: plan.eval(x32, f32, out=u))
        u1 = u.clone()
        plan.eval(x32, f32, out=u)
        torch.cuda.synchronize()
        same = bool(torch.equal(u, u1))
        plan.set_timing(True)
        plan.eval(x32, f32, out=u)
        torch.cuda.synchronize()
        st = plan.stage_times()
        plan.check()
        if "fp32" in checks:
            checks["deterministic"] = {"u": u1[torch.as_tensor(checks["fp32"]["idx"], device=u1.device)]
                                       .double().cpu().numpy()}
        out["stokeslet_deterministic"] = {
            "workload": "the headline workload (N = 1e6 uniform, FP32 at 2e-6, FFT <= 256^3) with "
                        "se_plan_set_deterministic on",
            "value": x32.shape[0] / (ms * 1e-3) / 1e6, "unit": "Mpoints/s", "ms_per_step": ms,
            "bit_identical_repeat": same, "stages_ms": st}
        plan.close()
    x, f, q = W.stresslet_blobs(500_000, 2)
    t = lambda a: torch.tensor(a, dtype=torch.float32, device=dev)  # noqa: E731
    x32 = f32_in_box(x)
    xd, fd, qd = torch.tensor(x32, device=dev), t(f), t(q)
    # parameters from the points (se_choose_params_points), beside the
    # selection that assumes uniform points
    t_sel = time.perf_counter()
    prm = se.choose_params_points("stresslet", x32, BOX, tol=2e-6)
    t_sel = time.perf_counter() - t_sel
    res = {}
    for name, kw in (("points", {k: prm[k] for k in ("xi", "M", "P", "rc", "cell_width")}), ("uniform", {})):
        plan = se.Plan("stresslet", len(x), BOX, prec="fp32", tol=2e-6, **kw)
        u = torch.empty_like(xd)
        ms = timed(lambda: plan.eval(xd, fd, qd, out=u))
        plan.set_timing(True)
        plan.eval(xd, fd, qd, out=u)
        torch.cuda.synchronize()
        st = plan.stage_times()
        plan.check()
        res[name] = (ms, {k: plan.params[k] for k in ("M", "P", "xi", "rc")}, st)
        plan.close()
    ms, pp, st = res["points"]
    # the output of the point-aware parameters at sampled targets (error check)
    plan = se.Plan("stresslet", len(x), BOX, prec="fp32", tol=2e-6,
                   **{k: prm[k] for k in ("xi", "M", "P", "rc", "cell_width")})
    us = plan.eval(xd, fd, qd, check=True).double().cpu().numpy()
    plan.close()
    sidx = np.sort(np.random.default_rng(19).choice(len(x), 512, replace=False))
    checks["stresslet"] = {"x": x32.astype(np.float64), "f": f.astype(np.float32).astype(np.float64),
                           "q": q.astype(np.float32).astype(np.float64), "idx": sidx, "u": us[sidx]}
    out["stresslet_clustered"] = {
        "workload": "stresslet sum, N = 5e5: 16 Gaussian blobs (sigma 0.05) + 20 % uniform, FP32 at 2e-6",
        "value": len(x) / (ms * 1e-3) / 1e6, "unit": "Mpoints/s", "ms_per_step": ms,
        "params": pp, "params_source": f"se_choose_params_points ({1e3 * t_sel:.0f} ms on the host)",
        "stages_ms": st, "uniform_params": res["uniform"][1], "uniform_params_ms_per_step": res["uniform"][0]}
    x, tq, g = W.rotlet_uniform(200_000, 3)
    xd, td, gd = torch.tensor(f32_in_box(x), device=dev), t(tq), t(g)
    plan = se.Plan("rotlet", len(x), BOX, prec="fp32", tol=2e-6)
    u = torch.empty_like(xd)
    ms_f = timed(lambda: plan.eval(xd, td, out=u))
    ms_b = timed(lambda: plan.backward(xd, td, gd))
    gf, gx = plan.backward(xd, td, gd)
    ridx = np.sort(np.random.default_rng(23).choice(len(x), 256, replace=False))
    checks["rotlet"] = {"x": f32_in_box(x).astype(np.float64), "f": tq.astype(np.float32).astype(np.float64),
                        "g": g.astype(np.float32).astype(np.float64), "idx": ridx,
                        "u": u.double().cpu().numpy()[ridx], "gf": gf.double().cpu().numpy()[ridx],
                        "gx": gx.double().cpu().numpy()[ridx]}
    plan.set_timing(True)
    plan.backward(xd, td, gd)
    torch.cuda.synchronize()
    st = plan.stage_times(backward=True)
    plan.check()
    out["rotlet_backward"] = {
        "workload": "rotlet sum, N = 2e5 uniform, FP32 at 2e-6: forward, and backward (du/df, du/dx, grid recomputed)",
        "forward_ms": ms_f, "backward_ms": ms_b, "value": len(x) / ((ms_f + ms_b) * 1e-3) / 1e6,
        "unit": "Mpoints/s (forward + backward)", "params": {k: plan.params[k] for k in ("M", "P", "xi", "rc")},
        "backward_stages_ms": st}
    plan.close()
    return out


def run_ours(args, rank, world, dist):
    import torch

    import paper_1607_04808_gb300 as se
    import workloads as W
    from paper_1607_04808_gb300 import _build

    _build.build()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    x64, f64 = W.stokeslet_uniform(N_POINTS, 1)
    x32 = torch.tensor(f32_in_box(x64), device=dev)
    f32 = torch.tensor(f64, dtype=torch.float32, device=dev)
    se.set_precompute_cache(False, None)  # time the precomputation itself
    t_plan = time.perf_counter()
    plan = se.Plan("stokeslet", N_POINTS, BOX, prec="fp32", tol=2e-6, max_fft=256)
    t_plan = time.perf_counter() - t_plan
    pre_ms, _ = plan.precompute_info()
    se.set_precompute_cache(True, None)
    prm = plan.params
    # timed steps overlap the Fourier part with the real-space sum; the per-stage
    # times come from a separate pass with stage timing on (stages in sequence)
    plan.set_timing(False)
    u = torch.empty_like(x32)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        plan.eval(x32, f32, out=u)
    plan.check()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    stage_acc = {}
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_wall = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()
            evs[k][0].record(stream)
            plan.eval(x32, f32, out=u)
            evs[k][1].record(stream)
            torch.cuda.synchronize()
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    launches_per_eval = plan.launch_count()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    ms = float(np.mean(step_ms))
    if dist:
        t = torch.tensor([ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    plan.check()
    checks = {}
    # the timed steps' output at sampled targets (error check after the timed regions)
    idx32 = np.sort(np.random.default_rng(29).choice(N_POINTS, 1024, replace=False))
    checks["fp32"] = {"x": f32_in_box(x64).astype(np.float64), "f": f64.astype(np.float32).astype(np.float64),
                      "idx": idx32, "u": u.double().cpu().numpy()[idx32]}
    plan.set_timing(True)
    seq_ms = []
    for _ in range(3):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        plan.eval(x32, f32, out=u)
        b.record(stream)
        torch.cuda.synchronize()
        seq_ms.append(a.elapsed_time(b))
        for name, v in plan.stage_times().items():
            stage_acc.setdefault(name, []).append(v)
    plan.set_timing(False)
    plan.check()
    stages = {k: float(np.mean(v)) for k, v in stage_acc.items()}

    # end to end through se_eval_host (pinned host buffers; copies inside the timed region)
    xh = torch.tensor(f32_in_box(x64)).pin_memory()
    fh = torch.tensor(f64, dtype=torch.float32).pin_memory()
    uh = torch.empty((N_POINTS, 3), dtype=torch.float32).pin_memory()
    plan.set_timing(False)
    for _ in range(3):
        plan.eval_host(xh, fh, out=uh)
    # each call is timed on the host clock (copies, evaluation, synchronisation);
    # the median over 20 calls is the value, robust to a stall of the host
    e2e_t = []
    for _ in range(20):
        t0 = time.perf_counter()
        plan.eval_host(xh, fh, out=uh)
        e2e_t.append(time.perf_counter() - t0)
    e2e_ms = 1e3 * float(np.median(e2e_t))
    e2e_mean_ms = 1e3 * float(np.mean(e2e_t))

    batched = None
    if not args.no_batch:
        batched, checks["batched"] = run_batched(args, rank, world, dist, dev, flush)

    # FP64 path on the same points
    fp64 = None
    if not args.no_fp64:
        x64d = torch.tensor(x64, device=dev)
        f64d = torch.tensor(f64, device=dev)
        se.set_precompute_cache(False, None)  # time the FP64 precomputation itself
        t64p = time.perf_counter()
        plan64 = se.Plan("stokeslet", N_POINTS, BOX, prec="fp64", tol=1e-10)
        t64p = time.perf_counter() - t64p
        pre64_ms, _ = plan64.precompute_info()
        se.set_precompute_cache(True, None)
        p64 = plan64.params
        plan64.set_timing(True)
        u64 = torch.empty_like(x64d)
        plan64.eval(x64d, f64d, out=u64)
        torch.cuda.synchronize()
        t64 = []
        st64 = {}
        for _ in range(2):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            plan64.eval(x64d, f64d, out=u64)
            b.record(stream)
            torch.cuda.synchronize()
            t64.append(a.elapsed_time(b))
            for name, v in plan64.stage_times().items():
                st64.setdefault(name, []).append(v)
        plan64.check()
        u64_host = u64.cpu().numpy()
        ms64 = float(np.mean(t64))
        fp64 = {"value": N_POINTS / (ms64 * 1e-3) / 1e6, "unit": "Mpoints/s", "ms_per_step": ms64,
                "tol": 1e-10, "params": {k: p64[k] for k in ("M", "P", "xi", "rc", "Mtilde")},
                "stages_ms": {k: float(np.mean(v)) for k, v in st64.items()},
                "fp32_speedup": ms64 / ms,
                "plan": {"create_ms": 1e3 * t64p, "precompute_ms": pre64_ms, "Mg": p64.get("Mg"),
                         "note": "FP64 precompute of Section 4.3 on the Mg^3 grid, outside the timed steps"}}
        plan64.close()

    # the triply periodic sum of the same points in the unit cube (FP32, same tolerance)
    periodic = None
    if not args.no_periodic:
        planp = se.Plan("stokeslet", N_POINTS, BOX, prec="fp32", tol=2e-6, periodic=True)
        pp = planp.params
        planp.set_timing(True)
        up = torch.empty_like(x32)
        planp.eval(x32, f32, out=up)
        torch.cuda.synchronize()
        tp, stp = [], {}
        for _ in range(3):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            planp.eval(x32, f32, out=up)
            b.record(stream)
            torch.cuda.synchronize()
            tp.append(a.elapsed_time(b))
            for name, v in planp.stage_times().items():
                stp.setdefault(name, []).append(v)
        planp.check()
        msp = float(np.mean(tp))
        periodic = {"value": N_POINTS / (msp * 1e-3) / 1e6, "unit": "Mpoints/s", "ms_per_step": msp,
                    "tol": 2e-6, "params": {k: pp[k] for k in ("M", "P", "xi", "rc")},
                    "stages_ms": {k: float(np.mean(v)) for k, v in stp.items()},
                    "workload": "the same points and forces, triply periodic stokeslet sum in the unit cube "
                                "(k = 0 mode left out), FFT M^3 unpadded, real space by nearest images"}
        planp.close()

    if rank != 0:
        return
    others = None if args.no_extra else run_other_configs(dev, flush, checks, x32, f32)
    value = world * N_POINTS / (ms * 1e-3) / 1e6
    peaks = read_peaks()
    clocks = clk.summary()
    sm_max = (peaks or {}).get("sm_max_mhz", 2070.0)
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    # FP32 peak from the unit counts: SMs x 128 FP32 lanes x 2 flop (FMA) x clock
    alu_peak = n_sm * 128 * 2 * sm_max * 1e6 / 1e12
    probe = se.measure_peaks()  # measured FMA rates (register-only kernels), after the timed regions
    pairs = N_POINTS * (N_POINTS - 1) * pair_fraction_unit_cube(prm["rc"] / BOX[3])
    real_ms = stages.get("real", float("nan"))
    achieved = pairs * FLOP_PER_PAIR / (real_ms * 1e-3) / 1e12
    hbm = (peaks or {}).get("hbm_gbs", 6800.0)
    Mt, Mf = prm["Mtilde"], 2 * prm["Mtilde"]
    nk = Mf * Mf * (Mf // 2 + 1)
    stage_bytes = {
        "spread": N_POINTS * 32 + 2 * 3 * Mt**3 * 4,
        # the fused z-transforms and scaling: the Mtilde nonzero z-planes of the
        # three spectra read and written once, and the kernel's octant
        "scale": 2 * 3 * Mt * Mf * (Mf // 2 + 1) * 8 + (Mt + 1) ** 3 * 4,
        "gather": 3 * Mt**3 * 4 + N_POINTS * (16 + 12 + 12),
        "real": N_POINTS * (32 + 24),
    }
    stage_gbs = {k: stage_bytes[k] / (stages[k] * 1e-3) / 1e9 for k in stage_bytes if stages.get(k)}
    # each hand-written stage against the roofline that binds it: spreading and
    # the gather are FP32 FMA work on register columns (3 P^3 FMA per point),
    # the scaling streams the spectrum through HBM, the real-space sum is FP32
    # ALU work (58 flop per pair); the FMA-bound stages also against the FMA
    # rate measured on this GPU
    P = prm["P"]
    grid_flop = N_POINTS * 3 * P**3 * 2
    stage_roofline = {}
    for k, bound, work, unit, peak in (
            ("spread", "fma", grid_flop, "TFLOP/s", alu_peak),
            ("gather", "fma", grid_flop, "TFLOP/s", alu_peak),
            ("scale", "hbm", stage_bytes["scale"], "GB/s", hbm),
            ("real", "alu", pairs * FLOP_PER_PAIR, "TFLOP/s", alu_peak)):
        if stages.get(k):
            a = work / (stages[k] * 1e-3) / (1e9 if unit == "GB/s" else 1e12)
            stage_roofline[k] = {"bound": bound, "achieved": a, "peak": peak, "unit": unit, "frac": a / peak}
            if unit == "TFLOP/s" and probe.get("fp32_fma_tflops"):
                stage_roofline[k]["frac_of_measured"] = a / probe["fp32_fma_tflops"]
    if "scale" in stage_roofline:
        stage_roofline["scale"]["note"] = ("the scaling fused with the transforms along z: its algorithmic bytes "
                                           "against the copy rate; the kernel is bound by its shared-memory passes "
                                           "(profiles/k_zscale_stokeslet_N1e6_fp32.md)")
    if batched is not None and batched.get("roofline", {}).get("achieved"):
        br = batched["roofline"]
        br.update(peak=alu_peak, frac=br["achieved"] / alu_peak, peak_measured=probe["fp32_fma_tflops"],
                  frac_of_measured=br["achieved"] / probe["fp32_fma_tflops"])
    cpu = None
    if not args.no_cpu:
        cpu, cidx, cref = cpu_baseline(x64, f64)
        if fp64 is not None:
            checks["fp64"] = {"idx": cidx, "ref": cref, "u": u64_host[cidx]}
    if fp64 is not None:
        # the FP64 stages against the measured FP64 FMA rate (the algorithmic
        # counts of the FP32 stages: 3 P^3 FMA per point in spreading and gather,
        # 58 flop per ordered pair within rc)
        P64, st64 = fp64["params"]["P"], fp64["stages_ms"]
        pairs64 = N_POINTS * (N_POINTS - 1) * pair_fraction_unit_cube(fp64["params"]["rc"] / BOX[3])
        work64 = {"spread": N_POINTS * 3 * P64**3 * 2, "gather": N_POINTS * 3 * P64**3 * 2,
                  "real": pairs64 * FLOP_PER_PAIR}
        fp64["stage_roofline"] = {
            k: {"bound": "fp64 fma", "achieved": w / (st64[k] * 1e-3) / 1e12, "unit": "TFLOP/s",
                "peak": probe["fp64_fma_tflops"], "peak_source": "measured (se_measure_peaks)",
                "frac": w / (st64[k] * 1e-3) / 1e12 / probe["fp64_fma_tflops"]}
            for k, w in work64.items() if st64.get(k)}
    errors = oracle_checks(checks) if not args.no_cpu else None
    if errors:
        for key, obj in (("fp64", fp64), ("batched", batched)):
            if obj is not None and key in errors:
                obj["error"] = errors[key]
        if others:
            for key in ("stresslet_clustered", "rotlet_backward", "stokeslet_deterministic"):
                if key in others and key in errors:
                    others[key]["error"] = errors[key]
    line = {
        "metric": METRIC, "value": value, "unit": "Mpoints/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": N_POINTS, "tol": 2e-6, "max_fft": 256,
                   "params": {k: prm[k] for k in ("M", "P", "xi", "rc", "Mtilde", "eta")},
                   "l2": "512 MB buffer zeroed between timed steps, outside the per-step events",
                   "parallelism": f"replicas x{world}", "wall_s_timed_region": t_wall},
        "stages_ms": stages,
        "stages_note": "per-stage times from 3 extra evaluations with stage timing on, stages in sequence "
                       f"({float(np.mean(seq_ms)):.3f} ms per evaluation); the timed steps run the Fourier part "
                       "on a second stream beside the real-space sum (se_plan_set_overlap)",
        "sequential_ms_per_step": float(np.mean(seq_ms)),
        "stage_algorithmic_gbs": stage_gbs,
        "stage_roofline": stage_roofline,
        "roofline": {"bound": "alu", "kernel": "k_real_symc (real-space pair sum, each pair once)", "achieved": achieved,
                     "peak": alu_peak, "unit": "TFLOP/s", "frac": achieved / alu_peak, "traffic": REAL_TRAFFIC_BYTES,
                     "peak_source": f"derived: {n_sm} SMs (device attribute) x 128 FP32 lanes x 2 flop x "
                                    f"{sm_max:.0f} MHz",
                     "peak_measured": probe["fp32_fma_tflops"],
                     "frac_of_measured": achieved / probe["fp32_fma_tflops"],
                     "work": "algorithmic: ordered pairs within rc (expected count for uniform points) x "
                             f"{FLOP_PER_PAIR} flop, as a direct evaluation of every ordered pair needs; the kernel "
                             "evaluates each unordered pair once",
                     "executed": REAL_EXECUTED,
                     "pairs_per_launch": pairs, "flop_per_pair": FLOP_PER_PAIR},
        "measured_peaks": dict(probe, source="se_measure_peaks: register-only FMA kernels on this GPU, "
                                             "after the timed regions"),
        "error": errors.get("fp32") if errors else None,
        "errors_note": ("relative L2 and relative max error against the oracle's FP64 direct sum at sampled "
                        "targets (FP32 results against the sums over the FP32-rounded inputs), taken after "
                        f"the timed regions ({errors['oracle_s']:.1f} s)") if errors else None,
        "hbm_peak_gbs": hbm,
        "plan": {"create_ms": 1e3 * t_plan, "precompute_ms": pre_ms,
                 "note": "plan creation (parameter choice, allocation, cuFFT plans, FP64 precompute of "
                         "Section 4.3) is outside the timed steps"},
        "fp64": fp64,
        "periodic": periodic,
        "batched": batched,
        "other_configs": others,
        "cpu_baseline": cpu,
        "e2e": {"value": N_POINTS / (e2e_ms * 1e-3) / 1e6, "unit": "Mpoints/s", "ms_per_step": e2e_ms,
                "mean_ms_per_step": e2e_mean_ms, "calls": len(e2e_t), "statistic": "median of host-clock call times",
                "h2d_bytes_per_step": 2 * N_POINTS * 3 * 4, "d2h_bytes_per_step": N_POINTS * 3 * 4},
        "gpu_launches": launches_per_eval * args.steps,
        "gpu_launches_note": f"kernels of libse.so launched in the timed region: {launches_per_eval} per step x "
                             f"{args.steps} steps (host-side count); cuFFT's own kernels come on top (4 per step "
                             "with the zero-padding-aware transforms and the fused z-kernel)",
        "clocks": clocks,
    }
    print(json.dumps(line))
    plan.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-periodic", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the clustered stresslet and rotlet backward lines")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        tdist.init_process_group("nccl")
        dist = tdist
    run_ours(args, rank, world, dist)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
