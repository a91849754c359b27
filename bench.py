#!/usr/bin/env python
"""Throughput of the fused meshless-LBM step on one GB300 (or N replicas under torchrun).

Workload (default ``tgv_large``): Taylor-Green vortex on a 2048 x 2048 lattice jittered by
+-0.3 h (seed 3), N_L = 30 nearest-neighbour stencils, cubic PHS + degree-4 polynomials,
FP64 shape vectors, dx_ml = h, tau = 0.8, u0 = 0.01 (lattice units).  One bench step = one
time step of the whole hot path (pull-stream, bounce-back, collide) over all 4,194,304 nodes.

Reported: GNUPS of the FP32 deviation-storage step (inputs resident in HBM), the FP64 step
beside it, the FP32-vs-FP64 relative L2 velocity error after a long run, the HBM roofline of
the step kernel, an end-to-end figure through host buffers, sampled GPU clocks and the CPU
oracle as a baseline.  ``--impl reference`` times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "MLBM GNUPS (node-steps/s) & % HBM peak, FP32 vs FP64 step at L2 err ≤1e-6"
UNIT = "GNUPS"
HBM_FALLBACK_GBS = 6800.0

WORKLOADS = {
    # name: (n_side, K, degree, tau, u0)
    "tgv_large": dict(n_side=2048, K=30, deg=4, tau=0.8, u0=0.01, seed=3),
    "tgv_512": dict(n_side=512, K=30, deg=4, tau=0.8, u0=0.01, seed=3),
    "tgv_small": dict(n_side=32, K=12, deg=2, tau=0.8, u0=0.01, seed=1),
}
# CPU baseline sample: the same recipe on a 128 x 128 cloud
CPU_SAMPLE = dict(n_side=128, K=30, deg=4, tau=0.8, u0=0.01, seed=3)


def step_bytes_per_node(K: int, dtype_bytes: int, nearest: bool = False) -> int:
    """Algorithmic bytes of one node update: the shape-vector entries of the 8 moving
    directions (FP32: the K - 1 members other than the stencil centre, whose weight follows
    from constant reproduction; FP64: all K members, the literal sum), the int32 stencil
    indices (own-node rule: K - 1 shared by all directions; nearest-node rule: K per direction),
    and the nine populations read once and written once."""
    members = K - 1 if dtype_bytes == 4 else K
    idx = 8 * K * 4 if nearest else 4 * (K - 1)
    return 8 * members * dtype_bytes + idx + 2 * 9 * dtype_bytes


def survey_bytes_per_node(K: int, dtype_bytes: int) -> int:
    """The roofline's per-node byte count as the scope table states it for a shared stencil:
    all K shape-vector entries of the 8 moving directions, K int32 indices, nine populations in
    and out (FP32: 36 K + 72, FP64: 68 K + 144).  The FP32 kernel reads 36 bytes fewer (the
    difference form needs neither the centre's weight nor its index): step_bytes_per_node."""
    return 8 * K * dtype_bytes + 4 * K + 2 * 9 * dtype_bytes


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d.get("hbm_gbs", HBM_FALLBACK_GBS)), "measured"
    return HBM_FALLBACK_GBS, "fallback"


def _step_source_hash():
    """Hash of the step kernel's source with comments and blank space removed, so that the
    committed DRAM-traffic figure is used only while the code it was measured on is unchanged."""
    import re

    h = hashlib.sha256()
    for f in ("step.cu", "d2q9_device.cuh", "tile_interp.cuh"):
        with open(os.path.join(ROOT, "paper_2306_01525_gb300", "csrc", f)) as fh:
            src = fh.read()
        if f == "step.cu":  # the step kernel and its launch, not the other kernels of the file
            src = src[src.index("struct StepArgs"):src.index("// Initial state")] + \
                src[src.index("size_t step_smem"):src.index("int launch_step(")]
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update("".join(src.split()).encode())
    return h.hexdigest()[:16]


def _ncu_traffic(dtype_name):
    """DRAM bytes per launch of the step kernel from the committed ncu summary, if the kernel
    source is unchanged since the capture; else None."""
    p = os.path.join(ROOT, "profiles", f"step_{dtype_name}_tgv_large.txt")
    if not os.path.exists(p):
        return None
    vals = {}
    with open(p) as fh:
        for line in fh:
            if ":" in line:
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
    if vals.get("kernel_source_hash") != _step_source_hash():
        return None
    try:
        return float(vals["dram_bytes_per_launch_full_size"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.tmp = None

    def start(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.tmp, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.tmp.flush()
        self.tmp.seek(0)
        rows = [r.split(",") for r in self.tmp.read().strip().splitlines() if r.strip()]
        self.tmp.close()
        os.unlink(self.tmp.name)
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax = max(smax, float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() in ("active", "1"):
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_oracle_gnups(seconds: float, steps=None, warmup: int = 0, threads=None):
    """Time the FP64 CPU oracle's step on the bounded sample cloud (all host cores, or the given
    number of threads)."""
    import mlbm_inputs as mi
    import oracle

    all_threads = oracle.num_threads()
    if threads:
        oracle.set_threads(threads)

    c = CPU_SAMPLE
    xy = mi.jittered_lattice(c["n_side"], 0.3, seed=c["seed"])
    dx = 1.0 / c["n_side"]
    sidx, W = oracle.weights(xy, c["K"], c["deg"], dx, box=(1.0, 1.0))
    st = oracle.Stepper(sidx, W, c["tau"])
    rho, u, v = mi.tgv_initial(xy, c["u0"])
    f = oracle.init_equilibrium(rho, u, v)
    for _ in range(warmup):
        f = st.step(f)
    n = xy.shape[1]
    done, t0 = 0, time.perf_counter()
    while True:
        f = st.step(f)
        done += 1
        el = time.perf_counter() - t0
        if (steps is not None and done >= steps) or (steps is None and el >= seconds and done >= 3):
            break
    cores = oracle.num_threads()
    if threads:
        oracle.set_threads(all_threads)
    return dict(value=n * done / el / 1e9, unit=UNIT, cores=cores, kind="oracle",
                sample=f"FP64 oracle step on a {c['n_side']}x{c['n_side']} jittered cloud of the "
                       f"same recipe (N_L={c['K']}, degree {c['deg']}), {done} steps, "
                       f"{el:.1f} s"), done, el


def _config(workload, world, ratio=1.0, stencil="own"):
    wl = WORKLOADS[workload]
    n_side, K, deg = wl["n_side"], wl["K"], wl["deg"]
    N = n_side * n_side
    return {
        "workload": f"tgv_{n_side}sq_k{K}_d{deg}",
        "nodes": N, "stencil": K, "degree": deg, "tau": wl["tau"], "u0": wl["u0"],
        "dx_ml": "h" if ratio == 1.0 else f"{ratio}h", "stencil_rule": stencil,
        "geometry": "periodic unit square, lattice jittered +-0.3h",
        "parallelism": "replicas" if world > 1 else "single",
        "l2_flush": "inputs larger than L2 (FP32 shape vectors %.2f GB + 2 states)" % (8 * K * 4 * N / 1e9),
    }


def _sample_config(workload, ratio=1.0, stencil="own"):
    """Config of what the CPU oracle is timed on: the bounded sample cloud (same recipe, stencil
    size and degree as the GPU workload, fewer nodes).  GNUPS is a per-node-update rate, so the
    sample's rate compares with the full workload's; the label names the cloud actually run."""
    c = CPU_SAMPLE
    N = c["n_side"] * c["n_side"]
    return {
        "workload": f"tgv_{c['n_side']}sq_k{c['K']}_d{c['deg']}",
        "nodes": N, "stencil": c["K"], "degree": c["deg"], "tau": c["tau"], "u0": c["u0"],
        "dx_ml": "h" if ratio == 1.0 else f"{ratio}h", "stencil_rule": stencil,
        "geometry": "periodic unit square, lattice jittered +-0.3h",
        "parallelism": "single",
        "sample_of": _config(workload, 1, ratio, stencil)["workload"],
    }


def measure_fp64_peak(local, launches=5, target_s=0.05):
    """The device's FP64 FMA rate, measured: the library's probe of independent FMA chains
    (mlbm_fp64_fma_rate) sized to about target_s per launch, timed with CUDA events on its
    stream after two warm-up launches, with the SM clock sampled meanwhile.  Returns the best
    launch's TFLOP/s and the median SM clock under load."""
    import torch

    import paper_2306_01525_gb300 as mlbm

    dev = torch.device("cuda", local)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    bps = 8
    sink = torch.zeros(16 * sms, dtype=torch.float64, device=dev)
    st = torch.cuda.Stream(device=dev)
    iters = 1 << 14
    with torch.cuda.stream(st):
        for _ in range(8):  # size the launch
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            mlbm.fp64_fma_rate(iters, bps, sink, stream=st)
            e1.record(st)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            if ms >= 0.5 * target_s * 1e3:
                break
            iters = int(iters * min(16.0, max(2.0, target_s * 1e3 / max(ms, 1e-3))))
        clocks = ClockSampler(local)
        clocks.start()
        rates, by_ctas = [], {}
        for c in (4, 8, 16):  # CTAs per SM (16 runs as two waves of 8)
            for it in range(2 + launches):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                flops = mlbm.fp64_fma_rate(iters * bps // c, c, sink, stream=st)
                e1.record(st)
                e1.synchronize()
                if it >= 2:
                    r = flops / (e0.elapsed_time(e1) * 1e-3) / 1e12
                    rates.append(r)
                    by_ctas[c] = max(by_ctas.get(c, 0.0), r)
        clk = clocks.stop()
    return {"tflops": max(rates), "tflops_median": statistics.median(rates), "launches": launches,
            "iters_per_chain_at_8_ctas": iters, "best_by_ctas_per_sm": by_ctas,
            "sm_mhz_median": clk["sm_mhz"] if clk else None, "clock_reasons": clk["reasons"] if clk else None,
            "how": "independent FP64 FMA chains (16 per thread, 256 threads x 4, 8 or 16 CTAs per SM), "
                   "CUDA events on the probe's stream, best of the timed launches"}


def annulus_profile(r, g, nu, r1, r2):
    """Analytic azimuthal speed of force-driven flow between two circles, eq. (bch_solution):
    u(r) = -G (r^2 - alpha r + beta / r), G = g / (3 nu), alpha = (r1^2 + r1 r2 + r2^2) / (r1 + r2),
    beta = r1^2 r2^2 / (r1 + r2); used only to report the error of a run."""
    G = g / (3.0 * nu)
    alpha = (r1 * r1 + r1 * r2 + r2 * r2) / (r1 + r2)
    beta = r1 * r1 * r2 * r2 / (r1 + r2)
    return -G * (r * r - alpha * r + beta / r)


def lattice_nu(tau):
    """Lattice viscosity c_s^2 (tau - 1/2) (Sec. 2.1, as fixed by the Sec. 3 parameters)."""
    return (tau - 0.5) / 3.0


def reduce_max(value: float, dist, device) -> float:
    """Maximum of a float over all ranks (identity without a process group)."""
    if dist is None:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def bench_batched(steps: int, warmup: int = 5):
    """The batched convergence sweep: 64 independent Taylor-Green runs (uneven N, N_L, degree,
    dx_ml) as segments of one cloud: one uneven FP64 solve launch, then FP32 steps of all runs
    in one persistent launch each, graph-captured."""
    import torch

    import mlbm_inputs as mi
    import paper_2306_01525_gb300 as mlbm

    runs = mi.sweep_runs()
    parts, segs, params, us, vs = [], [], [], [], []
    for r in runs:
        xy = mi.jittered_lattice(r["n_side"], 0.3, seed=r["seed"])
        parts.append(xy)
        segs.append(dict(geometry=mlbm.PERIODIC, lx=1.0, ly=1.0, k=r["K"], degree=r["degree"],
                         dx_ml=r["ratio"] / r["n_side"]))
        params.append((r["tau"], 0.0, 1.0))
        _, u, v = mi.tgv_initial(xy, r["u0"])
        us.append(u)
        vs.append(v)
    offs = np.cumsum([0] + [p.shape[1] for p in parts])
    xy = np.concatenate(parts, axis=1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    cloud = mlbm.build_cloud(xy, segs, offs, device=True)
    t_cloud = time.perf_counter() - t0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    w = mlbm.build_weights(cloud)
    torch.cuda.synchronize()
    t_weights = time.perf_counter() - t0
    dev = torch.device("cuda", torch.cuda.current_device())
    N = w.n
    td = lambda a: torch.as_tensor(a, dtype=torch.float64, device=dev)
    a = torch.empty(9 * N, dtype=torch.float32, device=dev)
    b = torch.empty_like(a)
    mlbm.init(w, params, mlbm.F32, td(np.ones(N)), td(np.concatenate(us)), td(np.concatenate(vs)), a)
    a = mlbm.run(w, params, mlbm.F32, a, b, warmup)
    b = b if a is not b else torch.empty_like(a)
    st = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    mlbm.run(w, params, mlbm.F32, a, b, steps)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    byts = sum(int(offs[i + 1] - offs[i]) * step_bytes_per_node(r["K"], 4) for i, r in enumerate(runs))
    peak, _ = _peaks()
    achieved = byts / (ms / steps * 1e-3) / 1e9
    # the paper's protocol (Sec. 3): every run to its own end time, the 10 % decay time of the
    # Taylor-Green vortex, exp(-2 nu k^2 t) = 0.9 with k = 2 pi dx_ml in lattice units; all runs in
    # one call, each segment stepping until its own count
    ends = [max(1, int(round(np.log(10.0 / 9.0) / (2.0 * lattice_nu(r["tau"]) *
                                                   (2.0 * np.pi * r["ratio"] / r["n_side"]) ** 2))))
            for r in runs]
    u0 = np.concatenate(us)
    v0 = np.concatenate(vs)
    mlbm.init(w, params, mlbm.F32, td(np.ones(N)), td(u0), td(v0), a)
    mlbm.run_until(w, params, mlbm.F32, a, b, [1] * len(runs))  # the sorted tile table, first use
    mlbm.init(w, params, mlbm.F32, td(np.ones(N)), td(u0), td(v0), a)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    res = mlbm.run_until(w, params, mlbm.F32, a, b, ends)
    e1.record(st)
    torch.cuda.synchronize()
    ms_p = e0.elapsed_time(e1)
    _, uu, vv = (t.cpu().numpy() for t in mlbm.moments(w, params, mlbm.F32, res))
    errs = []
    for i, r in enumerate(runs):
        sl = slice(int(offs[i]), int(offs[i + 1]))
        decay = np.exp(-2.0 * lattice_nu(r["tau"]) * (2.0 * np.pi * r["ratio"] / r["n_side"]) ** 2 * ends[i])
        ua, va = u0[sl] * decay, v0[sl] * decay
        e = float(np.sqrt(np.sum((uu[sl] - ua) ** 2 + (vv[sl] - va) ** 2) / np.sum(ua ** 2 + va ** 2)))
        errs.append([r["n_side"], r["degree"], r["ratio"], ends[i], e])
    node_steps = sum(int(offs[i + 1] - offs[i]) * ends[i] for i in range(len(runs)))
    return {"workload": "tgv_sweep_64runs", "runs": len(runs), "nodes": N,
            "stencils": sorted({r["K"] for r in runs}), "degrees": sorted({r["degree"] for r in runs}),
            "value": N * steps / (ms * 1e-3) / 1e9, "unit": UNIT, "steps": steps,
            "ms_per_step": ms / steps, "achieved_gbs": achieved, "frac_of_hbm": achieved / peak,
            "launches_per_step": 1, "setup_s": {"cloud_device": t_cloud, "weights_gpu": t_weights},
            "paper_protocol": {"steps_max": max(ends), "node_steps": node_steps, "ms": ms_p,
                               "value": node_steps / (ms_p * 1e-3) / 1e9, "unit": UNIT,
                               "l2_u_vs_analytic": errs,
                               "columns": ["sqrt_n", "degree", "dx_ml/h", "steps", "rel_l2_u"]}}


def bench_annulus(max_steps: int = 500000, chunk: int = 2000):
    """Annular channel, about 20k scattered nodes, N_L = 20, P_3, tau = 0.7, g = 1e-6, dx_ml =
    1/320, FP64, run until the relative velocity residual per step falls below 1e-10 or
    max_steps; L2 error of the speed vs the analytic profile."""
    import torch

    import mlbm_inputs as mi
    import paper_2306_01525_gb300 as mlbm

    dx, tau, g = 1.0 / 320, 0.7, 1e-6
    xy, _ = mi.annulus_cloud(h=mi.ANNULUS_H_FOR[20000], seed=2)
    cloud = mlbm.build_cloud(xy, dict(geometry=mlbm.ANNULUS, r_in=0.5, r_out=1.0, k=20, degree=3, dx_ml=dx))
    w = mlbm.build_weights(cloud)
    n = w.n
    dev = torch.device("cuda", torch.cuda.current_device())
    td = lambda x: torch.as_tensor(x, dtype=torch.float64, device=dev)
    params = [(tau, g, 1.0)]
    a = torch.empty(9 * n, dtype=torch.float64, device=dev)
    b = torch.empty_like(a)
    mlbm.init(w, params, mlbm.F64, td(np.ones(n)), td(np.zeros(n)), td(np.zeros(n)), a)
    # first use of every kernel of the loop below (on a machine with an empty kernel cache the
    # CUDA driver compiles torch's own kernels for this GPU on first use, outside the timed
    # region here)
    _, u, v = mlbm.moments(w, params, mlbm.F64, a)
    mlbm.norms(w, u, u.clone(), v, v.clone())
    prev, done, res = None, 0, float("inf")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    while done < max_steps:
        a = mlbm.run(w, params, mlbm.F64, a, b, chunk)
        b = b if a is not b else torch.empty_like(a)
        done += chunk
        _, u, v = mlbm.moments(w, params, mlbm.F64, a)
        if prev is not None:
            s = mlbm.norms(w, u, prev[0], v, prev[1])
            res = float(np.sqrt(s[0] / s[2]) / chunk)
            if res < 1e-10:
                break
        prev = (u.clone(), v.clone())
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    r = np.hypot(xy[0], xy[1])
    want = np.abs(annulus_profile(r / dx, g, lattice_nu(tau), 0.5 / dx, 1.0 / dx))
    uu, vv = u.cpu().numpy(), v.cpu().numpy()
    err = float(np.sqrt(np.sum((np.hypot(uu, vv) - want) ** 2) / np.sum(want ** 2)))
    return {"workload": "annulus_20k_k20_d3", "nodes": n, "steps": done,
            "residual_per_step": res if np.isfinite(res) else None,
            "l2_speed_vs_analytic": err, "value": n * done / el / 1e9, "unit": UNIT,
            "ms_per_step": el / done * 1e3, "dtype": "f64",
            "note": "wall time of the whole run incl. residual checks every %d steps" % chunk}


def bench_adjoint(steps: int = 2000):
    """Adjoint of the annulus with about 250k scattered nodes, N_L = 24, P_3, FP32 steps with
    sqrt(T) checkpointing: gradient of the velocity-profile mismatch w.r.t. tau, g and the
    initial fields; time of forward plus backward."""
    import torch

    import mlbm_inputs as mi
    import paper_2306_01525_gb300 as mlbm
    from paper_2306_01525_gb300.autograd import rollout

    dx, tau, g = 1.0 / 320, 0.7, 1e-5
    xy, _ = mi.annulus_cloud(h=mi.ANNULUS_H_FOR[250000], seed=5)
    cloud = mlbm.build_cloud(xy, dict(geometry=mlbm.ANNULUS, r_in=0.5, r_out=1.0, k=24, degree=3, dx_ml=dx))
    w = mlbm.build_weights(cloud)
    n = w.n
    dev = torch.device("cuda", torch.cuda.current_device())
    r = np.hypot(xy[0], xy[1])
    target = torch.as_tensor(np.abs(annulus_profile(r / dx, g, lattice_nu(tau), 0.5 / dx, 1.0 / dx)),
                             device=dev)
    tt = torch.tensor(tau, dtype=torch.float64, device=dev, requires_grad=True)
    gt = torch.tensor(g, dtype=torch.float64, device=dev, requires_grad=True)
    r0 = torch.ones(n, dtype=torch.float64, device=dev, requires_grad=True)
    a0 = torch.zeros(n, dtype=torch.float64, device=dev, requires_grad=True)
    b0 = torch.zeros(n, dtype=torch.float64, device=dev, requires_grad=True)
    # warm-up: a short rollout and its backward pass with the same loss (first use of the
    # library's kernels, of autograd and of every torch kernel the loss launches: with an empty
    # kernel cache the CUDA driver compiles torch's kernels for this GPU on first use, seconds
    # of host time)
    rw, uw, vw = rollout(w, tt, gt, r0, a0, b0, 10, dtype=mlbm.F32)
    ((torch.sqrt(uw * uw + vw * vw + 1e-30) - target) ** 2).sum().backward()
    for p_ in (tt, gt, r0, a0, b0):
        p_.grad = None
    torch.cuda.synchronize()
    torch.cuda.reset_peak_memory_stats()
    t0 = time.perf_counter()
    rho, u, v = rollout(w, tt, gt, r0, a0, b0, steps, dtype=mlbm.F32)
    loss = ((torch.sqrt(u * u + v * v + 1e-30) - target) ** 2).sum()
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    loss.backward()
    torch.cuda.synchronize()
    t_all = time.perf_counter() - t0
    peak_mem = torch.cuda.max_memory_allocated() / 1e9
    # one reverse step and one forward step on their own: CUDA events on the launching stream,
    # L2 flushed before every timed launch by a 256 MB write, then a 256 MB read of another
    # buffer (so that the timed kernel does not also pay the write-back of dirty flush lines)
    params = [(tau, g, 1.0)]
    s = torch.empty(9 * n, dtype=torch.float32, device=dev)
    mlbm.init(w, params, mlbm.F32, r0.detach(), a0.detach(), b0.detach(), s)
    sn = torch.empty_like(s)
    for _ in range(20):
        mlbm.step(w, params, mlbm.F32, s, sn)
        s, sn = sn, s
    mlbm.step(w, params, mlbm.F32, s, sn)
    lam = torch.randn(9 * n, dtype=torch.float32, device=dev, generator=torch.Generator(dev).manual_seed(3))
    lp = torch.empty_like(lam)
    gacc = torch.zeros(2, dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    clean = torch.ones(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    sink = torch.empty((), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def kernel_us(fn, reps=30):
        fn()
        total = 0.0
        for _ in range(reps):
            flush.zero_()
            torch.sum(clean, dim=0, out=sink)
            # a device-side delay (about 200 us at 2 GHz) before the start event, so that the
            # host has issued the call's launches before the device reaches the event and the
            # interval holds device time only, not the host's argument handling (about 30 us for
            # the reverse step); with 50 us the reverse step read 4 us longer
            torch.cuda._sleep(400_000)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            total += e0.elapsed_time(e1)
        return total / reps * 1e3

    rev_us = kernel_us(lambda: mlbm.adjoint_step(w, params, mlbm.F32, s, lam, lp, gacc, s_next=sn))
    rev_rc_us = kernel_us(lambda: mlbm.adjoint_step(w, params, mlbm.F32, s, lam, lp, gacc))
    fwd_us = kernel_us(lambda: mlbm.step(w, params, mlbm.F32, s, sn))
    # the same cloud under the nearest-node rule (each direction interpolated in the stencil of
    # its departure node): forward step and reverse step from s_next, timed the same way; the
    # first reverse step (not timed) builds the transposed tables
    wn = mlbm.build_weights(mlbm.build_cloud(
        xy, dict(geometry=mlbm.ANNULUS, r_in=0.5, r_out=1.0, k=24, degree=3, dx_ml=dx,
                 stencil_mode=mlbm.STENCIL_NEAREST), device=True))
    s_n = torch.empty(9 * n, dtype=torch.float32, device=dev)
    mlbm.init(wn, params, mlbm.F32, r0.detach(), a0.detach(), b0.detach(), s_n)
    sn_n = torch.empty_like(s_n)
    mlbm.step(wn, params, mlbm.F32, s_n, sn_n)
    rev_near_us = kernel_us(lambda: mlbm.adjoint_step(wn, params, mlbm.F32, s_n, lam, lp, gacc, s_next=sn_n))
    fwd_near_us = kernel_us(lambda: mlbm.step(wn, params, mlbm.F32, s_n, sn_n))
    del wn
    K = 24
    bpn = adjoint_bytes_per_node(K)
    peak, _ = _peaks()
    gbs = bpn * n / (rev_us * 1e-6) / 1e9
    # what a plain read of the same number of bytes takes, timed the same way (torch's sum over a
    # contiguous buffer): at a few hundred MB a launch's ramp-up and tail are a visible part of
    # its time, so this is the floor a kernel of this size can reach, below the copy peak
    plain = torch.ones(bpn * n // 4, dtype=torch.float32, device=dev)
    read_us = kernel_us(lambda: torch.sum(plain, dim=0, out=sink))
    del plain
    return {"workload": "annulus_250k_k24_d3_adjoint", "nodes": n, "steps": steps, "dtype": "f32",
            "checkpoint_every": int(np.ceil(np.sqrt(steps))), "forward_s": t_fwd,
            "forward_backward_s": t_all, "loss": float(loss.detach()),
            "dloss_dtau": float(tt.grad), "dloss_dg": float(gt.grad),
            "dloss_du0_norm": float(a0.grad.norm()),
            "peak_torch_mem_gb": peak_mem,
            "reverse_step": {"us": rev_us, "us_recompute_route": rev_rc_us, "forward_step_us": fwd_us,
                             "algorithmic_bytes_per_node": bpn, "achieved_gbs": gbs,
                             "frac_of_hbm": gbs / peak,
                             "plain_read_same_bytes": {"us": read_us, "gbs": bpn * n / (read_us * 1e-6) / 1e9,
                                                       "reverse_step_frac": read_us / rev_us},
                             "nearest_rule": {"us": rev_near_us, "forward_step_us": fwd_near_us},
                             "l2": "flushed before each launch (256 MB write, then 256 MB read)"}}


def adjoint_bytes_per_node(K: int) -> int:
    """Algorithmic bytes of one FP32 reverse step per node: the shape-vector entries of the 8
    moving directions for the K - 1 members other than the centre, their int32 stencil indices,
    the forward output and the incoming cotangent read once, the outgoing cotangent written
    once (nine populations each)."""
    return 8 * (K - 1) * 4 + 4 * (K - 1) + 3 * 9 * 4


def sc_bytes_per_node(K: int) -> int:
    """Algorithmic bytes of one FP32 Shan-Chen node update: both passes read the shape vectors
    and slot indices (as a plain step); pass 1 reads the nine populations and writes the
    streamed ones and psi, pass 2 reads psi and the streamed populations and writes the new
    ones."""
    per_pass = 8 * (K - 1) * 4 + 4 * (K - 1)
    return 2 * per_pass + (36 + 36 + 4) + (4 + 36 + 36)


def bench_shan_chen(n_side: int = 2048, steps: int = 200, warmup: int = 5):
    """Shan-Chen multiphase steps (two launches each) on the headline cloud: 2048^2 jittered,
    N_L = 30, P_4, dx_ml = h, G = -5.5, FP32, from a noisy uniform state at rho = ln 2."""
    import torch

    import mlbm_inputs as mi
    import paper_2306_01525_gb300 as mlbm

    K, deg = 30, 4
    xy = mi.jittered_lattice(n_side, 0.3, seed=3)
    seg = dict(geometry=mlbm.PERIODIC, lx=1.0, ly=1.0, k=K, degree=deg, dx_ml=1.0 / n_side)
    w = mlbm.build_weights(mlbm.build_cloud(xy, seg, device=True))
    N = w.n
    dev = torch.device("cuda", torch.cuda.current_device())
    rng = np.random.default_rng(9)
    td = lambda x: torch.as_tensor(x, dtype=torch.float64, device=dev)
    params, sc = [(1.0, 0.0, 1.0)], (-5.5, 1.0)
    a = torch.empty(9 * N, dtype=torch.float32, device=dev)
    b = torch.empty_like(a)
    mlbm.init(w, params, mlbm.F32, td(np.log(2.0) * (1 + 0.01 * rng.standard_normal(N))), td(np.zeros(N)),
              td(np.zeros(N)), a)
    for _ in range(warmup):
        mlbm.sc_step(w, params, sc, mlbm.F32, a, b)
        a, b = b, a
    st = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(steps):
        mlbm.sc_step(w, params, sc, mlbm.F32, a, b)
        a, b = b, a
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    peak, _ = _peaks()
    gbs = sc_bytes_per_node(K) * N / (ms * 1e-3) / 1e9
    return {"workload": f"shan_chen_{n_side}sq_k{K}_d{deg}", "nodes": N, "value": N / (ms * 1e-3) / 1e9,
            "unit": UNIT, "ms_per_step": ms, "launches_per_step": 2, "steps": steps,
            "algorithmic_bytes_per_node": sc_bytes_per_node(K), "achieved_gbs": gbs, "frac_of_hbm": gbs / peak,
            "dtype": "f32", "G": sc[0]}


def bench_tgv_4096(steps: int = 50, warmup: int = 5):
    """The large Taylor-Green recipe at four times the benchmark's node count: 4096^2 jittered
    nodes (16.8 M), N_L 30, P_4, dx_ml = h, FP32 tile layout only (about 50 GB on the device with
    the FP64 shape vectors); FP32 steps timed with CUDA events, inputs far larger than L2."""
    import torch

    import mlbm_inputs as mi
    import paper_2306_01525_gb300 as mlbm

    n_side, K, deg, tau, u0 = 4096, 30, 4, 0.8, 0.01
    xy = mi.jittered_lattice(n_side, 0.3, seed=7)
    dev = torch.device("cuda", torch.cuda.current_device())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    cloud = mlbm.build_cloud(xy, dict(geometry=mlbm.PERIODIC, lx=1.0, ly=1.0, k=K, degree=deg, dx_ml=1.0 / n_side),
                             device=True)
    torch.cuda.synchronize()
    t_cloud = time.perf_counter() - t0
    t0 = time.perf_counter()
    w = mlbm.build_weights(cloud, keep=mlbm.KEEP_W32)
    torch.cuda.synchronize()
    t_weights = time.perf_counter() - t0
    del cloud
    n = w.n
    params = [(tau, 0.0, 1.0)]
    rho, u, v = (torch.as_tensor(a, dtype=torch.float64, device=dev) for a in mi.tgv_initial(xy, u0))
    a = torch.empty(9 * n, dtype=torch.float32, device=dev)
    b = torch.empty_like(a)
    mlbm.init(w, params, mlbm.F32, rho, u, v, a)
    del rho, u, v
    a = mlbm.run(w, params, mlbm.F32, a, b, warmup)
    b = b if a is not b else torch.empty_like(a)
    st = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    mlbm.run(w, params, mlbm.F32, a, b, steps)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    peak, _ = _peaks()
    gbs = step_bytes_per_node(K, 4) * n / (ms * 1e-3) / 1e9
    out = {"workload": "tgv_4096sq_k30_d4", "nodes": n, "steps": steps, "dtype": "f32",
           "value": n / (ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": ms,
           "algorithmic_bytes_per_node": step_bytes_per_node(K, 4), "achieved_gbs": gbs, "frac_of_hbm": gbs / peak,
           "setup_s": {"cloud_device": t_cloud, "weights_gpu": t_weights},
           "device_memory_in_use_gb": (lambda fm: (fm[1] - fm[0]) / 1e9)(torch.cuda.mem_get_info())}
    del a, b, w
    return out


def bench_tgv_small(steps: int = 500, reps: int = 20):
    """The paper's Taylor-Green case as configured for plain MLBM in FP64: 32 x 32 jittered
    lattice (1024 nodes), N_L 12, P_2, tau 0.8, u0 0.01, dx_ml = h, 500 steps; a cloud this small
    is latency-bound, so the figure is the time of the whole 500-step run (graph-captured step
    loop), its GNUPS, and the L2 error of u against the analytic decay at the end."""
    import torch

    import mlbm_inputs as mi
    import paper_2306_01525_gb300 as mlbm

    wl = WORKLOADS["tgv_small"]
    n_side, K, deg, tau, u0 = wl["n_side"], wl["K"], wl["deg"], wl["tau"], wl["u0"]
    dx = 1.0 / n_side
    xy = mi.jittered_lattice(n_side, 0.3, seed=wl["seed"])
    w = mlbm.build_weights(mlbm.build_cloud(xy, dict(geometry=mlbm.PERIODIC, lx=1.0, ly=1.0, k=K,
                                                     degree=deg, dx_ml=dx)))
    dev = torch.device("cuda", torch.cuda.current_device())
    params = [(tau, 0.0, 1.0)]
    rho, u, v = (torch.as_tensor(a, dtype=torch.float64, device=dev) for a in mi.tgv_initial(xy, u0))
    a = torch.empty(9 * w.n, dtype=torch.float64, device=dev)
    b = torch.empty_like(a)
    mlbm.init(w, params, mlbm.F64, rho, u, v, a)
    mlbm.run(w, params, mlbm.F64, a, b, 64)  # graph capture and warm-up
    stream = torch.cuda.current_stream()
    times = []
    for _ in range(reps):
        mlbm.init(w, params, mlbm.F64, rho, u, v, a)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = mlbm.run(w, params, mlbm.F64, a, b, steps)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = float(np.median(times))
    _, uu, vv = mlbm.moments(w, params, mlbm.F64, res)
    decay = float(np.exp(-2.0 * lattice_nu(tau) * (2.0 * np.pi * dx) ** 2 * steps))
    sn = mlbm.norms(w, uu, u * decay, vv, v * decay)
    return {"workload": "tgv_32sq_k12_d2", "nodes": w.n, "steps": steps, "dtype": "f64",
            "run_ms": ms, "us_per_step": ms * 1e3 / steps, "value": w.n * steps / (ms * 1e-3) / 1e9,
            "unit": UNIT, "rel_l2_u_vs_analytic": float(np.sqrt(sn[0] / sn[1])),
            "timing": "median of %d runs, CUDA events" % reps}


def bench_lattice(n_side: int = 2048, steps: int = 200, warmup: int = 5):
    """Standard lattice LBM (index-shift streaming) on an n_side^2 periodic lattice, FP32: the
    paper's comparison method at the node count of the headline workload."""
    import torch

    import mlbm_inputs as mi
    import paper_2306_01525_gb300 as mlbm

    N = n_side * n_side
    dev = torch.device("cuda", torch.cuda.current_device())
    xy = mi.lattice(n_side)
    rho, u, v = mi.tgv_initial(xy, 0.01)
    td = lambda x: torch.as_tensor(x, dtype=torch.float64, device=dev)
    prm = (0.8, 0.0, 1.0)
    a = torch.empty(9 * N, dtype=torch.float32, device=dev)
    b = torch.empty_like(a)
    mlbm.lattice_init(n_side, n_side, prm, mlbm.F32, td(rho), td(u), td(v), a)
    for _ in range(warmup):
        mlbm.lattice_step(n_side, n_side, prm, mlbm.F32, a, b)
        a, b = b, a
    st = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(steps):
        mlbm.lattice_step(n_side, n_side, prm, mlbm.F32, a, b)
        a, b = b, a
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    peak, _ = _peaks()
    gbs = 72 * N / (ms * 1e-3) / 1e9
    return {"workload": f"lattice_lbm_{n_side}sq", "nodes": N, "value": N / (ms * 1e-3) / 1e9,
            "unit": UNIT, "ms_per_step": ms, "achieved_gbs": gbs, "frac_of_hbm": gbs / peak,
            "dtype": "f32"}


def bench_paper_sweep(dtype_name: str = "f64"):
    """The paper's Taylor-Green convergence study (Sec. 3, Fig. h_dx_explained and
    Fig. tgv_conv_P) on synthetic clouds: dx_ml in {1/10, 1/40, 1/160} x h in {1/10 .. 1/320} x
    {P_2, P_4}, N_L = 25, nearest-node stencils, tau = 0.8, dt = 1e-3 (10 dx_ml)^2 (diffusive
    scaling, U0 = 1, nu = 1), run to t_end; each dx_ml group is one batched cloud stepped by one
    launch per step.  Also the lattice LBM at dx in {1/10 .. 1/160}.  Returns the L2 map."""
    import torch

    import mlbm_inputs as mi
    import paper_2306_01525_gb300 as mlbm

    dtype = mlbm.F64 if dtype_name == "f64" else mlbm.F32
    tdt = torch.float64 if dtype == mlbm.F64 else torch.float32
    dev = torch.device("cuda", torch.cuda.current_device())
    td = lambda x: torch.as_tensor(x, dtype=torch.float64, device=dev)
    tau, nu_lat = 0.8, lattice_nu(0.8)
    hs = [10, 20, 40, 80, 160, 320]
    out = {"dx_ml": ["1/10", "1/40", "1/160"], "sqrt_n": hs, "stencil": 25, "dtype": dtype_name,
           "l2_u": {}, "lbm_l2_u": {}}
    node_steps, t_all = 0, 0.0
    for L in (10, 40, 160):
        steps = int(round(np.log(10.0) * L * L / (2.0 * nu_lat * (2 * np.pi) ** 2)))
        u0 = 0.01 * 10.0 / L  # U0 dt / dx_ml with dt = 1e-3 (10 dx_ml)^2
        parts, segs, us, vs = [], [], [], []
        for deg in (2, 4):
            for n in hs:
                xy = mi.jittered_lattice(n, 0.3, seed=1000 + n)
                parts.append(xy)
                segs.append(dict(geometry=mlbm.PERIODIC, lx=1.0, ly=1.0, k=25, degree=deg,
                                 dx_ml=1.0 / L, stencil_mode=mlbm.STENCIL_NEAREST))
                _, u, v = mi.tgv_initial(xy, u0)
                us.append(u)
                vs.append(v)
        offs = np.cumsum([0] + [q.shape[1] for q in parts])
        cloud = mlbm.build_cloud(np.concatenate(parts, axis=1), segs, offs)
        w = mlbm.build_weights(cloud)
        N = w.n
        params = [(tau, 0.0, 1.0)] * len(segs)
        a = torch.empty(9 * N, dtype=tdt, device=dev)
        b = torch.empty_like(a)
        mlbm.init(w, params, dtype, td(np.ones(N)), td(np.concatenate(us)), td(np.concatenate(vs)), a)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = mlbm.run(w, params, dtype, a, b, steps)
        torch.cuda.synchronize()
        t_all += time.perf_counter() - t0
        node_steps += N * steps
        _, ug, _ = mlbm.moments(w, params, dtype, res)
        ug = ug.cpu().numpy()
        decay = np.exp(-2.0 * nu_lat * (2 * np.pi / L) ** 2 * steps)
        for i, (deg, n) in enumerate([(d, n) for d in (2, 4) for n in hs]):
            xy = parts[i]
            ut = u0 * np.cos(2 * np.pi * xy[0]) * np.sin(2 * np.pi * xy[1]) * decay
            e = float(np.sqrt(np.sum((ug[offs[i]:offs[i + 1]] - ut) ** 2) / np.sum(ut ** 2)))
            out["l2_u"].setdefault(f"P{deg}", {}).setdefault(f"1/{L}", []).append(e)
        del w, cloud, a, b, res
        torch.cuda.empty_cache()
    for L in (10, 20, 40, 80, 160):
        steps = int(round(np.log(10.0) * L * L / (2.0 * nu_lat * (2 * np.pi) ** 2)))
        u0 = 0.01 * 10.0 / L
        xy = mi.lattice(L)
        _, u, v = mi.tgv_initial(xy, u0)
        a = torch.empty(9 * L * L, dtype=tdt, device=dev)
        b = torch.empty_like(a)
        mom = torch.empty(3 * L * L, dtype=tdt, device=dev)
        mlbm.lattice_init(L, L, (tau, 0.0, 1.0), dtype, td(np.ones(L * L)), td(u), td(v), a)
        for _ in range(steps):
            mlbm.lattice_step(L, L, (tau, 0.0, 1.0), dtype, a, b, mom)
            a, b = b, a
        ul = mom.view(3, -1)[1].double().cpu().numpy()
        decay = np.exp(-2.0 * nu_lat * (2 * np.pi / L) ** 2 * steps)
        ut = u0 * np.cos(2 * np.pi * xy[0]) * np.sin(2 * np.pi * xy[1]) * decay
        out["lbm_l2_u"][f"1/{L}"] = float(np.sqrt(np.sum((ul - ut) ** 2) / np.sum(ut ** 2)))
    out["value"] = node_steps / t_all / 1e9
    out["unit"] = UNIT
    out["seconds"] = t_all
    return out


def _dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args):
    world, rank, _ = _dist_setup()
    if rank != 0:
        return 0
    # the oracle: each step one oracle time step over the bounded sample cloud
    res, done, el = cpu_oracle_gnups(0.0, steps=args.steps, warmup=args.warmup)
    c = CPU_SAMPLE
    n = c["n_side"] ** 2
    line = {
        "impl": "reference", "metric": METRIC, "value": res["value"], "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": el / done * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _sample_config(args.workload, args.ratio, args.stencil),
        "cpu_baseline": res,
        "e2e": {"value": res["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_mlbm(args):
    import torch

    import mlbm_inputs as mi
    import paper_2306_01525_gb300 as mlbm

    world, rank, local = _dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    wl = WORKLOADS[args.workload]
    n_side, K, deg, tau, u0 = wl["n_side"], wl["K"], wl["deg"], wl["tau"], wl["u0"]
    dx = args.ratio / n_side
    xy = mi.jittered_lattice(n_side, 0.3, seed=wl["seed"])
    seg = dict(geometry=mlbm.PERIODIC, lx=1.0, ly=1.0, k=K, degree=deg, dx_ml=dx,
               stencil_mode=mlbm.STENCIL_NEAREST if args.stencil == "nearest" else mlbm.STENCIL_OWN)
    # stencil build on the device (first use of its kernels on a small cloud, then timed)
    mlbm.build_cloud(mi.jittered_lattice(32, 0.3, seed=1), dict(seg, k=min(K, 64)), device=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    cloud = mlbm.build_cloud(xy, seg, device=True)
    t_cloud = time.perf_counter() - t0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    w = mlbm.build_weights(cloud)
    torch.cuda.synchronize()
    t_weights = time.perf_counter() - t0
    N = w.n
    params = [(tau, 0.0, 1.0)]
    rho, u, v = mi.tgv_initial(xy, u0)
    td = lambda a: torch.as_tensor(a, dtype=torch.float64, device=dev)
    rho_d, u_d, v_d = td(rho), td(u), td(v)
    del cloud

    def fresh(dtype):
        tdt = torch.float32 if dtype == mlbm.F32 else torch.float64
        a = torch.empty(9 * N, dtype=tdt, device=dev)
        b = torch.empty_like(a)
        mlbm.init(w, params, dtype, rho_d, u_d, v_d, a)
        return a, b

    def timed_steps(dtype, steps, warmup, clocks=None):
        a, b = fresh(dtype)
        a2 = mlbm.run(w, params, dtype, a, b, warmup)
        b2 = b if a2 is a else a
        stream = torch.cuda.current_stream()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        if clocks:
            clocks.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        mlbm.run(w, params, dtype, a2, b2, steps)
        e1.record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop() if clocks else None
        ms = reduce_max(e0.elapsed_time(e1), dist, dev)
        if dist:
            dist.barrier()
        return ms, clk

    # ---------------------------------------------------------------- FP32 (headline)
    clocks = ClockSampler(local)
    ms32, clk = timed_steps(mlbm.F32, args.steps, args.warmup, clocks)
    ms_step32 = ms32 / args.steps
    gnups32 = N * world * args.steps / (ms32 * 1e-3) / 1e9
    # ---------------------------------------------------------------- FP64 beside it
    s64 = max(3, min(args.steps, 100))
    ms64, _ = timed_steps(mlbm.F64, s64, max(3, min(args.warmup, 5)))
    ms_step64 = ms64 / s64
    gnups64 = N * world * s64 / (ms64 * 1e-3) / 1e9
    # ---------------------------------------------------------------- precision after a run
    err = None
    err_an = None
    if args.err_steps > 0:
        a32, b32 = fresh(mlbm.F32)
        a64, b64 = fresh(mlbm.F64)
        r32 = mlbm.run(w, params, mlbm.F32, a32, b32, args.err_steps)
        r64 = mlbm.run(w, params, mlbm.F64, a64, b64, args.err_steps)
        _, u32, v32 = mlbm.moments(w, params, mlbm.F32, r32)
        _, u64, v64 = mlbm.moments(w, params, mlbm.F64, r64)
        s = mlbm.norms(w, u32, u64, v32, v64)
        err = float(np.sqrt(s[0] / s[1]))
        # the Taylor-Green decay in lattice units, eq. (tgv_eqs): the initial field times
        # exp(-2 nu (2 pi dx)^2 n), nu = (tau - 1/2) / 3, dx the streaming distance (unit box)
        decay = float(np.exp(-2.0 * lattice_nu(tau) * (2.0 * np.pi * dx) ** 2 * args.err_steps))
        ua, va = u_d * decay, v_d * decay
        err_an = {}
        for name, (uu, vv) in (("f32", (u32, v32)), ("f64", (u64, v64))):
            sa = mlbm.norms(w, uu, ua, vv, va)
            err_an[name] = float(np.sqrt(sa[0] / sa[1]))
        del a32, b32, a64, b64, r32, r64
    # ---------------------------------------------------------------- end to end
    # Through the C ABI with host buffers (mlbm_step_host): every step copies its input state
    # from pinned host memory, steps it and copies the result back; the batch's steps are
    # independent, so the library overlaps the copies of neighbouring steps with the compute.
    # 50 host-resident states per call (a batch the library pipelines: copy in, step, copy out of
    # neighbouring states overlap), whatever --steps is; each state is copied in, stepped once and
    # copied back inside the timed region
    e2e_steps = 50
    st_bytes = 9 * N * 4
    h_in = torch.empty(9 * N, dtype=torch.float32, pin_memory=True)
    h_out = [torch.empty(9 * N, dtype=torch.float32, pin_memory=True) for _ in range(2)]
    a, b = fresh(mlbm.F32)
    h_in.copy_(a)
    ins, outs = [h_in] * e2e_steps, [h_out[i % 2] for i in range(e2e_steps)]
    s_cmp = torch.cuda.Stream()
    mlbm.step_host(w, params, mlbm.F32, ins[:2], outs[:2], stream=s_cmp)  # buffers, streams
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s_cmp)
    mlbm.step_host(w, params, mlbm.F32, ins, outs, stream=s_cmp)
    e1.record(s_cmp)
    torch.cuda.synchronize()
    ms_e2e = reduce_max(e0.elapsed_time(e1) / e2e_steps, dist, dev)
    gnups_e2e = N * world / (ms_e2e * 1e-3) / 1e9
    # the results on the host equal a device-side step of the same input
    mlbm.step(w, params, mlbm.F32, a, b)
    e2e_ok = bool(torch.equal(b.cpu(), h_out[0]) and torch.equal(b.cpu(), h_out[1]))
    del h_in, h_out, ins, outs, a, b

    if rank != 0:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return 0
    peak, peak_kind = _peaks()
    fp64_peak = measure_fp64_peak(local)
    p64 = fp64_peak["tflops"]
    bpn32 = step_bytes_per_node(K, 4, args.stencil == "nearest")
    bpn_roof = bpn32 if args.stencil == "nearest" else survey_bytes_per_node(K, 4)
    achieved = bpn_roof * N / (ms_step32 * 1e-3) / 1e9
    default_workload = args.workload == "tgv_large" and args.stencil == "own" and args.ratio == 1.0
    traffic = _ncu_traffic("f32") if default_workload else None
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu, _, _ = cpu_oracle_gnups(args.cpu_seconds)
        one, _, _ = cpu_oracle_gnups(4.0, threads=1)
        cpu["single_thread"] = {"value": one["value"], "unit": UNIT, "cores": one["cores"], "sample": one["sample"]}
    extras = {}
    t_cloud_host = None
    if world == 1 and not args.no_extras:
        t0 = time.perf_counter()
        mlbm.build_cloud(xy, seg)  # the host build of the same cloud, for comparison
        t_cloud_host = time.perf_counter() - t0
        del w
        torch.cuda.empty_cache()
        extras["batched"] = bench_batched(1000)
        torch.cuda.empty_cache()
        extras["annulus"] = bench_annulus()
        torch.cuda.empty_cache()
        extras["adjoint"] = bench_adjoint(2000)
        torch.cuda.empty_cache()
        extras["lattice_lbm"] = bench_lattice()
        torch.cuda.empty_cache()
        extras["tgv_small"] = bench_tgv_small()
        torch.cuda.empty_cache()
        extras["tgv_4096"] = bench_tgv_4096()
        torch.cuda.empty_cache()
        extras["shan_chen"] = bench_shan_chen()
        torch.cuda.empty_cache()
        extras["paper_sweep"] = bench_paper_sweep("f64")
    line = {
        "metric": METRIC, "value": gnups32, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step32, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": _config(args.workload, world, args.ratio, args.stencil),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_source": peak_kind, "algorithmic_bytes_per_node": bpn_roof,
                     "kernel_bytes_per_node": bpn32,
                     "frac_by_kernel_bytes": bpn32 * N / (ms_step32 * 1e-3) / 1e9 / peak},
        "cpu_baseline": cpu,
        "e2e": {"value": gnups_e2e, "unit": UNIT, "h2d_bytes_per_step": st_bytes,
                "d2h_bytes_per_step": st_bytes, "ms_per_step": ms_e2e, "steps": e2e_steps,
                "api": "mlbm_step_host (C ABI, pinned host buffers)",
                "overlap": "copy in, step and copy out of neighbouring states on three streams, double-buffered",
                "result_matches_device_step": e2e_ok},
        "clocks": clk,
        "gpu_launches": args.steps,
        "fp64": {"value": gnups64, "unit": UNIT, "ms_per_step": ms_step64, "steps": s64,
                 "achieved_gbs": step_bytes_per_node(K, 8, args.stencil == "nearest") * N / (ms_step64 * 1e-3) / 1e9,
                 "bound": "fp64 alu", "achieved_tflops": (16 * K + 80) * N / (ms_step64 * 1e-3) / 1e12,
                 "peak_tflops": p64, "peak_source": "measured (fp64_peak)",
                 "frac": (16 * K + 80) * N / (ms_step64 * 1e-3) / 1e12 / p64},
        "fp64_peak": fp64_peak,
        "speedup_fp32_vs_fp64": gnups32 / gnups64,
        "fp32_vs_fp64_rel_l2_u": err, "error_steps": args.err_steps,
        "rel_l2_u_vs_analytic": err_an,
        "setup_s": {"cloud_device": t_cloud, "cloud_host": t_cloud_host, "weights_gpu": t_weights},
    }
    line.update(extras)
    print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="mlbm", choices=["mlbm", "reference"])
    ap.add_argument("--workload", default="tgv_large", choices=sorted(WORKLOADS))
    ap.add_argument("--err-steps", type=int, default=10000)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--stencil", default="own", choices=["own", "nearest"],
                    help="stencil rule of the main workload (own-node or nearest-node)")
    ap.add_argument("--ratio", type=float, default=1.0, help="dx_ml / h of the main workload")
    ap.add_argument("--leg", default=None,
                    choices=["batched", "annulus", "adjoint", "lattice_lbm", "shan_chen", "paper_sweep", "tgv_small",
                             "tgv_4096", "fp64_peak"],
                    help="run only this extra measurement and print it")
    ap.add_argument("--leg-steps", type=int, default=None,
                    help="with --leg: the leg's step count (annulus: its step cap), e.g. for a short ncu capture")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched-sweep, annulus and adjoint measurements")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.leg:
        import torch

        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        n = args.leg_steps
        legs = {"batched": lambda: bench_batched(n or 1000),
                "annulus": lambda: bench_annulus(n or 500000, min(2000, n or 2000)),
                "tgv_small": lambda: bench_tgv_small(n or 500),
                "tgv_4096": lambda: bench_tgv_4096(n or 50),
                "adjoint": lambda: bench_adjoint(n or 2000), "lattice_lbm": bench_lattice,
                "shan_chen": bench_shan_chen,
                "paper_sweep": lambda: bench_paper_sweep("f64"),
                "fp64_peak": lambda: measure_fp64_peak(int(os.environ.get("LOCAL_RANK", "0")))}
        print(json.dumps({args.leg: legs[args.leg]()}), flush=True)
        return 0
    return run_mlbm(args)


if __name__ == "__main__":
    sys.exit(main())
