#!/usr/bin/env python
"""Throughput benchmark of the fused explicit time step on one GB300.

Default workload: 2D Cahn-Hilliard (Model B, Eq. (model-b)), 4096 x 4096
periodic grid, FP64, h = 1, dt = 0.01, kappa = c1 = c2 = 1, 5-point Laplacian,
seeded uniform noise of +-0.01.  One benchmark step = SUB forward-Euler time
steps of the whole grid plus one FP64 mass reduction (the mass-drift check).

Prints one JSON line (rank 0).  `value` is GLUPS (grid points x time steps /
s / 1e9) with the fields resident in HBM, timed with CUDA events on the
launching stream; `e2e` is the same metric through the C ABI with host
buffers: every step writes the field from pinned host memory, steps, reduces
and reads the field back.  `--impl reference` times the FP64 CPU oracle on the
host cores instead (the reference arm).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# name -> (model, dims, shape (numpy order), dt, stencil, dtype, sub-steps per bench step
#          [, steps fused per launch: 0 = the library's choice [, kernel family]])
WORKLOADS = {
    "ch2d-4096-f64-lap5": (1, 2, (4096, 4096), 0.01, 0, 0, 100),
    "ch2d-4096-f64-lap9x4": (1, 2, (4096, 4096), 0.01, 2, 0, 100),
    "ch2d-4096-f32-lap5": (1, 2, (4096, 4096), 0.01, 0, 1, 100),
    "ch2d-16384-f32-lap5": (1, 2, (16384, 16384), 0.01, 0, 1, 20),
    "ch2d-16384-bf16-lap5": (1, 2, (16384, 16384), 0.01, 0, 2, 20),
    "ch2d-16384-f32-lap9x4": (1, 2, (16384, 16384), 0.01, 2, 1, 20),
    "gs2d-32768-bf16-lap5": (2, 2, (32768, 32768), 1.0, 0, 2, 10),
    "gs2d-8192-f32-lap5": (2, 2, (8192, 8192), 1.0, 0, 1, 10),
    "gs2d-32768-f32-lap5-k1": (2, 2, (32768, 32768), 1.0, 0, 1, 12, 1),
    "gs2d-32768-f32-lap5-k2": (2, 2, (32768, 32768), 1.0, 0, 1, 12, 2),
    "ch2d-16384-f32-lap5-k1": (1, 2, (16384, 16384), 0.01, 0, 1, 20, 1),
    "ch2d-16384-f32-lap5-k4": (1, 2, (16384, 16384), 0.01, 0, 1, 20, 4),
    "ch2d-16384-bf16-lap5-k4": (1, 2, (16384, 16384), 0.01, 0, 2, 20, 4),
    "ch2d-8192-f32-lap5": (1, 2, (8192, 8192), 0.01, 0, 1, 10),
    "ch3d-384-f32-lap7": (1, 3, (384, 384, 384), 0.005, 3, 1, 10),
    "ch3d-384-f64-lap27": (1, 3, (384, 384, 384), 0.005, 4, 0, 4),
    "ch3d-384-f64-lap7": (1, 3, (384, 384, 384), 0.005, 3, 0, 4),
    "ac2d-256-f64-lap5": (0, 2, (256, 256), 0.05, 0, 0, 1000),
    "gs2d-32768-f32-lap5": (2, 2, (32768, 32768), 1.0, 0, 1, 10),
    "gs2d-32768-f64-lap5": (2, 2, (32768, 32768), 1.0, 0, 0, 2),
    "ch3d-1024-f32-lap7": (1, 3, (1024, 1024, 1024), 0.005, 3, 1, 5),
    "ch3d-1024-bf16-lap7": (1, 3, (1024, 1024, 1024), 0.005, 3, 2, 5),
    "ch3d-1024-f64-lap7": (1, 3, (1024, 1024, 1024), 0.005, 3, 0, 2),
    "ch3d-1024-f32-lap27": (1, 3, (1024, 1024, 1024), 0.005, 4, 1, 5),
    "ch3d-1024-f64-lap27": (1, 3, (1024, 1024, 1024), 0.005, 4, 0, 2),
    "ch3d-1024-f64-lap27-zreg": (1, 3, (1024, 1024, 1024), 0.005, 4, 0, 2, 1, 2),
    "ac3d-512-f64-lap27": (0, 3, (512, 512, 512), 0.05, 4, 0, 10),
    "gs3d-512-f64-lap27": (2, 3, (512, 512, 512), 0.5, 4, 0, 5),
    "ch3d-1024-f32-lap13x4": (1, 3, (1024, 1024, 1024), 0.005, 5, 1, 5),
    "gs3d-512-f32-lap7": (2, 3, (512, 512, 512), 0.5, 3, 1, 10),
    "ac3d-1024-f32-lap27": (0, 3, (1024, 1024, 1024), 0.05, 4, 1, 5),
    "ac3d-1024-f32-lap7": (0, 3, (1024, 1024, 1024), 0.05, 3, 1, 6),
    # 3D temporal blocking: one step per launch against two (warp-row plane queues)
    "gs3d-512-f32-lap7-k1": (2, 3, (512, 512, 512), 0.5, 3, 1, 10, 1, 0),
    "gs3d-512-f32-lap7-k2": (2, 3, (512, 512, 512), 0.5, 3, 1, 10, 2),
    "gs3d-512-f32-lap7-async": (2, 3, (512, 512, 512), 0.5, 3, 1, 10, 1, 1),
    "gs3d-512-f32-lap7-tma": (2, 3, (512, 512, 512), 0.5, 3, 1, 10, 1, 6),
    "ch3d-1024-f32-lap7-async": (1, 3, (1024, 1024, 1024), 0.005, 3, 1, 5, 1, 1),
    "ch3d-1024-f32-lap7-tma": (1, 3, (1024, 1024, 1024), 0.005, 3, 1, 5, 1, 6),
    "ac3d-1024-f32-lap27-async": (0, 3, (1024, 1024, 1024), 0.05, 4, 1, 6, 1, 1),
    "ac3d-1024-f32-lap27-tma": (0, 3, (1024, 1024, 1024), 0.05, 4, 1, 6, 1, 6),
    "ac3d-1024-f32-lap27-k1": (0, 3, (1024, 1024, 1024), 0.05, 4, 1, 6, 1, 0),
    "ac3d-1024-f32-lap27-k2": (0, 3, (1024, 1024, 1024), 0.05, 4, 1, 6, 2),
    "ac3d-1024-f32-lap7-k2": (0, 3, (1024, 1024, 1024), 0.05, 3, 1, 6, 2),
    # Model C (phi coupled to a conserved rho), c3 = 0.5
    "mc2d-4096-f64-lap5": (3, 2, (4096, 4096), 0.02, 0, 0, 100),
    "mc2d-16384-f32-lap5": (3, 2, (16384, 16384), 0.02, 0, 1, 20),
    "mc3d-512-f64-lap7": (3, 3, (512, 512, 512), 0.02, 3, 0, 4),
    "mc3d-512-f32-lap7": (3, 3, (512, 512, 512), 0.02, 3, 1, 10),
    # semi-implicit Fourier spectral scheme (the library's own FFTs), the stencil entry unused
    "ch2d-4096-f64-spectral": (1, 2, (4096, 4096), 0.5, 0, 0, 20),
    "ac2d-4096-f64-spectral": (0, 2, (4096, 4096), 0.5, 0, 0, 20),
    "ch2d-8192-f32-spectral": (1, 2, (8192, 8192), 0.5, 0, 1, 20),
    "ch3d-256-f64-spectral": (1, 3, (256, 256, 256), 0.5, 3, 0, 10),
    # Model H (m and the d components of j), c3 = 0.5
    "mh2d-4096-f64-lap5": (4, 2, (4096, 4096), 0.01, 0, 0, 50),
    "mh2d-8192-f32-lap5": (4, 2, (8192, 8192), 0.01, 0, 1, 20),
    "mh3d-256-f64-lap7": (4, 3, (256, 256, 256), 0.005, 3, 0, 10),
    "mh3d-256-f32-lap7": (4, 3, (256, 256, 256), 0.005, 3, 1, 20),
    "mh3d-256-f32-lap27": (4, 3, (256, 256, 256), 0.005, 4, 1, 20),
    "mh3d-256-f32-lap13x4": (4, 3, (256, 256, 256), 0.005, 5, 1, 20),
    # generated cross Laplacians (accuracy order in the name), stencil entry 6
    "ch2d-4096-f64-gen8": (1, 2, (4096, 4096), 0.002, 6, 0, 50),
    "ac2d-4096-f64-gen6": (0, 2, (4096, 4096), 0.05, 6, 0, 50),
    "ch3d-256-f64-gen6": (1, 3, (256, 256, 256), 0.001, 6, 0, 10),
    "ch2d-8192-f32-gen8": (1, 2, (8192, 8192), 0.002, 6, 1, 20),
    # ablation: the unfused Cahn-Hilliard step (mu through a device-memory temporary)
    "ch2d-4096-f64-lap5-unfused": (1, 2, (4096, 4096), 0.01, 0, 0, 100, 1, 3),
    "ch2d-16384-f32-lap5-unfused": (1, 2, (16384, 16384), 0.01, 0, 1, 20, 1, 3),
    "ch3d-1024-f32-lap7-unfused": (1, 3, (1024, 1024, 1024), 0.005, 3, 1, 5, 1, 3),
}
DEFAULT = "ch2d-4096-f64-lap5"
MODEL_NAME = {0: "Allen-Cahn", 1: "Cahn-Hilliard", 2: "Gray-Scott", 3: "Model C", 4: "Model H"}
STENCIL_NAME = {0: "5-point", 1: "9-point box", 2: "4th-order 9-point cross", 3: "7-point", 4: "27-point",
                5: "4th-order 13-point cross", 6: "generated cross"}
DTYPE_NAME = {0: "f64", 1: "f32", 2: "bf16-storage/f32"}
ESIZE = {0: 8, 1: 4, 2: 2}

NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, nominal

# FP64 operations per stencil application with the fixed evaluation order and
# reuse of row/plane partial sums where the order permits it.
STENCIL_OPS = {0: 4, 1: 6, 2: 8, 3: 6, 4: 12, 5: 12}


# DRAM bytes (read + write) per step launch of the dominant kernel, from an ncu
# capture of the same kernel and workload (summaries in profiles/), keyed by
# (workload, steps per launch, kernel family); other pairs report null.
NCU_TRAFFIC = {
    ("ch2d-4096-f64-lap5", 1, 0): (242.47e6, "profiles/step2d_batch_ch_f64_lap5_4096.txt"),
    ("ch2d-4096-f64-lap5", 1, 4): (231.14e6, "profiles/step2d_batch_ch_f64_lap5_4096.txt"),
}


def spectral_ops_per_lup(npts: int) -> float:
    """FP64 operations per update of the spectral step: two real transforms at the
    radix-2 count of 2.5 log2(N) each, the cube (3) and the Fourier update (about
    6.5 per real point)."""
    import math

    return 5.0 * math.log2(npts) + 9.5


def spectral_bytes_per_lup_in_p(dims: int) -> int:
    """Algorithmic bytes per update of the spectral step, in units of the storage
    size P (a half spectrum holds about one P per real point): the x pass reads the
    spectrum and writes phi and the next step's transformed cubic term (3P); the
    last axis pass reads the transform and the resident spectrum and writes both
    (4P); in 3D the y passes before and after it read and write the transform
    (2P each)."""
    return 7 if dims == 2 else 11


def model_h_ops_per_lup(st: int) -> int:
    """Model H, fixed order: mu (s + 4), the m update (s + d (3 + dc) + 2) and each
    current component (s + dc + 4); dc = 1 or 3 FP64 operations per central
    difference of radius 1 or 2."""
    s = STENCIL_OPS[st]
    d = 3 if st >= 3 else 2
    dc = 3 if st in (2, 5) else 1
    return (2 + d) * s + d * (7 + 2 * dc) + 6


def generated_stencil_ops(order: int, dims: int) -> int:
    """Per application: r pair groups of 2d - 1 additions each, r + 1 multiplies /
    fused multiply-adds."""
    r = order // 2
    return r * (2 * dims - 1) + r + 1


def fp64_ops_per_lup(model: int, st: int, order: int = 0, dims: int = 2) -> int:
    if model == 4:
        return model_h_ops_per_lup(st)
    s = generated_stencil_ops(order, dims) if st == 6 else STENCIL_OPS[st]
    # Model C: mu of the density once per point (2), two stencils, the update (7)
    return {0: s + 5, 1: 2 * s + 5, 2: 2 * s + 9, 3: 2 * s + 9}[model]


def nfields(model: int, dims: int) -> int:
    return 1 + dims if model == 4 else (2 if model in (2, 3) else 1)


def hbm_bytes_per_lup(model: int, dtype: int, dims: int = 2) -> int:
    return 2 * nfields(model, dims) * ESIZE[dtype]


def load_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


# FP64 pipe: 152 SMs x 2 FP64 operations / clock x 2070 MHz (max SM clock).
FP64_PEAK_GOPS = 152 * 2 * 2.070


def roofline(model: int, dims: int, st: int, dtype: int, order: int, spectral: bool, npts: int, launch_ms: float,
             spl: int, traffic, peaks: dict) -> dict:
    """The roofline object of the dominant kernel: algorithmic work of one time step
    over the grid divided by the average step-kernel time (launch_ms per time step).
    FP64 kernels are bound by the FP64 pipe (ops against the derived peak), FP32/BF16
    kernels by HBM (algorithmic bytes against the measured copy bandwidth)."""
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    per_s = 1.0 / (launch_ms * 1e-3) / 1e9
    if spectral and dtype == 0:
        ops = spectral_ops_per_lup(npts)
        achieved = ops * npts * per_s
        return {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_GOPS, "unit": "FP64 Gop/s",
                "frac": achieved / FP64_PEAK_GOPS, "traffic": None,
                "note": f"semi-implicit spectral step, {ops:.1f} FP64 ops/LUP by the model 5 log2 N + 9.5 "
                        "(two real transforms at 2.5 log2 N each, cube, Fourier update)"}
    if spectral:
        bpl = spectral_bytes_per_lup_in_p(dims) * ESIZE[dtype]
        achieved = bpl * npts * per_s
        return {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                "frac_of_nominal": achieved / NOMINAL_HBM_GBS, "traffic": None,
                "note": f"semi-implicit spectral step, {bpl} bytes/LUP: one pass per transform axis (x pass "
                        "fused with the cube and the next step's forward transform, the last axis pass fused "
                        "with the Fourier update)"}
    if dtype == 0:
        ops = fp64_ops_per_lup(model, st, order, dims)
        achieved = ops * npts * per_s
        return {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_GOPS, "unit": "FP64 Gop/s",
                "frac": achieved / FP64_PEAK_GOPS, "traffic": traffic, "steps_per_launch": spl,
                "note": f"{ops} FP64 ops/LUP (fixed evaluation order); peak = 152 SMs x 2 FP64 ops/clk x 2.07 GHz; "
                        f"HBM side {hbm_bytes_per_lup(model, dtype, dims) * npts * per_s:.0f} GB/s"}
    bpl = hbm_bytes_per_lup(model, dtype, dims)
    achieved = bpl * npts * per_s
    return {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
            "frac_of_nominal": achieved / NOMINAL_HBM_GBS, "traffic": traffic, "steps_per_launch": spl,
            "note": f"{bpl} algorithmic bytes/LUP at one step per pass; peak = measured copy bandwidth"
                    + ("" if "hbm_gbs" in peaks else " (fallback)")
                    + (f"; {spl} steps per HBM pass, so this is an effective rate" if spl > 1 else "")}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        if not self.lines:
            return None
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def oracle_rate(model, dims, shape, dt, st, budget_s=15.0, max_steps=2000, spectral=False, order=0):
    """FP64 oracle GLUPS on the host cores over a bounded sample of the workload."""
    import numpy as np

    import oracle as O

    prm = O.params()
    npts = int(np.prod(shape))
    if spectral:
        from oracle import spectral as SO

        u = O.initial_condition(model, shape, seed=1, amp=0.01)
        t0 = time.perf_counter()
        SO.step(model, u, dt=dt, nsteps=1)
        t1 = time.perf_counter() - t0
        n = int(max(1, min(max_steps, budget_s / max(t1, 1e-6))))
        t0 = time.perf_counter()
        SO.step(model, u, dt=dt, nsteps=n)
        el = time.perf_counter() - t0
        return {"value": npts * n / el / 1e9, "unit": "GLUPS", "cores": 1, "kind": "oracle",
                "sample": f"{n} FP64 spectral oracle steps (numpy FFT) of the full {'x'.join(map(str, shape[::-1]))} "
                          f"grid ({el:.1f} s)"}
    if model == 4:
        m, js = O.initial_condition_h(shape, seed=1, amp=0.01)
        run = lambda n: O.step_h(st, m, js, dt=dt, prm=prm, nsteps=n)  # noqa: E731
    elif model in (2, 3):
        if model == 2:
            u, v = O.initial_condition(O.GS, shape, seed=2, amp=0.01, patches=64, patch=20)
        else:
            u, v = O.initial_condition(O.MC, shape, seed=1, amp=0.01)
        run = lambda n: O.step(model, st, u, v, dt=dt, prm=prm, nsteps=n)  # noqa: E731
    else:
        u = O.initial_condition(model, shape, seed=1, amp=0.01)
        run = lambda n: O.step(model, st, u, dt=dt, prm=prm, nsteps=n)  # noqa: E731
    if order and model in (0, 1):
        run = lambda n: O.step_gen(model, order, u, dt=dt, prm=prm, nsteps=n)  # noqa: E731

    run(1)  # start the OpenMP team
    t0 = time.perf_counter()
    run(2)
    t1 = (time.perf_counter() - t0) / 2
    n = int(max(1, min(max_steps, budget_s / max(t1, 1e-6))))
    t0 = time.perf_counter()
    run(n)
    el = time.perf_counter() - t0
    return {"value": npts * n / el / 1e9, "unit": "GLUPS", "cores": O.num_threads(), "kind": "oracle",
            "sample": f"{n} FP64 oracle time steps of the full {'x'.join(map(str, shape[::-1]))} grid "
                      f"({el:.1f} s, OpenMP)"}


# ------------------------------------------------------------ serving mix --

def served_requests(n_req: int, seed: int):
    """Seeded request stream with the shape of the served configuration: model
    uniform over Allen-Cahn / Cahn-Hilliard / Gray-Scott, 2D or 3D with equal
    probability, sides log-uniform in [64, 2048] (2D) or [32, 256] (3D), 100-5000
    steps, FP32 or FP64 storage, coefficients drawn in stable ranges, default
    stencils, dt inside the forward-Euler bound."""
    import numpy as np

    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_req):
        model = int(rng.integers(0, 3))
        dims = 2 if rng.random() < 0.5 else 3
        lo, hi = (64, 2048) if dims == 2 else (32, 256)
        side = int(round(float(np.exp(rng.uniform(np.log(lo), np.log(hi))))))
        shape = (side,) * dims
        nsteps = int(rng.integers(100, 5001))
        dtype = 1 if rng.random() < 0.5 else 0
        kw = dict(seed=1000 + i, dtype=dtype)
        if model == 2:
            kw.update(F=float(rng.uniform(0.02, 0.05)), k=float(rng.uniform(0.05, 0.065)), ic_amp=0.01,
                      gs_patches=int(rng.integers(1, 17)), gs_patch=min(8, side))
            dt = 1.0 if dims == 2 else 0.5
        else:
            kw.update(c1=float(rng.uniform(0.5, 1.5)), c2=float(rng.uniform(0.5, 1.5)), ic_amp=0.05)
            if model == 1:
                kw.update(kappa=float(rng.uniform(0.5, 1.5)))
                dt = 0.01 if dims == 2 else 0.005
            else:
                dt = 0.05
        out.append((model, shape, dt, nsteps, kw))
    return out


def run_served(sp, reqs, rate=None, budget=120 << 30, quantum=50):
    """Serve `reqs` (all at t=0 when rate is None, else Poisson arrivals at `rate`
    requests/s); returns (GLUPS over the makespan, latencies in s)."""
    import numpy as np

    rng = np.random.default_rng(7)
    lups = sum(int(np.prod(sh)) * n for _, sh, _, n, _ in reqs)
    with sp.Server(budget, max_slots=512, quantum_steps=quantum) as srv:
        t0 = time.perf_counter()
        arrivals = np.cumsum(rng.exponential(1.0 / rate, len(reqs))) if rate else np.zeros(len(reqs))
        tickets = []
        for (m, sh, dt, n, kw), ta in zip(reqs, arrivals):
            delay = ta - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            tickets.append(srv.submit(m, sh, dt=dt, nsteps=n, **kw))
        res = [srv.wait(t, timeout=3600) for t in tickets]
        el = time.perf_counter() - t0
    return lups / el / 1e9, [r.latency for r in res], el


def run_one_at_a_time_fp64(sp, reqs):
    """The same requests run one after another as plain FP64 grids."""
    import numpy as np

    lups = sum(int(np.prod(sh)) * n for _, sh, _, n, _ in reqs)
    t0 = time.perf_counter()
    for m, sh, dt, n, kw in reqs:
        kw = dict(kw, dtype=0)
        with sp.Simulation(m, sh, dt=dt, **kw) as s:
            s.step(n)
            s.reduce(sp.MASS)
    el = time.perf_counter() - t0
    return lups / el / 1e9, el


def served_summary_large(sp, n_req: int, seed=4, calib=100, baseline_sample=200):
    """The served stream at its stated size: capacities (burst GLUPS of the mixed
    stream and of its FP32 form) calibrated on the first `calib` requests, then
    all `n_req` requests arrive as a Poisson stream at 0.7 of the calibrated
    capacity, in both forms; the one-at-a-time FP64 baseline runs a seeded sample
    of `baseline_sample` requests of the same stream."""
    import numpy as np

    reqs = served_requests(n_req, seed)
    mean_lups = float(np.mean([np.prod(sh) * n for _, sh, _, n, _ in reqs]))
    cal = reqs[:calib]
    cal32 = [(m, sh, dt, n, dict(kw, dtype=1)) for m, sh, dt, n, kw in cal]
    burst_glups, _, burst_s = run_served(sp, cal)
    b32_glups, _, b32_s = run_served(sp, cal32)
    rate = 0.7 * burst_glups * 1e9 / mean_lups
    glups, lat, el = run_served(sp, reqs, rate=rate)
    reqs32 = [(m, sh, dt, n, dict(kw, dtype=1)) for m, sh, dt, n, kw in reqs]
    rate32 = 0.7 * b32_glups * 1e9 / mean_lups
    g32, lat32, el32 = run_served(sp, reqs32, rate=rate32)
    rng = np.random.default_rng(seed + 1)
    pick = sorted(rng.choice(n_req, size=min(baseline_sample, n_req), replace=False))
    fp64_glups, fp64_s = run_one_at_a_time_fp64(sp, [reqs[i] for i in pick])
    return {"requests": n_req, "mix": "AC/CH/GS x 2D (64^2-2048^2) / 3D (32^3-256^3) x FP32/FP64, 100-5000 steps",
            "budget_bytes": 120 << 30, "arrivals": "Poisson at 0.7 of the burst capacity of the first "
            f"{calib} requests", "calibration": {"burst_glups": burst_glups, "burst_makespan_s": burst_s,
                                                 "fp32_burst_glups": b32_glups, "fp32_burst_makespan_s": b32_s},
            "poisson_rate_per_s": rate, "glups": glups, "makespan_s": el,
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "fp32_form": {"poisson_rate_per_s": rate32, "glups": g32, "makespan_s": el32,
                          "p50_s": float(np.percentile(lat32, 50)), "p99_s": float(np.percentile(lat32, 99))},
            "fp64_one_at_a_time_glups": fp64_glups, "fp64_one_at_a_time_s": fp64_s,
            "fp64_one_at_a_time_sample": f"{len(pick)} requests drawn without replacement (seed {seed + 1})",
            "served_vs_fp64": glups / fp64_glups, "served_fp32_vs_fp64": g32 / fp64_glups}


def served_summary(sp, n_req=100, seed=4):
    import numpy as np

    if n_req > 1000:
        return served_summary_large(sp, n_req, seed)
    reqs = served_requests(n_req, seed)
    mean_lups = float(np.mean([np.prod(sh) * n for _, sh, _, n, _ in reqs]))
    burst_glups, _, burst_s = run_served(sp, reqs)
    rate = 0.7 * burst_glups * 1e9 / mean_lups
    glups, lat, el = run_served(sp, reqs, rate=rate)
    # the same stream served in its FP32 form (every request FP32 storage)
    reqs32 = [(m, sh, dt, n, dict(kw, dtype=1)) for m, sh, dt, n, kw in reqs]
    b32_glups, _, b32_s = run_served(sp, reqs32)
    rate32 = 0.7 * b32_glups * 1e9 / mean_lups
    g32, lat32, el32 = run_served(sp, reqs32, rate=rate32)
    fp64_glups, fp64_s = run_one_at_a_time_fp64(sp, reqs)
    return {"requests": n_req, "mix": "AC/CH/GS x 2D (64^2-2048^2) / 3D (32^3-256^3) x FP32/FP64, 100-5000 steps",
            "budget_bytes": 120 << 30, "burst_glups": burst_glups, "burst_makespan_s": burst_s,
            "poisson_rate_per_s": rate, "glups": glups, "makespan_s": el,
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "fp32_form": {"burst_glups": b32_glups, "burst_makespan_s": b32_s, "poisson_rate_per_s": rate32,
                          "glups": g32, "makespan_s": el32, "p50_s": float(np.percentile(lat32, 50)),
                          "p99_s": float(np.percentile(lat32, 99)),
                          "accuracy": "FP32 storage and arithmetic; relative L2 vs the FP64 oracle <= 2e-4 per "
                                      "field on served requests of ~5000 steps (Allen-Cahn and Cahn-Hilliard "
                                      "~1e-6, the Gray-Scott v field up to ~1e-4)"},
            "fp64_one_at_a_time_glups": fp64_glups, "fp64_one_at_a_time_s": fp64_s,
            "served_vs_fp64": burst_glups / fp64_glups, "served_fp32_vs_fp64": b32_glups / fp64_glups}


# The benchmark configurations beside the headline, measured in the same run with
# short timed regions: name -> (workload, bench steps timed).  One entry per
# configuration and stencil / storage type that the configuration names.
PER_CONFIG = [
    ("allen-cahn 256^2 f64 5-point", "ac2d-256-f64-lap5", 20),
    ("cahn-hilliard 4096^2 f64 9-point cross", "ch2d-4096-f64-lap9x4", 5),
    ("gray-scott 32768^2 f64 5-point", "gs2d-32768-f64-lap5", 4),
    ("gray-scott 32768^2 f32 5-point", "gs2d-32768-f32-lap5", 4),
    ("cahn-hilliard 1024^3 f64 7-point", "ch3d-1024-f64-lap7", 3),
    ("cahn-hilliard 1024^3 f64 27-point", "ch3d-1024-f64-lap27", 3),
    ("cahn-hilliard 1024^3 f32 7-point", "ch3d-1024-f32-lap7", 4),
    ("cahn-hilliard 1024^3 f32 27-point", "ch3d-1024-f32-lap27", 4),
]

# Error of each workload's result against the FP64 oracle, as the tests measure and
# bound it (relative L2 per field; tests/test_gpu_fullsize.py, test_gpu_serving.py).
def accuracy(name: str) -> str:
    dtype = WORKLOADS[name][5]
    if dtype == 0:
        if name.endswith("-spectral"):
            return "FP64: within 1e-12 of the field scale of the FP64 numpy oracle after 25 steps"
        return "FP64: bitwise equal to the FP64 oracle (fixed evaluation order)"
    if dtype == 2:
        return ("BF16 storage: no accuracy bound (created with SP_FLAG_BF16_NO_BOUND); relative L2 vs the FP64 "
                "oracle 0.04 to 1.0 over the benchmark runs (Cahn-Hilliard from +-0.01 noise stalls: 0.84 on "
                "128^3 after 2000 steps)")
    if name.startswith("ch2d") and "lap9x4" in name:
        return "FP32: relative L2 2.3e-6 vs the FP64 oracle after 10000 steps of 4096^2 (bound 1e-5)"
    if name.startswith("ch2d"):
        return "FP32: relative L2 4.1e-6 vs the FP64 oracle after 10000 steps of 4096^2 (bound 1e-5)"
    if name.startswith("gs2d"):
        return "FP32: relative L2 u 3.3e-6, v 1.0e-4 vs the FP64 oracle after 5000 steps of 2048^2 (bound 2e-4)"
    if name.startswith("ch3d"):
        return ("FP32: relative L2 4.1e-7 (7-point), 2.4e-7 (27-point), 1.8e-7 (13-point) vs the FP64 oracle "
                "after 2000 steps of 128^3 (bound 1e-6)")
    if name.startswith(("ac3d", "gs3d")):
        return ("FP32: relative L2 <= 2e-4 vs the FP64 oracle on served 3D requests of ~5000 steps "
                "(Allen-Cahn ~1e-7, Gray-Scott v ~3e-5)")
    return "FP32: relative L2 <= 1e-5 vs the FP64 oracle on the parity tests' runs"


def time_workload(sp, name: str, steps: int, warmup: int = 3, stream=None) -> dict:
    """GLUPS and roofline of one workload, autotuned, timed like the headline (CUDA
    events on the launching stream around each bench step, one mass reduction per
    bench step), with the clocks sampled during the timed region."""
    import numpy as np
    import torch

    model, dims, shape, dt, st, dtype, sub = WORKLOADS[name][:7]
    npts = int(np.prod(shape))
    kw = dict(stencil=st, dtype=dtype, seed=1, ic_amp=0.01, flags=sp.FLAG_BF16_NO_BOUND if dtype == 2 else 0)
    if model == 2:
        kw.update(seed=2, gs_patches=64, gs_patch=20)
    stream = stream or torch.cuda.Stream()
    with sp.Simulation(model, shape, dt=dt, **kw) as sim:
        sim.autotune(stream=stream)
        for _ in range(warmup):
            sim.step(sub, stream=stream)
            sim.reduce(sp.MASS, stream=stream)
        spl, variant = sim.launch_config
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * steps + 2)]
        torch.cuda.synchronize()
        with ClockSampler(torch.cuda.current_device()) as clocks:
            ev[0].record(stream)
            for i in range(steps):
                ev[2 * i + 1].record(stream)
                sim.step(sub, stream=stream)
                ev[2 * i + 2].record(stream)
                sim.reduce(sp.MASS, stream=stream)
            ev[-1].record(stream)
            torch.cuda.synchronize()
    total_ms = ev[0].elapsed_time(ev[-1])
    step_ms = sum(ev[2 * i + 1].elapsed_time(ev[2 * i + 2]) for i in range(steps))
    launch_ms = step_ms / (steps * sub)
    roof = roofline(model, dims, st, dtype, 0, False, npts, launch_ms, spl,
                    NCU_TRAFFIC.get((name, spl, variant), (None,))[0], load_peaks())
    return {"workload": workload_config(name)["workload"], "glups": npts * sub * steps / (total_ms * 1e-3) / 1e9,
            "kernel_glups": npts / (launch_ms * 1e-3) / 1e9, "ms_per_time_step": launch_ms,
            "roofline": {k: roof[k] for k in ("bound", "achieved", "peak", "unit", "frac")},
            "launch_config": {"steps_per_launch": spl, "kernel_family": variant},
            "accuracy": accuracy(name), "clocks": clocks.summary(),
            "timed": f"{steps} bench steps of {sub} time steps + one mass reduction each"}


def per_config_summary(sp, stream=None) -> dict:
    return {label: time_workload(sp, name, steps, stream=stream) for label, name, steps in PER_CONFIG}


def reduce_max_over_ranks(values, device="cpu"):
    """Element-wise maximum of `values` over all ranks (the job's time is the slowest
    rank's); identity when torch.distributed is not initialised."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t]


def replica_glups(lups_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job GLUPS of `world` independent replicas that each did `lups_per_rank`
    updates, over the slowest rank's time (weak scaling: work per GPU is fixed)."""
    return world * lups_per_rank / seconds / 1e9


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    model, dims, shape, dt, st, dtype, sub = WORKLOADS[args.workload][:7]
    import numpy as np

    import oracle as O

    npts = int(np.prod(shape))
    prm = O.params()
    if model == 2:
        u, v = O.initial_condition(O.GS, shape, seed=2, amp=0.01, patches=64, patch=20)
    elif model == 3:
        u, v = O.initial_condition(O.MC, shape, seed=1, amp=0.01)
    else:
        u, v = O.initial_condition(model, shape, seed=1, amp=0.01), None
    # one reference step = a bounded sample: `per` oracle time steps of the full grid
    t0 = time.perf_counter()
    O.step(model, st, u, v, dt=dt, prm=prm, nsteps=1) if v is not None else O.step(model, st, u, dt=dt, prm=prm, nsteps=1)
    t1 = time.perf_counter() - t0
    total_budget = 120.0
    per = int(max(1, min(sub, total_budget / max(t1, 1e-6) / max(1, args.steps + args.warmup))))
    for _ in range(args.warmup):
        O.step(model, st, u, v, dt=dt, prm=prm, nsteps=per) if v is not None else O.step(model, st, u, dt=dt, prm=prm, nsteps=per)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.step(model, st, u, v, dt=dt, prm=prm, nsteps=per) if v is not None else O.step(model, st, u, dt=dt, prm=prm, nsteps=per)
    el = time.perf_counter() - t0
    val = npts * per * args.steps / el / 1e9
    line = {"impl": "reference", "metric": "GLUPS", "value": val, "unit": "GLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded uniform noise)", "config": workload_config(args.workload),
            "e2e": {"value": val, "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "cpu_baseline": {"value": val, "unit": "GLUPS", "cores": O.num_threads(), "kind": "oracle",
                             "sample": f"each step = {per} FP64 oracle time steps of the full grid"}}
    print(json.dumps(line), flush=True)
    return 0


def workload_config(name):
    model, dims, shape, dt, st, dtype, sub = WORKLOADS[name][:7]
    if name.endswith("-spectral"):
        lap = "semi-implicit Fourier spectral scheme (continuous Laplacian)"
    elif "-gen" in name:
        lap = f"generated cross Laplacian of order {name.rsplit('-gen', 1)[1]}, forward Euler"
    else:
        lap = f"{STENCIL_NAME[st]} Laplacian, forward Euler"
    return {"workload": f"{MODEL_NAME[model]} {dims}D {'x'.join(map(str, shape[::-1]))} {DTYPE_NAME[dtype]}, "
                        f"{lap}, dt={dt}, h=1, periodic",
            "model": MODEL_NAME[model], "grid": list(shape[::-1]), "stencil": lap,
            "storage": DTYPE_NAME[dtype], "time_steps_per_bench_step": sub,
            "l2": "inputs larger than L2 (ping-pong field buffers exceed the 126 MB L2)"
            if int(__import__("numpy").prod(shape)) * ESIZE[dtype] * 2 > 126e6 else "L2-resident (small grid)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT, choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the library's default launch configuration")
    ap.add_argument("--served-requests", type=int, default=100)
    ap.add_argument("--no-per-config", action="store_true", help="skip the other benchmark configurations")
    ap.add_argument("--launch-config", default="", help="pin 'steps_per_launch,family' instead of autotuning")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2511_10508_gb300 as sp

    model, dims, shape, dt, st, dtype, sub = WORKLOADS[args.workload][:7]
    spl_req = WORKLOADS[args.workload][7] if len(WORKLOADS[args.workload]) > 7 else 0
    npts = int(np.prod(shape))
    spectral = args.workload.endswith("-spectral")
    order = int(args.workload.rsplit("-gen", 1)[1]) if "-gen" in args.workload else 0
    kw = dict(stencil=st, dtype=dtype, seed=1 + rank, ic_amp=0.01, steps_per_launch=spl_req,
              scheme=sp.SCHEME_SPECTRAL if spectral else sp.SCHEME_FD,
              flags=sp.FLAG_BF16_NO_BOUND if dtype == 2 else 0)  # BF16 storage: no accuracy bound
    if order:
        kw.update(stencil_order=order)
    if model == 2:
        kw.update(seed=2 + rank, gs_patches=64, gs_patch=20)
    sim = sp.Simulation(model, shape, dt=dt, **kw)
    stream = torch.cuda.Stream()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
            torch.cuda.synchronize()

    def bench_step():
        sim.step(sub, stream=stream)
        sim.reduce(sp.MASS, stream=stream)

    # warm-up (untimed); the library's autotuner picks the launch configuration
    # here unless the workload fixes the steps per launch
    family_req = WORKLOADS[args.workload][8] if len(WORKLOADS[args.workload]) > 8 else None
    if args.launch_config:
        sim.launch_config = tuple(int(x) for x in args.launch_config.split(","))
    elif family_req is not None:
        sim.launch_config = (max(spl_req, 1), family_req)
    elif not spl_req and not args.no_autotune:
        sim.autotune(stream=stream)
    for _ in range(args.warmup):
        bench_step()
    spl, variant = sim.launch_config
    barrier()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps + 2)]
    with ClockSampler(local) as clocks:
        barrier()
        ev[0].record(stream)
        for i in range(args.steps):
            ev[2 * i + 1].record(stream)
            sim.step(sub, stream=stream)
            ev[2 * i + 2].record(stream)
            sim.reduce(sp.MASS, stream=stream)
        ev[-1].record(stream)
        barrier()
    total_ms = ev[0].elapsed_time(ev[-1])
    per_step = [ev[2 * i + 1].elapsed_time(ev[2 * i + 2]) for i in range(args.steps)]
    step_ms = sum(per_step)
    best_ms, median_ms = min(per_step), float(np.median(per_step))
    total_ms, step_ms = reduce_max_over_ranks([total_ms, step_ms], device="cuda")
    lups = npts * sub * args.steps
    value = replica_glups(lups, world, total_ms * 1e-3)
    launch_ms = step_ms / (args.steps * sub)  # average duration of one step-kernel launch

    roof = roofline(model, dims, st, dtype, order, spectral, npts, launch_ms, spl,
                    NCU_TRAFFIC.get((args.workload, spl, variant), (None,))[0], load_peaks())
    achieved = roof["achieved"]
    if roof["unit"] == "FP64 Gop/s":
        # the device's sustained FP64 FMA rate (independent chains on every SM),
        # measured after the timed region: the attainable ceiling beside the nominal one
        measured = sp.probe_fp64_rate(stream=stream)
        roof["measured_fp64_gops"] = measured
        roof["frac_of_measured_fp64"] = achieved / measured if measured > 0 else None

    e2e = None
    if not args.no_e2e:
        n_fields = nfields(model, dims)
        host_in = [torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy() for _ in range(n_fields)]
        host_out = torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()
        for f in range(n_fields):
            host_in[f][...] = sim.read(f, stream=stream)
        e2e_steps = max(1, min(args.steps, 5))
        barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            for f in range(n_fields):
                sim.write(f, host_in[f], stream=stream)
            sim.step(sub, stream=stream)
            sim.reduce(sp.MASS, stream=stream)
            host_out[...] = 0
            N = sp._native
            N.check(N.lib().sp_read(sim.handle, 0, host_out.ctypes.data, host_out.nbytes, 1,
                                    stream.cuda_stream), "sp_read")
        barrier()
        el = reduce_max_over_ranks([time.perf_counter() - t0], device="cuda")[0]
        e2e = {"value": replica_glups(npts * sub * e2e_steps, world, el), "unit": "GLUPS",
               "h2d_bytes_per_step": npts * 8 * n_fields, "d2h_bytes_per_step": npts * 8 + 8, "steps": e2e_steps}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_rate(model, dims, shape, dt, st, spectral=spectral, order=order)

    served = None
    if rank == 0 and not args.no_served:
        served = served_summary(sp, n_req=args.served_requests)

    per_config = None
    if rank == 0 and world == 1 and not args.no_per_config and args.workload == DEFAULT:
        sim.close()
        per_config = per_config_summary(sp, stream=stream)

    # step kernels (one per spl time steps, plus a single-step remainder) and the
    # two reduction passes
    launches_per_step = (sub // spl + sub % spl) * (2 if variant == 3 else 1) + 2
    line = {"metric": "GLUPS", "value": value, "unit": "GLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": {0: "f64", 1: "f32", 2: "bf16"}[dtype],
            "data": "synthetic (seeded uniform noise, generated on device)",
            "config": dict(workload_config(args.workload), parallelism=f"replicas x{world}" if world > 1 else "1 GPU"),
            "roofline": roof, "accuracy": accuracy(args.workload), "cpu_baseline": cpu, "e2e": e2e,
            "clocks": clocks.summary(), "gpu_launches": launches_per_step * args.steps, "served": served,
            "per_config": per_config,
            "kernel_ms_per_time_step": launch_ms,
            "step_kernels_ms": {"mean": step_ms / args.steps, "median": median_ms, "best": best_ms,
                                "note": f"device time of the {sub} time steps of one bench step (CUDA events)"},
            "launch_config": {"steps_per_launch": spl, "kernel_family": variant,
                              "autotuned": bool(not spl_req and not args.no_autotune and not args.launch_config
                                                and family_req is None),
                              "ablation": "unfused two-pass Cahn-Hilliard step (5 field accesses per update)"
                              if variant == 3 else None}}
    sim.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
