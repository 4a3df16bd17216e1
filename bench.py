"""Benchmark of the DBFFT hot path on GB300.

Workload (one step): the effective stiffness of a 64^3 random-sphere composite
(non-overlapping spheres of radius 6 voxels to volume fraction 0.25, stiffness
contrast 100, nu = 0.3, seed 190512725 + 2) -- the six unit Mandel macro
strains solved as six right-hand sides of one batched, FP32-inner /
FP64-outer refined PCG to a true FP64 relative residual of 1e-6.

Metric: voxel * CG-iterations / s (inner CG iterations summed over the six
right-hand sides), and the time to a 1e-6 relative residual of the mixed
batched solve against FP64 PCG solving the six right-hand sides one after
another on the same GPU.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (launched by torch.distributed.run) every rank solves its own copy
of the workload (weak scaling, no collective on the data path); value is the
total work of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "voxel*CG-iters/s and time to 1e-6 rel. residual, mixed batched vs FP64 plain"
UNIT = "voxel*CG-iter/s"
N_GRID = 64
TOL = 1e-6
ETA_INNER = 1e-3
WORKLOAD = "64^3 random-sphere composite (r=6 vox, vf 0.25, contrast 100, nu 0.3), 6 unit Mandel strains"

# DRAM traffic per launch of the dominant kernel from an ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum), keyed by kernel; valid only
# for the kernel sources it was taken on (hash of KERNEL_SOURCES below).
# pass3_tangent_f32: the line-bulk k_axis3_lb<64, 6, OP_ISO, 1> of the 64^3 x 6 RHS
# step (warp lines, one right-hand side per CTA, the tuned form), ncu with caches
# flushed before the launch (39.50 MB read, nothing written back; inside the timed
# step the fields are L2-resident).
NCU_TRAFFIC = {"pass3_tangent_f32": {"bytes": 39500000, "src": "67fa03f4f67dfddf"},
               "fft_ax1_f32": {"bytes": 38940000 + 256, "src": "d1758b792b1f9b63"},
               "fft_ax2_f32": {"bytes": 38940000 + 256, "src": "d1758b792b1f9b63"}}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# sources that make up each profiled pass's kernels (a change invalidates its ncu counters)
KERNEL_SOURCES = {
    "pass3_tangent_f32": ["dbfft_dev.cuh", "fft.cuh", "passes.cuh", "constitutive.cuh", "pass3.cuh", "pass3_pipe.cuh",
                          "pass3_lb.cuh", "tma.cuh", "launch.h", "k_ax3_impl.cuh", "k_ax3_f32.cu", "k_ax3p_impl.cuh",
                          "k_ax3p_f32.cu", "k_ax3lb_f32.cu"],
    "fft_ax1_f32": ["dbfft_dev.cuh", "fft.cuh", "passes.cuh", "launch.h", "k_ax2.cu"],
    "fft_ax2_f32": ["dbfft_dev.cuh", "fft.cuh", "passes.cuh", "launch.h", "k_ax2.cu"],
}


def _sources_hash(files=None):
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1905_12725_gb300", "csrc")
    for n in sorted(files if files is not None else os.listdir(d)):
        with open(os.path.join(d, n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.time()  # the timed region starts once sampling runs
            while not self.lines and time.time() - t0 < 3.0 and self.proc.poll() is None:
                time.sleep(0.01)
            self.first = len(self.lines)
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        n_end = len(self.lines)
        t0 = time.time()  # one more sample after the region ends
        while len(self.lines) <= n_end and time.time() - t0 < 1.0:
            time.sleep(0.01)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def workload_inputs():
    from paper_1905_12725_gb300 import synth
    c = synth.config2(n=N_GRID)
    return c


# ------------------------------------------------------------------ CPU oracle sample
def oracle_sample(c, iters=40):
    """Time the FP64 oracle's PCG on the first right-hand side for a bounded number of iterations."""
    import oracle.dbfft_oracle as o
    shape = (N_GRID,) * 3
    lam, mu = o.lame(c["E"][c["phase"]], c["nu"][c["phase"]])
    T = o.IsoTangent(lam, mu)
    prob = o.Problem(shape)
    b = o.linear_rhs(prob, T, o.mandel_basis()[0])
    M = prob.make_preconditioner(T.mean())
    t0 = time.perf_counter()
    c0 = time.process_time()
    _, it, _ = o.pcg(prob, lambda v: prob.apply_K(T, v[0], v[1]), M, b, 1e-30, iters)
    dt = time.perf_counter() - t0
    cores = max(1, round((time.process_time() - c0) / dt))  # threads the sample kept busy
    V = N_GRID ** 3
    return V * it / dt, it, dt, cores


def _oracle_rhs_job(m, iters):
    """One unit Mandel strain of the headline workload through the oracle's PCG (a pool task)."""
    import oracle.dbfft_oracle as o
    c = workload_inputs()
    shape = (N_GRID,) * 3
    lam, mu = o.lame(c["E"][c["phase"]], c["nu"][c["phase"]])
    T = o.IsoTangent(lam, mu)
    prob = o.Problem(shape)
    b = o.linear_rhs(prob, T, o.mandel_basis()[m])
    M = prob.make_preconditioner(T.mean())
    t0 = time.perf_counter()
    _, it, _ = o.pcg(prob, lambda v: prob.apply_K(T, v[0], v[1]), M, b, 1e-30, iters)
    return it, time.perf_counter() - t0


def oracle_sample_all_cores(iters=20):
    """The oracle on every host core it can use: the six right-hand sides of the headline
    workload as six processes (spawned, so none inherits a CUDA context), each a bounded
    PCG sample; throughput = the iterations of all six over the longest of their PCG times
    (they run side by side; set-up outside the timed PCG is not counted)."""
    import multiprocessing as mp
    n = min(6, os.cpu_count() or 1)
    ctx = mp.get_context("spawn")
    with ctx.Pool(n) as pool:
        res = pool.starmap(_oracle_rhs_job, [(m, iters) for m in range(6)])
    dt = max(r[1] for r in res)
    its = sum(r[0] for r in res)
    return N_GRID ** 3 * its / dt, its, dt, n


def reference_arm(args, rank, world):
    if rank != 0:
        return
    c = workload_inputs()
    vals = []
    for _ in range(args.warmup):
        oracle_sample(c, iters=2)
    t_all = 0.0
    its = 0
    cores = 1
    for _ in range(args.steps):
        v, it, dt, nc = oracle_sample(c, iters=args.ref_iters)
        vals.append(v)
        t_all += dt
        its += it
        cores = max(cores, nc)
    value = N_GRID ** 3 * its / t_all
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_all / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "n": N_GRID, "batch": 6},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{args.ref_iters} PCG iterations of the FP64 numpy oracle on right-hand side 1 "
                                   f"per step (host cores: {os.cpu_count()})"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm
TUNE_CACHE = os.path.join(os.environ.get("TMPDIR", "/tmp"), "dbfft_tune_cache.txt")


def make_solver(c, precision, batch, targets=None, tol=TOL):
    from paper_1905_12725_gb300 import dbfft
    shape = (N_GRID,) * 3
    if targets is None:
        targets = np.zeros((batch, 3, 3))
    s = dbfft.Solver(shape, c["phase"], dbfft.iso_phases(c["E"], c["nu"]), targets, batch=batch,
                     precision=precision, tol=tol, eta_inner=ETA_INNER, max_iter=20000, max_newton=100)
    s.tuning = s.autotune(TUNE_CACHE)  # times launch shapes once, later contexts read the cache
    return s


def unit_mandel(m):
    pi = [0, 1, 2, 1, 0, 0]
    pj = [0, 1, 2, 2, 2, 1]
    t = np.zeros((3, 3))
    v = 1.0 if m < 3 else 1.0 / math.sqrt(2.0)
    t[pi[m], pj[m]] = t[pj[m], pi[m]] = v
    return t


def l2_roofline(dbfft, prof):
    """The FP32 passes of the step against the measured L2 copy bandwidth.

    At 64^3 x 6 right-hand sides the fields of a CG iteration (W 39 MB, CG
    vectors 20 MB) stay in the 126 MB L2 between passes, so L2, not HBM, is the
    memory ceiling of those passes; each pass's algorithmic bytes per second
    are reported against `dbfft_l2_copy_rate` (a 32 MB copy repeated in L2).
    """
    try:
        peak = dbfft.l2_copy_rate()
    except Exception as exc:  # measurement aid only
        return {"error": str(exc)[:200]}
    rows = {}
    for k, v in prof.items():
        if not k.endswith("_f32") or v["ms"] <= 0 or v["bytes"] <= 0:
            continue
        gbs = v["bytes"] / (v["ms"] * 1e-3) / 1e9
        rows[k] = {"GBps": gbs, "frac_of_l2": gbs / peak}
    return {"l2_copy_gbs": peak, "kernels": rows}


def fp64_roofline(dbfft, prof, hbm_peak, n, nc):
    """The FP64 residual chain against the measured FP64 FMA rate of this GPU.

    Flop model (stated, not counted): a complex transform of length n costs
    5 n log2 n flops, so 5 log2 n per complex element it reads and writes once
    (16 + 16 bytes in FP64); pass 3 runs two real transforms of length n per
    component and voxel (2.5 log2 n flops each) and about 36 flops of
    contraction per voxel. The element-wise passes are reported against HBM.
    """
    try:
        peak64 = dbfft.fp64_fma_rate()
    except Exception as exc:  # measurement aid only
        return {"error": str(exc)[:200]}
    lg = math.log2(n)
    tot = sum(v["ms"] for v in prof.values())
    rows, ms64 = {}, 0.0
    for k, v in prof.items():
        if not k.endswith("_f64") or not v["launches"] or v["ms"] <= 0:
            continue
        ms64 += v["ms"]
        row = {"launches": v["launches"], "ms_per_launch": v["ms"] / v["launches"],
               "GBps": v["bytes"] / (v["ms"] * 1e-3) / 1e9, "frac_of_hbm": v["bytes"] / (v["ms"] * 1e-3) / 1e9 / hbm_peak}
        if k.startswith("fft_"):
            flops = v["bytes"] / 32.0 * 5.0 * lg
        elif k.startswith("pass3"):
            voxels = (v["bytes"] / (2 * nc)) / 8.0  # bytes ~ 2 nc component passes of H * 16 B = V * 8 B each
            flops = voxels * (2 * nc * 2.5 * lg + 36.0)
        else:
            flops = None
        if flops is not None:
            row["tflops"] = flops / (v["ms"] * 1e-3) / 1e12
            row["frac_of_fp64_peak"] = row["tflops"] / peak64
        rows[k] = row
    return {"fma_peak_tflops": peak64, "share_of_step": ms64 / tot if tot else None, "kernels": rows,
            "flop_model": "5 log2 n flops per complex element per transform; pass 3: 2 nc x 2.5 log2 n + 36 per voxel"}


def operator_256(torch, dbfft, peak, iters=44):
    """FP32 inner-CG pass chain on a 256^3 linear two-phase RVE (one right-hand side)."""
    from paper_1905_12725_gb300 import synth
    n = 256
    # launch by launch, the inner CG runs in chunks of 4, 8, 16, 16, ... iterations; a cap on a
    # chunk boundary makes every profiled launch one of a working iteration
    b, c = 4, 4
    while b < iters:
        c = min(2 * c, 16)
        b += c
    iters = b
    rng = synth.Xoshiro256ss(synth.SEED_BASE + 42)
    g = np.random.default_rng(7)
    phase = (g.random((n, n, n)) < 0.3).astype(np.uint16)
    del rng
    eps = np.zeros((1, 3, 3))
    eps[0, 0, 0] = 1e-3
    s = dbfft.Solver((n, n, n), phase, dbfft.iso_phases([1.0, 100.0], [0.3, 0.3]), eps,
                     precision=dbfft.DBFFT_MIXED, tol=1e-30, eta_inner=1e-30, max_iter=iters, max_newton=1)
    tuning = s.autotune(TUNE_CACHE)
    s.solve_increment(0, allow_not_converged=True)  # warm-up (the next inner solves run as CUDA graphs)
    s.close()

    # graph-mode cost of one CG iteration: difference of two solves that differ only in the cap
    def graph_solve_ms(cap):
        sg = dbfft.Solver((n, n, n), phase, dbfft.iso_phases([1.0, 100.0], [0.3, 0.3]), eps,
                          precision=dbfft.DBFFT_MIXED, tol=1e-30, eta_inner=1e-30, max_iter=cap, max_newton=1)
        sg.autotune(TUNE_CACHE)
        sg.solve_increment(0, allow_not_converged=True)
        torch.cuda.synchronize()
        ts = []
        for _ in range(3):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(sg.stream)
            sg.solve_increment(0, allow_not_converged=True)
            e1.record(sg.stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        sg.close()
        return min(ts)

    t_lo, t_hi = graph_solve_ms(iters // 2), graph_solve_ms(iters + iters // 2)
    graph_ms_it = (t_hi - t_lo) / iters

    s = dbfft.Solver((n, n, n), phase, dbfft.iso_phases([1.0, 100.0], [0.3, 0.3]), eps,
                     precision=dbfft.DBFFT_MIXED, tol=1e-30, eta_inner=1e-30, max_iter=iters, max_newton=1)
    s.autotune(TUNE_CACHE)
    s.solve_increment(0, allow_not_converged=True)
    s.profile(True)
    t0 = time.perf_counter()
    rep = s.solve_increment(0, allow_not_converged=True)
    wall = time.perf_counter() - t0
    prof = s.profile_read()
    s.profile(False)
    s.close()
    names = ["pass1_grad_cg_f32", "pass1_grad_ax2_cg_f32", "fft_ax2_f32", "fft_ax1_f32", "pass3_tangent_f32",
             "pass5_div_cg_f32", "pass5_ax2_div_cg_f32"]
    rows = {}
    it_ms = 0.0
    it_bytes = 0.0
    for k in names:
        e = prof.get(k)
        if not e or not e["launches"]:
            continue
        gbs = e["bytes"] / (e["ms"] * 1e-3) / 1e9
        rows[k] = {"launches": e["launches"], "ms_per_launch": e["ms"] / e["launches"], "GBps": gbs,
                   "frac": gbs / peak}
        it_ms += e["ms"]
        it_bytes += e["bytes"]
    iters = rep["cg_iters"]
    bytes_it = it_bytes / max(iters, 1)
    # the method's algorithmic bytes of one FP32 CG iteration: the fused five-pass
    # operator (54 component passes) plus the CG vector work (21), one component
    # pass being one complex FP32 component over the half spectrum, plus 1 byte
    # of phase id per voxel
    H = n * n * (n // 2 + 1)
    method_bytes_it = 75 * H * 8 + n ** 3
    return {"grid": "256^3, 1 RHS, FP32 inner CG, iso two-phase (vf 0.3, contrast 100)", "tuning": tuning,
            "graph_ms_per_cg_iter": graph_ms_it,
            "graph_voxel_cg_iters_per_s": n ** 3 / (graph_ms_it * 1e-3),
            "method_bytes_per_cg_iter": method_bytes_it,
            "graph_method_GBps": method_bytes_it / (graph_ms_it * 1e-3) / 1e9,
            "graph_method_frac": method_bytes_it / (graph_ms_it * 1e-3) / 1e9 / peak,
            "impl_bytes_per_cg_iter": bytes_it,
            "graph_chain_GBps": bytes_it / (graph_ms_it * 1e-3) / 1e9,
            "graph_chain_frac": bytes_it / (graph_ms_it * 1e-3) / 1e9 / peak,
            "cg_iters": iters, "ms_per_cg_iter": it_ms / max(iters, 1),
            "voxel_cg_iters_per_s": n ** 3 * iters / (it_ms * 1e-3) if it_ms else None,
            "chain_GBps": it_bytes / (it_ms * 1e-3) / 1e9 if it_ms else None,
            "chain_frac": (it_bytes / (it_ms * 1e-3) / 1e9) / peak if it_ms else None,
            "method_frac": (method_bytes_it * iters / (it_ms * 1e-3) / 1e9) / peak if it_ms else None,
            "fracs_note": "*_method_frac: the method's 75 component passes + 1 B/voxel per CG iteration; "
                          "*_chain_frac: the bytes this implementation's kernels move",
            "passes": rows, "wall_s": wall}


def cufft_operator_256(torch, reps=10):
    """Comparison only: the same small-strain operator application K u at 256^3
    (FP32, one RHS, the two-phase map of operator_256) composed from torch
    element-wise ops and torch.fft (cuFFT) -- Fourier gradient, inverse 3-D
    real FFT of six components, isotropic stress, forward 3-D FFT,
    divergence. No part of the library uses it."""
    n = 256
    dev = torch.device("cuda")
    g = np.random.default_rng(7)
    phase = torch.from_numpy((g.random((n, n, n)) < 0.3).astype(np.int64)).to(dev)
    E = torch.tensor([1.0, 100.0], device=dev)
    nu = 0.3
    lam_t = (E * nu / ((1 + nu) * (1 - 2 * nu)))[phase].float()
    mu_t = (E / (2 * (1 + nu)))[phase].float()
    k = torch.fft.fftfreq(n, d=1.0 / n, device=dev).float() * 2 * math.pi
    k[n // 2] = 0.0
    kh = k[: n // 2 + 1].clone()
    kh[n // 2] = 0.0
    x1, x2, x3 = k[:, None, None], k[None, :, None], kh[None, None, :]
    u = (torch.randn(3, n, n, n // 2 + 1, device=dev) + 1j * torch.randn(3, n, n, n // 2 + 1, device=dev)).to(
        torch.complex64)
    pairs = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
    xs = [x1, x2, x3]

    def apply(u):
        eh = torch.stack([0.5j * (xs[i] * u[j] + xs[j] * u[i]) for i, j in pairs])
        e = torch.fft.irfftn(eh, s=(n, n, n), dim=(-3, -2, -1))
        tr = e[0] + e[1] + e[2]
        sig = torch.stack([lam_t * tr + 2 * mu_t * e[0], lam_t * tr + 2 * mu_t * e[1], lam_t * tr + 2 * mu_t * e[2],
                           2 * mu_t * e[3], 2 * mu_t * e[4], 2 * mu_t * e[5]])
        sh = torch.fft.rfftn(sig, dim=(-3, -2, -1))
        q0 = xs[0] * sh[0] + xs[1] * sh[5] + xs[2] * sh[4]
        q1 = xs[0] * sh[5] + xs[1] * sh[1] + xs[2] * sh[3]
        q2 = xs[0] * sh[4] + xs[1] * sh[3] + xs[2] * sh[2]
        return torch.stack([q0, q1, q2]) * (-1j / n ** 3)

    for _ in range(3):
        apply(u)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        apply(u)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    return {"what": "torch.fft (cuFFT) + torch element-wise ops, K u only (no CG vector work), FP32, 256^3, 1 RHS",
            "ms_per_application": ms, "voxel_applications_per_s": n ** 3 / (ms * 1e-3)}


# ------------------------------------------------------------------ other configurations
def _timed(fn):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return out, time.perf_counter() - t0


def case_c1():
    """16^3 centred sphere, E 1 / 10, nu 0.3, eps_xx = 1e-3, FP64 PCG to 1e-8."""
    from paper_1905_12725_gb300 import dbfft, synth
    c = synth.config1()
    s = dbfft.Solver((16,) * 3, c["phase"], dbfft.iso_phases(c["E"], c["nu"]), c["eps_bar"][None], tol=1e-8)
    s.solve_increment(0)
    rep, dt = _timed(lambda: s.solve_increment(0))
    return {"case": "c1 16^3 sphere FP64", "wall_ms": dt * 1e3, "report": rep,
            "sigma_bar": s.homogenized_stress()[0].tolist()}


NH_MASK_BITS = [(0, 1), (0, 2), (1, 2), (1, 1), (2, 2)]


def case_c3(precision, n=128, n_inc=20):
    """128^3 Neo-Hookean fibres (mu 1 / 20), F11 -> 1.2 in 20 increments, other macro stresses zero."""
    from paper_1905_12725_gb300 import dbfft, synth
    c = synth.config3(n=n)
    mask = np.zeros((3, 3), bool)
    for i, j in NH_MASK_BITS:
        mask[i, j] = True
    tgt = np.eye(3)
    tgt[0, 0] = 1.2
    tgt[mask] = 0.0
    s = dbfft.Solver((n,) * 3, c["phase"], dbfft.neo_hooke_phases(c["mu"], c["lam"]), tgt[None],
                     kinematics=dbfft.DBFFT_FINITE, precision=precision, stress_mask=mask.reshape(-1),
                     n_increments=n_inc, newton_tol=1e-8, load_tol=1e-10, eta_inner=1e-4, max_newton=30,
                     max_iter=5000)
    s.autotune(TUNE_CACHE)
    incs = []
    t_all = 0.0
    cg_all = 0
    for k in range(n_inc):
        rep, dt = _timed(lambda: s.solve_increment(k))
        t_all += dt
        cg_all += rep["cg_iters"]
        P = s.homogenized_stress()[0]
        incs.append({"inc": k, "newton": rep["newton_iters"], "cg": rep["cg_iters"], "eps_eq": rep["eps_eq"],
                     "load_res": rep["load_res"], "P11": P[0, 0], "ms": dt * 1e3})
    return {"case": f"c3 {n}^3 Neo-Hooke fibres vf {float(c['phase'].mean()):.3f}, n_fibres {c['n_fibres']}",
            "precision": "mixed" if precision else "fp64", "wall_s": t_all, "cg_iters": cg_all,
            "voxel_cg_iters_per_s": n ** 3 * cg_all / t_all, "increments": incs,
            "P_bar_final": s.homogenized_stress()[0].tolist(), "phase_sha256": synth.sha256(c["phase"])}


def case_porous(precision, n=64, n_inc=5, stretch=2.0):
    """Porous St. Venant-Kirchhoff matrix (E 70, nu 0.3; 5 pores of total porosity 0.2 with 1/100 of the
    stiffness), stretched to F11 = 2 in 5 increments with every other component of F held at its
    undeformed value; Newton to 1e-6."""
    from paper_1905_12725_gb300 import dbfft, synth
    c = synth.porous_svk(n=n)
    tgt = np.eye(3)
    tgt[0, 0] = stretch
    s = dbfft.Solver((n,) * 3, c["phase"], dbfft.svk_phases(c["mu"], c["lam"]), tgt[None],
                     kinematics=dbfft.DBFFT_FINITE, precision=precision, n_increments=n_inc, newton_tol=1e-6,
                     load_tol=1e-10, eta_inner=1e-3 if precision else 1e-4, max_newton=40, max_iter=20000)
    s.autotune(TUNE_CACHE)
    incs = []
    t_all = 0.0
    cg_all = 0
    for k in range(n_inc):
        rep, dt = _timed(lambda: s.solve_increment(k))
        t_all += dt
        cg_all += rep["cg_iters"]
        P = s.homogenized_stress()[0]
        incs.append({"inc": k, "newton": rep["newton_iters"], "cg": rep["cg_iters"], "eps_eq": rep["eps_eq"],
                     "P11": P[0, 0], "ms": dt * 1e3})
    Pfin = s.homogenized_stress()[0].tolist()
    s.close()
    # the other refresh policies of the preconditioner's reference stiffness (same solution,
    # other CG iteration counts; the paper's example keeps the initial tangent)
    policies = {}
    for name, pol in (("initial", dbfft.DBFFT_PRECOND_INITIAL), ("per_newton", dbfft.DBFFT_PRECOND_PER_NEWTON)):
        sp = dbfft.Solver((n,) * 3, c["phase"], dbfft.svk_phases(c["mu"], c["lam"]), tgt[None],
                          kinematics=dbfft.DBFFT_FINITE, precision=precision, n_increments=n_inc, newton_tol=1e-6,
                          load_tol=1e-10, eta_inner=1e-3 if precision else 1e-4, max_newton=40, max_iter=20000)
        sp.set_precond_refresh(pol)
        sp.autotune(TUNE_CACHE)
        cgs, wall = [], 0.0
        for k in range(n_inc):
            rep, dt = _timed(lambda: sp.solve_increment(k))
            cgs.append(rep["cg_iters"])
            wall += dt
        policies[name] = {"cg_per_increment": cgs, "wall_s": wall, "P11_final": sp.homogenized_stress()[0][0, 0]}
        sp.close()
    return {"case": f"porous SVK {n}^3, 5 pores, porosity {float(c['phase'].mean()):.4f}, F11 -> {stretch}",
            "precision": "mixed" if precision else "fp64", "wall_s": t_all, "cg_iters": cg_all,
            "voxel_cg_iters_per_s": n ** 3 * cg_all / t_all, "increments": incs,
            "P_bar_final": Pfin, "precond_refresh_per_increment_default": True,
            "other_precond_policies": policies, "phase_sha256": synth.sha256(c["phase"])}


def case_inclusion(n=63, tol=1e-8):
    """The paper's first and second benchmarks on its own odd grid: one centred spherical inclusion
    (vf 0.2) in a 63^3 box, matrix E 70 / nu 0.3, inclusion k E; uniaxial strain 0.1 % with every
    component prescribed, and uniaxial stress with every component stress-controlled; PCG to a
    relative residual of 1e-8 for contrasts k = 1e-5 .. 1e5, FP64 and mixed."""
    from paper_1905_12725_gb300 import dbfft, synth
    out = {"case": f"inclusion {n}^3 vf 0.2, contrast sweep", "tol": tol, "rows": []}
    for k in [1e-5, 1e-4, 1e-3, 1e-2, 1e-1, 1e1, 1e2, 1e3, 1e4, 1e5]:
        c = synth.inclusion(n, contrast=k)
        for control in ("strain", "stress"):
            if control == "strain":
                mask, target = None, np.diag([1e-3, 0.0, 0.0])
            else:
                mask, target = np.ones(9, bool), np.diag([70.0 * 1e-3, 0.0, 0.0])
            row = {"contrast": k, "control": control}
            for prec, name in ((dbfft.DBFFT_FP64, "fp64"), (dbfft.DBFFT_MIXED, "mixed")):
                s = dbfft.Solver((n,) * 3, c["phase"], dbfft.iso_phases(c["E"], c["nu"]), target[None],
                                 stress_mask=mask, tol=tol, precision=prec, eta_inner=1e-3, max_iter=20000)
                s.solve_increment(0)  # warm-up (graph capture, first-touch)
                rep, dt = _timed(lambda: s.solve_increment(0))
                sig = s.homogenized_stress()[0]
                row[name] = {"cg": rep["cg_iters"], "ms": dt * 1e3, "true_rel_res": rep["true_rel_res"],
                             "eps_eq": rep["eps_eq"], "sig_bar_11": sig[0, 0],
                             "eps_bar_11": float(s.get_solution()[1][0][0]) if control == "stress" else 1e-3}
                s.close()
            out["rows"].append(row)
    return out


def case_c4(precision, n=256, n_inc=40, only=None):
    """256^3 Voronoi polycrystal (500 grains), power-law CP, eps_xx to 2% at 1e-3/s in 40 increments."""
    from paper_1905_12725_gb300 import dbfft, synth
    t0 = time.perf_counter()
    c = synth.config4(n=n)
    t_gen = time.perf_counter() - t0
    mask = np.ones((3, 3), bool)
    mask[0, 0] = False
    tgt = np.zeros((3, 3))
    tgt[0, 0] = 0.02
    s = dbfft.Solver((n,) * 3, c["phase"], dbfft.cp_phases(c["quat"]), tgt[None], precision=precision,
                     stress_mask=mask.reshape(-1), n_increments=n_inc, total_time=20.0, newton_tol=1e-8,
                     load_tol=1e-10, eta_inner=1e-4, max_newton=40, max_iter=5000)
    s.autotune(TUNE_CACHE)
    incs = []
    t_all = 0.0
    cg_all = 0
    n_run = n_inc if only is None else only
    prof = None
    for k in range(n_run):
        if k == n_run - 1:
            s.profile(True)  # the last increment launch by launch, with per-kernel CUDA events
        rep, dt = _timed(lambda: s.solve_increment(k))
        if k == n_run - 1:
            prof = s.profile_read()
            s.profile(False)
        t_all += dt
        cg_all += rep["cg_iters"]
        sg = s.homogenized_stress()[0]
        incs.append({"inc": k, "newton": rep["newton_iters"], "cg": rep["cg_iters"], "eps_eq": rep["eps_eq"],
                     "sigma_xx": sg[0, 0], "ms": dt * 1e3})
    return {"case": f"c4 {n}^3 polycrystal 500 grains", "precision": "mixed" if precision else "fp64",
            "generate_s": t_gen, "wall_s": t_all, "cg_iters": cg_all,
            "last_increment_kernels (launch by launch)": {
                k: {"launches": v["launches"], "ms": v["ms"]} for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])},
            "voxel_cg_iters_per_s": n ** 3 * cg_all / t_all, "increments": incs,
            "phase_sha256": synth.sha256(c["phase"])}


def case_sens():
    """dC_eff,1111 / dE(x) of the headline composite for the per-voxel Young's modulus E(x)
    (dbfft_tangent_sensitivity): the six unit-strain solves (dbfft_homogenized_tangent) and
    the contraction of their strain fields, timed apart, with the Euler identity
    sum_x E(x) dC/dE(x) = C_eff,1111 (C_eff is homogeneous of degree one in the moduli)."""
    import torch
    from paper_1905_12725_gb300 import dbfft
    c = workload_inputs()
    shape = (N_GRID,) * 3
    G = np.zeros((1, 6, 6))
    G[0, 0, 0] = 1.0
    E_vox = np.asarray(c["E"], dtype=np.float64)[c["phase"]]
    out = {"case": "stiffness sensitivity, 64^3 composite, J = C_1111"}
    for prec, name in [(dbfft.DBFFT_MIXED, "mixed"), (dbfft.DBFFT_FP64, "fp64")]:
        s = dbfft.Solver(shape, c["phase"], dbfft.iso_phases(c["E"], c["nu"]), np.zeros((6, 3, 3)), batch=6,
                         E_scale=np.ones(shape), precision=prec, tol=TOL, eta_inner=ETA_INNER, max_iter=20000,
                         max_newton=100)
        s.autotune(TUNE_CACHE)
        s.homogenized_tangent()
        s.tangent_sensitivity(G)
        t_solve, t_sens = [], []
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s.homogenized_tangent()
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            dJ, C_eff, rep = s.tangent_sensitivity(G)  # reuses the six solves just made
            torch.cuda.synchronize()
            t_solve.append(t1 - t0)
            t_sens.append(time.perf_counter() - t1)
        tot = float(np.sum(dJ.cpu().numpy()[0] * E_vox))
        out[name] = {"solves_ms": 1e3 * float(np.median(t_solve)), "assembly_ms": 1e3 * float(np.median(t_sens)),
                     "C1111": float(C_eff[0, 0, 0]), "euler_rel": abs(tot - C_eff[0, 0, 0]) / abs(C_eff[0, 0, 0])}
        s.close()
    return out


def case_cpadj(n=64, n_inc=10):
    """Sensitivity of sigma_xx after a plastic loading path to every voxel's stiffness:
    the 500-grain Voronoi polycrystal of the 256^3 case generated on n^3, power-law CP,
    eps_xx at 1e-3/s (0.5 s increments) under uniaxial mixed control, FP64 Newton with
    checkpoints, then the reverse sweep (one FP64 adjoint solve per increment)."""
    from paper_1905_12725_gb300 import dbfft, synth
    c = synth.config4(n=n)
    mask = np.ones((3, 3), bool)
    mask[0, 0] = False
    tgt = np.zeros((3, 3))
    tgt[0, 0] = 1e-3 * 0.5 * n_inc
    s = dbfft.Solver((n,) * 3, c["phase"], dbfft.cp_phases(c["quat"]), tgt[None], precision=dbfft.DBFFT_FP64,
                     stress_mask=mask.reshape(-1), n_increments=n_inc, total_time=0.5 * n_inc, newton_tol=1e-10,
                     load_tol=1e-11, eta_inner=1e-6, max_newton=40, max_iter=5000, tol=1e-10)
    s.autotune(TUNE_CACHE)
    s.set_checkpointing(True)
    t_fwd, cg_fwd = 0.0, 0
    for k in range(n_inc):
        rep, dt = _timed(lambda: s.solve_increment(k))
        t_fwd += dt
        cg_fwd += rep["cg_iters"]
    sig = s.homogenized_stress()[0]
    g = np.zeros((1, 3, 3))
    g[0, 0, 0] = 1.0
    (dJ, rep), t_adj = _timed(lambda: s.cp_adjoint(g))
    d = dJ.cpu().numpy()[0]
    s.close()
    return {"case": f"cp adjoint {n}^3 polycrystal, {n_inc} increments", "precision": "fp64",
            "forward_s": t_fwd, "forward_cg_iters": cg_fwd, "adjoint_s": t_adj, "adjoint_cg_iters": rep["cg_iters"],
            "sigma_xx": sig[0, 0], "dJds_sum": float(d.sum()), "dJds_min": float(d.min()), "dJds_max": float(d.max()),
            "checkpoint_bytes": n ** 3 * 6 * 8 * n_inc}


def case_fcp(precision, n=64, n_grains=200, n_inc=40, rate=1e-3, dt=0.5):
    """n^3 Voronoi polycrystal, finite-strain CP (F = Fe Fp): F11 to 1.02 at 1e-3/s in
    40 increments, the lower off-diagonal F components held at zero and the other P
    components free (mixed control). With 1e-3 of stretch per increment the plain
    Newton iteration stalls on this grid; 5e-4, the step of the small-strain
    polycrystal case, converges."""
    from paper_1905_12725_gb300 import dbfft, synth
    t0 = time.perf_counter()
    rng = synth.Xoshiro256ss(1905)
    phase, _ = synth.periodic_voronoi(n, n_grains, rng)
    quats = synth.uniform_quaternions(n_grains, rng)
    t_gen = time.perf_counter() - t0
    mask = np.zeros((3, 3), bool)
    mask[0, 1] = mask[0, 2] = mask[1, 2] = mask[1, 1] = mask[2, 2] = True
    tgt = np.eye(3)
    tgt[0, 0] = 1.0 + rate * dt * n_inc
    tgt[mask] = 0.0
    s = dbfft.Solver((n,) * 3, phase, dbfft.cp_phases(quats, finite=True), tgt[None], kinematics=dbfft.DBFFT_FINITE,
                     precision=precision, stress_mask=mask.reshape(-1), n_increments=n_inc, total_time=n_inc * dt,
                     newton_tol=1e-8, load_tol=1e-10, eta_inner=1e-4, max_newton=40, max_iter=5000)
    s.autotune(TUNE_CACHE)
    incs = []
    t_all = 0.0
    cg_all = 0
    for k in range(n_inc):
        rep, el = _timed(lambda: s.solve_increment(k))
        t_all += el
        cg_all += rep["cg_iters"]
        P = s.homogenized_stress()[0]
        incs.append({"inc": k, "newton": rep["newton_iters"], "cg": rep["cg_iters"], "eps_eq": rep["eps_eq"],
                     "P_xx": P[0, 0], "ms": el * 1e3})
    s.close()
    return {"case": f"finite-strain CP {n}^3 polycrystal {n_grains} grains", "precision": "mixed" if precision else "fp64",
            "generate_s": t_gen, "wall_s": t_all, "cg_iters": cg_all,
            "voxel_cg_iters_per_s": n ** 3 * cg_all / t_all, "increments": incs,
            "phase_sha256": synth.sha256(phase)}


def case_c5(n=64, n_rve=32, n_fd=20):
    """32 RVEs of 64^3: d sigma_xx / dE(x) by the adjoint, checked by central differences on 20 voxels each."""
    from paper_1905_12725_gb300 import dbfft, synth
    c = synth.config5(n=n, n_rve=n_rve)
    E = c["E"][np.arange(n_rve)[:, None, None, None], c["phase"]]  # per-voxel Young's modulus
    ph = np.zeros_like(c["phase"])
    eps = np.zeros((n_rve, 3, 3))
    eps[:, 0, 0] = 1e-3
    g = np.zeros((n_rve, 9))
    g[:, 0] = 1.0
    out = {"case": f"c5 {n_rve} x {n}^3 adjoint", "vf_target": c["vf_target"].tolist()}
    for prec, name in [(dbfft.DBFFT_MIXED, "mixed"), (dbfft.DBFFT_FP64, "fp64")]:
        s = dbfft.Solver((n,) * 3, ph, dbfft.iso_phases([1.0], [0.3]), eps, E_scale=E, precision=prec,
                         tol=1e-10 if prec == dbfft.DBFFT_FP64 else 1e-7, eta_inner=1e-3)
        s.autotune(TUNE_CACHE)
        s.adjoint(g)
        (dJ, rep), dt = _timed(lambda: s.adjoint(g))
        out[name] = {"wall_ms": dt * 1e3, "report": rep, "dJdE": dJ}
        s.close()
    dJ64 = out["fp64"]["dJdE"].cpu().numpy()
    dJmx = out["mixed"]["dJdE"].cpu().numpy()
    out["mixed_vs_fp64_rel"] = float(np.abs(dJmx - dJ64).max() / np.abs(dJ64).max())
    # central differences, delta = 1e-3 E(x), batched over the RVEs (one voxel per RVE per solve pair)
    rng = synth.Xoshiro256ss(synth.SEED_BASE + 55)
    vox = np.array([synth.random_voxels(n ** 3, n_fd, rng) for _ in range(n_rve)])
    errs = []
    t0 = time.perf_counter()
    for k in range(n_fd):
        Js = []
        for sgn in (+1.0, -1.0):
            Ep = E.copy().reshape(n_rve, -1)
            d = 1e-3 * Ep[np.arange(n_rve), vox[:, k]]
            Ep[np.arange(n_rve), vox[:, k]] += sgn * d
            sp = dbfft.Solver((n,) * 3, ph, dbfft.iso_phases([1.0], [0.3]), eps, E_scale=Ep.reshape(E.shape),
                              precision=dbfft.DBFFT_MIXED, tol=1e-12, eta_inner=1e-3)
            sp.autotune(TUNE_CACHE)
            sp.solve_increment(0)
            Js.append(sp.homogenized_stress()[:, 0, 0])
            sp.close()
        d = 1e-3 * E.reshape(n_rve, -1)[np.arange(n_rve), vox[:, k]]
        fd = (Js[0] - Js[1]) / (2 * d)
        adj = dJ64.reshape(n_rve, -1)[np.arange(n_rve), vox[:, k]]
        errs.append(np.abs(fd - adj) / np.abs(adj))
    errs = np.array(errs)
    out["fd_check"] = {"voxels_per_rve": n_fd, "max_rel_err": float(errs.max()), "median_rel_err": float(np.median(errs)),
                       "pass_1e-4": bool(errs.max() < 1e-4), "wall_s": time.perf_counter() - t0}
    for name in ["mixed", "fp64"]:
        out[name].pop("dJdE")
    return out


def reduce_over_ranks(dist, t_local, work_local, device):
    """Whole-job timing across replicas: the slowest rank's time and the work
    of all ranks (max and sum over the process group); identity on one rank."""
    if dist is None:
        return float(t_local), float(work_local)
    import torch
    t = torch.tensor([float(t_local)], dtype=torch.float64, device=device)
    w = torch.tensor([float(work_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t.item()), float(w.item())


def our_arm(args, rank, world, local_rank):
    import torch
    from paper_1905_12725_gb300 import dbfft

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
    dev = torch.device("cuda", local_rank)
    peak, peak_kind = _peaks()
    c = workload_inputs()
    V = N_GRID ** 3
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def l2_flush():
        flush.fill_(1.0)

    # --- mixed batched: the timed step
    s = make_solver(c, dbfft.DBFFT_MIXED, 6)
    for _ in range(args.warmup):
        s.homogenized_tangent()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local_rank)
    clocks.start()
    launches0 = s.launch_count()
    stream = torch.cuda.current_stream(dev)
    ms_steps, iters_steps, res_steps = [], [], []
    for _ in range(args.steps):
        l2_flush()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        Ceff, rep = s.homogenized_tangent()
        e1.record(stream)
        torch.cuda.synchronize()
        ms_steps.append(e0.elapsed_time(e1))
        iters_steps.append(rep["cg_iters"])
        res_steps.append(rep["true_rel_res"])
    gpu_launches = s.launch_count() - launches0
    clk = clocks.stop()
    # per-kernel device times: the same steps again with every launch bracketed by
    # CUDA events on the context stream (launched one by one instead of as a graph)
    s.profile(True)
    for _ in range(args.steps):
        l2_flush()
        s.homogenized_tangent()
    prof = s.profile_read()
    s.profile(False)
    t_total, work = reduce_over_ranks(dist, sum(ms_steps) * 1e-3, V * sum(iters_steps), dev)
    value = work / t_total
    Ceff = Ceff[0]

    # --- dominant kernel roofline (live, CUDA events on the context stream)
    dom = max(prof.items(), key=lambda kv: kv[1]["ms"])
    dname, de = dom
    per_launch_ms = de["ms"] / de["launches"]
    per_launch_bytes = de["bytes"] / de["launches"]
    achieved = per_launch_bytes / (per_launch_ms * 1e-3) / 1e9
    tr = NCU_TRAFFIC.get(dname)
    traffic = (tr["bytes"] if tr and dname in KERNEL_SOURCES and tr.get("src") == _sources_hash(KERNEL_SOURCES[dname])
               else None)
    kernels = {k: {"launches": v["launches"], "ms": v["ms"],
                   "GBps": (v["bytes"] / (v["ms"] * 1e-3) / 1e9) if v["ms"] > 0 and v["bytes"] > 0 else None}
               for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])}
    fp64 = fp64_roofline(dbfft, prof, peak, N_GRID, 6)
    l2 = l2_roofline(dbfft, prof)

    # --- FP64 plain: six right-hand sides one after another, FP64 PCG to 1e-6
    plain = [make_solver(c, dbfft.DBFFT_FP64, 1, targets=unit_mandel(m)[None]) for m in range(6)]
    for p in plain:
        p.solve_increment(0)
    l2_flush()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    it64 = 0
    res64 = 0.0
    for p in plain:
        r = p.solve_increment(0)
        it64 += r["cg_iters"]
        res64 = max(res64, r["true_rel_res"])
    e1.record(stream)
    torch.cuda.synchronize()
    t64 = e0.elapsed_time(e1)
    C64 = np.zeros((6, 6))
    for m, p in enumerate(plain):
        sg = p.homogenized_stress()[0]
        C64[:, m] = [sg[0, 0], sg[1, 1], sg[2, 2], math.sqrt(2) * sg[1, 2], math.sqrt(2) * sg[0, 2],
                     math.sqrt(2) * sg[0, 1]]
        p.close()

    # --- end to end through the C ABI with host buffers (create from host map, solve, read C_eff)
    e2e_ms = []
    e2e_iters = []
    for k in range(args.warmup + args.steps):
        l2_flush()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        se = make_solver(c, dbfft.DBFFT_MIXED, 6)
        Ce, r = se.homogenized_tangent()
        se.close()
        torch.cuda.synchronize()
        if k >= args.warmup:
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
            e2e_iters.append(r["cg_iters"])
    e2e_t, e2e_work = reduce_over_ranks(dist, sum(e2e_ms) * 1e-3, V * sum(e2e_iters), dev)

    op256 = None
    if rank == 0 and not args.skip_256:
        op256 = operator_256(torch, dbfft, peak)
        try:
            op256["cufft_comparison"] = cufft_operator_256(torch)
        except Exception as exc:  # comparison only; never fails the benchmark
            op256["cufft_comparison"] = {"error": str(exc)[:200]}

    cpu = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        v, it, dt, nc = oracle_sample(c, iters=args.ref_iters)
        cpu = {"value": v, "unit": UNIT, "cores": nc, "kind": "oracle",
               "sample": f"{it} PCG iterations of the FP64 numpy oracle on right-hand side 1 of the same "
                         f"workload ({dt:.1f} s; cores = CPU time / wall time of the sample; host has "
                         f"{os.cpu_count()} cores)"}
        try:
            v6, it6, dt6, n6 = oracle_sample_all_cores()
            cpu["all_cores"] = {"value": v6, "unit": UNIT, "cores": n6,
                                "sample": f"the six right-hand sides as {n6} spawned processes side by side, "
                                          f"{it6} PCG iterations in all, the longest taking {dt6:.1f} s"}
        except Exception as exc:  # a reported baseline only
            cpu["all_cores"] = {"error": str(exc)[:200]}

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": float(np.mean(ms_steps)), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 inner / f64 outer",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N_GRID, "batch": 6, "tol": TOL, "eta_inner": ETA_INNER,
                   "seed": 190512725 + 2, "l2": "flushed (512 MiB write) before every step",
                   "parallelism": f"replicas x{world}"},
        "time_to_1e-6_ms": {"mixed_batched": float(np.mean(ms_steps)), "fp64_plain_sequential": t64,
                            "speedup": t64 / float(np.mean(ms_steps))},
        "cg_iters_per_step": {"mixed_batched": int(np.mean(iters_steps)), "fp64_plain": it64},
        "true_rel_res": {"mixed_batched": max(res_steps), "fp64_plain": res64},
        "fp64_plain_value": V * it64 / (t64 * 1e-3),
        "C_eff_rel_diff_mixed_vs_fp64": float(np.abs(Ceff - C64).max() / np.abs(C64).max()),
        "roofline": {"bound": "hbm", "kernel": dname, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_source": peak_kind,
                     "algorithmic_bytes_per_launch": per_launch_bytes, "ms_per_launch": per_launch_ms},
        "kernels": kernels,
        "fp64": fp64,
        "l2": l2,
        "tuning": s.tuning,
        "gpu_launches": int(gpu_launches),
        "e2e": {"value": e2e_work / e2e_t, "unit": UNIT, "h2d_bytes_per_step": int(c["phase"].nbytes + 6 * 9 * 8),
                "d2h_bytes_per_step": 36 * 8, "ms_per_step": float(np.mean(e2e_ms)),
                "path": "dbfft_create from host phase map + dbfft_homogenized_tangent + dbfft_destroy"},
        "clocks": clk,
        "operator_256": op256,
        "cpu_baseline": cpu,
        "src": _sources_hash(),
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-iters", type=int, default=40)
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-256", action="store_true")
    ap.add_argument("--case", default="",
                    choices=["", "op256", "c2", "c1", "c3", "c3fp64", "c4", "c4fp64", "c5", "porous",
                             "porousfp64", "porous63", "porous63fp64", "inclusion", "fcp", "fcpfp64", "fcp63",
                             "fcp63fp64", "cpadj", "sens"],
                    help="run one sub-measurement only: op256 = 256^3 FP32 CG pass chain, c2 = one mixed "
                         "batched 64^3 solve (profiler captures); c1, c3[fp64], c4[fp64], c5 = the other "
                         "configurations at full size; porous[fp64] = the porous St. Venant-Kirchhoff "
                         "stretch (64^3; porous63[fp64] on the paper's 63^3 grid); inclusion = the 63^3 inclusion contrast sweep; "
                         "fcp[fp64] = the 64^3 finite-strain crystal-plasticity stretch (fcp63[fp64] on 63^3)")
    args = ap.parse_args()
    if args.case:
        import torch
        from paper_1905_12725_gb300 import dbfft
        torch.cuda.set_device(0)
        if args.case == "op256":
            r = operator_256(torch, dbfft, _peaks()[0], iters=args.steps)
            r["cufft_comparison"] = cufft_operator_256(torch)
            print(json.dumps(r), flush=True)
        elif args.case in ("porous63", "porous63fp64"):
            prec = dbfft.DBFFT_FP64 if args.case.endswith("fp64") else dbfft.DBFFT_MIXED
            print(json.dumps(case_porous(prec, n=63), default=float), flush=True)
        elif args.case == "sens":
            print(json.dumps(case_sens(), default=float), flush=True)
        elif args.case == "cpadj":
            print(json.dumps(case_cpadj(), default=float), flush=True)
        elif args.case == "inclusion":
            print(json.dumps(case_inclusion(), default=float), flush=True)
        elif args.case in ("fcp", "fcpfp64", "fcp63", "fcp63fp64"):
            prec = dbfft.DBFFT_FP64 if args.case.endswith("fp64") else dbfft.DBFFT_MIXED
            print(json.dumps(case_fcp(prec, n=63 if "63" in args.case else 64), default=float), flush=True)
        elif args.case in ("c1", "c3", "c3fp64", "c4", "c4fp64", "c5", "porous", "porousfp64"):
            prec = dbfft.DBFFT_FP64 if args.case.endswith("fp64") else dbfft.DBFFT_MIXED
            res = {"c1": lambda: case_c1(), "c3": lambda: case_c3(prec), "c3fp64": lambda: case_c3(prec),
                   "c4": lambda: case_c4(prec), "c4fp64": lambda: case_c4(prec, only=args.steps),
                   "c5": lambda: case_c5(), "porous": lambda: case_porous(prec),
                   "porousfp64": lambda: case_porous(prec)}[args.case]()
            print(json.dumps(res, default=float), flush=True)
        else:
            s = make_solver(workload_inputs(), dbfft.DBFFT_MIXED, 6)
            for _ in range(max(args.steps, 1)):
                _, rep = s.homogenized_tangent()
            print(json.dumps(rep), flush=True)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    our_arm(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
