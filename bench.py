"""Benchmark of the fused DUGKS step on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload nonuniform|burgers] [--substeps S]

A bench step is one output interval of S DUGKS time steps (default 50) on
the workload's full grid; every DUGKS time step is one launch of the fused
step kernel, i.e. one pass of the whole method over the grid.

* value      : cell-velocity updates per second with the state resident in
               HBM (K intervals timed with CUDA events on the solver's stream).
* e2e        : the same metric through the C ABI with host buffers: each
               interval uploads phi0 from pinned host memory
               (dugks_init_phi_host), steps S times, and reads phi back to
               host memory (dugks_get_phi_host).
* roofline   : the fused step kernel against the measured HBM copy
               bandwidth (and the nominal 7.9 TB/s); algorithmic bytes = read
               ftilde once + write once = 2 * 9 * sizeof(T) per cell; the
               launch time is the looped interval time over its launches.
* cpu_baseline (rank 0, N = 1): the FP64 CPU oracle on a bounded sample, on
               all host cores and on one, with the CPU model.
* batched    : the 256-instance workload, 1000 steps as 20 graph replays,
               against the single-instance step's rate, bit-identity checked,
               16 sampled instances against stored FP64 oracle runs.
* parity     : the single-instance workloads run for their configured steps
               against stored FP64 oracle runs (tests/golden); the adjoint
               gradient against stored FP64 central differences.

--impl reference times that oracle as it stands on the host cores.
Multi-GPU runs are independent replicas (one per rank, weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DUGKS cell-velocity updates/sec and % HBM roofline (FP32, 1 GB300); adjoint/step ratio"
UNIT = "cell-velocity updates/s"
Q = 9
PROFILE = os.path.join(ROOT, "profiles", "fused_step_nonuniform_2048.txt")
# the files that define the FP32 step kernel (step_vp) and what it includes
KERNEL_SOURCES = [os.path.join(ROOT, "paper_1906_11036_gb300", "csrc", f)
                  for f in ("dugks_step_vp.cuh", "dugks_kernels.cuh", "dugks_device.cuh")]
NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, nominal


def workload(name: str):
    from paper_1906_11036_gb300 import inputs as I

    if name == "nonuniform":
        return I.nonuniform()
    if name == "burgers":
        return I.burgers()
    raise SystemExit(f"unknown workload {name}")


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def profile_traffic(workload_name: str):
    """dram bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source and this workload; else None."""
    if not os.path.exists(PROFILE):
        return None
    kv = {}
    for line in open(PROFILE):
        if ":" in line and not line.startswith(" "):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("kernel_source_hash") != kernel_source_hash() or kv.get("workload") != workload_name:
        return None
    try:
        return float(kv["dram_bytes_per_launch_full_grid"])
    except (KeyError, ValueError):
        return None


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return float(json.load(open(path))["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.p is not None:
            time.sleep(0.2)
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
                self.out, _ = self.p.communicate()

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for _, _, flags in rows for n, f in zip(names, flags) if f.lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def cpu_model() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform

    return platform.processor() or platform.machine()


def oracle_rate(p, phi0, seconds: float, threads: int, max_rows: int | None = None):
    """Time the FP64 oracle as it stands on a horizontal band of the workload
    (all columns, the first `rows` rows, walls as in the workload) for about
    `seconds`; returns (CVU/s, sample description, threads)."""
    from oracle import Oracle

    rows = p.ny if max_rows is None else min(p.ny, max_rows)
    band = p.with_(yf=p.yf[: rows + 1])
    o = Oracle(band)
    f = o.init(np.ascontiguousarray(phi0[:rows]))
    t0 = time.perf_counter()
    f = o.run(f, 1, threads)  # calibration step (also first-touch of the workspace)
    one = time.perf_counter() - t0
    n = max(1, int(seconds / max(one, 1e-6)))
    t0 = time.perf_counter()
    o.run(f, n, threads)
    el = time.perf_counter() - t0
    cvu = band.nx * rows * Q * n
    return cvu / el, f"{n} oracle steps on a {band.nx}x{rows} band of the {p.nx}x{p.ny} workload", threads


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle

    oracle.build()
    p, phi0 = workload(args.workload)
    threads = os.cpu_count() or 1
    # each bench step: one oracle time step on a band sized so that warmup+steps take ~2 minutes
    from oracle import Oracle

    rows = min(p.ny, 64)
    band = p.with_(yf=p.yf[: rows + 1])
    o = Oracle(band)
    f = o.init(np.ascontiguousarray(phi0[:rows]))
    t0 = time.perf_counter()
    f = o.run(f, 1, threads)
    per_row = (time.perf_counter() - t0) / rows
    total = args.steps + args.warmup
    rows = int(max(4, min(p.ny, 120.0 / max(total, 1) / max(per_row, 1e-9))))
    band = p.with_(yf=p.yf[: rows + 1])
    o = Oracle(band)
    f = o.init(np.ascontiguousarray(phi0[:rows]))
    f = o.run(f, args.warmup, threads)
    t0 = time.perf_counter()
    o.run(f, args.steps, threads)
    el = time.perf_counter() - t0
    value = band.nx * rows * Q * args.steps / el
    sample = f"each step: one FP64 oracle time step on a {band.nx}x{rows} band of the {p.nx}x{p.ny} {args.workload} workload"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(args, p),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def adjoint_ratio(args):
    """Adjoint/step ratio on the adjoint workload (512^2 periodic Burgers-type
    NCDE, FP32, 400 steps checkpointed every 20): time of one adjoint step
    against one forward step, and of the whole checkpointed gradient against
    the forward run."""
    import torch

    from paper_1906_11036_gb300 import inputs as I
    from paper_1906_11036_gb300.dugks import Solver

    p, phi0 = I.burgers(512, steps=400)
    s = Solver(p, precision=32)
    phi0_t = torch.tensor(phi0, dtype=torch.float32, device="cuda")
    s.init_phi(phi0_t)
    s.step(20)
    f = s.save_state().clone()
    mu = torch.randn_like(f)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    torch.cuda.synchronize()
    ev[0].record(s.stream)
    s.step(200)
    ev[1].record(s.stream)
    # one adjoint step as a reverse sweep runs it: the kernel alone (the sweep sums the FP64
    # partials once at its end)
    for _ in range(3):
        lam, _ = s.adjoint_step(f, mu, with_alpha=False)
    torch.cuda.synchronize()
    ev[2].record(s.stream)
    for _ in range(50):
        lam, _ = s.adjoint_step(f, mu, with_alpha=False)
    ev[3].record(s.stream)
    ev[3].synchronize()
    t_fwd = ev[0].elapsed_time(ev[1]) / 200
    t_adj = ev[2].elapsed_time(ev[3]) / 50
    # the whole gradient of the misfit J = 1/2 sum |V| (phi^N - target)^2 w.r.t. phi0, alpha and u
    _, _, target, area = I.adjoint_workload(512, p.steps)
    s.init_phi(phi0_t)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.step(p.steps)
    phiN = s.get_phi().double().cpu().numpy()
    torch.cuda.synchronize()
    t_run = time.perf_counter() - t0
    gN = torch.tensor(area * (phiN - target), dtype=torch.float32, device="cuda")
    t0 = time.perf_counter()
    s.gradient(phi0_t, p.steps, gN, checkpoint_every=20, with_u=True)  # allocates the context's workspace
    t_grad_first = time.perf_counter() - t0
    t0 = time.perf_counter()
    g0, dalpha, du = s.gradient(phi0_t, p.steps, gN, checkpoint_every=20, with_u=True)
    t_grad = time.perf_counter() - t0
    g0 = g0.double().cpu().numpy()
    s.close()
    out = {"workload": "burgers_512x512, 400 FP32 steps, checkpoint every 20; gradient w.r.t. phi0, alpha, u",
           "forward_ms_per_step": t_fwd, "adjoint_ms_per_step": t_adj, "adjoint_step_ratio": t_adj / t_fwd,
           "forward_run_s": t_run, "gradient_s": t_grad, "gradient_to_forward_ratio": t_grad / t_run,
           "gradient_first_call_s": t_grad_first,
           "gradient_timing": "second call on the context (its workspace allocated by the first)"}
    path = os.path.join(GOLDEN, "oracle_adjoint_fd.npz")
    if os.path.exists(path):
        # against FP64 central differences of the oracle (eps = 1e-4) stored by make_adjoint_fd.py
        z = np.load(path)
        dirs = I.unit_directions(phi0.shape, int(z["ndir"]), seed=5)
        gd = np.array([float((g0 * d).sum()) for d in dirs])
        out["vs_fp64_fd"] = {
            "directions": int(z["ndir"]), "eps": float(z["eps"]),
            "max_rel_err_dirs": float(np.max(np.abs(gd - z["fd_dirs"]) / np.abs(z["fd_dirs"]))),
            "rel_err_dalpha": abs(dalpha - float(z["fd_alpha"])) / abs(float(z["fd_alpha"])),
            "max_rel_err_du": float(np.max(np.abs(np.asarray(du) - z["fd_u"]) / np.abs(z["fd_u"]))),
            "rel_l2_vs_oracle_adjoint_sampled": _rel_l2(g0.reshape(-1)[z["grad_sample_idx"]], z["grad_sample"])}
    # the same step on 2048^2 (state, mu and lambda larger than L2): roofline of the adjoint step,
    # algorithmic bytes = read ftilde^n and mu, write lambda = 3 x 36 B per cell in FP32
    p, phi0 = I.burgers(2048, steps=20)
    s = Solver(p, precision=32)
    s.init_phi(torch.tensor(phi0, dtype=torch.float32, device="cuda"))
    s.step(5)
    f = s.save_state().clone()
    mu = torch.randn_like(f)
    for _ in range(3):
        lam, _ = s.adjoint_step(f, mu, with_alpha=False)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record(s.stream)
    s.step(20)
    ev[1].record(s.stream)
    ev[2].record(s.stream)
    for _ in range(20):
        lam, _ = s.adjoint_step(f, mu, with_alpha=False)
    ev[3].record(s.stream)
    ev[3].synchronize()
    t_fwd2, t_adj2 = ev[0].elapsed_time(ev[1]) / 20, ev[2].elapsed_time(ev[3]) / 20
    s.close()
    peak, peak_kind = measured_peak()
    alg = 2048 * 2048 * 3 * Q * 4
    out["large"] = {"workload": "burgers_2048x2048, FP32", "forward_ms_per_step": t_fwd2,
                    "adjoint_ms_per_step": t_adj2, "adjoint_step_ratio": t_adj2 / t_fwd2,
                    "algorithmic_bytes_per_adjoint_step": alg,
                    "roofline_frac": alg / (t_adj2 * 1e-3) / 1e9 / peak, "peak_kind": peak_kind}
    # the same on the non-uniform mesh with Dirichlet walls (mirrored ghosts folded back)
    p, phi0 = I.nonuniform(2048, steps=20)
    s = Solver(p, precision=32)
    s.init_phi(torch.tensor(phi0, dtype=torch.float32, device="cuda"))
    s.step(5)
    f = s.save_state().clone()
    mu = torch.randn_like(f)
    for _ in range(3):
        lam, _ = s.adjoint_step(f, mu, with_alpha=False)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record(s.stream)
    s.step(20)
    ev[1].record(s.stream)
    ev[2].record(s.stream)
    for _ in range(20):
        lam, _ = s.adjoint_step(f, mu, with_alpha=False)
    ev[3].record(s.stream)
    ev[3].synchronize()
    t_fwd3, t_adj3 = ev[0].elapsed_time(ev[1]) / 20, ev[2].elapsed_time(ev[3]) / 20
    s.close()
    out["large_walls"] = {"workload": "nonuniform_2048x2048 (tanh mesh, Dirichlet walls), FP32",
                          "forward_ms_per_step": t_fwd3, "adjoint_ms_per_step": t_adj3,
                          "adjoint_step_ratio": t_adj3 / t_fwd3, "algorithmic_bytes_per_adjoint_step": alg,
                          "roofline_frac": alg / (t_adj3 * 1e-3) / 1e9 / peak, "peak_kind": peak_kind}
    return out


def batched_run(single_value: float | None, steps: int = 1000, check: int = 8):
    """The batched workload (256 periodic Burgers-type instances, sides drawn from
    64..512, seed 7): the configured 1000 steps of every instance as 20 replays of
    the 50-step CUDA graph of the batched persistent step (one launch per step of
    all instances), timed with CUDA events on the batch's stream.  Reported against
    the single-instance step's cell-velocity rate of the main run (same GPU, same
    accuracy: every instance equals the single-instance step bit for bit, checked
    here on `check` instances stepped on their own for the same steps)."""
    import torch

    from paper_1906_11036_gb300 import inputs as I
    from paper_1906_11036_gb300.dugks import BatchSolver, Solver

    items = I.batched()
    cells = sum(p.nx * p.ny for p, _ in items)
    stream = torch.cuda.Stream()
    b = BatchSolver([p for p, _ in items], stream=stream)
    for i, (_, phi0) in enumerate(items):
        b.init_phi(i, phi0)
    rows, _ = b.autotune(20)  # trials run on snapshots and restore the states
    b.sync()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    b.step(steps)
    ev1.record(stream)
    ev1.synchronize()
    b.sync()
    t_batch = ev0.elapsed_time(ev1) / 1e3
    # bit-identity against the single-instance step on a spread of instance sizes
    order = sorted(range(len(items)), key=lambda i: items[i][0].nx)
    picks = [order[int(k * (len(order) - 1) / max(1, check - 1))] for k in range(check)]
    same = 0
    for i in picks:
        p, phi0 = items[i]
        fb = b.save_state(i)
        s = Solver(p, precision=32)
        s.init_phi(torch.tensor(phi0, device="cuda"))
        s.step(steps)
        fs = s.save_state()
        torch.cuda.synchronize()
        same += int(torch.equal(fb, fs))
        s.close()
    # the 16 sampled instances against the FP64 oracle's runs stored by make_batched_oracle.py
    vs_oracle = None
    path = os.path.join(GOLDEN, "oracle_batched16.npz")
    if os.path.exists(path) and steps == 1000:
        z = np.load(path)
        errs = []
        for i in (int(v) for v in z["ids"]):
            phi_t = b.get_phi(i)
            b.sync()  # the copy runs on the batch's stream
            phi = phi_t.double().cpu().numpy().reshape(-1)
            errs.append(_rel_l2(phi[z[f"sample_{i}"]], z[f"phi_{i}"]))
        vs_oracle = {"instances": len(errs), "max_rel_l2": max(errs), "median_rel_l2": float(np.median(errs))}
    b.close()
    v_b = cells * Q * steps / t_batch
    peak, peak_kind = measured_peak()
    out = {"workload": "256 periodic Burgers-type instances, sides 64-512 (seed 7), FP32",
           "steps": steps, "graph_replays": steps // 50, "cells": cells, "value": v_b, "unit": UNIT,
           "ms_per_step": 1e3 * t_batch / steps, "tile_rows": rows,
           "roofline_frac": v_b * 8 / 1e9 / peak, "peak_kind": peak_kind,
           "bit_identical_to_single_instance": f"{same}/{len(picks)} instances checked"}
    if vs_oracle is not None:
        out["vs_fp64_oracle"] = vs_oracle
    if single_value:
        out["single_instance_value"] = single_value
        out["batched_to_single_instance"] = v_b / single_value
    return out


def sources_vs_plain(steps: int = 100):
    """The source-term workload (Example 4.5 scaled to 2048^2: B = phi^2 u,
    D = diag(phi^2, phi^3), six-term source F, FP32): per-step device time of the
    step with F and R against the plain step on the same problem, and the
    fraction of the measured HBM bandwidth its algorithmic bytes reach
    (72 B/cell for ftilde + 4 B per source field + 8 B for the phi history)."""
    import torch

    from paper_1906_11036_gb300 import inputs as I
    from paper_1906_11036_gb300.dugks import Solver

    p, phi0 = I.nonlinear_source(2048)
    cells = p.nx * p.ny
    out = {"workload": f"{p.name} (Example 4.5 at 2048^2), FP32, {len(p.source)} source terms", "steps": steps}
    for name, q in (("source", p), ("plain", p.with_(source=()))):
        s = Solver(q, precision=32)
        s.init_phi(torch.tensor(phi0, device="cuda"))
        s.step(5)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        s.step(steps)
        e1.record(s.stream)
        e1.synchronize()
        out[f"{name}_us_per_step"] = e0.elapsed_time(e1) / steps * 1e3
        s.close()
    peak, peak_kind = measured_peak()
    alg = cells * (2 * Q * 4 + 4 * len(p.source) + 8)
    out["source_value"] = cells * Q / (out["source_us_per_step"] * 1e-6)
    out["unit"] = UNIT
    out["algorithmic_bytes_per_step"] = alg
    out["roofline_frac"] = alg / (out["source_us_per_step"] * 1e-6) / 1e9 / peak
    out["peak_kind"] = peak_kind
    out["source_to_plain_ratio"] = out["source_us_per_step"] / out["plain_us_per_step"]
    return out


def three_d(n: int = 256, steps: int = 20):
    """The 3-D step (periodic Burgers-type workload on n^3 cells, FP32) with the
    D3Q19 and D3Q15 velocity sets: device time per step (CUDA events on the
    solver's stream, state of 2 x Q x 4 B per cell, larger than L2 at 256^3),
    cell-velocity updates/s, and the fraction of the measured HBM bandwidth that
    the algorithmic bytes (read and write ftilde once: 8 Q B per cell) reach."""
    import torch

    from paper_1906_11036_gb300 import inputs as I
    from paper_1906_11036_gb300.dugks import Solver3

    peak, peak_kind = measured_peak()
    out = {}
    for q in (19, 15):
        p, phi0 = I.burgers3d(n, lattice=q)
        s = Solver3(p, precision=32)
        s.init_phi(phi0)
        s.step(3)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        s.step(steps)
        e1.record(s.stream)
        e1.synchronize()
        t = e0.elapsed_time(e1) / steps * 1e-3
        _, mass = s.get_phi(mass=True)
        info = s.info()
        s.close()
        cells = p.cells
        alg = cells * q * 8
        out[f"d3q{q}"] = {"workload": p.name, "steps": steps, "us_per_step": t * 1e6, "value": cells * q / t,
                          "unit": UNIT, "algorithmic_bytes_per_step": alg, "achieved_gbs": alg / t / 1e9,
                          "roofline_frac": alg / t / 1e9 / peak, "peak_kind": peak_kind, "mass": mass,
                          "grid": list(info["grid"]), "zseg": info["zseg"], "block": info["block_threads"]}
    return out


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden")


def _rel_l2(a, b) -> float:
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def parity_vs_stored_oracle():
    """Error of the GPU path against the FP64 oracle on the full-size, full-length
    single-instance workloads: each is run from its initial field for its
    configured steps and phi is compared, at the stored sample cells, with the
    oracle's run stored under tests/golden (written by make_oracle_runs.py there,
    which calls only the oracle): relative L2 over the samples and the relative
    change of the mass against the oracle's."""
    import torch

    from paper_1906_11036_gb300 import inputs as I
    from paper_1906_11036_gb300.dugks import Solver

    out = {}
    for name, precs in (("gaussian_hill", (64, 32)), ("burgers", (32,)), ("nonuniform", (32,))):
        path = os.path.join(GOLDEN, f"oracle_{name}.npz")
        if not os.path.exists(path):
            out[name] = "no stored oracle run"
            continue
        g = np.load(path)
        p, phi0 = I.PRESETS[name]()
        for prec in precs:
            s = Solver(p, precision=prec)
            s.init_phi(torch.tensor(phi0, dtype=s.dtype, device="cuda"))
            s.step(p.steps)
            phi, m = s.get_phi(mass=True)
            s.close()
            full = phi.double().cpu().numpy()
            got = full.reshape(-1)[g["sample"]]
            out[f"{name}_fp{prec}"] = {"workload": f"{p.name}, {p.steps} steps, FP{prec}",
                                       "rel_l2_vs_oracle": _rel_l2(got, g["phi"]), "samples": int(got.size),
                                       "mass_rel_vs_oracle": abs(m - float(g["mass"])) / abs(float(g["mass"]))}
            if name == "gaussian_hill":
                # GRE (Eq. 4.1.1) against the closed form of Eq. 4.4.3; the oracle's stored run (every
                # cell) beside it: the kinetic scheme's own distance from the PDE at this c
                xc, yc = p.centres()
                ex = I.gaussian_hill_exact(xc, yc, p.steps * p.dt, p.u, p.alpha)
                ref = np.zeros(p.nx * p.ny)
                ref[g["sample"]] = g["phi"]
                out[f"{name}_fp{prec}"]["gre_vs_closed_form"] = I.gre(full, ex)
                out[f"{name}_fp{prec}"]["oracle_gre_vs_closed_form"] = I.gre(ref.reshape(p.ny, p.nx), ex)
    return out


def configs_table(args):
    """One row per workload configuration (Gaussian hill 64^2 FP64, Burgers 1024^2
    FP32, non-uniform 2048^2 FP32, 256 batched instances, the 512^2 adjoint):
    the GPU rate and its error against the stored FP64 oracle runs, next to the
    oracle as it stands timed on one host thread and on all of them (bounded
    samples of the same workload).  `bench.py --configs` prints it as one JSON line."""
    import torch

    import oracle
    from oracle import Oracle
    from paper_1906_11036_gb300 import inputs as I
    from paper_1906_11036_gb300.dugks import Solver

    oracle.build()
    nproc = os.cpu_count() or 1
    sec = args.cpu_seconds
    peak, peak_kind = measured_peak()
    par = parity_vs_stored_oracle()
    rows = []

    def gpu_rate(p, phi0, prec, steps):
        s = Solver(p, precision=prec)
        s.init_phi(torch.tensor(phi0, dtype=s.dtype, device="cuda"))
        s.step(min(steps, 20))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        s.step(steps)
        e1.record(s.stream)
        e1.synchronize()
        s.close()
        t = e0.elapsed_time(e1) / 1e3
        return p.nx * p.ny * Q * steps / t, t / steps

    for key, name, prec, big in (("1", "gaussian_hill", 64, False), ("2", "burgers", 32, True),
                                 ("3", "nonuniform", 32, True)):
        p, phi0 = I.PRESETS[name]()
        v, t_step = gpu_rate(p, phi0, prec, p.steps)
        r1, smp1, _ = oracle_rate(p, phi0, sec, 1, max_rows=64 if big else None)
        rn, smpn, thr = oracle_rate(p, phi0, sec, nproc, max_rows=256 if big else None)
        esz = 8 if prec == 64 else 4
        pr = par.get(f"{name}_fp{prec}", {})
        rows.append({"config": key, "workload": f"{p.name}, {p.steps} steps, FP{prec}", "gpu_cvu_s": v,
                     "us_per_step": t_step * 1e6, "hbm_frac": 2 * Q * esz * p.nx * p.ny / t_step / 1e9 / peak,
                     "l2_resident": 2 * Q * esz * p.nx * p.ny < 126e6,
                     "rel_l2_vs_oracle": pr.get("rel_l2_vs_oracle"), "mass_rel_vs_oracle": pr.get("mass_rel_vs_oracle"),
                     "oracle_cvu_s_1_thread": r1, "oracle_cvu_s_nproc": rn, "oracle_threads": thr,
                     "oracle_sample_1_thread": smp1, "oracle_sample_nproc": smpn})
    # 4: the batched workload; the oracle on one 512^2 instance of it
    b = batched_run(None)
    items = I.batched()
    p4, phi4 = next(it for it in items if it[0].nx == 512)
    r1, smp1, _ = oracle_rate(p4, phi4, sec, 1, max_rows=64)
    rn, smpn, thr = oracle_rate(p4, phi4, sec, nproc)
    rows.append({"config": "4", "workload": b["workload"] + ", 1000 steps", "gpu_cvu_s": b["value"],
                 "us_per_step": b["ms_per_step"] * 1e3, "hbm_frac": b["roofline_frac"],
                 "rel_l2_vs_oracle": (b.get("vs_fp64_oracle") or {}).get("max_rel_l2"),
                 "oracle_cvu_s_1_thread": r1, "oracle_cvu_s_nproc": rn, "oracle_threads": thr,
                 "oracle_sample_1_thread": "one 512^2 instance: " + smp1, "oracle_sample_nproc": "one 512^2 instance: " + smpn})
    # 5: the adjoint workload; the oracle's adjoint step (single-threaded as it stands) on the full grid
    a = adjoint_ratio(args)
    p5, phi5 = I.burgers(512, steps=400)
    o = Oracle(p5)
    f = o.init(phi5)
    mu = np.random.default_rng(3).standard_normal(f.shape)
    t0 = time.perf_counter()
    n5 = 0
    while time.perf_counter() - t0 < sec:
        o.adjoint_step_full(f, mu)
        n5 += 1
    r_adj = p5.nx * p5.ny * Q * n5 / (time.perf_counter() - t0)
    fd = a.get("vs_fp64_fd", {})
    rows.append({"config": "5", "workload": a["workload"], "gpu_adjoint_cvu_s": p5.nx * p5.ny * Q / (a["adjoint_ms_per_step"] * 1e-3),
                 "adjoint_step_ratio": a["adjoint_step_ratio"], "gradient_to_forward_ratio": a["gradient_to_forward_ratio"],
                 "hbm_frac_2048": a["large"]["roofline_frac"], "adjoint_step_ratio_2048": a["large"]["adjoint_step_ratio"],
                 "max_rel_err_vs_fd_32_dirs": fd.get("max_rel_err_dirs"), "rel_err_dalpha_vs_fd": fd.get("rel_err_dalpha"),
                 "max_rel_err_du_vs_fd": fd.get("max_rel_err_du"),
                 "rel_l2_vs_oracle_adjoint_sampled": fd.get("rel_l2_vs_oracle_adjoint_sampled"),
                 "oracle_adjoint_cvu_s_1_thread": r_adj,
                 "oracle_sample": f"{n5} FP64 oracle adjoint steps on the full 512^2 grid (one thread: it is not threaded)"})
    return {"configs": rows, "peak_gbs": peak, "peak_kind": peak_kind, "cpu_model": cpu_model(), "nproc": nproc}


def max_over_ranks(times, world: int, device="cpu"):
    """Element-wise maximum of per-rank timings over all ranks (the slowest
    replica sets the job's time); identity for a single process."""
    if world <= 1:
        return list(times)
    import torch
    import torch.distributed as dist

    t = torch.tensor(list(times), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def replica_value(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput of independent replicas: all ranks' units over the
    slowest rank's time."""
    return world * units_per_rank / seconds


def config_dict(args, p):
    return {"workload": f"{args.workload}_{p.nx}x{p.ny}", "nx": p.nx, "ny": p.ny, "velocity_set": "D2Q9",
            "mesh": "tanh-stretched k=2, Dirichlet walls" if args.workload == "nonuniform" else "uniform periodic",
            "dt": p.dt, "c": p.c, "step": f"{args.substeps} DUGKS time steps (one output interval)",
            "l2": "state larger than L2 (two 9-plane FP32 buffers)", "parallelism": "replicas"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="nonuniform", choices=["nonuniform", "burgers"])
    ap.add_argument("--substeps", type=int, default=50)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-sources", action="store_true")
    ap.add_argument("--no-3d", action="store_true")
    ap.add_argument("--no-parity", action="store_true")
    ap.add_argument("--configs", action="store_true", help="print the per-configuration table instead")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.configs:
        import __graft_entry__

        __graft_entry__.build()
        print(json.dumps(configs_table(args)), flush=True)
        return 0

    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__

    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
        __graft_entry__.build()
    from paper_1906_11036_gb300.dugks import Solver

    p, phi0 = workload(args.workload)
    S = args.substeps
    cells = p.nx * p.ny
    cvu_per_step = cells * Q * S
    stream = torch.cuda.Stream()
    solver = Solver(p, precision=32, stream=stream)
    info = solver.info()
    with torch.cuda.stream(stream):
        solver.init_phi(torch.tensor(phi0, device="cuda"))
        for _ in range(args.warmup):
            solver.step(S)
    stream.synchronize()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # ---- device-resident throughput --------------------------------------------
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    with Clocks(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            solver.step(S)
        ev1.record(stream)
        ev1.synchronize()
    barrier()
    t_dev = ev0.elapsed_time(ev1) / 1e3
    solver.sync()
    # ---- per-launch kernel duration (events around each launch) ------------------
    nl = min(200, max(20, args.steps * S // 4))
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nl)]
    for a, b in evs:
        a.record(stream)
        solver.step(1)
        b.record(stream)
    stream.synchronize()
    launch_s = statistics.median(a.elapsed_time(b) for a, b in evs) / 1e3
    # ---- end to end through host buffers ------------------------------------------
    phi_host = torch.tensor(phi0, dtype=torch.float64).pin_memory()
    out_host = torch.empty((p.ny, p.nx), dtype=torch.float64).pin_memory()
    phi_np, out_np = phi_host.numpy(), out_host.numpy()
    e2e_steps = max(1, min(args.steps, 10))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        solver.init_phi(phi_np)
        solver.step(S)
        solver.get_phi_host(out_np)
    barrier()
    t_e2e = time.perf_counter() - t0
    solver.close()
    adjoint = adjoint_ratio(args) if (world == 1 and not args.no_adjoint) else None
    batched = None  # after the main line's value is known
    sources = sources_vs_plain() if (world == 1 and not args.no_sources) else None
    d3 = three_d() if (world == 1 and not args.no_3d) else None
    parity = parity_vs_stored_oracle() if (world == 1 and not args.no_parity) else None

    t_dev, t_e2e = max_over_ranks([t_dev, t_e2e], world, device="cuda")
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0

    value = replica_value(cvu_per_step * args.steps, world, t_dev)
    e2e = replica_value(cvu_per_step * e2e_steps, world, t_e2e)
    peak, peak_kind = measured_peak()
    alg_bytes = 2 * Q * 4 * cells
    # one launch per DUGKS time step: its duration from the looped timing (CUDA events around
    # the K timed intervals of S launches each); the median of per-launch event pairs, which
    # carry their own overhead, is reported beside it
    launch_loop_s = t_dev / (args.steps * S)
    achieved = alg_bytes / launch_loop_s / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config_dict(args, p),
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": 8 * cells, "d2h_bytes_per_step": 8 * cells + 8},
        "gpu_launches": args.steps * S,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": profile_traffic(args.workload), "peak_kind": peak_kind,
                     "frac_of_nominal": achieved / NOMINAL_HBM_GBS, "nominal_peak": NOMINAL_HBM_GBS,
                     "kernel": "step_vp", "kernel_ms": launch_loop_s * 1e3,
                     "kernel_ms_from": "looped timing: interval time / launches",
                     "kernel_ms_events": launch_s * 1e3,
                     "algorithmic_bytes_per_launch": alg_bytes},
        "clocks": clk.summary(),
        "launch": {"block": info["block_threads"], "grid": info["grid_blocks"]},
    }
    if adjoint is not None:
        line["adjoint"] = adjoint
    if world == 1 and not args.no_batched:
        line["batched"] = batched_run(value)
    if sources is not None:
        line["sources"] = sources
    if d3 is not None:
        line["three_d"] = d3
    if parity is not None:
        line["parity"] = parity
    if world == 1 and not args.no_cpu_baseline:
        import oracle

        oracle.build()
        rate, sample, thr = oracle_rate(p, phi0, args.cpu_seconds, os.cpu_count() or 1, max_rows=256)
        rate1, sample1, _ = oracle_rate(p, phi0, args.cpu_seconds, 1, max_rows=64)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": thr, "kind": "oracle", "sample": sample,
                                "cpu_model": cpu_model(), "value_1_thread": rate1, "sample_1_thread": sample1}
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
