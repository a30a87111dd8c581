"""Benchmark of the MRT lattice Boltzmann hot path on one GB300 (or N replicas).

Workload: the synthetic four-directional braided cell 128x128x256 (interior
braiding angle 30 deg, yarn fraction 0.45, seed 42, yarn tensor
k_axial = 6.0 / k_trans = 0.8 rotated per family, matrix 0.2), temperature
difference along z, periodic laterals, FP32 distributions.

One bench step = one pass of the hot path over the cell: ITERS fused
collide-stream iterations in check intervals of K = 100 (each interval ends
with an FP64 plane-flux / residual check and the k_eff finalize), launched as
one CUDA graph with a device-side while condition.  FP32 plain iterations run
two per launch (temporal blocking, identical results; --no-fuse: one).
Metric: GLUPS (giga lattice updates per second).  Each step is timed by its own
CUDA events; between steps a 256 MB write (outside the timed region) evicts
the 129 MB L2.

`value`: device time (CUDA events on the solver's stream) with the state
resident.  `e2e`: the same metric through the public C ABI with pinned host
buffers: upload the phase map and tensors, solve ITERS iterations from the
linear start, download the temperature field, every step.

Outside the timed region (--legs, default all): per-config lines (the 32^3
layered cell, the bench cell's six solves, the 192-solve batched sweep, the
256x256x512 precision cell with its oracle error), time to k_eff within 1e-4
of the FP64 oracle's converged value, the combined batched + warm-started +
BF16 form against plain FP32, the learned warm start on 128x128x256 cells
and the tensor-core convolution's throughput.

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NX, NY, NZ = 128, 128, 256
G_DEG, PHI, SEED, NMAX = 30.0, 0.45, 42, 128
K = 100
ITERS = 1000
# the state is four stored fields per node (th and jhat / 2; the seven
# populations follow from them exactly): 4 values read + 4 written + 1 B
# phase id per update (a seven-population state would move 57 B in FP32)
BYTES_PER_LUP = {"f32": 33, "bf16": 17, "f16": 17}
# DRAM bytes (read + write) per launch of the dominant kernel, from one ncu
# capture of this workload (dram__bytes_read.sum + dram__bytes_write.sum),
# keyed by (kernel, storage) and stamped with the SHA-256 prefix of the
# kernel source it was taken on; a stamp that no longer matches the source
# reports null instead of a stale figure.
TRAFFIC = {("fused2", "f32"): (92.21e6, "6059c6de3e622a6f")}   # mean of 3 launches
KERNEL_SOURCE = os.path.join(ROOT, "paper_1503_08718_gb300", "csrc", "lbm_kernels.cuh")
STORAGE = {"f32": 0, "bf16": 1, "f16": 2}
WORKLOAD = (f"braid {NX}x{NY}x{NZ} g=30deg phi=0.45 seed=42, dT along z, periodic laterals, "
            f"FP32 D3Q7 MRT")


def kernel_source_sha16():
    import hashlib
    with open(KERNEL_SOURCE, "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


def traffic_for(key):
    """DRAM bytes per launch for (kernel, storage) if captured on the current
    kernel source, else None."""
    ent = TRAFFIC.get(key)
    if ent is None or ent[1] != kernel_source_sha16():
        return None
    return ent[0]


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def bf16_sustained_tflops():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["bf16_tflops_sustained"]), "measured"
    except Exception:
        return 1700.0, "fallback"


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (getattr(self, "out", "") or "").splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def make_cell(lbm, I, device):
    S = lbm.Solver(NX, NY, NZ, device=device)
    anchors = I.braid_anchors(NX, NY, SEED, n_max=NMAX)
    used, frac = S.set_geometry_braid(math.radians(G_DEG), anchors, PHI)
    lam = I.braid_tensors(G_DEG)
    S.set_tensors(lam)
    return S, lam, used, frac


def kernel_launch_us(S, opts, stream, steps_per_launch, n=200, warm=20, axis=2, lateral=0):
    """Average device time of one launch of the plain step kernel (two steps
    per launch when fused): n launches issued by lbm_advance are captured
    into a CUDA graph on the solver's stream (so stream-launch gaps are not
    counted) and one replay is timed with CUDA events on that stream.  n is
    even, so a replay ends in the buffer it started from.  Falls back to
    timing the launches directly if capture is unavailable."""
    import torch
    S.start(axis, lateral, opts)
    S.advance(warm * steps_per_launch)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    try:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            S.advance(n * steps_per_launch)
        with torch.cuda.stream(stream):
            g.replay()
            e0.record(stream)
            g.replay()
            e1.record(stream)
        torch.cuda.synchronize()
        mode = "graph"
    except Exception:
        torch.cuda.synchronize()
        e0.record(stream)
        S.advance(n * steps_per_launch)
        e1.record(stream)
        torch.cuda.synchronize()
        mode = "stream"
    return e0.elapsed_time(e1) * 1000.0 / n, n, mode


REFERENCE_FILE = os.path.join(ROOT, "tests", "golden", "keff_reference.json")


def reference_keff(label, phase):
    """Converged FP64 oracle value k* of a cell, written by
    tests/golden/make_keff_reference.py, if that file holds the cell and its
    phase map hash matches the one voxelised here."""
    import hashlib
    try:
        with open(REFERENCE_FILE) as fh:
            ent = json.load(fh)["cells"][label]
    except (OSError, KeyError, ValueError):
        return None
    if not ent.get("converged") or ent["phase_sha256"] != hashlib.sha256(phase.tobytes()).hexdigest():
        return None
    return ent


def first_within(h, k_ref, rel):
    """Index of the first check after which every later k_eff stays within
    rel of k_ref, or None."""
    err = np.abs(h[:, 1] / k_ref - 1.0)
    bad = np.nonzero(err > rel)[0]
    first = 0 if bad.size == 0 else int(bad[-1]) + 1
    return first if first < len(h) else None


def time_to_keff(lbm, S, stream, iters=60_000, rel=1e-4):
    """Time to k_eff within `rel` of the converged FP64 oracle value k* on the
    bench cell from the linear start, for FP32 and 16-bit storage: the first
    check after which every later k_eff stays within rel of k*, times the
    measured device time per iteration (every check interval is the same
    work).  Without a stored k* for this cell, the FP32 value after 250 000
    iterations stands in (k_ref_source says which)."""
    ref = reference_keff("braid128x128x256_z", S.geometry())
    out = {"rel": rel}
    if ref is not None:
        k_ref = ref["k_star"]
        out.update(k_ref=k_ref, k_ref_source="FP64 oracle, converged to R_Q <= %g in %d iterations"
                   % (ref["rq_tol"], ref["iters"]))
    else:
        o = S.opts(tol=0.0, max_iters=250_000, check_every=K)
        o.stream = int(stream.cuda_stream)
        S.start(2, 0, o)
        k_ref = S.run().k_eff
        out.update(k_ref=k_ref, k_ref_source="GPU FP32 after 250000 iterations (no oracle k* stored)")
    for name in ("f32", "bf16", "f16"):
        o = S.opts(tol=0.0, max_iters=iters, check_every=K, storage=STORAGE[name])
        o.stream = int(stream.cuda_stream)
        S.start(2, 0, o)
        info = S.run()
        h = S.history()
        first = first_within(h, k_ref, rel)
        ms_per_iter = info.elapsed_ms / info.iters
        n_it = int(h[first, 0]) if first is not None else None
        out[name] = {"iters": n_it, "ms": n_it * ms_per_iter if n_it else None,
                     "ms_per_iter": ms_per_iter, "iters_run": int(info.iters),
                     "k_final": float(h[-1, 1]),
                     "k_final_rel_vs_ref": float(h[-1, 1] / k_ref - 1.0)}
    if out["f32"]["ms"] and out["bf16"]["ms"]:
        out["speedup_bf16_vs_f32"] = out["f32"]["ms"] / out["bf16"]["ms"]
    return out


def solve_glups(S, axis, lateral, opts, n_vox):
    """GLUPS of one solve (lbm_start + lbm_run), device time from the
    solver's CUDA events."""
    S.start(axis, lateral, opts)
    info = S.run()
    return n_vox * info.iters / info.elapsed_ms / 1e6, info


def config1_layered(lbm, I, stream):
    """The 32^3 layered cell (z layers of 8 voxels, matrix 0.2, yarn 6.0 /
    0.8 at 30 deg from z in the xz-plane), z axis, periodic laterals, to
    R_T <= 1e-8: iterations, device time, GLUPS and k_eff against the exact
    94/245.  The state (1.9 MB) is L2-resident: GLUPS, no HBM roofline."""
    yarn = I.transversely_isotropic(6.0, 0.8, I.axis_in_xz_from_z(30.0))
    lam = np.stack([I.isotropic(0.2), yarn])
    with lbm.Solver(32, 32, 32) as S:
        S.set_geometry(I.layered_phase(32, 32, 32), 2)
        S.set_tensors(lam)
        o = S.opts(tol=1e-8)
        o.stream = int(stream.cuda_stream)
        S.start(2, 0, o)                      # warm-up (graph build)
        S.run()
        g, info = solve_glups(S, 2, 0, o, 32 ** 3)
        exact = 94.0 / 245.0
        return {"workload": "layered 32^3, z axis, periodic, FP32, to R_T <= 1e-8",
                "glups": g, "iters": int(info.iters), "ms": info.elapsed_ms,
                "k_eff": info.k_eff, "k_rel_vs_exact": info.k_eff / exact - 1.0,
                "plan": S.launch_plan(), "l2_resident": True}


def config2_all_solves(lbm, S, stream, n_vox, iters=1000):
    """The bench cell along x, y and z with periodic and adiabatic laterals
    (FP32, fused pairs where the rows allow them): GLUPS of each solve."""
    rows = []
    for axis in (0, 1, 2):
        for lateral in (0, 1):
            o = S.opts(tol=0.0, max_iters=iters)
            o.stream = int(stream.cuda_stream)
            solve_glups(S, axis, lateral, o, n_vox)       # warm-up (graph build)
            g, info = solve_glups(S, axis, lateral, o, n_vox)
            rows.append({"axis": "xyz"[axis], "lateral": ("periodic", "adiabatic")[lateral],
                         "glups": g, "iters": int(info.iters), "k_eff": info.k_eff,
                         "steps_per_launch": S.launch_plan()["steps_per_launch"]})
    return rows


def config4_precision(lbm, I, stream, peak, with_oracle, iters=2000, n_check=20):
    """The 256x256x512 braid (35 deg, yarn fraction 0.50, seed 7), every axis,
    periodic laterals, FP32 / BF16 / FP16 storage: GLUPS over `iters`
    iterations, the dominant kernel's average launch time and roofline
    fraction (33 or 17 B per update), and the k_eff error against the FP64
    oracle after n_check iterations from the linear start."""
    n = (256, 256, 512)
    n_vox = n[0] * n[1] * n[2]
    anchors = I.braid_anchors(n[0], n[1], 7, n_max=1024)
    lam = I.braid_tensors(35.0)
    out = {"workload": "braid 256x256x512 g=35deg phi=0.50 seed=7, periodic laterals",
           "per_axis": []}
    ph_ref = None
    if with_oracle:
        from oracle import oracle as O
        ph_ref, _, _ = O.braid_phase(*n, math.radians(35.0), anchors, 0.50)
    with lbm.Solver(*n) as S:
        S.set_geometry_braid(math.radians(35.0), anchors, 0.50)
        S.set_tensors(lam)
        if ph_ref is not None:
            out["voxeliser_bit_exact"] = bool(np.array_equal(S.geometry(), ph_ref))
        for axis in (0, 1, 2):
            k_oracle = None
            if ph_ref is not None:
                L = O.Lattice(ph_ref, lam, O.lattice_scale(lam), axis, 0)
                L.init_linear()
                L.step(n_check)
                k_oracle = L.k_eff()[0]
                del L
            for name in ("f32", "bf16", "f16"):
                o = S.opts(tol=0.0, max_iters=iters, storage=STORAGE[name])
                o.stream = int(stream.cuda_stream)
                solve_glups(S, axis, 0, o, n_vox)             # warm-up
                g, info = solve_glups(S, axis, 0, o, n_vox)
                spl = S.launch_plan()["steps_per_launch"]
                us, _, _ = kernel_launch_us(S, o, stream, spl, n=100, warm=10, axis=axis)
                moved = BYTES_PER_LUP[name] * n_vox
                row = {"axis": "xyz"[axis], "storage": name, "glups": g,
                       "steps_per_launch": spl, "dominant_kernel_us": us,
                       "roofline_frac": moved * spl / (us * 1e-6) / 1e9 / peak,
                       "frac_moved": moved / (us * 1e-6) / 1e9 / peak}
                if k_oracle is not None:
                    o2 = S.opts(storage=STORAGE[name])
                    o2.stream = int(stream.cuda_stream)
                    S.start(axis, 0, o2)
                    S.advance(n_check - 1)
                    k = S.check().k_eff
                    row["k_rel_vs_oracle_at_%d" % n_check] = k / k_oracle - 1.0
                out["per_axis"].append(row)
    return out


def sweep(lbm, I, n_cells=64, iters=500):
    """The braid sweep of uneven cells (N_xy 64..160, N_z up to 320, yarn
    fraction 0.30-0.60, braiding angle 20-45 deg), every cell along x, y and
    z: one batched graph launch against the same solves run one by one."""
    cells = I.braid_sweep_cells(n_cells)
    phases = []
    for c in cells:
        with lbm.Solver(c["nx"], c["ny"], c["nz"]) as V:
            V.set_geometry_braid(math.radians(c["g_deg"]),
                                 I.braid_anchors(c["nx"], c["ny"], c["seed"], n_max=256), c["phi"])
            phases.append((V.geometry(), I.braid_tensors(c["g_deg"])))
    opts = lbm.Solver.opts(tol=0.0, max_iters=iters)
    B = lbm.Batch()
    for ph, lam in phases:
        for axis in (0, 1, 2):
            B.add(ph, lam, axis)
    info = B.solve(0, opts)
    batched = info.total_updates / info.elapsed_ms / 1e6
    B.close()
    plans = []
    seq_ms, seq_upd = 0.0, 0
    for ph, lam in phases:
        nz, ny, nx = ph.shape
        with lbm.Solver(nx, ny, nz) as S1:
            S1.set_geometry(ph, 5)
            S1.set_tensors(lam)
            for axis in (0, 1, 2):
                S1.solve(axis, 0, opts)                   # warm-up (graph build)
                r = S1.solve(axis, 0, opts)
                seq_ms += r.elapsed_ms
                seq_upd += r.iters * ph.size
                plans.append(S1.launch_plan()["steps_per_launch"])
    return {"solves": 3 * len(cells), "cells": len(cells),
            "voxels_per_axis": int(sum(p.size for p, _ in phases)), "iters_per_solve": iters,
            "batched_glups": batched, "sequential_glups": seq_upd / seq_ms / 1e6,
            "batched_ms": info.elapsed_ms, "sequential_ms": seq_ms,
            "block_threads": info.block_threads,
            "batched_steps_per_launch": info.steps_per_launch,
            "sequential_fused_solves": int(sum(p == 2 for p in plans)),
            "batched_over_sequential": batched / (seq_upd / seq_ms / 1e6), "unit": "GLUPS"}


WARM_WEIGHTS = os.path.join(ROOT, "paper_1503_08718_gb300", "weights", "warmnet_braid64.npz")
COMBINED_SEEDS = tuple(range(7000, 7016))


def combined_form(lbm, I, stream, rel=1e-4, budget=40_000):
    """The combined form against the plain FP32 solver on 16 held-out 64^3
    braided cells (seeds 7000..7015 of the warm-start distribution, z axis,
    periodic laterals), each with its converged FP64 oracle value k*.

    plain: the single-solve FP32 path (two steps per launch), one cell after
    another from the linear start; per cell the device time until k_eff stays
    within rel of k* (history x device time per iteration), summed.
    Batched variants: one graph launch for all 16 cells; their time is the
    device time (per-check timestamps) at which the last solve entered the
    band for good, plus, for warm starts, the network's batched inference
    (one forward pass over the 16 cells, CUDA events).  Reported: batched
    FP32 linear start, batched FP32 warm start, and the combined form,
    batched + warm start + BF16 storage."""
    import torch
    from paper_1503_08718_gb300 import warmstart as W

    if not os.path.exists(WARM_WEIGHTS):
        return {"unavailable": "no trained warm-start weights"}
    cells = []
    for s in COMBINED_SEEDS:
        g, phi = I.warm_cell_params(s)
        with lbm.Solver(64, 64, 64) as V:
            V.set_geometry_braid(math.radians(g), I.braid_anchors(64, 64, s, n_max=256), phi)
            ph = V.geometry()
        ref = reference_keff(f"warm64_{s}", ph)
        if ref is not None:
            cells.append((ph, I.braid_tensors(g), ref["k_star"]))
    if len(cells) < 4:
        return {"unavailable": "fewer than 4 of the cells have a converged oracle k* stored"}
    out = {"workload": f"{len(cells)} held-out braids 64^3 (seeds 7000-7015 with a stored k*), "
                       "z axis, periodic",
           "rel": rel, "budget_iters": budget}
    # plain FP32, one cell at a time
    tot, iters = 0.0, []
    for ph, lam, kst in cells:
        with lbm.Solver(64, 64, 64) as S:
            S.set_geometry(ph, 5)
            S.set_tensors(lam)
            o = S.opts(tol=0.0, max_iters=budget)
            o.stream = int(stream.cuda_stream)
            S.start(2, 0, o)
            S.run()                                   # warm-up (graph build)
            S.start(2, 0, o)
            info = S.run()
            h = S.history()
            f = first_within(h, kst, rel)
            if f is None:
                return {"unavailable": "plain FP32 did not reach the band within the budget"}
            tot += info.elapsed_ms / info.iters * h[f, 0]
            iters.append(int(h[f, 0]))
    out["plain_f32_sequential"] = {"ms": tot, "iters_mean": float(np.mean(iters))}
    # network inference for all cells at once
    net = W.WarmNet.from_file(WARM_WEIGHTS)
    phs = np.stack([c[0] for c in cells])
    x0, tl = net.make_input(phs, [c[1] for c in cells])
    vol = (len(cells), 64, 64, 64)
    net.forward(x0, vol, tl)                          # warm-up (module load)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    pred, _ = net.forward(x0, vol, tl)
    e1.record()
    torch.cuda.synchronize()
    infer_ms = e0.elapsed_time(e1)
    T0 = pred.view(*vol).cpu().numpy().astype(np.float32)
    out["inference_ms"] = infer_ms

    def batched(storage, warm):
        B = lbm.Batch()
        for i, (ph, lam, _) in enumerate(cells):
            B.add(ph, lam, 2)
            if warm:
                B.set_initial(i, np.ascontiguousarray(T0[i]))
        info = B.solve(0, lbm.Solver.opts(tol=0.0, max_iters=budget, storage=storage))
        worst, its, kerr = 0.0, [], []
        for i, (_, _, kst) in enumerate(cells):
            h = B.history(i)
            f = first_within(h, kst, rel)
            if f is None:
                B.close()
                return None
            worst = max(worst, h[f, 4])
            its.append(int(h[f, 0]))
            kerr.append(abs(h[-1, 1] / kst - 1.0))
        B.close()
        return {"ms": worst + (infer_ms if warm else 0.0), "batch_ms_to_band": worst,
                "iters_mean": float(np.mean(its)), "iters_max": int(max(its)),
                "k_final_max_rel_err": float(max(kerr)),
                "steps_per_launch": info.steps_per_launch, "block_threads": info.block_threads}

    out["batched_f32_linear"] = batched(lbm.LBM_STORE_F32, False)
    out["batched_f32_warm"] = batched(lbm.LBM_STORE_F32, True)
    out["combined_bf16_warm_batched"] = batched(lbm.LBM_STORE_BF16, True)
    c = out["combined_bf16_warm_batched"]
    if c:
        out["combined_over_plain_time"] = c["ms"] / out["plain_f32_sequential"]["ms"]
        out["warm_iters_saved"] = (1.0 - out["batched_f32_warm"]["iters_mean"] /
                                   out["batched_f32_linear"]["iters_mean"]) if out["batched_f32_warm"] else None
    return out


def warm_start_config5(lbm, I, stream, seeds=tuple(range(5000, 5010)), tol=1e-8):
    """Learned warm start on 128x128x256 braided cells of the warm-start
    distribution (seeds 5000.., z axis, periodic laterals, FP32): iterations
    and device time to R_T <= tol from the linear profile and from the
    network's prediction (inference time included), and the k_eff of both."""
    import torch
    from paper_1503_08718_gb300 import warmstart as W

    if not os.path.exists(WARM_WEIGHTS):
        return {"unavailable": "no trained warm-start weights"}
    net = W.WarmNet.from_file(WARM_WEIGHTS)
    rows = []
    for s in seeds:
        g, phi = I.warm_cell_params(s)
        lam = I.braid_tensors(g)
        with lbm.Solver(128, 128, 256) as S:
            S.set_geometry_braid(math.radians(g), I.braid_anchors(128, 128, s, n_max=512), phi)
            S.set_tensors(lam)
            ph = S.geometry()
            o = S.opts(tol=tol, max_iters=3_000_000)
            o.stream = int(stream.cuda_stream)
            S.start(2, 0, o)
            lin = S.run(allow=())
            h_lin = S.history()
            net.predict(ph, lam, as_tensor=True)              # warm-up (module load)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            T0 = net.predict(ph, lam, as_tensor=True)
            e1.record()
            torch.cuda.synchronize()
            inf_ms = e0.elapsed_time(e1)
            T0h = np.ascontiguousarray(T0.cpu().numpy(), dtype=np.float32)
            o.t_init = T0h.ctypes.data_as(lbm.ctypes.POINTER(lbm.ctypes.c_float))
            S.start(2, 0, o)
            warm = S.run(allow=())
            h_warm = S.history()
            # iterations until k_eff stays within 1e-4 of the converged value
            # (the linear start's, run to R_T <= tol)
            i1, i2 = first_within(h_lin, lin.k_eff, 1e-4), first_within(h_warm, lin.k_eff, 1e-4)
            k1 = int(h_lin[i1, 0]) if i1 is not None else None
            k2 = int(h_warm[i2, 0]) if i2 is not None else None
            rows.append({"seed": s, "g_deg": g, "phi": phi,
                         "linear": {"iters": int(lin.iters), "ms": lin.elapsed_ms, "k_eff": lin.k_eff,
                                    "iters_to_keff_1e-4": k1},
                         "warm": {"iters": int(warm.iters), "ms": warm.elapsed_ms + inf_ms,
                                  "inference_ms": inf_ms, "k_eff": warm.k_eff, "iters_to_keff_1e-4": k2},
                         "iters_saved": 1.0 - warm.iters / lin.iters,
                         "iters_saved_to_keff_1e-4": (1.0 - k2 / k1) if k1 and k2 else None,
                         "k_rel_diff": warm.k_eff / lin.k_eff - 1.0})
    return {"workload": "braids 128x128x256 (warm-start distribution), z axis, periodic, FP32, "
                        "to R_T <= %g" % tol, "cells": rows,
            "iters_saved_mean": float(np.mean([r["iters_saved"] for r in rows])),
            "iters_saved_to_keff_1e-4_mean": float(np.mean([r["iters_saved_to_keff_1e-4"] or 0.0 for r in rows])),
            "time_ratio_mean": float(np.mean([r["warm"]["ms"] / r["linear"]["ms"] for r in rows]))}


def conv_throughput(lbm, sustained_tflops, n=4, d=64, h=64, w=64, cin=64, cout=64, reps=10):
    """The warm-start network's 3x3x3 convolution at 4 cells of 64^3 with 64
    input and 64 output channels: the tcgen05 forward and weight-gradient
    kernels against the mma.sync ones (CUDA events), TFLOP/s and the fraction
    of the sustained BF16 peak."""
    import torch
    V = n * d * h * w
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    x = torch.randn(V, cin, device="cuda", generator=g).to(torch.bfloat16)
    gy = torch.randn(V, cout, device="cuda", generator=g).to(torch.bfloat16)
    W = (torch.randn(27, cin, cout, device="cuda", generator=g) / math.sqrt(27 * cin)).to(torch.bfloat16)
    b = torch.zeros(cout, device="cuda")
    y = torch.empty(V, cout, dtype=torch.bfloat16, device="cuda")
    dw = torch.zeros(27, cin, cout, device="cuda")
    wk = torch.empty(27 * cin * cout, dtype=torch.bfloat16, device="cuda")
    lbm.lbm_nn_weights_kmajor(W.data_ptr(), wk.data_ptr(), cin, cout, 0, None)
    flop = 2.0 * V * 27 * cin * cout

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        return {"ms": ms, "tflops": flop / ms / 1e9, "frac_sustained": flop / ms / 1e9 / sustained_tflops}

    out = {"shape": f"{n} x {d}x{h}x{w}, {cin} -> {cout} channels, 3x3x3", "gflop": flop / 1e9,
           "peak_sustained_tflops": sustained_tflops}
    out["fwd_tcgen05"] = timed(lambda: lbm.lbm_nn_conv3d_tc(x.data_ptr(), cin, wk.data_ptr(), b.data_ptr(),
                                                             y.data_ptr(), cout, n, d, h, w, 1, 0, None))
    out["fwd_mma_sync"] = timed(lambda: lbm.lbm_nn_conv3d(x.data_ptr(), cin, W.data_ptr(), b.data_ptr(),
                                                           y.data_ptr(), cout, n, d, h, w, 3, 1, 0, None))
    out["wgrad_tcgen05"] = timed(lambda: lbm.lbm_nn_conv3d_wgrad_tc(x.data_ptr(), cin, gy.data_ptr(), cout,
                                                                     dw.data_ptr(), n, d, h, w, None))
    out["wgrad_mma_sync"] = timed(lambda: lbm.lbm_nn_conv3d_wgrad(x.data_ptr(), cin, gy.data_ptr(), cout,
                                                                   dw.data_ptr(), n, d, h, w, 3, None))
    out["tc_error"] = lbm.lbm_nn_tc_error(True)
    return out


def cpu_oracle_sample(seconds_target=15.0):
    """Times the FP64 oracle on the host cores on the same cell: a fixed
    number of iterations of the full 128x128x256 lattice."""
    from oracle import oracle as O
    from paper_1503_08718_gb300 import inputs as I

    anchors = I.braid_anchors(NX, NY, SEED, n_max=NMAX)
    phase, _, _ = O.braid_phase(NX, NY, NZ, math.radians(G_DEG), anchors, PHI)
    lam = I.braid_tensors(G_DEG)
    L = O.Lattice(phase, lam, O.lattice_scale(lam), 2, 0)
    L.init_linear()
    t0 = time.perf_counter()
    L.step(2)
    dt = time.perf_counter() - t0
    n = max(2, min(200, int(seconds_target / max(dt / 2, 1e-6))))
    t0 = time.perf_counter()
    L.step(n)
    dt = time.perf_counter() - t0
    glups = NX * NY * NZ * n / dt / 1e9
    return glups, O.max_threads(), n, dt


def cpu_oracle_one_core(seconds_target=3.0):
    """The same oracle sample on one host core (iterations of the full cell)."""
    from oracle import oracle as O
    from paper_1503_08718_gb300 import inputs as I

    anchors = I.braid_anchors(NX, NY, SEED, n_max=NMAX)
    phase, _, _ = O.braid_phase(NX, NY, NZ, math.radians(G_DEG), anchors, PHI)
    lam = I.braid_tensors(G_DEG)
    all_cores = O.max_threads()
    O.set_threads(1)
    try:
        L = O.Lattice(phase, lam, O.lattice_scale(lam), 2, 0)
        L.init_linear()
        t0 = time.perf_counter()
        L.step(1)
        dt1 = time.perf_counter() - t0
        n = max(1, min(50, int(seconds_target / max(dt1, 1e-6))))
        t0 = time.perf_counter()
        L.step(n)
        dt = time.perf_counter() - t0
    finally:
        O.set_threads(all_cores)
    return NX * NY * NZ * n / dt / 1e9, n, dt


def oracle_extras():
    """Further oracle timings on the host cores: the 32^3 layered cell solved to
    R_T <= 1e-8, 500 iterations of the 256x256x512 braid, and the time the
    oracle would need for the bench cell's 33 400 iterations to k_eff within
    1e-4, extrapolated from its measured rate."""
    from oracle import oracle as O
    from paper_1503_08718_gb300 import inputs as I

    out = {"cores": O.max_threads()}
    yarn = I.transversely_isotropic(6.0, 0.8, I.axis_in_xz_from_z(30.0))
    lam = np.stack([I.isotropic(0.2), yarn])
    L = O.Lattice(I.layered_phase(32, 32, 32), lam, O.lattice_scale(lam), 2, 0)
    L.init_linear()
    t0 = time.perf_counter()
    rc, rt = L.solve(tol=1e-8, check_every=K)
    dt = time.perf_counter() - t0
    out["layered_32_converged"] = {"iters": L.iter, "seconds": dt, "k_eff": L.k_eff()[0],
                                   "exact": 94.0 / 245.0, "residual_T": rt}
    n4 = (256, 256, 512)
    anchors = I.braid_anchors(n4[0], n4[1], 7, n_max=1024)
    phase, _, _ = O.braid_phase(*n4, math.radians(35.0), anchors, 0.50)
    lam4 = I.braid_tensors(35.0)
    L4 = O.Lattice(phase, lam4, O.lattice_scale(lam4), 2, 0)
    L4.init_linear()
    t0 = time.perf_counter()
    L4.step(500)
    dt4 = time.perf_counter() - t0
    out["braid_256x256x512_500_iters"] = {"seconds": dt4, "glups": n4[0] * n4[1] * n4[2] * 500 / dt4 / 1e9}
    g, _, n, dt2 = cpu_oracle_sample(seconds_target=5.0)
    out["bench_cell_time_to_keff_1e-4_s"] = NX * NY * NZ * 33_400 / (g * 1e9)
    out["bench_cell_rate_glups"] = g
    return out


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle as O  # noqa: F401  (builds on first use)
    per_step = []
    glups_all = []
    cores = None
    sample = None
    for i in range(args.warmup + args.steps):
        glups, cores, n, dt = cpu_oracle_sample(seconds_target=args.ref_seconds)
        if i >= args.warmup:
            per_step.append(dt)
            glups_all.append(glups)
            sample = f"{n} FP64 oracle iterations of the full {NX}x{NY}x{NZ} cell per step"
    value = statistics.mean(glups_all)
    line = {
        "impl": "reference", "metric": "GLUPS", "value": value, "unit": "GLUPS",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * statistics.mean(per_step), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "iters_per_step": "bounded sample"},
        "cpu_baseline": {"value": value, "unit": "GLUPS", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "GLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    if args.oracle_extras:
        line["oracle_extras"] = oracle_extras()
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch

    from paper_1503_08718_gb300 import build as B
    from paper_1503_08718_gb300 import inputs as I
    from paper_1503_08718_gb300 import lbm, replicas

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    B.build()
    lbm.load()

    S, lam, used, frac = make_cell(lbm, I, dev)
    stream = torch.cuda.Stream(device=dev)
    iters = args.iters
    opts = S.opts(tol=0.0, max_iters=iters, check_every=K, host_loop=int(args.launch == "host"),
                  storage=STORAGE[args.storage], fuse=int(args.fuse))
    opts.stream = int(stream.cuda_stream)

    def one_step():
        S.start(2, 0, opts)
        info = S.run()
        assert info.iters == iters, info.as_dict()
        return info

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    # each step is bracketed by its own events; between steps (outside the
    # timed region) a 256 MB write evicts the L2, so no step starts on data
    # the previous one left there
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    with ClockSampler(dev) as clk:
        t0 = time.perf_counter()
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(k & 255)
            evs[k][0].record(stream)
            info = one_step()
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    ms = sum(a.elapsed_time(b) for a, b in evs)
    del flush
    if ws > 1:
        torch.distributed.barrier()
    ms = replicas.max_over_ranks(ms, device=f"cuda:{dev}")
    n_vox = NX * NY * NZ
    lups = n_vox * iters * args.steps * ws
    glups = lups / (ms / 1000.0) / 1e9
    # per check interval: the first step, fused pairs (FP32, the cell's 128 x
    # 128 rows allow them), the remaining single steps and the check step
    plan = S.launch_plan()
    R = K - 2
    pairs = 2 * (R // 4) if plan["steps_per_launch"] == 2 else 0
    launches_per_interval = 2 + pairs + (R - 2 * pairs)
    launches_per_step = (iters // K) * launches_per_interval + 2   # + permute, init
    # roofline of the dominant kernel: the fused two-step kernel in FP32,
    # else the single step.  Algorithmic bytes per launch follow the
    # per-update figure (33 B/LUP FP32, 17 B/LUP 16-bit: 4 fields read, 4
    # written, 1 B phase id) times the updates one launch performs
    # (voxels x 2 for the two-step kernel).  A two-step launch moves the state
    # through HBM once (33 B per voxel for two updates), so its `frac` exceeds
    # 1 by construction; `frac_moved` divides the bytes it actually has to
    # move by the same time (its bandwidth efficiency).  Its average launch
    # time is measured with CUDA events on the solver's stream over a run of
    # its launches alone (lbm_advance); frac_whole_step charges every launch
    # of the timed bench step to it instead (a lower bound).
    upd = 2 if pairs else 1
    if pairs:
        dom_launches = args.steps * (iters // K) * pairs
        dominant = "fused2_kernel (2 updates per launch)"
        dom_key = ("fused2", "f32")
    else:
        dom_launches = args.steps * iters
        dominant = "step_kernel"
        dom_key = ("step", args.storage)
    moved_bytes = BYTES_PER_LUP[args.storage] * n_vox
    dom_bytes = moved_bytes * upd
    per_launch_s = (ms / 1000.0) / dom_launches
    achieved_step = dom_bytes / per_launch_s / 1e9
    launch_us, n_timed, timing_mode = kernel_launch_us(S, opts, stream, upd)
    achieved = dom_bytes / (launch_us * 1e-6) / 1e9
    peak, peak_kind = peaks()
    traffic = args.traffic if args.traffic is not None else traffic_for(dom_key)

    # the same step with 16-bit distribution storage (FP32 collision,
    # stochastic rounding): GLUPS and the roofline at 29 B/LUP
    variants = {}
    if args.storage == "f32" and not args.no_variants:
        for name in ("bf16", "f16"):
            o16 = S.opts(tol=0.0, max_iters=iters, check_every=K, storage=STORAGE[name],
                         host_loop=int(args.launch == "host"))
            o16.stream = int(stream.cuda_stream)
            for _ in range(args.warmup):
                S.start(2, 0, o16)
                S.run()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            n16 = max(3, args.steps // 2)
            e0.record(stream)
            for _ in range(n16):
                S.start(2, 0, o16)
                i16 = S.run()
            e1.record(stream)
            torch.cuda.synchronize()
            ms16 = e0.elapsed_time(e1)
            g16 = n_vox * iters * n16 / (ms16 / 1000.0) / 1e9
            us16, _, _ = kernel_launch_us(S, o16, stream, 1)
            a16 = BYTES_PER_LUP[name] * n_vox / (us16 * 1e-6) / 1e9
            variants[name] = {"value": g16, "unit": "GLUPS", "steps": n16,
                              "ms_per_step": ms16 / n16, "bytes_per_lup": BYTES_PER_LUP[name],
                              "step_kernel_us": us16, "roofline_frac": a16 / peak,
                              "k_eff_after_step": i16.k_eff,
                              "k_eff_rel_vs_f32": (i16.k_eff - info.k_eff) / info.k_eff}

    extras = {}
    legs = set() if args.no_extras else set(args.legs.split(","))
    if "all" in legs:
        legs = {"configs", "time_to_keff", "combined", "cfg5", "conv"}
    if "configs" in legs:
        extras["configs"] = {
            "cfg1_layered32": config1_layered(lbm, I, stream),
            "cfg2_bench_cell_all_solves": config2_all_solves(lbm, S, stream, n_vox),
            "cfg3_sweep": sweep(lbm, I),
            "cfg4_braid256x256x512": config4_precision(lbm, I, stream, peak,
                                                       with_oracle=not args.skip_cpu),
        }
    if "time_to_keff" in legs:
        extras["time_to_keff"] = time_to_keff(lbm, S, stream)
    if "combined" in legs:
        extras["combined_form"] = combined_form(lbm, I, stream)
    if "cfg5" in legs:
        extras.setdefault("configs", {})["cfg5_warm_start"] = warm_start_config5(lbm, I, stream)
    if "conv" in legs:
        sus, sus_kind = bf16_sustained_tflops()
        extras["warmnet_conv"] = conv_throughput(lbm, sus)
        extras["warmnet_conv"]["peak_source"] = sus_kind

    # end to end through the public API with host buffers
    anchors = I.braid_anchors(NX, NY, SEED, n_max=NMAX)
    # host buffers in pinned memory (the copies DMA straight to and from it)
    phase_h = torch.empty((NZ, NY, NX), dtype=torch.uint8, pin_memory=True).numpy()
    phase_h[...] = S.geometry()
    T_h = torch.empty((NZ, NY, NX), dtype=torch.float32, pin_memory=True).numpy()
    e2e_ms = []
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S.set_geometry(phase_h, 5)
        S.set_tensors(lam)
        S.start(2, 0, opts)
        S.run()
        S.temperature(out=T_h)
        S.k_eff()
        t1 = time.perf_counter()
        if i >= args.warmup:
            e2e_ms.append((t1 - t0) * 1000)
    e2e_total_ms = replicas.max_over_ranks(sum(e2e_ms), device=f"cuda:{dev}")
    e2e_glups = n_vox * iters * len(e2e_ms) * ws / (e2e_total_ms / 1000.0) / 1e9
    del anchors

    if rank == 0:
        cpu = None
        if not args.skip_cpu:
            g, cores, n, dt = cpu_oracle_sample(seconds_target=args.ref_seconds)
            g1, n1, dt1 = cpu_oracle_one_core()
            cpu = {"value": g, "unit": "GLUPS", "cores": cores, "kind": "oracle",
                   "sample": f"{n} FP64 oracle iterations of the full {NX}x{NY}x{NZ} cell "
                             f"({dt:.1f} s)",
                   "one_core": {"value": g1, "unit": "GLUPS",
                                "sample": f"{n1} iterations of the same cell ({dt1:.1f} s)"}}
        line = {
            "metric": "GLUPS", "value": glups, "unit": "GLUPS", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.storage == "f32" else f"f32 (storage {args.storage})",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "iters_per_step": iters, "check_every": K,
                       "storage": args.storage, "fuse": bool(args.fuse),
                       "launch": args.launch,
                       "yarns": used, "yarn_fraction": round(frac, 6),
                       "l2": "flushed between steps (256 MB write outside the timed region)",
                       "parallelism": f"replicas{ws}"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_source": peak_kind, "kernel": dominant,
                         "updates_per_launch": upd,
                         "bytes_per_launch": dom_bytes,
                         "frac_basis": (f"{BYTES_PER_LUP[args.storage]} B/LUP x {n_vox} voxels x "
                                        f"{upd} updates per launch"),
                         "moved_bytes_per_launch": moved_bytes,
                         "frac_moved": moved_bytes / (launch_us * 1e-6) / 1e9 / peak,
                         "traffic_over_moved": (traffic / moved_bytes) if traffic else None,
                         "kernel_source_sha16": kernel_source_sha16(),
                         "launch_us": launch_us,
                         "launches_timed": n_timed, "launch_timing": timing_mode,
                         "frac_whole_step": achieved_step / peak,
                         # the state is four fields per node; a state of seven
                         # populations would move 57 B per update (FP32), 29 B
                         # (16-bit): the same launch against that figure
                         "seven_population_equivalent": {
                             "bytes_per_lup": 57 if args.storage == "f32" else 29,
                             "frac": (57 if args.storage == "f32" else 29) * n_vox * upd
                             / (launch_us * 1e-6) / 1e9 / peak}},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_glups, "unit": "GLUPS",
                    "h2d_bytes_per_step": n_vox + lam.nbytes,
                    "d2h_bytes_per_step": 4 * n_vox + 8},
            "gpu_launches": launches_per_step * args.steps,
            "launch_plan": plan,
            "clocks": clk.summary(),
            "k_eff_after_step": info.k_eff,
            "storage_variants": variants or None,
            **extras,
            "wall_s_timed": wall,
        }
        print(json.dumps(line), flush=True)
    S.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--iters", type=int, default=ITERS, help="iterations per step (multiple of 100)")
    ap.add_argument("--launch", default="graph", choices=["graph", "host"],
                    help="graph: one CUDA graph per step with a device-side while node; "
                         "host: the same kernels launched from the host (for profilers)")
    ap.add_argument("--storage", default="f32", choices=["f32", "bf16", "f16"],
                    help="distribution storage (collision is FP32 in every mode)")
    ap.add_argument("--no-fuse", action="store_true",
                    help="run FP32 plain steps one per launch (default: two, temporal blocking)")
    ap.add_argument("--no-variants", action="store_true",
                    help="omit the BF16/FP16 storage variants of the step")
    ap.add_argument("--no-extras", action="store_true",
                    help="omit every leg outside the timed region")
    ap.add_argument("--legs", default="all",
                    help="comma list of the legs outside the timed region: configs, time_to_keff, "
                         "combined, cfg5, conv (default all)")
    ap.add_argument("--skip-cpu", action="store_true", help="omit the CPU oracle baseline leg")
    ap.add_argument("--ref-seconds", type=float, default=15.0)
    ap.add_argument("--oracle-extras", action="store_true",
                    help="reference arm: also time the oracle on the layered 32^3 cell to "
                         "convergence and on 500 iterations of the 256x256x512 braid")
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per fused-step launch from an ncu capture")
    args = ap.parse_args()
    args.fuse = not args.no_fuse
    if args.iters % K:
        ap.error("--iters must be a multiple of 100")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
