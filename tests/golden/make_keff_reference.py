"""Writes keff_reference.json: converged FP64 oracle values k* of Eq. 22 for
the cells whose time-to-k_eff the benchmark measures.

Only the oracle (and the seeded input generators) run here.  Each cell is
voxelised by the oracle's own voxeliser and iterated from the linear start
(the initial field of the method's reading 11) in chunks of `chunk` steps;
after each chunk the plane fluxes give k_eff and the spread R_Q (Eq. 22 and
Fig. 8: all plane fluxes are equal at the steady state).  The run stops
when R_Q <= rq_tol, or (--dk-tol, for cells too large to iterate that far on
the host) when k_eff changed by at most dk_tol over the last chunk: the
error decays geometrically, so what remains is a few times the last change.
The record keeps the iteration count, the final R_Q and the change of k_eff
over the last chunk, and the SHA-256 of the phase map so that a consumer can
check it voxelised the same cell.

Usage: python tests/golden/make_keff_reference.py [--only LABEL] [--threads N]
Cells:
  braid128x128x256_z: the 128x128x256 braid (angle 30 deg, yarn fraction
      0.45, seed 42, 128 anchors), temperature difference along z,
      periodic laterals;
  warm64_<seed>, seed 7000..7015: held-out 64^3 braids of the warm-start
      distribution (inputs.warm_cell_params), z axis, periodic laterals.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_1503_08718_gb300 import inputs as I  # noqa: E402

OUT = os.path.join(HERE, "keff_reference.json")
WARM_SEEDS = tuple(range(7000, 7016))


def cells():
    yield dict(label="braid128x128x256_z", shape=(128, 128, 256), g_deg=30.0, phi=0.45,
               seed=42, n_anchors=128, axis=2, lateral=0)
    for s in WARM_SEEDS:
        g, phi = I.warm_cell_params(s)
        yield dict(label=f"warm64_{s}", shape=(64, 64, 64), g_deg=g, phi=phi, seed=s,
                   n_anchors=256, axis=2, lateral=0)


def solve(c, rq_tol, dk_tol, chunk, max_iters, log):
    nx, ny, nz = c["shape"]
    anchors = I.braid_anchors(nx, ny, c["seed"], n_max=c["n_anchors"])
    phase, used, frac = O.braid_phase(nx, ny, nz, math.radians(c["g_deg"]), anchors, c["phi"])
    lam = I.braid_tensors(c["g_deg"])
    s = O.lattice_scale(lam)
    L = O.Lattice(phase, lam, s, c["axis"], c["lateral"])
    L.init_linear()
    k_prev, t0 = None, time.time()
    while True:
        L.step(chunk)
        k, rq = L.k_eff()
        dk = None if k_prev is None else abs(k / k_prev - 1.0)
        log(f"{c['label']}: iter {L.iter} k {k:.12f} R_Q {rq:.3e} dk {dk}")
        if rq <= rq_tol or (dk is not None and dk <= dk_tol) or L.iter >= max_iters:
            break
        k_prev = k
    return dict(c, shape=list(c["shape"]), phase_sha256=hashlib.sha256(phase.tobytes()).hexdigest(),
                yarns=used, yarn_fraction=frac, lattice_scale=s, k_star=k, iters=L.iter,
                residual_Q=rq, dk_last_chunk=dk,
                converged=bool(rq <= rq_tol or (dk is not None and dk <= dk_tol)),
                seconds=time.time() - t0, threads=O.max_threads())


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", default=None)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--rq-tol", type=float, default=1e-10)
    ap.add_argument("--dk-tol", type=float, default=0.0,
                    help="also stop once k_eff changes by at most this (relative) over a chunk")
    ap.add_argument("--chunk", type=int, default=1000)
    ap.add_argument("--max-iters", type=int, default=2_000_000)
    a = ap.parse_args()
    if a.threads:
        O.set_threads(a.threads)
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as fh:
            data = json.load(fh)
    data.setdefault("how", "FP64 oracle (oracle/lbm_oracle.c) from the linear start, "
                           "stopped at R_Q <= rq_tol; written by make_keff_reference.py")
    data.setdefault("cells", {})
    for c in cells():
        if a.only and not c["label"].startswith(a.only):
            continue
        if c["label"] in data["cells"] and data["cells"][c["label"]].get("converged"):
            continue
        r = solve(c, a.rq_tol, a.dk_tol, a.chunk, a.max_iters, lambda m: print(m, flush=True))
        r["rq_tol"] = a.rq_tol
        r["dk_tol"] = a.dk_tol
        data["cells"][c["label"]] = r
        with open(OUT + ".tmp", "w") as fh:
            json.dump(data, fh, indent=1, sort_keys=True)
        os.replace(OUT + ".tmp", OUT)


if __name__ == "__main__":
    main()
