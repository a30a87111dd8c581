"""Measurements beyond the benchmark line, each printed as one JSON object.

precision: the 256 x 256 x 512 braided cell (interior braiding angle 35 deg,
yarn fraction 0.50, seed 7) solved along x, y and z with FP32, BF16 and FP16
distribution storage for the same iteration budget from the linear start.
The FP32 path equals the FP64 oracle to 1e-5 in k_eff (parity tests), so the
16-bit results are reported against FP32 at the same iteration: that
difference is the storage error.  Also GLUPS per storage and direction.

Usage: python -m paper_1503_08718_gb300.experiments precision [--iters N]
"""
from __future__ import annotations

import argparse
import json
import math

from . import build
from . import inputs as I
from . import lbm


def precision(iters: int = 20_000, shape=(256, 256, 512), g_deg=35.0, phi=0.50, seed=7,
              device: int = 0):
    build.build()
    nx, ny, nz = shape
    S = lbm.Solver(nx, ny, nz, device)
    used, frac = S.set_geometry_braid(math.radians(g_deg), I.braid_anchors(nx, ny, seed, n_max=1024),
                                      phi)
    S.set_tensors(I.braid_tensors(g_deg))
    out = {"cell": f"braid {nx}x{ny}x{nz} g={g_deg}deg phi={phi} seed={seed}", "yarns": used,
           "yarn_fraction": frac, "iters": iters, "directions": {}}
    for axis, name in ((0, "x"), (1, "y"), (2, "z")):
        row = {}
        k32 = None
        for st_name, st in (("f32", lbm.LBM_STORE_F32), ("bf16", lbm.LBM_STORE_BF16),
                            ("f16", lbm.LBM_STORE_F16)):
            info = S.solve(axis, 0, S.opts(tol=0.0, max_iters=iters, storage=st))
            glups = nx * ny * nz * info.iters / info.elapsed_ms / 1e6
            if k32 is None:
                k32 = info.k_eff
            row[st_name] = {"k_eff": info.k_eff, "glups": glups, "ms": info.elapsed_ms,
                            "k_rel_vs_f32": info.k_eff / k32 - 1.0,
                            "residual_T": info.residual_T}
        out["directions"][name] = row
    S.close()
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("what", choices=["precision"])
    ap.add_argument("--iters", type=int, default=20_000)
    a = ap.parse_args(argv)
    if a.what == "precision":
        print(json.dumps(precision(a.iters)))


if __name__ == "__main__":
    main()
