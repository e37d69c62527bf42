"""Writes tests/golden/large161_reference.json: the FP64 oracle's per-source power on
the 161x161 near-field scene (S = 25921, M = 128, 6 kHz, 8 sources), full grid,
2050 Gauss-Seidel sweeps from x = 0 (Eq. (13)-(14)), formulation E, x scaled to
power by 1/||g||^2.  Per source: the power summed over grid points within half the
Rayleigh beamwidth (Eq. (25)) of the source, in dB.

Calls only the oracle and the scene generator.  Needs about 6 GB of memory (A in
FP64) and some 15-30 minutes of one CPU core:
    python tests/golden/make_large161_reference.py
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
import synth  # noqa: E402

SWEEPS = 2050


def region_power_db(x_full, grid, src_xyz, radius):
    pts = grid.points()
    out = []
    for s in src_xyz:
        m = np.linalg.norm(pts[:, :2] - s[None, :2], axis=1) <= radius
        out.append(10.0 * np.log10(max(float(x_full[m].sum()), 1e-30)))
    return out


def main():
    t0 = time.time()
    sc = synth.scene_large_161()
    pts = sc.grid.points()
    b = O.das_map(sc.mics, pts, sc.freq, sc.c, sc.C)
    A, g2 = O.psf_matrix(sc.mics, pts, sc.freq, sc.c)
    t1 = time.time()
    x = O.gauss_seidel(A, b, SWEEPS)
    t2 = time.time()
    power = O.to_power(x, g2)
    beam = 1.22 * 1.5 * sc.c / (1.5 * sc.freq)   # Rayleigh beamwidth at the plane, z0 = D = 1.5 m
    out = {
        "scene": "synth.scene_large_161() (seed 3)", "S": int(sc.grid.S), "M": int(sc.M), "freq_hz": sc.freq,
        "sweeps": SWEEPS, "formulation": "E", "radius_m": beam / 2,
        "source_xyz": np.asarray(sc.src_xyz).tolist(), "source_power": np.asarray(sc.powers).tolist(),
        "region_power_db": region_power_db(power, sc.grid, sc.src_xyz, beam / 2),
        "total_power": float(power.sum()),
        "seconds": {"build": round(t1 - t0, 1), "sweeps": round(t2 - t1, 1)},
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "large161_reference.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path, out["region_power_db"], out["seconds"])


if __name__ == "__main__":
    main()
