"""Oracle-side helpers of the end-to-end parity tests (test infrastructure).

Two facts about the method set how an end-to-end result is compared with the
oracle's:

1. Algorithm 1 is a threshold decision.  The GPU's DAS map differs from the
   oracle's FP64 map (rounded to FP32) by at most DAS_TOL * max|b| (the DAS
   kernel's tested bound); a prediction averages map values, so every wavelet
   detail moves by at most twice that.  A threshold inside a gap of the sorted
   |detail| values wider than four times the bound therefore selects the same
   points from either map: `margin_threshold` finds one.

2. The Gauss-Seidel iterate after a fixed number of sweeps is ill-conditioned:
   A is singular (the paper notes that DAMAS has no unique solution), and the
   clamped iteration drifts along directions the data barely fix.  Rounding A
   and b to FP32 alone moves the oracle's own 1000-sweep iterate by about 2e-4
   on the compressed 81x81 system (1.5e-3 on the full grid), while A x (the map
   the solution reproduces) and the integrated power move by about 3e-7.
   `iterate_tolerance` measures that response s_round on the system at hand,
   with the oracle only, and states the tolerance on the iterate as
   PARITY + K_ROUND * s_round: rounding is the least any FP32 implementation
   perturbs its inputs by, and the GPU's inputs (a 3xTF32 Gram with truncating
   FP32 accumulation, FP32 DAS sums of M^2 terms) carry errors a few times
   larger.  The well-conditioned quantities are held to the benchmark spec's figure
   1e-4 directly.  The response to the Gram's truncation bias (s_bias) is
   measured and reported beside it.
"""
from __future__ import annotations

from concurrent.futures import ThreadPoolExecutor

import numpy as np

import oracle as O

DAS_TOL = 2e-5         # max |b_gpu - b| <= DAS_TOL * max |b| (the DAS kernel's test bound)
PARITY = 1e-4          # the solver's relative L2 bound on identical FP32 inputs
GRAM_BIAS = 3e-6       # relative truncation bias of the tensor-core Gram's FP32 accumulation
K_ROUND = 8.0          # stated multiple of the iterate's response to FP32 rounding of A and b


def rel(a, b) -> float:
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = float(np.linalg.norm(b))
    return float(np.linalg.norm(a - b)) / (nb if nb > 0 else 1.0)


def margin_threshold(b32, nx: int, ny: int, levels: int, predictor: int, keep_lo: float, keep_hi: float):
    """An absolute threshold (EPS_ABS) keeping between keep_lo and keep_hi of the
    nx*ny points, at the midpoint of the widest gap between consecutive |detail|
    values there.  Returns (eps, gap in units of DAS_TOL * max|b|); a gap above 4
    makes the selection identical for every map within the DAS bound."""
    b32 = np.asarray(b32, np.float32).reshape(-1)
    _, det, lev, _ = O.wavelet_select(b32, nx, ny, levels, predictor, O.EPS_ABS, 0.0)
    S = nx * ny
    n0 = int(np.sum(lev == 0))
    d = np.sort(np.abs(det[lev > 0]).astype(np.float64))[::-1]
    k0 = max(int(np.ceil(keep_lo * S)) - n0, 1)
    k1 = min(int(np.floor(keep_hi * S)) - n0, len(d) - 1)
    if k1 <= k0:
        raise ValueError("keep range holds no rank")
    gaps = d[k0 - 1:k1 - 1] - d[k0:k1]        # gap below rank r (1-based) for r in k0..k1-1
    i = int(np.argmax(gaps))
    eps = 0.5 * (d[k0 - 1 + i] + d[k0 + i])
    unit = DAS_TOL * float(np.max(b32))
    return float(np.float32(eps)), float(gaps[i]) / unit


def _gs(A, b, iters):
    return O.gauss_seidel(A, b, iters)


def sensitivity_inputs(A64, b64):
    """The two perturbed systems whose iterates set the tolerance: (A, b) rounded
    to FP32, and A with its off-diagonal entries scaled by (1 - GRAM_BIAS)."""
    A32 = A64.astype(np.float32).astype(np.float64)
    b32 = np.asarray(b64).astype(np.float32).astype(np.float64)
    Ab = A64 * (1.0 - GRAM_BIAS)
    np.fill_diagonal(Ab, 1.0)
    return [(A32, b32), (Ab, np.asarray(b64, np.float64))]


def tolerance_from(x_round, x_bias, x_ref):
    s_round, s_bias = rel(x_round, x_ref), rel(x_bias, x_ref)
    return PARITY + K_ROUND * s_round, {"s_round": s_round, "s_bias": s_bias}


def iterate_tolerance(A64, b64, iters: int, x_ref=None, threads: int = 3):
    """Tolerance on the relative L2 error of the iterate (in the units of x_ref's
    system) after `iters` sweeps:  PARITY + K_ROUND * s_round, where s_round is
    the oracle's response to A and b rounded to FP32; s_bias, its response to
    the off-diagonal entries of A scaled by (1 - GRAM_BIAS), is reported beside
    it.  x_ref (the oracle's iterate on A64, b64) is computed when not given.
    Returns (tol, details)."""
    jobs = sensitivity_inputs(A64, b64)
    if x_ref is None:
        jobs.append((A64, np.asarray(b64, np.float64)))
    with ThreadPoolExecutor(threads) as ex:          # the oracle's C loops release the GIL
        res = list(ex.map(lambda ab: _gs(ab[0], ab[1], iters), jobs))
    if x_ref is None:
        x_ref = res[2]
    tol, det = tolerance_from(res[0], res[1], x_ref)
    det["x_ref"] = x_ref
    return tol, det


def conditioned_errors(A64, x_sub, x_ref_sub, g2, g2_ref):
    """Errors of the well-conditioned outputs: the reproduced map A x (relative L2,
    with the oracle's A for both) and the integrated power sum x / ||g||^2."""
    r = rel(A64 @ np.asarray(x_sub, np.float64), A64 @ np.asarray(x_ref_sub, np.float64))
    p = float(np.sum(np.asarray(x_sub, np.float64) / np.asarray(g2, np.float64)))
    p_ref = float(np.sum(np.asarray(x_ref_sub, np.float64) / np.asarray(g2_ref, np.float64)))
    return r, abs(p - p_ref) / abs(p_ref)
