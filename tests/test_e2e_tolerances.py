"""Pins of the two facts the end-to-end parity tests rest on (oracle only, CPU).

1. A threshold from e2e_util.margin_threshold selects the same compressed grid
   from every map within the DAS kernel's error bound: checked by perturbing the
   oracle's map at the full bound (random signs, and the adversarial pattern
   that pushes every detail towards the threshold) and re-running Algorithm 1.
2. The iterate after 1000 sweeps is ill-conditioned while the reproduced map A x
   and the integrated power are not: rounding A and b to FP32 moves the FP64
   iterate by 1e-5..1e-3 but those two by less than 1e-6.
"""
import numpy as np
import pytest

import oracle as O
import synth
from e2e_util import DAS_TOL, conditioned_errors, iterate_tolerance, margin_threshold, rel


@pytest.fixture(scope="module")
def scene81():
    sc = synth.scene_spiral_81()
    b64 = O.das_map(sc.mics, sc.grid.points(), sc.freq, sc.c, sc.C)
    return sc, b64


def test_margin_threshold_is_stable_under_map_errors_within_the_bound(scene81):
    sc, b64 = scene81
    b32 = b64.astype(np.float32)
    eps, gap = margin_threshold(b32, 81, 81, 2, O.PRED_HAAR, 0.08, 0.12)
    assert gap > 4.0
    idx0, det, lev, _ = O.wavelet_select(b32, 81, 81, 2, O.PRED_HAAR, O.EPS_ABS, eps)
    assert 0.08 * 6561 <= len(idx0) <= 0.12 * 6561
    delta = DAS_TOL * float(b32.max())
    rng = np.random.default_rng(3)
    for _ in range(4):
        bp = (b64 + delta * rng.choice([-1.0, 1.0], size=b64.shape)).astype(np.float32)
        idx, _, _, _ = O.wavelet_select(bp, 81, 81, 2, O.PRED_HAAR, O.EPS_ABS, eps)
        assert np.array_equal(idx, idx0)
    # Haar predicts from the lower-left coarse neighbour: lowering the map there and
    # raising the point (or the reverse) moves a detail by 2 delta towards eps
    sign = np.where(np.abs(det) >= eps, -1.0, 1.0)          # kept: shrink |d|; dropped: grow it
    push = np.zeros_like(b64)
    kept_or_not = (lev > 0)
    push[kept_or_not] = -sign[kept_or_not] * np.sign(det[kept_or_not]) * delta
    bp = (b64 + push).astype(np.float32)
    idx, _, _, _ = O.wavelet_select(bp, 81, 81, 2, O.PRED_HAAR, O.EPS_ABS, eps)
    assert np.array_equal(idx, idx0)
    # and a threshold placed at a detail value itself is not stable: moving that one
    # point's map value by delta towards its prediction drops it (the pin bites)
    p = int(np.flatnonzero(lev > 0)[np.argsort(-np.abs(det[lev > 0]), kind="stable")][len(idx0) - int(np.sum(lev == 0))])
    eps_bad = float(abs(det[p]))
    i1, _, _, _ = O.wavelet_select(b32, 81, 81, 2, O.PRED_HAAR, O.EPS_ABS, eps_bad)
    bq = b64.copy()
    bq[p] += delta * np.sign(det[p])
    i2, _, _, _ = O.wavelet_select(bq.astype(np.float32), 81, 81, 2, O.PRED_HAAR, O.EPS_ABS, eps_bad)
    assert p in set(i1.tolist()) and p not in set(i2.tolist())


def test_iterate_is_ill_conditioned_but_reproduced_map_and_power_are_not(scene81):
    sc, b64 = scene81
    eps, _ = margin_threshold(b64.astype(np.float32), 81, 81, 2, O.PRED_HAAR, 0.08, 0.12)
    idx, _, _, _ = O.wavelet_select(b64.astype(np.float32), 81, 81, 2, O.PRED_HAAR, O.EPS_ABS, eps)
    A, g2 = O.psf_matrix(sc.mics, sc.grid.points()[idx], sc.freq, sc.c)
    bs = b64[idx]
    tol, det = iterate_tolerance(A, bs, 1000)
    x = det["x_ref"]
    assert 1e-5 <= det["s_round"] <= 1e-3, det["s_round"]
    assert det["s_bias"] <= 1e-2
    assert tol == pytest.approx(1e-4 + 8.0 * det["s_round"])
    xr = O.gauss_seidel(A.astype(np.float32).astype(np.float64), bs.astype(np.float32).astype(np.float64), 1000)
    assert rel(xr, x) == pytest.approx(det["s_round"])
    e_reconv, e_pow = conditioned_errors(A, xr, x, g2, g2)
    assert e_reconv < 1e-6 and e_pow < 1e-6
