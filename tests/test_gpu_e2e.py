"""End-to-end parity: the §5 procedure on the GPU (DAS map, Algorithm 1, PSF of
the kept points, Gauss-Seidel from x = 0, power map), every step in the CUDA
library, against the oracle's FP64 procedure (oracle.solve_bin) on the same
scene.

What is compared and why (tests/e2e_util.py):
  - the compressed grid: identical, with a threshold whose margin exceeds four
    times the DAS kernel's error bound (so any map within that bound selects
    the same points);
  - the reproduced map A x and the integrated power: relative error <= 1e-4,
    the benchmark spec's figure (both are well-conditioned);
  - the power map itself: relative L2 <= 1e-4 + 8 s_round, where s_round is the
    oracle's own response, on this system, to A and b rounded to FP32: after a
    fixed number of sweeps the iterate of the singular system is
    ill-conditioned (measured on GB300: 4.4 s_round on the compressed grid,
    4.6 s_round on the full grid).
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import torch

import oracle as O
import synth
from e2e_util import (DAS_TOL, PARITY, conditioned_errors, iterate_tolerance, margin_threshold, rel,
                      sensitivity_inputs, tolerance_from)

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_1608_05179_gb300")
D = P.damas


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = D.Context(0)
    yield c
    c.close()


def _report(name, **kw):
    print(f"[e2e] {name}: " + ", ".join(f"{k}={v:.3e}" for k, v in kw.items()))


def _check(name, out, orc, A64, tol, iters_detail):
    """The end-to-end assertions shared by the compressed and the full grid."""
    x_gpu = out["x"].cpu().numpy().astype(np.float64)
    xs_gpu = out["x_sub"].cpu().numpy().astype(np.float64)
    g2_gpu = out["gnorm2"].cpu().numpy().astype(np.float64)
    e_map = rel(x_gpu, orc["x"])
    e_reconv, e_pow = conditioned_errors(A64, xs_gpu, orc["x_sub"], g2_gpu, orc["gnorm2"])
    e_tot = abs(out["total_power"].item() - orc["x"].sum()) / orc["x"].sum()
    _report(name, map=e_map, map_tol=tol, s_round=iters_detail["s_round"], s_bias=iters_detail["s_bias"],
            reconv=e_reconv, power=e_pow, total=e_tot)
    assert e_reconv <= PARITY
    assert e_pow <= PARITY and e_tot <= PARITY
    assert e_map <= tol


def test_end_to_end_compressed_bin(ctx):
    """81x81 spiral scene (M = 64, 2 kHz), Haar L = 2, a threshold keeping 8-12% of
    the points placed with a provable margin, 1000 sweeps."""
    sc = synth.scene_spiral_81()
    pts = sc.grid.points()
    b64 = O.das_map(sc.mics, pts, sc.freq, sc.c, sc.C)
    eps, gap = margin_threshold(b64.astype(np.float32), 81, 81, 2, O.PRED_HAAR, 0.08, 0.12)
    assert gap > 4.0, gap
    g = D.Geometry.from_scene(sc.mics, sc.grid, sc.c)
    out = D.solve_bin(ctx, g, sc.freq, D.csm_tensor(sc.C), 1000, compressed=True, levels=2,
                      predictor=O.PRED_HAAR, eps_mode=O.EPS_ABS, eps=eps)
    torch.cuda.synchronize()
    orc = O.solve_bin(sc.mics, sc.grid, sc.freq, sc.c, sc.C, 1000, compressed=True, levels=2,
                      predictor=O.PRED_HAAR, eps_mode=O.EPS_ABS, eps=eps)
    # the grid, bit-exact
    assert np.array_equal(out["idx"].cpu().numpy(), orc["idx"])
    # each kernel within its own bound on this bin
    b_gpu = out["b"].cpu().numpy()
    assert np.max(np.abs(b_gpu - b64)) <= DAS_TOL * np.max(b64)
    A_gpu = out["A"][:, :out["S_sub"]].cpu().numpy()
    assert np.max(np.abs(A_gpu - orc["A"])) <= 5e-6
    tol, det = iterate_tolerance(orc["A"], orc["b"][orc["idx"]], 1000, x_ref=orc["x_sub"])
    _check("compressed 81x81", out, orc, orc["A"], tol, det)


@pytest.mark.slow
def test_end_to_end_full_grid_81x81(ctx):
    """The full 81x81 grid (S = 6561): GPU-built b and A, 1000 sweeps, against
    oracle.solve_bin(compressed=False).  The oracle runs take about a minute; its
    three Gauss-Seidel runs go on host threads side by side."""
    sc = synth.scene_spiral_81()
    g = D.Geometry.from_scene(sc.mics, sc.grid, sc.c)
    out = D.solve_bin(ctx, g, sc.freq, D.csm_tensor(sc.C), 1000, compressed=False)
    torch.cuda.synchronize()
    pts = sc.grid.points()
    with ThreadPoolExecutor(3) as ex:                # the oracle's C loops release the GIL
        f_orc = ex.submit(O.solve_bin, sc.mics, sc.grid, sc.freq, sc.c, sc.C, 1000, False)
        A64, _ = O.psf_matrix(sc.mics, pts, sc.freq, sc.c)
        b64 = O.das_map(sc.mics, pts, sc.freq, sc.c, sc.C)
        f_sens = [ex.submit(O.gauss_seidel, A, b, 1000) for A, b in sensitivity_inputs(A64, b64)]
        orc = f_orc.result()
        x_round, x_bias = f_sens[0].result(), f_sens[1].result()
    assert np.array_equal(orc["A"], A64)
    tol, det = tolerance_from(x_round, x_bias, orc["x_sub"])
    assert np.max(np.abs(out["b"].cpu().numpy() - b64)) <= DAS_TOL * np.max(b64)
    _check("full 81x81", out, orc, A64, tol, det)


def test_selection_near_threshold_flips_only_near_points(ctx):
    """With the keep-fraction threshold of the benchmark (10%), the GPU map and the
    oracle's map may select differently only at points whose detail lies within
    the DAS bound of the threshold (an FP32 decision on maps that differ within
    that bound); everything else agrees."""
    sc = synth.scene_spiral_81()
    g = D.Geometry.from_scene(sc.mics, sc.grid, sc.c)
    b = D.das_map(ctx, g, sc.freq, D.csm_tensor(sc.C))
    idx, n, _, _ = D.wavelet_compress_grid(ctx, b, 81, 81, 2, O.PRED_HAAR, O.EPS_KEEP_FRAC, 0.1)
    gi = set(idx[: int(n.item())].cpu().numpy().tolist())
    bo32 = O.das_map(sc.mics, sc.grid.points(), sc.freq, sc.c, sc.C).astype(np.float32)
    io, det, _, ea = O.wavelet_select(bo32, 81, 81, 2, O.PRED_HAAR, O.EPS_KEEP_FRAC, 0.1)
    oi = set(io.tolist())
    unit = DAS_TOL * float(bo32.max())
    near = {p for p in (gi ^ oi) if abs(abs(float(det[p])) - ea) <= 4 * unit}
    assert gi ^ oi == near
    # and the GPU's selection on the oracle's own FP32 map is bit-exact
    idx2, n2, _, _ = D.wavelet_compress_grid(ctx, torch.as_tensor(bo32, device="cuda"), 81, 81, 2, O.PRED_HAAR,
                                             O.EPS_KEEP_FRAC, 0.1)
    assert np.array_equal(idx2[: int(n2.item())].cpu().numpy(), io)
