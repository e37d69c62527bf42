"""Diagonal removal (§2) through the C-ABI: the map without the CSM diagonal, the
PSF without the m = m' microphone pairs rescaled to a unit diagonal, and the
solve on that system, against the oracle's literal double sums."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import synth

pytestmark = pytest.mark.gpu

D = pytest.importorskip("paper_1608_05179_gb300").damas


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = D.Context(0)
    yield c
    c.close()


def rel_l2(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    e = float(np.linalg.norm(a - b) / np.linalg.norm(b))
    print(f"[rel_l2] {e:.3e}")
    return e


@pytest.mark.parametrize("form", [O.FORM_E, O.FORM_P])
def test_dr_map_matches_oracle(ctx, form):
    sc = synth.scene_monopole_small()
    g = D.Geometry.from_scene(sc.mics, sc.grid, sc.c, form, diag_removal=1)
    b = D.das_map(ctx, g, sc.freq, D.csm_tensor(sc.C)).cpu().numpy()
    pts = sc.grid.points()
    bo = O.das_map(sc.mics, pts, sc.freq, sc.c, sc.C, form, diag_removal=True)
    full = O.das_map(sc.mics, pts, sc.freq, sc.c, sc.C, form)
    # FP32 quadratic form: the error scales with the map before the diagonal terms cancel
    assert np.abs(b - bo).max() <= 2e-5 * np.abs(full).max()


@pytest.mark.parametrize("form", [O.FORM_E, O.FORM_P])
def test_dr_psf_matches_oracle(ctx, form):
    sc = synth.scene_monopole_small()
    g = D.Geometry.from_scene(sc.mics, sc.grid, sc.c, form, diag_removal=1)
    A, g2, dsc = D.damas_build_psf_dr(ctx, g, sc.freq)
    torch.cuda.synchronize()
    S = sc.grid.S
    Ad, _ = O.psf_matrix(sc.mics, sc.grid.points(), sc.freq, sc.c, form, diag_removal=True)
    d = np.sqrt(np.diag(Ad))
    Aw = Ad / d[:, None] / d[None, :]
    Ag = A.cpu().numpy()
    assert np.allclose(dsc.cpu().numpy(), d, rtol=2e-6, atol=0)
    assert np.all(np.diag(Ag[:, :S]) == 1.0) and np.all(Ag[:, S:] == 0.0)
    # the tensor-core Gram's bound (M = 16) plus the FP32 correction, over d_n d_s ~ 1 - 1/M
    assert np.abs(Ag[:, :S] - Aw).max() <= 1e-5
    if form == O.FORM_E:
        assert np.array_equal(Ag[:, :S], Ag[:, :S].T)


def test_dr_system_sweeps_on_same_inputs(ctx):
    """The unit-diagonal form has negative entries: the solver checks for them and
    runs every row (no candidate skipping).  Same FP32 inputs on both sides."""
    sc = synth.scene_monopole_small()
    pts = sc.grid.points()
    Ad, _ = O.psf_matrix(sc.mics, pts, sc.freq, sc.c, diag_removal=True)
    b = O.das_map(sc.mics, pts, sc.freq, sc.c, sc.C, diag_removal=True)
    d = np.sqrt(np.diag(Ad))
    A1 = (Ad / d[:, None] / d[None, :]).astype(np.float32)
    np.fill_diagonal(A1, 1.0)
    b1 = (b / d).astype(np.float32)
    S = len(b)
    lda = D.damas_lda(S)
    At = torch.zeros((S, lda), device="cuda")
    At[:, :S] = torch.as_tensor(A1, device="cuda")
    x = torch.zeros(S, device="cuda")
    D.damas_solve(ctx, D.System(At, torch.as_tensor(b1, device="cuda"), x, 100))
    xo = O.gauss_seidel(A1.astype(np.float64), b1.astype(np.float64), 100)
    assert rel_l2(x.cpu().numpy(), xo) <= 1e-4


def test_dr_bin_end_to_end(ctx):
    """solve_bin with diagonal removal (full grid) against the oracle's iteration on
    the unscaled system (A_ii != 1, divided as Eq. (14) says)."""
    sc = synth.scene_monopole_small()
    g = D.Geometry.from_scene(sc.mics, sc.grid, sc.c, diag_removal=1)
    out = D.solve_bin(ctx, g, sc.freq, D.csm_tensor(sc.C), 100, compressed=False)
    torch.cuda.synchronize()
    pts = sc.grid.points()
    Ad, g2 = O.psf_matrix(sc.mics, pts, sc.freq, sc.c, diag_removal=True)
    b = O.das_map(sc.mics, pts, sc.freq, sc.c, sc.C, diag_removal=True)
    xo = O.to_power(O.gauss_seidel(Ad, b, 100), g2)
    x = out["x"].cpu().numpy()
    assert rel_l2(x, xo) <= 2e-3
    assert int(np.argmax(x)) == int(np.argmax(xo))


def test_dr_rejections(ctx):
    sc = synth.scene_monopole_small()
    g = D.Geometry.from_scene(sc.mics, sc.grid, sc.c, diag_removal=1)
    with pytest.raises(D.DamasError):
        D.damas_build_psf(ctx, g, sc.freq)          # the plain PSF has a unit diagonal
    g0 = D.Geometry.from_scene(sc.mics, sc.grid, sc.c)
    with pytest.raises(D.DamasError):
        D.damas_build_psf_dr(ctx, g0, sc.freq)      # needs diag_removal = 1
    one = D.Geometry.from_scene(sc.mics[:1], sc.grid, sc.c, diag_removal=1)
    with pytest.raises(D.DamasError):
        D.das_map(ctx, one, sc.freq, D.csm_tensor(sc.C[:1, :1]))   # no pairs with one microphone
