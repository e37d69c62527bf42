"""Pins for the oracle's steering vectors, PSF matrix and DAS map (§2-§3).

Each check is tied to something other than the oracle's own formula: a
two-element interferometer closed form, invariants that the definitions force
(unit norm, reciprocity, Cauchy-Schwarz, Schur-product PSD), the far-field
shift invariance the paper discusses in §1, and the scene generator's
independent monopole model (a unit source on a grid point must give b = A e_s).
"""
import math

import numpy as np
import pytest

import oracle as O
import synth


def _small_scene():
    return synth.scene_monopole_small(seed=0)


def test_e_vectors_unit_norm_and_gnorm():
    sc = _small_scene()
    pts = sc.grid.points()
    E, g2 = O.vectors(sc.mics, pts, sc.freq, sc.c, "e")
    assert np.allclose(np.linalg.norm(E, axis=1), 1.0, atol=1e-14)
    d = np.linalg.norm(pts[:, None, :] - sc.mics[None, :, :], axis=2)
    r = np.linalg.norm(pts, axis=1)
    assert np.allclose(g2, ((r[:, None] / d) ** 2).sum(1), rtol=1e-14)


def test_v_g_reciprocity():
    """v_n^H g_n = sum_m (d/|r|)(|r|/d) = M exactly (Eq. (4) with Eq. (7))."""
    sc = _small_scene()
    pts = sc.grid.points()[:50]
    V, _ = O.vectors(sc.mics, pts, sc.freq, sc.c, "v")
    G, _ = O.vectors(sc.mics, pts, sc.freq, sc.c, "g")
    ip = (V.conj() * G).sum(1)
    assert np.allclose(ip, sc.M, atol=1e-12)


def test_phase_sign_convention():
    """One microphone at the origin, point on the axis at distance z:
    g = exp(-j k z) (Eq. (7) with |r| = d)."""
    mics = np.zeros((1, 3))
    z = 1.2345
    G, _ = O.vectors(mics, np.array([[0.0, 0.0, z]]), 1000.0, 343.0, "g")
    k = 2 * math.pi * 1000.0 / 343.0
    assert abs(G[0, 0] - np.exp(-1j * k * z)) < 1e-13


def test_psf_e_unit_diag_symmetric_bounded_psd():
    sc = _small_scene()
    A, _ = O.psf_matrix(sc.mics, sc.grid.points(), sc.freq, sc.c, O.FORM_E)
    assert np.all(np.diag(A) == 1.0)
    assert np.array_equal(A, A.T)
    assert A.min() >= 0.0 and A.max() <= 1.0 + 1e-12          # Cauchy-Schwarz on unit vectors
    assert np.linalg.eigvalsh(A).min() >= -1e-12              # Schur product of a Gram and its conjugate


def test_psf_p_unit_diag_not_symmetric():
    sc = _small_scene()
    A, _ = O.psf_matrix(sc.mics, sc.grid.points()[:60], sc.freq, sc.c, O.FORM_P)
    assert np.all(np.diag(A) == 1.0)
    assert np.abs(A - A.T).max() > 1e-6


def _two_mic_setup():
    mics = np.array([[-0.3, 0.05, 0.0], [0.25, -0.1, 0.0]])
    grid = synth.square_plane(7, 1.0, 1.5)
    return mics, grid.points(), 3000.0, 343.0


def test_psf_e_two_element_closed_form():
    """Two microphones: |e_n^H e_m|^2 = (w1n w1m)^2 + (w2n w2m)^2
    + 2 w1n w1m w2n w2m cos(k[(d1n - d1m) - (d2n - d2m)]), w_in = (1/d_in)/sqrt(sum_i 1/d_in^2)."""
    mics, pts, f, c = _two_mic_setup()
    A, _ = O.psf_matrix(mics, pts, f, c, O.FORM_E)
    k = 2 * math.pi * f / c
    d = np.linalg.norm(pts[:, None, :] - mics[None, :, :], axis=2)       # (S, 2)
    w = (1 / d) / np.sqrt((1 / d ** 2).sum(1, keepdims=True))
    w1, w2, d1, d2 = w[:, 0], w[:, 1], d[:, 0], d[:, 1]
    ref = ((w1[:, None] * w1[None, :]) ** 2 + (w2[:, None] * w2[None, :]) ** 2
           + 2 * w1[:, None] * w1[None, :] * w2[:, None] * w2[None, :]
           * np.cos(k * ((d1[:, None] - d1[None, :]) - (d2[:, None] - d2[None, :]))))
    np.fill_diagonal(ref, 1.0)
    assert np.abs(A - ref).max() < 1e-13


def test_psf_p_two_element_closed_form():
    """Two microphones, formulation P: PSF(r_n|r_s) = |a1 e^{jk(d1n-d1s)} + a2 e^{jk(d2n-d2s)}|^2 / 4,
    a_i = (d_in/|r_n|)(|r_s|/d_is)."""
    mics, pts, f, c = _two_mic_setup()
    A, _ = O.psf_matrix(mics, pts, f, c, O.FORM_P)
    k = 2 * math.pi * f / c
    d = np.linalg.norm(pts[:, None, :] - mics[None, :, :], axis=2)
    r = np.linalg.norm(pts, axis=1)
    tot = 0
    for i in range(2):
        a = (d[:, i][:, None] / r[:, None]) * (r[None, :] / d[:, i][None, :])
        tot = tot + a * np.exp(1j * k * (d[:, i][:, None] - d[:, i][None, :]))
    ref = np.abs(tot) ** 2 / 4
    np.fill_diagonal(ref, 1.0)
    assert np.abs(A - ref).max() < 1e-13


def test_single_microphone_psf_is_all_ones():
    mics = np.array([[0.1, -0.2, 0.0]])
    pts = synth.square_plane(5, 1.0, 1.0).points()
    A, _ = O.psf_matrix(mics, pts, 2000.0, 343.0, O.FORM_E)
    assert np.allclose(A, 1.0, atol=1e-14)


def test_far_field_shift_invariance():
    """Far from a small array the PSF depends only on the offset r_n - r_m (the
    shift-invariance assumption of spectral methods, §1); close to the array it
    does not (the case the paper's method is built for)."""
    rng = np.random.default_rng(3)
    mics = synth.mic_disc(12, 0.2, rng)
    n = lambda ix, iy: iy * 9 + ix

    def shift_err(grid):
        A, _ = O.psf_matrix(mics, grid.points(), 8000.0, 343.0, O.FORM_E)
        err = max(abs(A[n(ix, iy), n(ix + 2, iy + 1)] - A[n(ix + 1, iy + 2), n(ix + 3, iy + 3)])
                  for ix in range(4) for iy in range(4))
        return err, np.ptp(A)

    far, spread = shift_err(synth.square_plane(9, 40.0, 400.0))
    assert far < 2e-3 and spread > 0.5
    near, _ = shift_err(synth.square_plane(9, 1.0, 0.5))
    assert near > 0.05


@pytest.mark.parametrize("form", [O.FORM_E, O.FORM_P])
def test_das_of_on_grid_monopole_is_psf_column(form):
    """Eq. (9)-(11): a unit-power monopole at grid point s (noise-free CSM from the
    scene generator's own propagation model) gives b = PSF(. | r_s) = A[:, s]
    (formulation P) or ||g_s||^2 A[:, s] (formulation E)."""
    sc = synth.scene_monopole_small(seed=0, snr_db=None)
    pts = sc.grid.points()
    s = sc.extra["src_index"]
    A, g2 = O.psf_matrix(sc.mics, pts, sc.freq, sc.c, form)
    b = O.das_map(sc.mics, pts, sc.freq, sc.c, sc.C, form)
    col = A[:, s] * (g2[s] if form == O.FORM_E else 1.0)
    assert np.abs(b - col).max() <= 1e-12 * np.abs(b).max()
    assert int(np.argmax(b)) == s


def test_das_identity_csm_and_hermitian_real():
    sc = _small_scene()
    pts = sc.grid.points()
    b = O.das_map(sc.mics, pts, sc.freq, sc.c, np.eye(sc.M), O.FORM_E)
    assert np.allclose(b, 1.0, atol=1e-13)                       # e_n^H I e_n = |e_n|^2
    bp = O.das_map(sc.mics, pts, sc.freq, sc.c, np.eye(sc.M), O.FORM_P)
    d = np.linalg.norm(pts[:, None, :] - sc.mics[None, :, :], axis=2)
    r = np.linalg.norm(pts, axis=1)
    assert np.allclose(bp, ((d / r[:, None]) ** 2).sum(1) / sc.M ** 2, rtol=1e-13)
    _, bim = O.das_map(sc.mics, pts, sc.freq, sc.c, sc.C, O.FORM_E, return_imag=True)
    bre = O.das_map(sc.mics, pts, sc.freq, sc.c, sc.C, O.FORM_E)
    assert np.abs(bim).max() < 1e-12 * np.abs(bre).max()


def test_das_linear_in_csm_and_nonnegative():
    sc = _small_scene()
    pts = sc.grid.points()
    rng = np.random.default_rng(7)
    src = sc.grid.points()[rng.choice(sc.grid.S, 3)]
    C2 = synth.simulate_csm(sc.mics, src, np.array([0.3, 0.2, 0.1]), sc.freq, sc.c, None, None)
    b1 = O.das_map(sc.mics, pts, sc.freq, sc.c, sc.C)
    b2 = O.das_map(sc.mics, pts, sc.freq, sc.c, C2)
    b12 = O.das_map(sc.mics, pts, sc.freq, sc.c, sc.C + C2)
    assert np.allclose(b12, b1 + b2, rtol=1e-12)
    assert b1.min() > 0 and b2.min() >= -1e-12


def test_incoherent_superposition_equals_A_times_powers():
    """Eq. (11)-(12): for sources on grid points, b = A x with x the source powers
    (formulation E: x'_s = P_s ||g_s||^2)."""
    sc = synth.scene_monopole_small(seed=0, snr_db=None)
    pts = sc.grid.points()
    sel = np.array([17, 220, 301])
    pw = np.array([1.0, 0.4, 0.7])
    C = synth.simulate_csm(sc.mics, pts[sel], pw, sc.freq, sc.c, None, None)
    A, g2 = O.psf_matrix(sc.mics, pts, sc.freq, sc.c, O.FORM_E)
    b = O.das_map(sc.mics, pts, sc.freq, sc.c, C, O.FORM_E)
    x = np.zeros(sc.grid.S)
    x[sel] = pw * g2[sel]
    assert np.abs(A @ x - b).max() < 1e-12 * b.max()


# ----------------------------------------------------------------------------- diagonal removal (§2)
@pytest.mark.parametrize("form", [O.FORM_E, O.FORM_P])
def test_dr_map_of_uncorrelated_noise_is_zero(form):
    """Removing the CSM diagonal removes any uncorrelated (diagonal) noise exactly."""
    sc = synth.scene_monopole_small()
    rng = np.random.default_rng(7)
    C = np.diag(rng.uniform(0.1, 2.0, sc.M)).astype(complex)
    b = O.das_map(sc.mics, sc.grid.points(), sc.freq, sc.c, C, form, diag_removal=True)
    assert np.abs(b).max() == 0.0
    b_full = O.das_map(sc.mics, sc.grid.points(), sc.freq, sc.c, C, form)
    assert np.abs(b_full).min() > 0.0


@pytest.mark.parametrize("form", [O.FORM_E, O.FORM_P])
def test_dr_psf_is_the_full_psf_less_the_pair_diagonal(form):
    """The double sum over m != m' equals |sum_m conj(l_m) r_m|^2 - sum_m |l_m|^2 |r_m|^2
    (a different computation: the full PSF and an explicit correction), and its
    diagonal is 1 - sum_m |e_m|^4 (E) or 1 - 1/M (P)."""
    sc = synth.scene_monopole_small()
    pts = sc.grid.points()
    A, _ = O.psf_matrix(sc.mics, pts, sc.freq, sc.c, form)
    Ad, _ = O.psf_matrix(sc.mics, pts, sc.freq, sc.c, form, diag_removal=True)
    if form == O.FORM_E:
        L, _ = O.vectors(sc.mics, pts, sc.freq, sc.c, "e")
        R, scale = L, 1.0
    else:
        L, _ = O.vectors(sc.mics, pts, sc.freq, sc.c, "v")
        R, _ = O.vectors(sc.mics, pts, sc.freq, sc.c, "g")
        scale = 1.0 / sc.M ** 2
    corr = scale * (np.abs(L) ** 2) @ (np.abs(R) ** 2).T
    assert np.allclose(Ad, A - corr, atol=1e-12, rtol=0)
    want = 1.0 - (np.abs(L) ** 4).sum(1) if form == O.FORM_E else np.full(sc.grid.S, 1.0 - 1.0 / sc.M)
    assert np.allclose(np.diag(Ad), want, atol=1e-12, rtol=0)


def test_dr_psf_symmetric_psd_and_signed():
    """Formulation E: a Gram matrix of the pair vectors (conj(e_m) e_m')_{m != m'}, so
    symmetric PSD; unlike the full PSF it has negative entries."""
    sc = synth.scene_monopole_small()
    Ad, _ = O.psf_matrix(sc.mics, sc.grid.points(), sc.freq, sc.c, diag_removal=True)
    assert np.array_equal(Ad, Ad.T)
    assert np.linalg.eigvalsh(Ad).min() > -1e-12
    assert (Ad < 0).any()


@pytest.mark.parametrize("form", [O.FORM_E, O.FORM_P])
def test_dr_map_of_an_on_grid_monopole_is_its_psf_column(form):
    sc = synth.scene_monopole_small()
    pts = sc.grid.points()
    s = sc.grid.S // 2 + 3
    g, g2 = O.vectors(sc.mics, pts[s:s + 1], sc.freq, sc.c, "g")
    C = np.outer(g[0], np.conj(g[0]))
    b = O.das_map(sc.mics, pts, sc.freq, sc.c, C, form, diag_removal=True)
    Ad, _ = O.psf_matrix(sc.mics, pts, sc.freq, sc.c, form, diag_removal=True)
    col = Ad[:, s] * (g2[0] if form == O.FORM_E else 1.0)
    assert np.allclose(b, col, atol=1e-12 * np.abs(col).max(), rtol=0)


def test_gauss_seidel_unit_diagonal_rescaling():
    """The clamped iteration on (A, b) equals, step for step, the one on
    (D^-1/2 A D^-1/2, D^-1/2 b) with x = D^-1/2 y, D = diag(A): the update
    x_i - r_i / A_ii becomes y_i - r'_i with r' = D^-1/2 r, and x >= 0 iff y >= 0."""
    sc = synth.scene_monopole_small()
    pts = sc.grid.points()
    Ad, _ = O.psf_matrix(sc.mics, pts, sc.freq, sc.c, diag_removal=True)
    b = O.das_map(sc.mics, pts, sc.freq, sc.c, sc.C, diag_removal=True)
    d = np.sqrt(np.diag(Ad))
    x = O.gauss_seidel(Ad, b, 40)
    y = O.gauss_seidel(Ad / d[:, None] / d[None, :], b / d, 40)
    assert np.abs(x).max() > 0
    assert np.allclose(y / d, x, atol=1e-10 * np.abs(x).max(), rtol=0)
