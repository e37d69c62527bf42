"""Oracle: plain FP64 CPU implementation of the DAMAS-on-a-compressed-grid hot path.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's CPU
baseline leg may import this package; the CUDA library never does, and the two
share no code.  The arithmetic lives in damas_oracle.c (built by oracle.build);
this module marshals numpy arrays into it and adds the small pieces that are
plain numpy (restriction, scatter, integrated power, KKT residual, objective).

Paper equations are numbered in order of appearance:
(2) DAS map, (4) steering v, (7) propagation g, (10) PSF, (12) Ax=b,
(13)-(14) Gauss-Seidel with clamp, (15) nested grids, (22) compressed grid,
(23) interpolating wavelet coefficient, (24) compressed system; Algorithm 1.

Formulations of the PSF matrix:
  E (default): e_n = g_n / ||g_n||, A_nm = |e_n^H e_m|^2, b_n = Re(e_n^H C e_n);
     A is symmetric, PSD, unit diagonal.  The solution x' is in units of
     power * ||g_n||^2; the power map is x_n = x'_n / ||g_n||^2.
  P: the paper's literal v (Eq. (4)) and g (Eq. (7)): A_ns = |v_n^H g_s|^2 / M^2,
     b_n = Re(v_n^H C v_n) / M^2; unit diagonal, not symmetric.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import build as _build

FORM_E = 0
FORM_P = 1
PRED_LINEAR = 0
PRED_HAAR = 1
EPS_ABS = 0
EPS_REL_MAX = 1
EPS_KEEP_FRAC = 2

_VEC_G, _VEC_V, _VEC_E = 0, 1, 2

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        fp = ctypes.POINTER(ctypes.c_float)
        ip = ctypes.POINTER(ctypes.c_int32)
        bp = ctypes.POINTER(ctypes.c_int8)
        lib.orc_vectors.argtypes = [ctypes.c_int, dp, ctypes.c_int, dp, ctypes.c_double, ctypes.c_int, dp, dp, dp]
        lib.orc_psf.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, ctypes.c_double, dp, ctypes.c_int]
        lib.orc_das.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, ctypes.c_double, dp, dp]
        lib.orc_das_dr.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, ctypes.c_double, dp]
        lib.orc_psf_dr.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, ctypes.c_double, dp, ctypes.c_int]
        lib.orc_gauss_seidel.argtypes = [ctypes.c_int, dp, ctypes.c_int, dp, dp, ctypes.c_int]
        lib.orc_wavelet_select.argtypes = [ctypes.c_int, ctypes.c_int, fp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_double, ip, fp, bp, fp]
        lib.orc_wavelet_select.restype = ctypes.c_int
        for f in (lib.orc_vectors, lib.orc_psf, lib.orc_das, lib.orc_gauss_seidel, lib.orc_das_dr, lib.orc_psf_dr):
            f.restype = None
        _lib = lib
    return _lib


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def wavenumber(freq: float, c: float) -> float:
    """k = omega / c0 (§2)."""
    return 2.0 * math.pi * freq / c


def vectors(mics, pts, freq, c, kind: str):
    """Vectors of each point towards the microphones: kind 'g' (Eq. (7)),
    'v' (Eq. (4)) or 'e' (g normalised).  Returns (S, M) complex128 and ||g||^2."""
    lib = _load()
    mics = _c64(mics)
    pts = _c64(pts)
    M, S = mics.shape[0], pts.shape[0]
    re = np.empty((S, M))
    im = np.empty((S, M))
    g2 = np.empty(S)
    code = {"g": _VEC_G, "v": _VEC_V, "e": _VEC_E}[kind]
    lib.orc_vectors(M, _d(mics), S, _d(pts), wavenumber(freq, c), code, _d(re), _d(im), _d(g2))
    return re + 1j * im, g2


def psf_matrix(mics, pts, freq, c, form: int = FORM_E, diag_removal: bool = False):
    """A (S x S, FP64) of Eq. (10)/(12) with unit diagonal; also ||g_n||^2.
    diag_removal: the PSF without the m = m' microphone pairs (orc_psf_dr); its
    diagonal is then computed, not 1."""
    lib = _load()
    M = np.asarray(mics).shape[0]
    if form == FORM_E:
        L, g2 = vectors(mics, pts, freq, c, "e")
        R, scale = L, 1.0
    else:
        L, g2 = vectors(mics, pts, freq, c, "v")
        R, _ = vectors(mics, pts, freq, c, "g")
        scale = 1.0 / (M * M)
    S = L.shape[0]
    A = np.empty((S, S))
    lre, lim = _c64(L.real), _c64(L.imag)
    rre, rim = _c64(R.real), _c64(R.imag)
    if diag_removal:
        lib.orc_psf_dr(S, M, _d(lre), _d(lim), _d(rre), _d(rim), scale, _d(A), S)
    else:
        lib.orc_psf(S, M, _d(lre), _d(lim), _d(rre), _d(rim), scale, _d(A), S)
    return A, g2


def das_map(mics, pts, freq, c, C, form: int = FORM_E, return_imag: bool = False, diag_removal: bool = False):
    """DAS map b of Eq. (2) (FP64); diag_removal: without the CSM diagonal (orc_das_dr)."""
    lib = _load()
    M = np.asarray(mics).shape[0]
    if form == FORM_E:
        L, _ = vectors(mics, pts, freq, c, "e")
        scale = 1.0
    else:
        L, _ = vectors(mics, pts, freq, c, "v")
        scale = 1.0 / (M * M)
    S = L.shape[0]
    Ci = np.empty((M, M, 2))
    Ci[..., 0] = np.real(C)
    Ci[..., 1] = np.imag(C)
    b = np.empty(S)
    bi = np.empty(S)
    lre, lim = _c64(L.real), _c64(L.imag)
    if diag_removal:
        lib.orc_das_dr(S, M, _d(lre), _d(lim), _d(Ci), scale, _d(b))
        bi[:] = 0.0
    else:
        lib.orc_das(S, M, _d(lre), _d(lim), _d(Ci), scale, _d(b), _d(bi))
    return (b, bi) if return_imag else b


def csm_welch(p, K: int, hop: int, bins):
    """Cross-spectral matrix (Eq. (1)) of each FFT bin in `bins` estimated from
    microphone time series p (M x T, FP64): blocks of K samples every `hop`
    samples, periodic Hann window w, averaged over the L = (T - K) // hop + 1
    blocks (Welch):
        C_f = sum_l X_lf X_lf^H / (L * sum_t w(t)^2),
        X_lf[m] = sum_t w(t) p[m, l*hop + t] exp(-2 pi i f t / K).
    The FFT is numpy's (a library primitive used as one step)."""
    p = np.asarray(p, np.float64)
    M, T = p.shape
    L = (T - K) // hop + 1
    w = 0.5 - 0.5 * np.cos(2.0 * np.pi * np.arange(K) / K)
    bins = np.asarray(bins, int)
    C = np.zeros((len(bins), M, M), complex)
    for l in range(L):
        X = np.fft.fft(p[:, l * hop:l * hop + K] * w, axis=1)[:, bins]   # M x F
        for i in range(len(bins)):
            C[i] += np.outer(X[:, i], X[:, i].conj())
    return C / (L * np.sum(w * w))


def gauss_seidel(A, b, iters: int, x0=None):
    """DAMAS Gauss-Seidel with the non-negativity clamp, Eq. (13)-(14), FP64."""
    lib = _load()
    A = _c64(A)
    b = _c64(b)
    S = b.shape[0]
    x = np.zeros(S) if x0 is None else _c64(x0).copy()
    lib.orc_gauss_seidel(S, _d(A), A.shape[1], _d(b), _d(x), int(iters))
    return x


def wavelet_select(b, nx: int, ny: int, levels: int, predictor: int = PRED_HAAR,
                   eps_mode: int = EPS_REL_MAX, eps: float = 0.1):
    """Algorithm 1 on the FP32 map b.  Returns (idx int32 ascending, detail,
    level, eps_abs) with detail = interpolated - actual (FP32, 0 on G^0) and
    level 0 on G^0, j+1 on G^{j+1} minus G^j."""
    lib = _load()
    bf = np.ascontiguousarray(np.asarray(b, dtype=np.float32).reshape(-1))
    S = nx * ny
    if bf.size != S:
        raise ValueError("b has the wrong size")
    idx = np.empty(S, np.int32)
    ad = np.empty(S, np.float32)
    lv = np.empty(S, np.int8)
    ea = np.empty(1, np.float32)
    n = lib.orc_wavelet_select(nx, ny, bf.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), int(levels),
                               int(predictor), int(eps_mode), float(eps),
                               idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                               ad.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                               lv.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)),
                               ea.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    return idx[:n].copy(), ad, lv, float(ea[0])


def default_levels(N: int) -> int:
    """Largest L <= floor(log2 N) with 2^L dividing N - 1 (every coarse
    neighbour then exists); the paper's own choice is floor(log2 N)."""
    J = int(math.floor(math.log2(N)))
    for L in range(J, 0, -1):
        if (N - 1) % (1 << L) == 0:
            return L
    return 1


def pad_grid(idx, nx: int, ny: int, radius: int):
    """Neighbour padding of a compressed grid (an extension of Algorithm 1 aimed
    at the aliasing §5 reports on the compressed grid): every grid point within
    Chebyshev distance radius of a listed point, ascending.  Entries outside the
    grid are ignored.  Plain loops over the listed points and the offsets."""
    S = nx * ny
    keep = np.zeros(S, dtype=bool)
    for p in np.asarray(idx, dtype=np.int64).ravel():
        if p < 0 or p >= S:
            continue
        ix, iy = int(p) % nx, int(p) // nx
        for dy in range(-radius, radius + 1):
            for dx in range(-radius, radius + 1):
                x, y = ix + dx, iy + dy
                if 0 <= x < nx and 0 <= y < ny:
                    keep[y * nx + x] = True
    return np.nonzero(keep)[0].astype(np.int32)


# ----------------------------------------------------------------------------- numpy helpers
def restrict(b, idx):
    """b~ = b[idx] (Eq. (24))."""
    return np.asarray(b)[np.asarray(idx)]


def scatter(x_sub, idx, S):
    """Compressed-grid solution back onto the full grid, zero elsewhere (§5)."""
    out = np.zeros(S)
    out[np.asarray(idx)] = x_sub
    return out


def to_power(x, gnorm2, form: int = FORM_E):
    """Power map: x_n = x'_n / ||g_n||^2 under formulation E, unchanged under P."""
    return np.asarray(x) / np.asarray(gnorm2) if form == FORM_E else np.asarray(x)


def objective(A, b, x):
    """0.5 x^T A x - b^T x: the quadratic the clamped Gauss-Seidel descends for symmetric PSD A."""
    return 0.5 * x @ (A @ x) - b @ x


def kkt_residual(A, b, x):
    """Largest violation of the complementarity conditions of the clamped
    iteration's fixed points: x >= 0, (Ax - b)_n = 0 where x_n > 0,
    (Ax - b)_n >= 0 where x_n = 0."""
    g = A @ x - b
    pos = x > 0
    v1 = np.abs(g[pos]).max() if pos.any() else 0.0
    v2 = (-g[~pos]).clip(min=0).max() if (~pos).any() else 0.0
    v3 = (-x).clip(min=0).max()
    return max(v1, v2, v3)


def solve_bin(mics, grid, freq, c, C, iters, compressed: bool, levels=None,
              predictor=PRED_HAAR, eps_mode=EPS_KEEP_FRAC, eps=0.1, form=FORM_E, b_f32=None, pad_radius=0):
    """One frequency bin end to end (§5 procedure): DAS map, optional wavelet
    compression (Algorithm 1), PSF matrix on the kept points, Gauss-Seidel from
    x^0 = 0, scatter to the full grid and convert to power.  b_f32, when given,
    is the FP32 map the grid selection is taken from (the selection is an FP32
    decision); otherwise the FP64 map rounded to FP32 is used.  pad_radius > 0
    adds the neighbours of the kept points (pad_grid)."""
    pts = grid.points()
    b = das_map(mics, pts, freq, c, C, form)
    if compressed:
        bsel = np.asarray(b, np.float32) if b_f32 is None else np.asarray(b_f32, np.float32)
        L = default_levels(grid.nx) if levels is None else levels
        idx, _, _, eps_abs = wavelet_select(bsel, grid.nx, grid.ny, L, predictor, eps_mode, eps)
        if pad_radius:
            idx = pad_grid(idx, grid.nx, grid.ny, pad_radius)
    else:
        idx, eps_abs = np.arange(grid.S, dtype=np.int32), None
    A, g2 = psf_matrix(mics, pts[idx], freq, c, form)
    x_sub = gauss_seidel(A, b[idx], iters)
    x_full = scatter(to_power(x_sub, g2, form), idx, grid.S)
    return {"b": b, "idx": idx, "A": A, "gnorm2": g2, "x_sub": x_sub, "x": x_full, "eps_abs": eps_abs}
