"""Seeded synthetic inputs shared by the oracle-side tests, the GPU tests and the bench.

This module builds *scenes*: microphone array layouts, scan-plane grids, source
positions and powers, and the cross-spectral matrix (CSM) a free-field array
would measure from them.  It holds none of the beamforming/deconvolution
method itself (steering vectors of grid points, DAS map, PSF matrix, wavelet
compression, Gauss-Seidel): those live in the oracle and in the CUDA library,
which never import each other.

Geometry convention (paper §2, Fig. 1): the array lies in the plane z = 0 with
its centre at the origin; the scan plane is parallel to it at distance z.  A grid
point has index n = iy * nx + ix (0-based, x fastest).

Measurement model: incoherent monopoles with mean-square pressure P_s at the
array centre.  The expected CSM (§2 Eq. (1) with §3 Eq. (8)) is
C = sum_s P_s a_s a_s^H + N, where the microphone transfer vector of a source at
r_s is a_m = |r_s| / |r_s - r_m| * exp(-j k |r_s - r_m|) (free-field spherical
spreading referenced to the array centre, time convention exp(+j w t)), and N is
diagonal Gaussian self-noise N_mm = sigma^2 |z_m|^2, z_m ~ CN(0, 1), with
sigma^2 = 10^(-SNR/10) * tr(C_signal) / M.  The paper adds "Gaussian white noise
at the microphone array" (§5) without fixing its form; this diagonal form is the
reading used throughout.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SPEED_OF_SOUND = 343.0


# ----------------------------------------------------------------------------- arrays
def mic_disc(M: int, radius: float, rng: np.random.Generator) -> np.ndarray:
    """M microphones uniformly distributed over a disc of the given radius (z = 0)."""
    u = rng.random(M)
    t = rng.random(M) * 2.0 * math.pi
    r = radius * np.sqrt(u)
    return np.stack([r * np.cos(t), r * np.sin(t), np.zeros(M)], axis=1)


def mic_log_spiral(M: int, arms: int, aperture: float, spiral_deg: float = 70.0) -> np.ndarray:
    """Multi-arm logarithmic spiral: M/arms microphones per arm, radii log-spaced
    from 0.1 R to R (R = aperture / 2), arm a rotated by 2 pi a / arms, angle
    growing as cot(spiral_deg) * ln(r / r0)."""
    if M % arms:
        raise ValueError("M must be a multiple of the arm count")
    K = M // arms
    R = 0.5 * aperture
    r0 = 0.1 * R
    cot = 1.0 / math.tan(math.radians(spiral_deg))
    out = []
    for a in range(arms):
        for k in range(K):
            r = r0 * (R / r0) ** (k / (K - 1)) if K > 1 else R
            th = 2.0 * math.pi * a / arms + cot * math.log(r / r0)
            out.append((r * math.cos(th), r * math.sin(th), 0.0))
    return np.asarray(out, dtype=np.float64)


# ----------------------------------------------------------------------------- grids
@dataclass(frozen=True)
class Grid:
    """Equidistant nx x ny scan grid in the plane at distance z (paper §2)."""
    nx: int
    ny: int
    x0: float
    y0: float
    dx: float
    dy: float
    z: float

    @property
    def S(self) -> int:
        return self.nx * self.ny

    def points(self, idx=None) -> np.ndarray:
        ix = np.arange(self.nx)
        iy = np.arange(self.ny)
        X, Y = np.meshgrid(self.x0 + ix * self.dx, self.y0 + iy * self.dy)
        p = np.stack([X.ravel(), Y.ravel(), np.full(self.S, self.z)], axis=1)
        return p if idx is None else p[np.asarray(idx)]

    def point(self, ix: int, iy: int) -> np.ndarray:
        return np.array([self.x0 + ix * self.dx, self.y0 + iy * self.dy, self.z])


def square_plane(N: int, width: float, z: float) -> Grid:
    """N x N grid spanning width x width metres, centred on the array axis."""
    d = width / (N - 1)
    return Grid(N, N, -0.5 * width, -0.5 * width, d, d, z)


# ----------------------------------------------------------------------------- scene
def _transfer(mics: np.ndarray, src: np.ndarray, k: float) -> np.ndarray:
    """Free-field transfer vectors of sources (rows of src) to the microphones,
    referenced to the array centre: shape (n_src, M)."""
    diff = src[:, None, :] - mics[None, :, :]
    d = np.sqrt((diff * diff).sum(-1))
    r0 = np.sqrt((src * src).sum(-1))[:, None]
    return (r0 / d) * np.exp(-1j * k * d)


def simulate_csm(mics: np.ndarray, src_xyz: np.ndarray, powers: np.ndarray, freq: float,
                 c: float, snr_db: float | None, rng: np.random.Generator | None) -> np.ndarray:
    """Expected cross-spectral matrix of incoherent monopoles plus diagonal noise (M x M, complex128)."""
    k = 2.0 * math.pi * freq / c
    a = _transfer(np.asarray(mics, float), np.atleast_2d(np.asarray(src_xyz, float)), k)
    p = np.asarray(powers, float).reshape(-1)
    C = (a.T * p) @ a.conj()
    if snr_db is not None:
        M = mics.shape[0]
        sig2 = 10.0 ** (-snr_db / 10.0) * np.real(np.trace(C)) / M
        z = (rng.standard_normal(M) + 1j * rng.standard_normal(M)) / math.sqrt(2.0)
        C = C + np.diag(sig2 * np.abs(z) ** 2)
    return 0.5 * (C + C.conj().T)


def simulate_timeseries(mics: np.ndarray, src_xyz: np.ndarray, powers: np.ndarray, fs: float, T: int, c: float,
                        snr_db: float | None, rng: np.random.Generator) -> np.ndarray:
    """Microphone signals (M x T, float64) of incoherent monopoles emitting white
    Gaussian noise of variance powers[s] per sample, each delayed by d/c and
    scaled by |r_s|/d (the transfer of _transfer, so the expected CSM of a bin is
    simulate_csm's); the delays are applied exactly (circularly) in the frequency
    domain.  Plus white noise at snr_db below the mean signal power."""
    mics = np.asarray(mics, float)
    src = np.atleast_2d(np.asarray(src_xyz, float))
    f = np.fft.rfftfreq(T, 1.0 / fs)
    out = np.zeros((mics.shape[0], T))
    for s_xyz, pw in zip(src, np.asarray(powers, float).reshape(-1)):
        sig = np.fft.rfft(rng.standard_normal(T) * math.sqrt(pw))
        d = np.sqrt(((s_xyz[None, :] - mics) ** 2).sum(1))
        r0 = math.sqrt((s_xyz * s_xyz).sum())
        for m in range(mics.shape[0]):
            out[m] += (r0 / d[m]) * np.fft.irfft(sig * np.exp(-2j * math.pi * f * d[m] / c), T)
    if snr_db is not None:
        sig2 = 10.0 ** (-snr_db / 10.0) * float(np.mean(out * out))
        out += rng.standard_normal(out.shape) * math.sqrt(sig2)
    return out


def csm_to_f32_interleaved(C: np.ndarray) -> np.ndarray:
    """Row-major M x M complex -> float32 array (M, M, 2) holding (re, im)."""
    out = np.empty(C.shape + (2,), np.float32)
    out[..., 0] = C.real
    out[..., 1] = C.imag
    return out


# ----------------------------------------------------------------------------- configs
@dataclass
class Scene:
    """One frequency bin of one measurement: array, grid, sources and CSM."""
    name: str
    mics: np.ndarray
    grid: Grid
    freq: float
    c: float
    src_xyz: np.ndarray
    powers: np.ndarray
    C: np.ndarray
    extra: dict = field(default_factory=dict)

    @property
    def M(self) -> int:
        return self.mics.shape[0]


def _offgrid_sources(rng, n, patch, z):
    xy = (rng.random((n, 2)) - 0.5) * patch
    return np.concatenate([xy, np.full((n, 1), z)], axis=1)


def scene_monopole_small(seed: int = 0, snr_db: float | None = 20.0) -> Scene:
    """M=16 mics uniform in a 0.5 m-radius disc; 21x21 grid over 1x1 m at z=1 m
    (S=441); f=4 kHz; one unit-power monopole on the centre grid point (10, 10)."""
    rng = np.random.default_rng(seed)
    mics = mic_disc(16, 0.5, rng)
    grid = square_plane(21, 1.0, 1.0)
    src = grid.point(10, 10)[None, :]
    pw = np.array([1.0])
    C = simulate_csm(mics, src, pw, 4000.0, SPEED_OF_SOUND, snr_db, rng)
    return Scene("monopole_21x21_M16", mics, grid, 4000.0, SPEED_OF_SOUND, src, pw, C,
                 {"src_index": 10 * 21 + 10, "iters": 100})


def scene_spiral_81(seed: int = 1, snr_db: float | None = 20.0) -> Scene:
    """M=64 mics on a 4-arm log spiral of 1 m aperture; 81x81 grid over 2x2 m at
    z=2 m (S=6561); f=2 kHz; three incoherent monopoles with powers 1, 0.5, 0.25 at
    uniform-random off-grid positions in a 0.4x0.4 m patch on the axis."""
    rng = np.random.default_rng(seed)
    mics = mic_log_spiral(64, 4, 1.0)
    grid = square_plane(81, 2.0, 2.0)
    src = _offgrid_sources(rng, 3, 0.4, 2.0)
    pw = np.array([1.0, 0.5, 0.25])
    C = simulate_csm(mics, src, pw, 2000.0, SPEED_OF_SOUND, snr_db, rng)
    return Scene("spiral_81x81_M64", mics, grid, 2000.0, SPEED_OF_SOUND, src, pw, C,
                 {"iters": 1000, "levels": 2, "keep_frac": 0.10})


def band_freqs(n_bins: int = 64, f_lo: float = 1000.0, f_hi: float = 8000.0) -> np.ndarray:
    """Log-spaced analysis frequencies of a band (§6 band processing)."""
    return np.geomspace(f_lo, f_hi, n_bins)


def scene_band_121(seed: int = 2, n_bins: int = 64, snr_db: float | None = 20.0):
    """Band workload: the 64-mic spiral and 2x2 m plane at z=2 m with a 121x121
    grid (S=14641), five incoherent sources with powers log-uniform over 10 dB,
    bins log-spaced 1-8 kHz.  Returns a list of per-bin Scenes sharing geometry."""
    rng = np.random.default_rng(seed)
    mics = mic_log_spiral(64, 4, 1.0)
    grid = square_plane(121, 2.0, 2.0)
    src = _offgrid_sources(rng, 5, 0.8, 2.0)
    pw = 10.0 ** (-rng.random(5))
    out = []
    for f in band_freqs(n_bins):
        C = simulate_csm(mics, src, pw, float(f), SPEED_OF_SOUND, snr_db, rng)
        out.append(Scene(f"band_121x121_{f:.0f}Hz", mics, grid, float(f), SPEED_OF_SOUND, src, pw, C,
                         {"iters": 1000, "levels": 3}))
    return out


def scene_large_161(seed: int = 3, snr_db: float | None = 20.0) -> Scene:
    """M=128 mics on an 8-arm log spiral of 1.5 m aperture; 161x161 grid over
    3x3 m at z=1.5 m (S=25921, near field); f=6 kHz; eight incoherent sources
    with powers log-uniform over 20 dB."""
    rng = np.random.default_rng(seed)
    mics = mic_log_spiral(128, 8, 1.5)
    grid = square_plane(161, 3.0, 1.5)
    src = _offgrid_sources(rng, 8, 2.0, 1.5)
    pw = 10.0 ** (-2.0 * rng.random(8))
    C = simulate_csm(mics, src, pw, 6000.0, SPEED_OF_SOUND, snr_db, rng)
    return Scene("spiral_161x161_M128", mics, grid, 6000.0, SPEED_OF_SOUND, src, pw, C,
                 {"iters_bulk": 2000, "iters_refine": 50})


def scene_paper_image(seed: int = 4, n_src: int = 70, snr_db: float | None = 15.0) -> Scene:
    """The paper's experimental setup (§5): M = 60 microphones within a 1 m
    aperture (here a 3-arm log spiral; the layout figure is not available), scan
    plane at z0 = 5 m covering a 60 degree opening (2 z0 tan 30 deg wide), 50 x 50
    grid, f = 3 kHz, c0 = 340 m/s, 15 dB SNR; a 70-point extended "image" source
    (here a ring and a bar of unit-power incoherent monopoles standing in for the
    unavailable Case-4 pattern)."""
    rng = np.random.default_rng(seed)
    mics = mic_log_spiral(60, 3, 1.0)
    width = 2.0 * 5.0 * math.tan(math.radians(30.0))
    grid = square_plane(50, width, 5.0)
    n_ring = n_src * 3 // 5
    t = np.arange(n_ring) * 2.0 * math.pi / n_ring
    ring = np.stack([-0.6 + 0.45 * np.cos(t), 0.3 + 0.45 * np.sin(t)], axis=1)
    n_bar = n_src - n_ring
    bar = np.stack([np.linspace(0.3, 1.2, n_bar), np.full(n_bar, -0.6)], axis=1)
    xy = np.concatenate([ring, bar]) + 0.01 * (rng.random((n_src, 2)) - 0.5)
    src = np.concatenate([xy, np.full((n_src, 1), 5.0)], axis=1)
    pw = np.ones(n_src)
    C = simulate_csm(mics, src, pw, 3000.0, 340.0, snr_db, rng)
    return Scene("paper_image_50x50_M60", mics, grid, 3000.0, 340.0, src, pw, C, {"levels": 5, "iters": 1000})


def scene_random(rng: np.random.Generator, M: int, N: int, n_src: int, freq: float,
                 width: float = 2.0, z: float = 2.0, snr_db: float | None = 20.0) -> Scene:
    """A random request-sized scene (spiral array, N x N plane, off-grid sources)."""
    arms = 4 if M <= 64 else 8
    mics = mic_log_spiral(M, arms, 1.0)
    grid = square_plane(N, width, z)
    src = _offgrid_sources(rng, n_src, 0.5 * width, z)
    pw = 10.0 ** (-rng.random(n_src))
    C = simulate_csm(mics, src, pw, freq, SPEED_OF_SOUND, snr_db, rng)
    return Scene(f"req_M{M}_N{N}_{freq:.0f}Hz", mics, grid, freq, SPEED_OF_SOUND, src, pw, C)


def serve_requests(seed: int = 5, n: int = 64, rate_hz: float = 200.0):
    """Poisson request stream: arrival times plus per-request (M, N, bins, keep
    fraction, source count), drawn as the serving workload describes."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, n))
    reqs = []
    for i in range(n):
        reqs.append({
            "t_arrive": float(t[i]),
            "M": int(rng.choice([32, 64, 128])),
            "N": int(rng.choice([41, 81, 121, 161])),
            "n_bins": int(rng.integers(1, 33)),
            "f_lo": 1000.0, "f_hi": 10000.0,
            "keep_frac": float(rng.uniform(0.02, 0.30)),
            "n_src": int(rng.integers(1, 7)),
            "seed": int(rng.integers(0, 2**31 - 1)),
        })
    return reqs


def random_psd_system(rng: np.random.Generator, S: int, rank: int | None = None):
    """A random symmetric positive semi-definite matrix with unit diagonal and
    non-negative entries (a normalised Gram matrix of non-negative random rows),
    plus a right-hand side b = A x_true with sparse non-negative x_true.  Plain
    linear algebra on random draws, used only as a solver input."""
    rank = rank or max(2, S // 2)
    Y = rng.random((S, rank)) ** 4
    Y /= np.linalg.norm(Y, axis=1, keepdims=True)
    A = Y @ Y.T
    np.fill_diagonal(A, 1.0)
    x_true = np.zeros(S)
    nz = rng.choice(S, size=max(1, S // 8), replace=False)
    x_true[nz] = rng.random(nz.size)
    b = A @ x_true
    return A, b
