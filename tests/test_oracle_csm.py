"""Pins of the oracle's CSM estimate from time series (Welch averaging, Eq. (1))."""
import math

import numpy as np

import oracle as O
import synth


def test_pure_tone_on_a_bin_closed_form():
    """p_m(t) = a_m cos(2 pi k0 t / K - phi_m): with the periodic Hann window the
    bin-k0 spectrum of every block is (a_m / 2) e^{-i phi_m} sum_t w (times a
    common block phase), so C = (sum w)^2 / (4 sum w^2) v v^H = (K / 6) v v^H,
    v_m = a_m e^{-i phi_m}; a bin three away holds nothing."""
    rng = np.random.default_rng(1)
    M, K, hop, T, k0 = 5, 256, 96, 256 * 12, 37
    a = rng.uniform(0.5, 2.0, M)
    phi = rng.uniform(0, 2 * math.pi, M)
    t = np.arange(T)
    p = a[:, None] * np.cos(2 * math.pi * k0 * t[None, :] / K - phi[:, None])
    C = O.csm_welch(p, K, hop, [k0, k0 + 3])
    v = a * np.exp(-1j * phi)
    assert np.allclose(C[0], (K / 6.0) * np.outer(v, v.conj()), atol=1e-9 * K, rtol=0)
    assert np.abs(C[1]).max() < 1e-9 * K


def test_hermitian_psd_and_block_count():
    rng = np.random.default_rng(2)
    p = rng.standard_normal((6, 5000))
    C = O.csm_welch(p, 512, 200, [3, 40, 255, 256])
    for Cf in C:
        assert np.allclose(Cf, Cf.conj().T, atol=1e-12)
        assert np.linalg.eigvalsh(Cf).min() > -1e-9
    # one block: C is the rank-one outer product of the windowed block's spectrum
    C1 = O.csm_welch(p[:, :512], 512, 512, [40])
    w = 0.5 - 0.5 * np.cos(2 * np.pi * np.arange(512) / 512)
    X = np.fft.fft(p[:, :512] * w, axis=1)[:, 40]
    assert np.allclose(C1[0], np.outer(X, X.conj()) / np.sum(w * w), atol=1e-12, rtol=0)


def test_monopole_noise_estimate_approaches_the_expected_csm():
    """White-noise monopole: the estimate converges to simulate_csm's expected CSM."""
    rng = np.random.default_rng(3)
    mics = synth.mic_disc(8, 0.3, rng)
    src = np.array([[0.1, -0.05, 1.0]])
    fs, K, c = 16000.0, 256, 343.0
    p = synth.simulate_timeseries(mics, src, [1.0], fs, 256 * 400, c, None, rng)
    k = 40
    C = O.csm_welch(p, K, K // 2, [k])[0]
    Ce = synth.simulate_csm(mics, src, [1.0], k * fs / K, c, None, None)
    assert np.linalg.norm(C - Ce) / np.linalg.norm(Ce) < 0.1
