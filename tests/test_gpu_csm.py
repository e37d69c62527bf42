"""CSM estimate from time series (Welch) through the C-ABI against the oracle,
and the acquisition-to-map path: time series -> CSM -> DAS map -> DAMAS."""
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


def _series(M, T, seed=0, snr_db=20.0):
    rng = np.random.default_rng(seed)
    mics = synth.mic_log_spiral(M, 4 if M % 4 == 0 else 1, 1.0) if M >= 8 else synth.mic_disc(M, 0.5, rng)
    src = np.array([[0.2, -0.1, 1.5], [-0.3, 0.25, 1.5]])
    p = synth.simulate_timeseries(mics, src, [1.0, 0.5], 16000.0, T, 343.0, snr_db, rng)
    return mics, src, p


@pytest.mark.parametrize("M,K,hop,T,bins", [
    (16, 512, 256, 512 * 100, [16, 40, 64, 100, 128, 200, 255, 256]),
    (100, 256, 100, 256 * 60, list(range(3, 3 + 70))),          # ragged tiles on both kernels
    (8, 1024, 1024, 1024 * 4, [0, 1, 511, 512]),                 # no overlap; DC and Nyquist bins
])
def test_csm_matches_oracle(ctx, M, K, hop, T, bins):
    _, _, p = _series(M, T)
    pt = torch.as_tensor(p.astype(np.float32), device="cuda")
    bt = torch.as_tensor(np.array(bins, np.int32), device="cuda")
    C = D.damas_csm(ctx, pt, K, hop, bt)
    torch.cuda.synchronize()
    Cg = C.cpu().numpy()
    Cg = Cg[..., 0].astype(np.float64) + 1j * Cg[..., 1]
    Co = O.csm_welch(p.astype(np.float32).astype(np.float64), K, hop, bins)
    err = np.abs(Cg - Co).max() / np.abs(Co).max()
    print(f"[csm] M={M} K={K}: max |dC| / max |C| = {err:.2e}")
    assert err <= 2e-5
    assert np.array_equal(Cg, np.conj(np.transpose(Cg, (0, 2, 1))))   # exactly Hermitian


def test_acquisition_to_map(ctx):
    """A monopole's time series through the whole path finds its grid point."""
    rng = np.random.default_rng(5)
    mics = synth.mic_log_spiral(32, 4, 1.0)
    grid = synth.square_plane(41, 1.6, 1.5)
    s = 17 * 41 + 25
    src = grid.points()[s:s + 1]
    fs, K = 16000.0, 512
    p = synth.simulate_timeseries(mics, src, [1.0], fs, K * 200, 343.0, 25.0, rng)
    kbin = 96                                         # 3 kHz
    C = D.damas_csm(ctx, torch.as_tensor(p.astype(np.float32), device="cuda"), K, K // 2,
                    torch.tensor([kbin], dtype=torch.int32, device="cuda"))
    geom = D.Geometry.from_scene(mics, grid, 343.0)
    out = D.solve_bin(ctx, geom, kbin * fs / K, C[0], 300, compressed=True, levels=3, eps=0.15)
    x = out["x"].cpu().numpy()
    assert int(np.argmax(x)) == s
    assert 0.7 < float(out["total_power"].item()) < 1.3
