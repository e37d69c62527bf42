"""GPU neighbour padding of compressed grids against the oracle: bit-exact index
sets and counts over grid shapes, radii, repeats, out-of-range entries, clamped
counts and in-place output; then the padded pipeline on the 81x81 scene."""
import numpy as np
import pytest
import torch

import oracle as O
import synth

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


def _gpu_pad(ctx, idx, nx, ny, r, count=None, inplace=False):
    cap = max(nx * ny, len(idx), 1)
    buf = torch.zeros(cap, dtype=torch.int32, device="cuda")
    if len(idx):
        buf[: len(idx)] = torch.as_tensor(np.asarray(idx, np.int32), device="cuda")
    n = torch.tensor([len(idx) if count is None else count], dtype=torch.int32, device="cuda")
    out = buf if inplace else None
    o, m = D.damas_pad_grid(ctx, buf, n, nx, ny, r, out_idx=out)
    torch.cuda.synchronize()
    k = int(m.item())
    return o[:k].cpu().numpy()


@pytest.mark.parametrize("nx,ny", [(1, 1), (1, 37), (29, 1), (21, 21), (50, 50), (81, 81), (161, 161), (200, 33)])
@pytest.mark.parametrize("r", [0, 1, 3])
def test_pad_matches_oracle(ctx, nx, ny, r):
    rng = np.random.default_rng(nx * 1000 + ny * 10 + r)
    S = nx * ny
    k = max(1, S // 15)
    idx = rng.choice(S, min(k, S), replace=False).astype(np.int32)
    np.testing.assert_array_equal(_gpu_pad(ctx, idx, nx, ny, r), O.pad_grid(idx, nx, ny, r))


def test_pad_edge_cases(ctx):
    nx, ny = 19, 13
    S = nx * ny
    # empty input
    assert _gpu_pad(ctx, [], nx, ny, 2).size == 0
    # every point, large radius: the whole grid
    np.testing.assert_array_equal(_gpu_pad(ctx, np.arange(S), nx, ny, 8), np.arange(S))
    # repeats and unsorted input, corners
    idx = np.array([S - 1, 0, 0, nx - 1, S - nx, 100, 100], np.int32)
    for r in (0, 1, 2):
        np.testing.assert_array_equal(_gpu_pad(ctx, idx, nx, ny, r), O.pad_grid(idx, nx, ny, r))
    # entries outside the grid are ignored
    idx = np.array([-7, 5, S, S + 100, 40], np.int32)
    np.testing.assert_array_equal(_gpu_pad(ctx, idx, nx, ny, 1), O.pad_grid(idx, nx, ny, 1))
    # a count above the capacity of the grid is clamped to nx*ny, a negative one to 0
    idx = np.arange(S, dtype=np.int32)[::7]
    assert _gpu_pad(ctx, idx, nx, ny, 0, count=-3).size == 0
    full = np.concatenate([idx, np.zeros(S - len(idx), np.int32)])   # the buffer beyond the list holds zeros
    np.testing.assert_array_equal(_gpu_pad(ctx, idx, nx, ny, 1, count=S + 50), O.pad_grid(full, nx, ny, 1))
    # in place
    idx = np.array([3, 77, 150], np.int32)
    np.testing.assert_array_equal(_gpu_pad(ctx, idx, nx, ny, 2, inplace=True), O.pad_grid(idx, nx, ny, 2))


def test_pad_rejects_bad_arguments(ctx):
    idx = torch.zeros(16, dtype=torch.int32, device="cuda")
    n = torch.ones(1, dtype=torch.int32, device="cuda")
    for args in [(4, 4, -1), (4, 4, 9), (0, 4, 1), (70000, 1, 1)]:
        with pytest.raises(D.DamasError) as ei:
            D.damas_pad_grid(ctx, idx, n, *args)
        assert ei.value.code == P._lib.DAMAS_EINVAL


def test_padded_pipeline_81x81(ctx):
    """Compressed grid of the 81x81 scene (Haar L=2, keep 10%), padded by one
    point, through the PSF and 1000 sweeps: the padded set is the oracle's
    padding of the GPU's own selection, and the integrated power agrees with the
    oracle run on that set."""
    sc = synth.scene_spiral_81()
    g = D.Geometry.from_scene(sc.mics, sc.grid, sc.c)
    C = D.csm_tensor(sc.C)
    plain = D.solve_bin(ctx, g, sc.freq, C, 10, compressed=True, levels=2, eps=0.1)
    out = D.solve_bin(ctx, g, sc.freq, C, 1000, compressed=True, levels=2, eps=0.1, pad_radius=1)
    torch.cuda.synchronize()
    sel = plain["idx"].cpu().numpy()
    want = O.pad_grid(sel, 81, 81, 1)
    np.testing.assert_array_equal(out["idx"].cpu().numpy(), want)
    assert out["S_sub"] > plain["S_sub"]
    pts = sc.grid.points()
    A, g2 = O.psf_matrix(sc.mics, pts[want], sc.freq, sc.c)
    b = O.das_map(sc.mics, pts, sc.freq, sc.c, sc.C)
    x = O.gauss_seidel(A, b[want], 1000)
    tot = float(np.sum(O.to_power(x, g2)))
    assert abs(out["total_power"].item() - tot) <= 2e-3 * tot
