"""The allocation-free compressed-grid entry point (wavelet_compress_grid_noalloc).

It exists for callers that cannot allocate device memory when they need a
compressed grid (real-time threads, plug-ins confined to memory their host
application gave them, fixed device-memory budgets).  Through the C ABI it must
give exactly the results of wavelet_compress_grid, on consecutive calls that
share its fixed work array, and refuse grids larger than that array.  The file
is named to be collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

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


def _maps():
    rng = np.random.default_rng(21)
    sc = synth.scene_spiral_81()
    # a DAS-like smooth map and a rough one; the second call must not see the first's leftovers
    iy, ix = np.mgrid[0:81, 0:81]
    smooth = np.exp(-((ix - 40.3) ** 2 + (iy - 38.7) ** 2) / 90.0).astype(np.float32) + np.float32(0.01)
    rough = rng.random((97, 113)).astype(np.float32)
    return [(smooth.reshape(-1), 81, 81, 2, D.PRED_HAAR, D.EPS_KEEP_FRAC, 0.10),
            (rough.reshape(-1), 113, 97, 3, D.PRED_LINEAR, D.EPS_REL_MAX, 0.05)], sc


def _outputs(n_pts):
    return (torch.full((n_pts,), -7, dtype=torch.int32, device="cuda"),
            torch.full((1,), -7, dtype=torch.int32, device="cuda"),
            torch.full((n_pts,), float("nan"), dtype=torch.float32, device="cuda"),
            torch.full((1,), float("nan"), dtype=torch.float32, device="cuda"))


def test_noalloc_matches_context_entry_point_on_two_calls(ctx):
    cases, _ = _maps()
    for b, nx, ny, L, pred, mode, eps in cases:
        bt = torch.as_tensor(b, device="cuda")
        ref = _outputs(nx * ny)
        D.wavelet_compress_grid(ctx, bt, nx, ny, L, pred, mode, eps, *ref)
        got = _outputs(nx * ny)
        D.wavelet_compress_grid_noalloc(ctx, bt, nx, ny, L, pred, mode, eps, *got)
        torch.cuda.synchronize()
        n = int(ref[1].item())
        assert int(got[1].item()) == n
        assert torch.equal(got[0][:n], ref[0][:n])
        assert torch.equal(got[2].view(torch.int32), ref[2].view(torch.int32))
        assert torch.equal(got[3].view(torch.int32), ref[3].view(torch.int32))


def test_noalloc_rejects_grids_beyond_its_work_array(ctx):
    from paper_1608_05179_gb300 import _lib
    lib = _lib.load()
    nx, ny = 1024, 257                                    # 263168 points > 262144
    b = torch.zeros(nx * ny, device="cuda")
    idx = torch.empty(nx * ny, dtype=torch.int32, device="cuda")
    cnt = torch.empty(1, dtype=torch.int32, device="cuda")
    cfg = _lib.damas_wavelet_cfg(3, D.PRED_LINEAR, D.EPS_ABS, 0.1)
    rc = lib.wavelet_compress_grid_noalloc(ctx.handle, ctypes.c_void_p(b.data_ptr()), nx, ny, ctypes.byref(cfg),
                                           ctypes.c_void_p(idx.data_ptr()), ctypes.c_void_p(cnt.data_ptr()),
                                           None, None, None)
    assert rc == _lib.DAMAS_EINVAL
    assert b"allocation-free" in lib.damas_last_error(ctx.handle)


def test_noalloc_has_the_limits_of_the_context_entry_point(ctx):
    """A 262144 x 1 grid fits the work array, but a side above 65535 is refused by
    both entry points alike."""
    from paper_1608_05179_gb300 import _lib
    lib = _lib.load()
    nx, ny = 262144, 1
    b = torch.zeros(nx * ny, device="cuda")
    idx = torch.empty(nx * ny, dtype=torch.int32, device="cuda")
    cnt = torch.empty(1, dtype=torch.int32, device="cuda")
    cfg = _lib.damas_wavelet_cfg(1, D.PRED_LINEAR, D.EPS_ABS, 0.1)
    args = (ctx.handle, ctypes.c_void_p(b.data_ptr()), nx, ny, ctypes.byref(cfg), ctypes.c_void_p(idx.data_ptr()),
            ctypes.c_void_p(cnt.data_ptr()), None, None, None)
    assert lib.wavelet_compress_grid(*args) == _lib.DAMAS_EINVAL
    assert lib.wavelet_compress_grid_noalloc(*args) == _lib.DAMAS_EINVAL
    assert b"65535" in lib.damas_last_error(ctx.handle)
