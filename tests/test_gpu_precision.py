"""Storage precision of A (BF16 bulk sweeps + FP32 refinement) against the FP64 oracle.

The iteration's solution set is not a point (A is singular), so two runs whose
A differ in rounding follow different paths through it; what stays put is the
power the map assigns to each source region.  The test compares that power, in
dB, per source, on the 161x161 near-field scene compressed to about 10% of its
points (the oracle's selection is used on both sides)."""
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


def region_power_db(x_full, grid, src_xyz, radius):
    pts = grid.points()
    out = []
    for s in src_xyz:
        m = np.linalg.norm(pts[:, :2] - s[None, :2], axis=1) <= radius
        out.append(10 * np.log10(max(x_full[m].sum(), 1e-30)))
    return np.array(out)


def test_bf16_bulk_with_fp32_refinement_per_source_db(ctx):
    sc = synth.scene_large_161()
    pts = sc.grid.points()
    b = O.das_map(sc.mics, pts, sc.freq, sc.c, sc.C)
    idx, _, _, _ = O.wavelet_select(b.astype(np.float32), 161, 161, 5, O.PRED_LINEAR, O.EPS_KEEP_FRAC, 0.10)
    A64, g2 = O.psf_matrix(sc.mics, pts[idx], sc.freq, sc.c)
    T = 400
    x_orc = O.to_power(O.gauss_seidel(A64, b[idx], T), g2)
    S = len(idx)
    geom = D.Geometry.from_scene(sc.mics, sc.grid, sc.c)
    it = torch.as_tensor(idx, device="cuda")
    A32, g2d = D.damas_build_psf(ctx, geom, sc.freq, it, S)
    Abf, _ = D.damas_build_psf(ctx, geom, sc.freq, it, S, a_dtype=D.BF16)
    bt = torch.as_tensor(b[idx].astype(np.float32), device="cuda")
    runs = {}
    for name, (nb, nr) in {"fp32": (0, T), "bf16": (T, 0), "bf16+fp32": (T - 50, 50)}.items():
        x = torch.zeros(S, device="cuda")
        D.solve_mixed(ctx, Abf, A32, bt, x, nb, nr)
        runs[name] = O.scatter(x.cpu().numpy() / g2d.cpu().numpy(), idx, sc.grid.S)
    beam = 1.22 * 1.5 * sc.c / (1.5 * sc.freq)      # Rayleigh beamwidth at the plane (§5), z0 = D = 1.5 m
    ref = region_power_db(O.scatter(x_orc, idx, sc.grid.S), sc.grid, sc.src_xyz, beam / 2)
    err = {k: np.abs(region_power_db(v, sc.grid, sc.src_xyz, beam / 2) - ref) for k, v in runs.items()}
    print("per-source |dB error| vs FP64 oracle:", {k: np.round(v, 3).tolist() for k, v in err.items()})
    assert err["fp32"].max() <= 0.05, err["fp32"]
    assert err["bf16+fp32"].max() <= 0.5, err["bf16+fp32"]
    assert err["bf16+fp32"].max() <= err["bf16"].max() + 1e-6


def _padded(A64, dtype):
    S = A64.shape[0]
    out = np.zeros((S, D.damas_lda(S)), np.float32)
    out[:, :S] = A64
    return torch.as_tensor(out, device="cuda").to(dtype)


@pytest.mark.parametrize("nb,nr", [(300, 50), (0, 120), (200, 0)])
def test_solve_mixed_in_one_call_equals_the_two_solves(ctx, nb, nr):
    """damas_solve_mixed through the C ABI, two systems in one call, against the
    two damas_solve calls it stands for (BF16 from zero, then FP32 from the
    exact residual): bit for bit."""
    import ctypes
    from paper_1608_05179_gb300 import _lib
    lib = _lib.load()
    systems = [synth.random_psd_system(np.random.default_rng(s), S) for s, S in ((1, 300), (2, 701))]
    ms, xs, refs = [], [], []
    for A64, b64 in systems:
        A32, Abf = _padded(A64, torch.float32), _padded(A64, torch.bfloat16)
        b = torch.as_tensor(b64.astype(np.float32), device="cuda")
        x = torch.full((len(b64),), 3.0, device="cuda")
        ms.append(_lib.damas_mixed_system(Abf.data_ptr(), None, A32.data_ptr(), None, A32.shape[1], len(b64),
                                          b.data_ptr(), x.data_ptr(), nb, nr, 0))
        xs.append((x, A32, Abf, b))
        xr = torch.zeros(len(b64), device="cuda")
        if nb:
            D.damas_solve(ctx, D.System(Abf, b, xr, nb, init=D.INIT_ZERO))
        if nr or not nb:
            D.damas_solve(ctx, D.System(A32, b, xr, nr, init=D.INIT_X if nb else D.INIT_ZERO))
        refs.append(xr)
    arr = (_lib.damas_mixed_system * 2)(*ms)
    rc = lib.damas_solve_mixed(ctx.handle, arr, 2, None, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, lib.damas_last_error(ctx.handle)
    for (x, *_), xr in zip(xs, refs):
        assert torch.equal(x, xr)
    # the binding (one system) gives the same
    x, A32, Abf, b = xs[0]
    x2 = torch.zeros_like(x)
    D.solve_mixed(ctx, Abf, A32, b, x2, nb, nr)
    assert torch.equal(x2, refs[0])


def test_psf_in_both_storage_types_equals_the_two_builds(ctx):
    """damas_build_psf_f32_bf16: the FP32 matrix of damas_build_psf(F32) and the BF16
    matrix of damas_build_psf(BF16), bit for bit, from one build (ragged size)."""
    sc = synth.scene_spiral_81()
    geom = D.Geometry.from_scene(sc.mics, sc.grid, sc.c)
    idx = torch.as_tensor(np.arange(5, 6561, 9, dtype=np.int32), device="cuda")    # 729 points
    A32, g2 = D.damas_build_psf(ctx, geom, sc.freq, idx, int(idx.numel()))
    Abf, _ = D.damas_build_psf(ctx, geom, sc.freq, idx, int(idx.numel()), a_dtype=D.BF16)
    B32, Bbf, h2 = D.damas_build_psf_f32_bf16(ctx, geom, sc.freq, idx)
    torch.cuda.synchronize()
    assert torch.equal(A32, B32) and torch.equal(g2, h2)
    assert torch.equal(Abf.view(torch.int16), Bbf.view(torch.int16))
