"""The C ABI refuses, with DAMAS_EINVAL and before any launch, device pointers that
its kernels could not use: A (and At) not 16-byte aligned for the solver's TMA
and vector reads, complex matrices not 8-byte aligned, and the two outputs of the
dual-storage PSF build overlapping.  Every case is host-side validation only; a
valid call on the same context afterwards still works and gives the usual result."""
import ctypes

import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

D = pytest.importorskip("paper_1608_05179_gb300").damas
L = pytest.importorskip("paper_1608_05179_gb300")._lib


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = D.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def small():
    sc = synth.scene_monopole_small()
    return sc


def _einval(ctx, rc):
    assert rc == L.DAMAS_EINVAL, rc
    assert ctx.lib.damas_last_error(ctx.handle)


def test_solve_rejects_misaligned_matrix(ctx, small):
    g = D.Geometry.from_scene(small.mics, small.grid, small.c)
    b = D.das_map(ctx, g, small.freq, D.csm_tensor(small.C))
    A, _ = D.damas_build_psf(ctx, g, small.freq)
    S = small.grid.S
    x = torch.zeros(S, device="cuda")
    for shift_A, shift_x in ((4, 0), (8, 0), (0, 2)):
        st = D.System(A, b, x, 10).cstruct()
        st.A_dev = A.data_ptr() + shift_A
        st.x_dev = x.data_ptr() + shift_x
        arr = (L.damas_system * 1)(st)
        _einval(ctx, ctx.lib.damas_solve(ctx.handle, arr, 1, None, None))
    # the same system, aligned, on the same context
    x_ref = torch.zeros(S, device="cuda")
    D.damas_solve(ctx, D.System(A, b, x_ref, 10))
    assert torch.isfinite(x_ref).all() and float(x_ref.sum()) > 0


def test_das_map_rejects_misaligned_csm(ctx, small):
    g = D.Geometry.from_scene(small.mics, small.grid, small.c)
    C = D.csm_tensor(small.C)
    big = torch.zeros(C.numel() + 2, dtype=torch.float32, device="cuda")
    big[1:1 + C.numel()] = C.reshape(-1)
    b = torch.empty(g.S, dtype=torch.float32, device="cuda")
    gs = g.cstruct()
    _einval(ctx, ctx.lib.das_map(ctx.handle, ctypes.byref(gs), float(small.freq), big.data_ptr() + 4, b.data_ptr(),
                                 None))
    ref = D.das_map(ctx, g, small.freq, C)
    assert torch.isfinite(ref).all()


def test_dual_psf_rejects_overlap_and_misalignment(ctx, small):
    g = D.Geometry.from_scene(small.mics, small.grid, small.c)
    S = g.S
    lda = D.damas_lda(S)
    gs = g.cstruct()
    buf = torch.empty(S * lda * 2, dtype=torch.float32, device="cuda")
    g2 = torch.empty(S, dtype=torch.float32, device="cuda")
    p = buf.data_ptr()
    call = lambda a32, a16: ctx.lib.damas_build_psf_f32_bf16(ctx.handle, ctypes.byref(gs), float(small.freq), None,
                                                            S, a32, a16, lda, g2.data_ptr(), None)
    _einval(ctx, call(p, p))                                # same start
    _einval(ctx, call(p, p + S * lda * 4 - 64))             # BF16 copy starts inside the FP32 matrix
    _einval(ctx, call(p + S * lda * 2 - 64, p))             # FP32 matrix starts inside the BF16 copy
    _einval(ctx, call(p, p + S * lda * 4 + 8))              # adjacent but not 16-byte aligned
    _einval(ctx, call(p + 4, p + S * lda * 4 + 16))         # FP32 matrix not 16-byte aligned
    # adjacent and aligned: accepted, and equal to the two separate builds
    A32 = buf[:S * lda].view(S, lda)
    A16 = buf[S * lda:].view(torch.bfloat16)[:S * lda].view(S, lda)
    ctx.check(call(A32.data_ptr(), A16.data_ptr()))
    r32, _ = D.damas_build_psf(ctx, g, small.freq)
    r16, _ = D.damas_build_psf(ctx, g, small.freq, a_dtype=D.BF16)
    torch.cuda.synchronize()
    assert torch.equal(A32, r32) and torch.equal(A16, r16)


def test_context_hbm_budget_refuses_scratch_beyond_it(small):
    """DAMAS_OPT_HBM_BUDGET_BYTES: scratch that would take the context above the
    cap is refused with DAMAS_ENOMEM (the context stays usable); a cap below what
    it holds, or a negative one, is refused with DAMAS_EINVAL; 0 lifts the cap."""
    c = D.Context(0)
    try:
        sc = synth.scene_spiral_81()
        g = D.Geometry.from_scene(sc.mics, sc.grid, sc.c)
        with pytest.raises(D.DamasError):
            D.damas_set_option(c, L.OPT_HBM_BUDGET_BYTES, -1)
        D.damas_set_option(c, L.OPT_HBM_BUDGET_BYTES, 2 << 20)   # 2 MiB: below the 81x81 PSF's planes
        A = torch.empty((g.S, D.damas_lda(g.S)), dtype=torch.float32, device="cuda")
        g2 = torch.empty(g.S, dtype=torch.float32, device="cuda")
        with pytest.raises(D.DamasError) as e:
            D.damas_build_psf(c, g, sc.freq, A=A, gnorm2=g2)
        assert e.value.code == L.DAMAS_ENOMEM
        # the small grid's scratch fits the same cap
        gs = D.Geometry.from_scene(small.mics, small.grid, small.c)
        As, _ = D.damas_build_psf(c, gs, small.freq)
        assert torch.isfinite(As).all()
        with pytest.raises(D.DamasError):
            D.damas_set_option(c, L.OPT_HBM_BUDGET_BYTES, (1 << 20) - 4096)   # below what the context holds now
        D.damas_set_option(c, L.OPT_HBM_BUDGET_BYTES, 0)
        D.damas_build_psf(c, g, sc.freq, A=A, gnorm2=g2)
        torch.cuda.synchronize()
        c2 = D.Context(0)
        try:
            ref, _ = D.damas_build_psf(c2, g, sc.freq)
            torch.cuda.synchronize()
        finally:
            c2.close()
        assert torch.equal(A, ref)
    finally:
        c.close()
