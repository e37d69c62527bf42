"""Bounded waits of the PSF build (tensor-core Gram): a wait that runs out is
reported, marks the output, stops a later solve on the same context, and
leaves the device usable.

The wait is made to run out from the host: the context's test hook makes the
Gram's operand loader wait for a device flag that nothing sets.  No GPU fault
is involved."""
import numpy as np
import pytest
import torch

import oracle as O
import synth

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_1608_05179_gb300")
D = P.damas
L = P._lib


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = D.Context(0)
    yield c
    c.close()


def test_psf_wait_that_runs_out_is_reported_and_the_device_stays_usable(ctx):
    sc = synth.scene_monopole_small()
    g = D.Geometry.from_scene(sc.mics, sc.grid, sc.c)
    S = sc.grid.S
    A_ref, g2 = D.damas_build_psf(ctx, g, sc.freq)
    D.damas_check(ctx)                                   # nothing ran out
    b = D.das_map(ctx, g, sc.freq, D.csm_tensor(sc.C))

    D.damas_set_option(ctx, L.OPT_BUILD_TIMEOUT_MS, 20)
    D.damas_set_option(ctx, L.OPT_TEST_HOLD_BUILD, 1)
    try:
        A_bad, _ = D.damas_build_psf(ctx, g, sc.freq)    # returns once enqueued
        with pytest.raises(D.DamasError) as e:
            D.damas_check(ctx)
        assert e.value.code == L.DAMAS_ETIMEDOUT
        assert torch.isnan(A_bad[:, :S]).any()          # the aborted tiles are marked
        D.damas_check(ctx)                               # the check cleared the status

        # a solve after a failed build on the context reports it and leaves x alone
        D.damas_build_psf(ctx, g, sc.freq, A=A_bad)
        x = torch.full((S,), 7.0, device="cuda")
        with pytest.raises(D.DamasError) as e:
            D.damas_solve(ctx, D.System(A_ref, b, x, 10))
        assert e.value.code == L.DAMAS_ETIMEDOUT
        assert bool(torch.all(x == 7.0))
        with pytest.raises(D.DamasError):
            D.damas_check(ctx)
    finally:
        D.damas_set_option(ctx, L.OPT_TEST_HOLD_BUILD, 0)
        D.damas_set_option(ctx, L.OPT_BUILD_TIMEOUT_MS, 2000)

    # back to normal on the same context: the same matrix bit for bit, and a solve
    A2, _ = D.damas_build_psf(ctx, g, sc.freq)
    D.damas_check(ctx)
    assert torch.equal(A2, A_ref)
    x = torch.zeros(S, device="cuda")
    D.damas_solve(ctx, D.System(A2, b, x, 20))
    A64, _ = O.psf_matrix(sc.mics, sc.grid.points(), sc.freq, sc.c)
    assert float(np.max(np.abs(A2[:, :S].cpu().numpy() - A64))) <= 5e-6


def test_options_are_validated(ctx):
    with pytest.raises(D.DamasError):
        D.damas_set_option(ctx, L.OPT_BUILD_TIMEOUT_MS, 0)
    with pytest.raises(D.DamasError):
        D.damas_set_option(ctx, L.OPT_TEST_HOLD_BUILD, 2)
    with pytest.raises(D.DamasError):
        D.damas_set_option(ctx, 99, 1)
