"""Band processing: all bins' iterations in one launch (§6 band processing).

- every bin of a batched launch equals the same bin solved alone, bit for bit;
- a captured CUDA graph of phase 2 reproduces the eager run bit for bit;
- the batched solve matches the oracle iteration on oracle-built systems.
"""
import numpy as np
import pytest
import torch

import oracle as O
import synth

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_1608_05179_gb300")
D = P.damas
from paper_1608_05179_gb300 import band as B  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = D.Context(0)
    yield c
    c.close()


def _band(n_bins, N=81):
    scenes = synth.scene_band_121(n_bins=n_bins)
    sc0 = scenes[0]
    grid = synth.square_plane(N, 2.0, 2.0)
    Cs = [synth.simulate_csm(sc0.mics, sc0.src_xyz, sc0.powers, s.freq, s.c, 20.0, np.random.default_rng(i))
          for i, s in enumerate(scenes)]
    return sc0.mics, grid, [s.freq for s in scenes], Cs


def test_batched_equals_solo_and_graph_replay(ctx):
    mics, grid, freqs, Cs = _band(6)
    geom = D.Geometry.from_scene(mics, grid, synth.SPEED_OF_SOUND)
    C = torch.stack([D.csm_tensor(c) for c in Cs])
    grids, bs = B.solve_band(ctx, geom, freqs, C, 60, levels=4, eps=2e-3, rows_per_cta=256)
    assert len(set(grids.S_f)) > 1                       # uneven compressed sizes
    x_batch = [x.clone() for x in bs.x]
    # each bin alone, default team size
    for f in range(len(freqs)):
        solo = torch.zeros_like(bs.x[f])
        D.damas_solve(ctx, D.System(bs.A[f], bs.b_sub[f], solo, 60))
        assert torch.equal(solo, x_batch[f]), f
    # graph replay of phase 2, several times (each replay starts from clean mailboxes),
    # with an eager solve on the same context in between
    bs.capture(grids)
    for rep in range(3):
        bs.replay()
        bs.check()
        for f in range(len(freqs)):
            assert torch.equal(bs.x[f], x_batch[f]), (rep, f)
        solo = torch.zeros_like(bs.x[0])
        D.damas_solve(ctx, D.System(bs.A[0], bs.b_sub[0], solo, 60))
        assert torch.equal(solo, x_batch[0])


def test_batched_solve_matches_oracle(ctx):
    """Systems built by the oracle (one per bin, uneven sizes), solved in one launch."""
    mics, grid, freqs, Cs = _band(4)
    pts = grid.points()
    systems, refs = [], []
    for fr, Cf in zip(freqs, Cs):
        b = O.das_map(mics, pts, fr, synth.SPEED_OF_SOUND, Cf)
        idx, _, _, _ = O.wavelet_select(b.astype(np.float32), 81, 81, 4, O.PRED_LINEAR, O.EPS_REL_MAX, 5e-3)
        A, _ = O.psf_matrix(mics, pts[idx], fr, synth.SPEED_OF_SOUND)
        A32, b32 = A.astype(np.float32), b[idx].astype(np.float32)
        S = len(idx)
        Ap = np.zeros((S, D.damas_lda(S)), np.float32)
        Ap[:, :S] = A32
        systems.append(D.System(torch.as_tensor(Ap, device="cuda"), torch.as_tensor(b32, device="cuda"),
                                torch.zeros(S, device="cuda"), 200, ctas=max(1, S // 512)))
        refs.append(O.gauss_seidel(A32.astype(np.float64), b32.astype(np.float64), 200))
    assert len({s.b.numel() for s in systems}) == len(systems)
    D.damas_solve(ctx, systems)
    for s, xo in zip(systems, refs):
        err = np.linalg.norm(s.x.cpu().numpy() - xo) / np.linalg.norm(xo)
        assert err <= 1e-4


def test_autotuner_picks_a_candidate(ctx):
    mics, grid, freqs, Cs = _band(3)
    geom = D.Geometry.from_scene(mics, grid, synth.SPEED_OF_SOUND)
    C = torch.stack([D.csm_tensor(c) for c in Cs])
    grids = B.compress_band(ctx, geom, freqs, C, 4, D.PRED_LINEAR, D.EPS_REL_MAX, 2e-3)
    grids.S_f = [int(v) for v in grids.S_f_dev.cpu().tolist()]
    best, timings = B.autotune_rows(ctx, geom, freqs, grids, iters_probe=5, candidates=(256, 1024),
                                    balance=(512,))
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert best in timings and min(timings, key=timings.get) == best
    assert {(p, v) for p, v, _ in timings} <= {("rows", 256), ("rows", 1024), ("balance", 512)}
    assert {cap for _, _, cap in timings} <= {sms, 2 * sms}
    assert ("rows", 256, sms) in timings and ("rows", 1024, sms) in timings and ("balance", 512, sms) in timings
    # the chosen plan solves the band like any other
    bs = B.plan_solver(ctx, geom, freqs, grids.S_f, 30, D.F32, best)
    bs.run(grids)
    bs.check()
