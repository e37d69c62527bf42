"""Serving loop: continuous batching of independent requests.

Each request's result is the same bit for bit whether it runs alone or in a mix
of overlapping requests, and equals the plain per-bin path of the library."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_1608_05179_gb300")
D = P.damas
from paper_1608_05179_gb300 import serve as SV  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = D.Context(0)
    yield c
    c.close()


def _requests(n=6, seed=5):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        M = int(rng.choice([32, 64]))
        N = int(rng.choice([41, 81]))
        F = int(rng.integers(1, 4))
        freqs = np.sort(rng.uniform(1000, 6000, F))
        sc = synth.scene_random(rng, M, N, int(rng.integers(1, 4)), float(freqs[0]))
        C = np.stack([synth.simulate_csm(sc.mics, sc.src_xyz, sc.powers, f, sc.c, 20.0, rng) for f in freqs])
        reqs.append(SV.Request(sc.mics, sc.grid, freqs, C, iters=int(rng.integers(50, 150)), levels=3,
                               eps=float(rng.uniform(0.05, 0.3))))
    return reqs


def test_alone_equals_mix_and_plain_path(ctx):
    reqs = _requests()
    srv = SV.Server(ctx, max_inflight=4)
    alone = [srv.wait(srv.submit(r)) for r in reqs]                 # one at a time
    tickets = [srv.submit(r) for r in reqs]                          # all at once: overlapping
    mix = [srv.wait(t) for t in tickets]
    srv.stop()
    for a, m in zip(alone, mix):
        assert np.array_equal(a.x, m.x)
        assert np.array_equal(a.total_power, m.total_power)
        assert np.array_equal(a.S_sub, m.S_sub)
        assert a.t_submit <= a.t_admit <= a.t_done
    # overlapping requests: some were admitted before the previous one finished
    assert any(mix[i + 1].t_admit < mix[i].t_done for i in range(len(mix) - 1))
    # the plain per-bin path gives the same maps
    r = reqs[0]
    geom = D.Geometry.from_scene(r.mics, r.grid, r.c)
    for f, fr in enumerate(r.freqs):
        out = D.solve_bin(ctx, geom, float(fr), D.csm_tensor(r.C[f]), r.iters, compressed=True, levels=r.levels,
                          predictor=r.predictor, eps_mode=r.eps_mode, eps=r.eps)
        assert np.array_equal(out["x"].cpu().numpy(), alone[0].x[f])


def test_full_grid_request_and_release(ctx):
    reqs = _requests(1, seed=9)
    reqs[0].levels = 0
    srv = SV.Server(ctx, max_inflight=2)
    res = srv.wait(srv.submit(reqs[0]))
    srv.stop()
    assert np.all(res.S_sub == reqs[0].grid.nx * reqs[0].grid.ny)
    assert res.x.min() >= 0 and np.all(res.total_power > 0)


def test_submit_after_stop_is_refused(ctx):
    srv = SV.Server(ctx, max_inflight=1)
    srv.stop()
    with pytest.raises(D.DamasError):
        srv.submit(_requests(1)[0])
