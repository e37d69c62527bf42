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


# ----------------------------------------------------------------------------- against the oracle
def _oracle_requests():
    """Single-bin compressed requests of several sizes with thresholds placed with a
    provable margin (tests/e2e_util.py), plus one three-bin full-grid request."""
    import oracle as O
    from e2e_util import margin_threshold
    rng = np.random.default_rng(17)
    reqs = []
    for M, N, L, iters in ((16, 21, 2, 200), (32, 41, 3, 300), (64, 41, 3, 150), (32, 33, 2, 250)):
        f = float(rng.uniform(1500, 5000))
        sc = synth.scene_random(rng, M, N, int(rng.integers(1, 4)), f)
        C = synth.simulate_csm(sc.mics, sc.src_xyz, sc.powers, f, sc.c, 20.0, rng)
        b64 = O.das_map(sc.mics, sc.grid.points(), f, sc.c, C)
        eps, gap = margin_threshold(b64.astype(np.float32), N, N, L, O.PRED_LINEAR, 0.10, 0.30)
        assert gap > 4.0, (M, N, gap)
        reqs.append(SV.Request(sc.mics, sc.grid, np.array([f]), C[None], iters=iters, levels=L,
                               eps_mode=D.EPS_ABS, eps=eps))
    freqs = np.sort(rng.uniform(1500, 5000, 3))
    sc = synth.scene_random(rng, 32, 21, 2, float(freqs[0]))
    Cs = np.stack([synth.simulate_csm(sc.mics, sc.src_xyz, sc.powers, f, sc.c, 20.0, rng) for f in freqs])
    reqs.append(SV.Request(sc.mics, sc.grid, freqs, Cs, iters=200, levels=0))
    return reqs


def test_served_bins_match_the_oracle(ctx):
    """Every bin of every served request against oracle.solve_bin (the §5
    procedure in FP64): identical compressed grid, reproduced map and integrated
    power within 1e-4, power map within the oracle's own conditioning bound."""
    import oracle as O
    from e2e_util import PARITY, conditioned_errors, iterate_tolerance, rel
    reqs = _oracle_requests()
    srv = SV.Server(ctx, max_inflight=4)
    tickets = [srv.submit(r) for r in reqs]                  # overlapping on the device
    res = [srv.wait(t) for t in tickets]
    srv.stop()
    for r, got in zip(reqs, res):
        for f, fr in enumerate(r.freqs):
            orc = O.solve_bin(r.mics, r.grid, float(fr), r.c, r.C[f], r.iters, compressed=r.levels > 0,
                              levels=r.levels or None, predictor=r.predictor, eps_mode=r.eps_mode, eps=r.eps)
            assert int(got.S_sub[f]) == len(orc["idx"])
            x = got.x[f].astype(np.float64)
            assert np.all(x[np.setdiff1d(np.arange(r.grid.S), orc["idx"])] == 0.0)
            xs = x[orc["idx"]] * orc["gnorm2"]             # back to the solver's unknowns (formulation E)
            tol, det = iterate_tolerance(orc["A"], orc["b"][orc["idx"]], r.iters, x_ref=orc["x_sub"])
            e_map = rel(x, orc["x"])
            e_reconv, e_pow = conditioned_errors(orc["A"], xs, orc["x_sub"], orc["gnorm2"], orc["gnorm2"])
            e_tot = abs(got.total_power[f] - orc["x"].sum()) / orc["x"].sum()
            print(f"[serve-oracle] S={r.grid.S} S~={len(orc['idx'])} iters={r.iters}: map {e_map:.2e} "
                  f"(tol {tol:.2e}) reconv {e_reconv:.2e} power {e_pow:.2e} total {e_tot:.2e}")
            assert e_map <= tol
            assert e_reconv <= PARITY and e_pow <= 2 * PARITY and e_tot <= PARITY


# ----------------------------------------------------------------------------- admission
def _same_shape_requests(n=4):
    rng = np.random.default_rng(23)
    reqs = []
    for _ in range(n):
        freqs = np.sort(rng.uniform(2000, 4000, 2))
        sc = synth.scene_random(rng, 32, 41, 2, float(freqs[0]))
        C = np.stack([synth.simulate_csm(sc.mics, sc.src_xyz, sc.powers, f, sc.c, 20.0, rng) for f in freqs])
        reqs.append(SV.Request(sc.mics, sc.grid, freqs, C, iters=300, levels=3, eps=0.2))
    return reqs


def test_hbm_budget_admits_one_request_at_a_time(ctx):
    """A budget that holds one request's device memory but not two: every request
    is admitted only after the previous one is done, and the results are the
    same bit for bit as with a budget that holds them all."""
    reqs = _same_shape_requests()
    srv = SV.Server(ctx, max_inflight=4)                      # default budget: half the free memory
    free = [srv.wait(t) for t in [srv.submit(r) for r in reqs]]
    srv.stop()
    assert all(a.hbm_bytes > 0 for a in free)
    assert any(free[i + 1].t_admit < free[i].t_done for i in range(len(free) - 1))   # they overlapped there
    budget = min(a.hbm_bytes for a in free)                   # one request fits, two never do
    assert 2 * budget > max(a.hbm_bytes for a in free)
    srv = SV.Server(ctx, hbm_budget_bytes=budget, max_inflight=4)
    tight = [srv.wait(t) for t in [srv.submit(r) for r in reqs]]
    srv.stop()
    for i in range(1, len(tight)):
        assert tight[i].t_admit >= tight[i - 1].t_done
    for a, b in zip(free, tight):
        assert a.hbm_bytes == b.hbm_bytes
        assert np.array_equal(a.x, b.x) and np.array_equal(a.total_power, b.total_power)


def test_single_cta_solve_is_charged_a_whole_sm(ctx):
    """A request whose bins solve in the single-CTA form (each CTA fills an SM)
    is charged two half-SM units per bin; with four units (two SMs) two such
    single-bin requests may solve at once but a third waits for one to finish."""
    reqs = _same_shape_requests(3)
    for r in reqs:
        r.freqs, r.C = r.freqs[:1], r.C[:1]
    srv = SV.Server(ctx, max_inflight=4, sm_slots=4)
    res = [srv.wait(t) for t in [srv.submit(r) for r in reqs]]
    srv.stop()
    plan = [D.damas_solve_plan(ctx, int(a.S_sub[0])) for a in res]
    assert all(p[0] == 1 and a.S_sub[0] >= 97 for p, a in zip(plan, res)), plan   # single-CTA form
    assert all(a.sm_units == 2 for a in res)
    # stage-2 intervals: never three at once
    iv = sorted((a.t_solve, a.t_done) for a in res)
    assert not (iv[2][0] < iv[0][1] and iv[2][0] < iv[1][1])
