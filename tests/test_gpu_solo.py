"""The single-CTA form of the Gauss-Seidel launch (Eq. (13)-(14)): one CTA per
system, A streamed, no hand-overs between CTAs.  Its fold schedule differs from
the team form's, but every row receives every dx in step order through the same
arithmetic, so iterates and saved states are bit-identical to the team form's;
the tests hold it to that and to the oracle iteration (relative L2 <= 1e-4 after
the same number of sweeps)."""
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


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    e = float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
    print(f"[rel_l2] {e:.3e}")
    return e


def padded(A64, dtype=torch.float32):
    S = A64.shape[0]
    out = np.zeros((S, D.damas_lda(S)), np.float32)
    out[:, :S] = A64
    return torch.as_tensor(out).to("cuda", dtype)


def oracle_iterate(A64, b64, iters, bf16=False, x0=None):
    A32 = A64.astype(np.float32)
    if bf16:
        A32 = torch.as_tensor(A32).to(torch.bfloat16).float().numpy()
    return O.gauss_seidel(A32.astype(np.float64), b64.astype(np.float32).astype(np.float64), iters, x0=x0)


def compressed_system():
    sc = synth.scene_spiral_81()
    pts = sc.grid.points()
    b = O.das_map(sc.mics, pts, sc.freq, sc.c, sc.C)
    idx, _, _, _ = O.wavelet_select(b.astype(np.float32), 81, 81, 2, O.PRED_HAAR, O.EPS_KEEP_FRAC, 0.1)
    A, _ = O.psf_matrix(sc.mics, pts[idx], sc.freq, sc.c)
    return A, b[idx]


def solve(ctx, A, b, iters, ctas, place=0, **kw):
    x = kw.pop("x", None)
    if x is None:
        x = torch.zeros(b.numel(), device="cuda")
    D.damas_solve(ctx, D.System(A, b, x, iters, **kw), ctas_per_system=ctas, a_placement=place)
    return x


def test_solo_plan(ctx):
    for S in (97, 657, 1000):
        ncta, R, res = D.damas_solve_plan(ctx, S, ctas=1)
        assert (ncta, R, res) == (1, (S + 31) // 32 * 32, 0)
    # three blocks or fewer: the team form's single-CTA launch
    assert D.damas_solve_plan(ctx, 96, ctas=1)[0] == 1


@pytest.mark.parametrize("bf16", [False, True])
def test_solo_equals_team_bit_for_bit(ctx, bf16):
    """The compressed 81x81 system (S~ = 657): the single-CTA form gives the team
    form's x exactly (resident 11-CTA team, streamed 5-CTA team) and matches the
    oracle on the same (FP32 or BF16-rounded) A."""
    A64, b64 = compressed_system()
    dt = torch.bfloat16 if bf16 else torch.float32
    iters = 500 if bf16 else 1000
    A = padded(A64, dt)
    b = torch.as_tensor(b64.astype(np.float32), device="cuda")
    x1 = solve(ctx, A, b, iters, 1)
    for ctas, place in ((0, 0), (5, 2)):
        xt = solve(ctx, A, b, iters, ctas, place)
        assert torch.equal(x1, xt), (ctas, place)
    assert rel_l2(x1.cpu().numpy(), oracle_iterate(A64, b64, iters, bf16=bf16)) <= 1e-4


@pytest.mark.parametrize("S", [97, 100, 127, 128, 129, 257, 431])
def test_solo_ragged_sizes(ctx, S):
    A64, b64 = synth.random_psd_system(np.random.default_rng(S), S)
    A = padded(A64)
    b = torch.as_tensor(b64.astype(np.float32), device="cuda")
    x1 = solve(ctx, A, b, 60, 1)
    x3 = solve(ctx, A, b, 60, 3, 2)
    assert torch.equal(x1, x3)
    assert rel_l2(x1.cpu().numpy(), oracle_iterate(A64, b64, 60)) <= 1e-4


def test_solo_resume_across_forms(ctx):
    """300 + 200 sweeps through the saved state equal 500 sweeps, in either order of
    the two forms."""
    A64, b64 = compressed_system()
    S = len(b64)
    A = padded(A64)
    b = torch.as_tensor(b64.astype(np.float32), device="cuda")
    ref = solve(ctx, A, b, 500, 1)
    assert torch.equal(ref, solve(ctx, A, b, 500, 4, 2))
    for first, second in ((1, 2), (2, 1), (1, 1)):
        st = torch.zeros(D.damas_state_floats(S), device="cuda")
        x = solve(ctx, A, b, 300, first, 2 if first > 1 else 0, state=st)
        solve(ctx, A, b, 200, second, 2 if second > 1 else 0, x=x, state=st, init=D.INIT_STATE)
        assert torch.equal(x, ref), (first, second)


def test_solo_states_equal(ctx):
    """The state a single-CTA call leaves (residual pair and pending dx blocks) is
    the team form's, bit for bit."""
    A64, b64 = compressed_system()
    S = len(b64)
    A = padded(A64)
    b = torch.as_tensor(b64.astype(np.float32), device="cuda")
    s1 = torch.zeros(D.damas_state_floats(S), device="cuda")
    s2 = torch.zeros_like(s1)
    solve(ctx, A, b, 37, 1, state=s1)
    solve(ctx, A, b, 37, 3, 2, state=s2)
    assert torch.equal(s1, s2)


def test_solo_warm_start_from_x(ctx):
    A64, b64 = compressed_system()
    xh = oracle_iterate(A64, b64, 200).astype(np.float32)
    A = padded(A64)
    b = torch.as_tensor(b64.astype(np.float32), device="cuda")
    x1 = solve(ctx, A, b, 300, 1, x=torch.as_tensor(xh, device="cuda"), init=D.INIT_X)
    x3 = solve(ctx, A, b, 300, 3, x=torch.as_tensor(xh, device="cuda"), init=D.INIT_X)
    assert torch.equal(x1, x3)
    assert rel_l2(x1.cpu().numpy(), oracle_iterate(A64, b64, 300, x0=xh.astype(np.float64))) <= 1e-4


def test_solo_negative_entries(ctx):
    """A matrix with negative entries (no row skipping) gives the same x in both forms."""
    rng = np.random.default_rng(8)
    S = 150
    Y = rng.standard_normal((S, 2 * S))
    A64 = Y @ Y.T / (2 * S)
    dg = np.sqrt(np.diag(A64))
    A64 = A64 / dg[:, None] / dg[None, :]
    np.fill_diagonal(A64, 1.0)
    b64 = A64 @ np.abs(rng.standard_normal(S)) * (rng.random(S) < 0.3)
    A = padded(A64)
    b = torch.as_tensor(b64.astype(np.float32), device="cuda")
    x1 = solve(ctx, A, b, 80, 1)
    assert torch.equal(x1, solve(ctx, A, b, 80, 2, 2))
    assert rel_l2(x1.cpu().numpy(), oracle_iterate(A64, b64, 80)) <= 1e-4


def test_solo_nonsymmetric_with_transpose(ctx):
    """Formulation P: columns are read through the transpose."""
    sc = synth.scene_monopole_small()
    pts = sc.grid.points()
    A64, _ = O.psf_matrix(sc.mics, pts, sc.freq, sc.c, O.FORM_P)
    b64 = O.das_map(sc.mics, pts, sc.freq, sc.c, sc.C, O.FORM_P)
    A, At = padded(A64), padded(np.ascontiguousarray(A64.T))
    b = torch.as_tensor(b64.astype(np.float32), device="cuda")
    x1 = solve(ctx, A, b, 100, 1, At=At)
    assert torch.equal(x1, solve(ctx, A, b, 100, 3, 2, At=At))
    assert rel_l2(x1.cpu().numpy(), oracle_iterate(A64, b64, 100)) <= 1e-4


def test_solo_batch_beyond_one_launch(ctx):
    """70 single-CTA systems of mixed sizes in one call (two launches of at most
    64 systems) equal the same systems solved one at a time."""
    rng = np.random.default_rng(70)
    made = [synth.random_psd_system(rng, int(S)) for S in rng.integers(97, 700, 70)]
    batch, alone = [], []
    for A64, b64 in made:
        A = padded(A64)
        b = torch.as_tensor(b64.astype(np.float32), device="cuda")
        batch.append(D.System(A, b, torch.zeros(len(b64), device="cuda"), 40, ctas=1))
        alone.append(solve(ctx, A, b, 40, 1))
    D.damas_solve(ctx, batch)
    for s, x in zip(batch, alone):
        assert torch.equal(s.x, x)
    assert rel_l2(batch[5].x.cpu().numpy(), oracle_iterate(*made[5], 40)) <= 1e-4


def test_solo_zero_iterations_keep_the_state(ctx):
    A64, b64 = synth.random_psd_system(np.random.default_rng(3), 200)
    A = padded(A64)
    b = torch.as_tensor(b64.astype(np.float32), device="cuda")
    st = torch.zeros(D.damas_state_floats(200), device="cuda")
    x = solve(ctx, A, b, 25, 1, state=st)
    st0, x0 = st.clone(), x.clone()
    solve(ctx, A, b, 0, 1, x=x, state=st, init=D.INIT_STATE)
    assert torch.equal(st, st0) and torch.equal(x, x0)


def test_solo_graph_replays(ctx):
    """A recorded single-CTA solve replays to the eager result every time."""
    A64, b64 = compressed_system()
    A = padded(A64)
    b = torch.as_tensor(b64.astype(np.float32), device="cuda")
    ref = solve(ctx, A, b, 200, 1)
    x = torch.zeros_like(ref)
    solve(ctx, A, b, 200, 1, x=x)  # sizes the scratch before recording
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            D.damas_solve(ctx, D.System(A, b, x, 200), ctas_per_system=1, stream=s,
                          status=torch.zeros(1, dtype=torch.int32, device="cuda"))
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(3):
        x.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(x, ref)


def test_solo_and_team_systems_in_one_call(ctx):
    """A call mixing systems the single-CTA form would take with systems that need
    teams runs them all as teams in one launch; every result equals the system
    solved alone."""
    rng = np.random.default_rng(5)
    made = [synth.random_psd_system(rng, S) for S in (300, 1500, 657, 64)]
    batch, alone = [], []
    for (A64, b64), ctas in zip(made, (1, 0, 0, 0)):
        A = padded(A64)
        b = torch.as_tensor(b64.astype(np.float32), device="cuda")
        batch.append(D.System(A, b, torch.zeros(len(b64), device="cuda"), 50, ctas=ctas))
        alone.append(solve(ctx, A, b, 50, ctas))
    D.damas_solve(ctx, batch)
    for s, x in zip(batch, alone):
        assert torch.equal(s.x, x)


def test_solve_statistics_agree_between_forms(ctx):
    """The launch statistics (blocks solved, rows that entered a chain, nonzero
    dx) count the iteration itself, so the single-CTA form and a team report the
    same numbers; blocks solved = sweeps x blocks."""
    A64, b64 = compressed_system()
    S, iters = len(b64), 200
    nb = -(-S // 32)
    out = []
    for ctas, place in ((1, 2), (5, 2), (0, 1)):
        A = padded(A64)
        b = torch.as_tensor(b64.astype(np.float32), device="cuda")
        x = torch.zeros(S, device="cuda")
        st = torch.zeros(3, dtype=torch.int64, device="cuda")
        D.damas_solve(ctx, D.System(A, b, x, iters), ctas_per_system=ctas, a_placement=place, stats=st)
        out.append(st.cpu().numpy().tolist())
    print("[stats]", out)
    assert out[0] == out[1] == out[2]
    solves, cand, nnz = out[0]
    assert solves == iters * nb
    assert 0 < nnz <= cand <= solves * 32


def test_chain_probe(ctx):
    t_cand, t_bar = D.damas_chain_probe(ctx, 20000)
    print(f"[chain probe] {t_cand:.1f} ns per candidate, {t_bar:.1f} ns per barrier step")
    assert 1.0 < t_cand < 1000.0 and 1.0 < t_bar < 5000.0
