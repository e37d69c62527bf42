"""GPU parity: every hot-path step through the C-ABI library against the oracle.

Tolerances (the numbers are derived in the design notes):
  - A (FP32): max |A_gpu - A_oracle| <= 5e-6 (entries lie in [0, 1]; FP32 vectors
    and an FP32 Gram of M terms); BF16 storage: relative 2^-8 per entry.
  - DAS map: max |b_gpu - b| <= 2e-5 * max |b|.
  - Compressed grid: bit-exact indices, count and threshold on an identical FP32 map.
  - Sweeps, identical FP32 inputs: ||x_gpu - x_oracle||_2 <= 1e-4 ||x_oracle||_2
    after the same number of sweeps (the oracle iterates in FP64 on the same A, b).
"""
import math

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
    """Relative L2 error of a against b; the value is printed (pytest -s) so a run records it."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    e = float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))
    import inspect
    print(f"[rel_l2] {inspect.stack()[1].function}: {e:.3e}")
    return e


def geom_of(sc, form=O.FORM_E):
    return D.Geometry.from_scene(sc.mics, sc.grid, sc.c, form)


def padded(A64, dtype=torch.float32):
    S = A64.shape[0]
    lda = D.damas_lda(S)
    out = np.zeros((S, lda), np.float32)
    out[:, :S] = A64
    return torch.as_tensor(out).to("cuda", dtype)


# ----------------------------------------------------------------------------- a1 + a4
@pytest.mark.parametrize("form", [O.FORM_E, O.FORM_P])
def test_psf_full_grid_matches_oracle(ctx, form):
    sc = synth.scene_monopole_small()
    g = geom_of(sc, form)
    A, g2 = D.damas_build_psf(ctx, g, sc.freq)
    torch.cuda.synchronize()
    Ao, g2o = O.psf_matrix(sc.mics, sc.grid.points(), sc.freq, sc.c, form)
    Ag = A.cpu().numpy()
    S = sc.grid.S
    assert np.abs(Ag[:, :S] - Ao).max() <= 5e-6
    assert np.all(np.diag(Ag) == 1.0)
    assert np.all(Ag[:, S:] == 0.0)
    assert np.allclose(g2.cpu().numpy(), g2o, rtol=1e-6)
    if form == O.FORM_E:
        assert np.array_equal(Ag[:, :S], Ag[:, :S].T)      # exactly symmetric, as the solver assumes


def test_psf_selected_points_and_bf16(ctx):
    sc = synth.scene_spiral_81()
    g = geom_of(sc)
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(sc.grid.S, 333, replace=False)).astype(np.int32)
    it = torch.as_tensor(idx, device="cuda")
    A, g2 = D.damas_build_psf(ctx, g, sc.freq, it, len(idx))
    Ab, _ = D.damas_build_psf(ctx, g, sc.freq, it, len(idx), a_dtype=D.BF16)
    torch.cuda.synchronize()
    Ao, g2o = O.psf_matrix(sc.mics, sc.grid.points()[idx], sc.freq, sc.c)
    assert np.abs(A.cpu().numpy()[:, :333] - Ao).max() <= 5e-6
    assert torch.equal(A[:, :333], A[:, :333].T) and torch.equal(Ab[:, :333], Ab[:, :333].T)
    Abf = Ab.float().cpu().numpy()[:, :333]
    assert np.all(np.abs(Abf - Ao) <= 2.0 ** -8 * np.abs(Ao) + 1e-6)
    assert np.allclose(g2.cpu().numpy(), g2o, rtol=1e-6)


def gram_tolerance(M):
    """Bound on max |A_gpu - A| (entries in [0, 1]) for the 3xTF32 tensor-core Gram.

    Every partial sum of G = e_n^H e_m has modulus <= 1 (Cauchy-Schwarz on unit
    vectors; the same after the 1/M scaling of formulation P); each of the
    12 * ceil(M / 16) MMA accumulations into Re G or Im G loses at most one FP32
    ulp of such a value (2^-23, the accumulator truncates); the dropped lo*lo
    products and the rounding of the lo parts add at most 2^-21; A = |G|^2
    doubles the error of |G|; 1e-6 covers the FP32 vectors themselves."""
    return 2.0 * (12 * math.ceil(M / 16) * 2.0 ** -23 + 2.0 ** -21) + 1e-6


@pytest.mark.parametrize("M", [128, 256])
@pytest.mark.parametrize("form", [O.FORM_E, O.FORM_P])
def test_psf_large_arrays(ctx, M, form):
    mics = synth.mic_log_spiral(M, 8, 1.5)
    grid = synth.square_plane(21, 2.0, 1.5)
    g = D.Geometry.from_scene(mics, grid, synth.SPEED_OF_SOUND, form)
    A, _ = D.damas_build_psf(ctx, g, 3000.0)
    torch.cuda.synchronize()
    Ao, _ = O.psf_matrix(mics, grid.points(), 3000.0, synth.SPEED_OF_SOUND, form)
    Ag = A.cpu().numpy()[:, :grid.S]
    assert np.abs(Ag - Ao).max() <= gram_tolerance(M)
    assert np.all(np.diag(Ag) == 1.0)
    if form == O.FORM_E:
        assert np.array_equal(Ag, Ag.T)


def test_psf_tiles_ragged_and_tiny(ctx):
    """Sizes around the 128 x 256 tile edges and a single point."""
    sc = synth.scene_spiral_81()
    g = geom_of(sc)
    pts = sc.grid.points()
    rng = np.random.default_rng(3)
    for n in (1, 2, 127, 128, 129, 255, 256, 257, 300, 513):
        idx = np.sort(rng.choice(sc.grid.S, n, replace=False)).astype(np.int32)
        A, _ = D.damas_build_psf(ctx, g, sc.freq, torch.as_tensor(idx, device="cuda"), n)
        torch.cuda.synchronize()
        Ao, _ = O.psf_matrix(sc.mics, pts[idx], sc.freq, sc.c)
        Ag = A.cpu().numpy()
        assert np.abs(Ag[:, :n] - Ao).max() <= 5e-6, n
        assert np.all(Ag[:, n:] == 0.0) and np.array_equal(Ag[:, :n], Ag[:, :n].T), n


# ----------------------------------------------------------------------------- a2
@pytest.mark.parametrize("form", [O.FORM_E, O.FORM_P])
@pytest.mark.parametrize("which", ["small", "spiral"])
def test_das_map_matches_oracle(ctx, form, which):
    sc = synth.scene_monopole_small() if which == "small" else synth.scene_spiral_81()
    b = D.das_map(ctx, geom_of(sc, form), sc.freq, D.csm_tensor(sc.C))
    torch.cuda.synchronize()
    bo = O.das_map(sc.mics, sc.grid.points(), sc.freq, sc.c, sc.C, form)
    assert np.abs(b.cpu().numpy() - bo).max() <= 2e-5 * np.abs(bo).max()


def test_das_map_large_array(ctx):
    rng = np.random.default_rng(4)
    sc = synth.scene_random(rng, 128, 41, 3, 5000.0)
    b = D.das_map(ctx, geom_of(sc), sc.freq, D.csm_tensor(sc.C))
    torch.cuda.synchronize()
    bo = O.das_map(sc.mics, sc.grid.points(), sc.freq, sc.c, sc.C)
    assert np.abs(b.cpu().numpy() - bo).max() <= 2e-5 * np.abs(bo).max()


# ----------------------------------------------------------------------------- a3
WAVELET_CASES = [
    # (scene, N, levels, predictor, mode, eps)
    ("spiral", 81, 2, O.PRED_HAAR, O.EPS_KEEP_FRAC, 0.10),
    ("spiral", 81, 4, O.PRED_LINEAR, O.EPS_REL_MAX, 0.05),
    ("spiral", 81, 4, O.PRED_HAAR, O.EPS_ABS, 0.5),
    ("spiral", 81, 2, O.PRED_LINEAR, O.EPS_KEEP_FRAC, 0.30),
    ("spiral", 81, 2, O.PRED_LINEAR, O.EPS_KEEP_FRAC, 0.02),
    ("spiral", 81, 2, O.PRED_LINEAR, O.EPS_KEEP_FRAC, 1.0),
    ("paper50", 50, 5, O.PRED_LINEAR, O.EPS_REL_MAX, 0.1),
    ("paper50", 50, 5, O.PRED_HAAR, O.EPS_KEEP_FRAC, 0.07),
    ("small", 21, 2, O.PRED_LINEAR, O.EPS_REL_MAX, 0.01),
    ("rect", 0, 3, O.PRED_LINEAR, O.EPS_KEEP_FRAC, 0.15),
]


def _wavelet_map(which):
    if which == "spiral":
        sc = synth.scene_spiral_81()
        return O.das_map(sc.mics, sc.grid.points(), sc.freq, sc.c, sc.C).astype(np.float32), 81, 81
    if which == "small":
        sc = synth.scene_monopole_small()
        return O.das_map(sc.mics, sc.grid.points(), sc.freq, sc.c, sc.C).astype(np.float32), 21, 21
    if which == "paper50":
        mics = synth.mic_disc(60, 0.5, np.random.default_rng(0))
        g = synth.square_plane(50, 5.77, 5.0)
        C = synth.simulate_csm(mics, np.array([g.point(24, 24)]), np.array([1.0]), 3000.0, 340.0, 15.0,
                               np.random.default_rng(1))
        return O.das_map(mics, g.points(), 3000.0, 340.0, C).astype(np.float32), 50, 50
    rng = np.random.default_rng(9)                       # rectangular grid with a ragged edge
    return rng.random(37 * 70).astype(np.float32), 70, 37


@pytest.mark.parametrize("case", WAVELET_CASES)
def test_wavelet_bit_exact(ctx, case):
    which, _, L, pred, mode, eps = case
    b, nx, ny = _wavelet_map(which)
    bt = torch.as_tensor(b, device="cuda")
    det = torch.empty(nx * ny, dtype=torch.float32, device="cuda")
    ea = torch.empty(1, dtype=torch.float32, device="cuda")
    idx, n, _, _ = D.wavelet_compress_grid(ctx, bt, nx, ny, L, pred, mode, eps, detail=det, eps_abs=ea)
    torch.cuda.synchronize()
    io, do, lo, eo = O.wavelet_select(b, nx, ny, L, pred, mode, eps)
    n = int(n.item())
    assert n == len(io)
    assert np.array_equal(idx[:n].cpu().numpy(), io)
    assert np.array_equal(det.cpu().numpy().view(np.uint32), do.view(np.uint32))
    assert ea.item() == eo or (math.isinf(eo) and math.isinf(ea.item()))


def test_wavelet_ties_and_constant(ctx):
    for b in (np.zeros((21, 21), np.float32), np.tile(np.float32([1, 0]), (33, 17))[:, :33].copy()):
        ny, nx = b.shape
        bt = torch.as_tensor(b.reshape(-1), device="cuda")
        for mode, eps in ((O.EPS_KEEP_FRAC, 0.1), (O.EPS_ABS, 0.0), (O.EPS_REL_MAX, 0.5)):
            idx, n, _, _ = D.wavelet_compress_grid(ctx, bt, nx, ny, 2, O.PRED_LINEAR, mode, eps)
            io, _, _, _ = O.wavelet_select(b, nx, ny, 2, O.PRED_LINEAR, mode, eps)
            assert np.array_equal(idx[:int(n.item())].cpu().numpy(), io)


# ----------------------------------------------------------------------------- a5, a7
def test_gather_and_scatter_power(ctx):
    rng = np.random.default_rng(3)
    S = 1000
    b = rng.random(S).astype(np.float32)
    idx = np.sort(rng.choice(S, 77, replace=False)).astype(np.int32)
    it = torch.as_tensor(idx, device="cuda")
    sub = D.damas_gather(ctx, torch.as_tensor(b, device="cuda"), it, 77)
    assert np.array_equal(sub.cpu().numpy(), b[idx])
    g2 = (1.0 + rng.random(77)).astype(np.float32)
    xf, tot = D.damas_scatter_power(ctx, sub, it, torch.as_tensor(g2, device="cuda"), 77, S)
    ref = O.scatter(O.to_power(b[idx].astype(np.float64), g2.astype(np.float64)), idx, S)
    assert np.allclose(xf.cpu().numpy(), ref, rtol=1e-7)
    assert abs(tot.item() - ref.sum()) <= 1e-6 * ref.sum()


# ----------------------------------------------------------------------------- a6
def _solve_gpu(ctx, A64, b64, iters, dtype=torch.float32, **kw):
    S = len(b64)
    A = padded(A64, dtype)
    b = torch.as_tensor(b64.astype(np.float32), device="cuda")
    x = torch.zeros(S, dtype=torch.float32, device="cuda")
    D.damas_solve(ctx, D.System(A, b, x, iters), **kw)
    return x.cpu().numpy()


def _oracle_fp32_inputs(A64, b64, iters, bf16=False):
    if bf16:
        A32 = torch.as_tensor(A64.astype(np.float32)).to(torch.bfloat16).float().numpy()
    else:
        A32 = A64.astype(np.float32)
    return O.gauss_seidel(A32.astype(np.float64), b64.astype(np.float32).astype(np.float64), iters)


def _compressed_system():
    sc = synth.scene_spiral_81()
    pts = sc.grid.points()
    b = O.das_map(sc.mics, pts, sc.freq, sc.c, sc.C)
    idx, _, _, _ = O.wavelet_select(b.astype(np.float32), 81, 81, 2, O.PRED_HAAR, O.EPS_KEEP_FRAC, 0.1)
    A, _ = O.psf_matrix(sc.mics, pts[idx], sc.freq, sc.c)
    return A, b[idx]


@pytest.mark.slow
def test_sweep_full_grid_81x81_1000_sweeps(ctx):
    """The benchmark's full-grid solve (S = 6561, 1000 sweeps, the automatic
    launch plan) against the FP64 oracle on the same FP32 inputs."""
    sc = synth.scene_spiral_81()
    pts = sc.grid.points()
    A, _ = O.psf_matrix(sc.mics, pts, sc.freq, sc.c)
    b = O.das_map(sc.mics, pts, sc.freq, sc.c, sc.C)
    x = _solve_gpu(ctx, A, b, 1000)
    xo = _oracle_fp32_inputs(A, b, 1000)
    assert rel_l2(x, xo) <= 1e-4


@pytest.mark.parametrize("ctas", [0, 1, 3, 7])
def test_sweep_small_full_grid(ctx, ctas):
    sc = synth.scene_monopole_small()
    pts = sc.grid.points()
    A, _ = O.psf_matrix(sc.mics, pts, sc.freq, sc.c)
    b = O.das_map(sc.mics, pts, sc.freq, sc.c, sc.C)
    x = _solve_gpu(ctx, A, b, 100, ctas_per_system=ctas)
    xo = _oracle_fp32_inputs(A, b, 100)
    assert rel_l2(x, xo) <= 1e-4


@pytest.mark.parametrize("ctas,place", [(0, 0), (11, 1), (1, 2), (1, 0), (2, 2), (5, 2), (0, 2)])
def test_sweep_compressed_1000(ctx, ctas, place):
    A, b = _compressed_system()
    x = _solve_gpu(ctx, A, b, 1000, ctas_per_system=ctas, a_placement=place)
    xo = _oracle_fp32_inputs(A, b, 1000)
    assert rel_l2(x, xo) <= 1e-4


@pytest.mark.parametrize("S", [1, 5, 31, 32, 33, 95, 257])
def test_sweep_ragged_sizes(ctx, S):
    A, b = synth.random_psd_system(np.random.default_rng(S), S)
    xo = _oracle_fp32_inputs(A, b, 60)
    for ctas, place in ((0, 0), (2, 0), (0, 2), (3, 2)):
        x = _solve_gpu(ctx, A, b, 60, ctas_per_system=ctas, a_placement=place)
        assert rel_l2(x, xo) <= 1e-4, (S, ctas, place)


def test_sweep_bf16_storage(ctx):
    """BF16-stored A: parity with the oracle iterating on the same BF16-rounded A.
    (Against the FP32 trajectory the iterate differs by far more than the
    rounding: the system is singular and the iteration follows a different path
    through the solution set, which the precision study quantifies.)"""
    A, b = _compressed_system()
    x = _solve_gpu(ctx, A, b, 500, dtype=torch.bfloat16)
    assert rel_l2(x, _oracle_fp32_inputs(A, b, 500, bf16=True)) <= 1e-4


@pytest.mark.parametrize("ctas,place", [(5, 1), (3, 2), (1, 2)])
def test_sweep_nonsymmetric_with_transpose(ctx, ctas, place):
    """Formulation P gives a non-symmetric A: the solver reads its columns through
    the transpose when A's rows are streamed, and from shared memory otherwise."""
    sc = synth.scene_monopole_small()
    pts = sc.grid.points()
    A64, _ = O.psf_matrix(sc.mics, pts, sc.freq, sc.c, O.FORM_P)
    b64 = O.das_map(sc.mics, pts, sc.freq, sc.c, sc.C, O.FORM_P)
    S = len(b64)
    A = padded(A64)
    At = padded(np.ascontiguousarray(A64.T))
    b = torch.as_tensor(b64.astype(np.float32), device="cuda")
    x = torch.zeros(S, device="cuda")
    D.damas_solve(ctx, D.System(A, b, x, 100, At=At), ctas_per_system=ctas, a_placement=place)
    assert rel_l2(x.cpu().numpy(), _oracle_fp32_inputs(A64, b64, 100)) <= 1e-4


def test_sweep_negative_entries_solved_in_full(ctx):
    """Rows are skipped only when A >= 0 guarantees they cannot move; a matrix with
    negative entries is solved row by row (still the same iteration)."""
    rng = np.random.default_rng(8)
    S = 150
    Y = rng.standard_normal((S, 2 * S))
    A64 = Y @ Y.T / (2 * S)
    dg = np.sqrt(np.diag(A64))
    A64 = A64 / dg[:, None] / dg[None, :]
    np.fill_diagonal(A64, 1.0)
    b64 = A64 @ np.abs(rng.standard_normal(S)) * (rng.random(S) < 0.3)
    for ctas, place in ((0, 0), (2, 2)):
        x = _solve_gpu(ctx, A64, b64, 80, ctas_per_system=ctas, a_placement=place)
        assert rel_l2(x, _oracle_fp32_inputs(A64, b64, 80)) <= 1e-4


def test_sweep_zero_rhs_and_zero_iters(ctx):
    A, _ = synth.random_psd_system(np.random.default_rng(1), 100)
    x = _solve_gpu(ctx, A, np.zeros(100), 10)
    assert np.all(x == 0)
    A2, b2 = synth.random_psd_system(np.random.default_rng(2), 70)
    assert np.all(_solve_gpu(ctx, A2, b2, 0) == 0)


@pytest.mark.parametrize("ctas,place", [(4, 0), (11, 1), (3, 2)])
def test_sweep_resume_is_bit_exact_and_deterministic(ctx, ctas, place):
    """300 + 200 sweeps through the saved state equal 500 sweeps bit for bit, whatever
    the team layout of the second call; repeated runs are bit-identical."""
    A64, b64 = _compressed_system()
    S = len(b64)
    A = padded(A64)
    b = torch.as_tensor(b64.astype(np.float32), device="cuda")
    x1 = torch.zeros(S, device="cuda")
    st = torch.zeros(D.damas_state_floats(S), device="cuda")
    D.damas_solve(ctx, D.System(A, b, x1, 300, state=st), ctas_per_system=ctas, a_placement=place)
    D.damas_solve(ctx, D.System(A, b, x1, 200, state=st, init=D.INIT_STATE), ctas_per_system=2, a_placement=2)
    x2 = torch.zeros(S, device="cuda")
    D.damas_solve(ctx, D.System(A, b, x2, 500), ctas_per_system=ctas, a_placement=place)
    x3 = torch.zeros(S, device="cuda")
    D.damas_solve(ctx, D.System(A, b, x3, 500), ctas_per_system=5, a_placement=2)
    assert torch.equal(x1, x2) and torch.equal(x2, x3)


def test_sweep_warm_start_from_x(ctx):
    A64, b64 = _compressed_system()
    S = len(b64)
    xo_half = _oracle_fp32_inputs(A64, b64, 200)
    A = padded(A64)
    b = torch.as_tensor(b64.astype(np.float32), device="cuda")
    x = torch.as_tensor(xo_half.astype(np.float32), device="cuda")
    D.damas_solve(ctx, D.System(A, b, x, 300, init=D.INIT_X), ctas_per_system=3)
    xo = O.gauss_seidel(A64.astype(np.float32).astype(np.float64), b64.astype(np.float32).astype(np.float64), 300,
                        x0=xo_half.astype(np.float32).astype(np.float64))
    assert rel_l2(x.cpu().numpy(), xo) <= 1e-4


def test_batched_systems_equal_solo(ctx):
    rng = np.random.default_rng(11)
    systems, solo = [], []
    for S in (40, 257, 600, 96):
        A64, b64 = synth.random_psd_system(rng, S)
        A = padded(A64)
        b = torch.as_tensor(b64.astype(np.float32), device="cuda")
        systems.append(D.System(A, b, torch.zeros(S, device="cuda"), 150))
        solo.append(D.System(A, b, torch.zeros(S, device="cuda"), 150))
    D.damas_solve(ctx, systems)
    for s in solo:
        D.damas_solve(ctx, s)
    for a, s in zip(systems, solo):
        assert torch.equal(a.x, s.x)


def test_many_systems_one_call(ctx):
    """40 systems of different sizes in one call (more than one launch used to hold):
    each equals its solo solve bit for bit and matches the oracle iteration."""
    rng = np.random.default_rng(31)
    made = [synth.random_psd_system(rng, int(S)) for S in rng.integers(40, 200, size=40)]
    systems, solo = [], []
    for A64, b64 in made:
        A = padded(A64)
        b = torch.as_tensor(b64.astype(np.float32), device="cuda")
        systems.append(D.System(A, b, torch.zeros(len(b64), device="cuda"), 80))
        solo.append(D.System(A, b, torch.zeros(len(b64), device="cuda"), 80))
    D.damas_solve(ctx, systems)
    for s_ in solo:
        D.damas_solve(ctx, s_)
    for (A64, b64), a, s_ in zip(made, systems, solo):
        assert torch.equal(a.x, s_.x)
    for q in (0, 17, 39):
        assert rel_l2(systems[q].x.cpu().numpy(), _oracle_fp32_inputs(*made[q], 80)) <= 1e-4


def test_large_batch_streamed_equals_solo(ctx):
    """A batch whose resident teams would need more than one launch is streamed so
    that all teams run side by side; every system still equals its solo solve (held
    in shared memory) bit for bit."""
    rng = np.random.default_rng(21)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    S = 1050                               # BF16 A: a resident team (larger than the single-CTA default)
    n, R, res = D.damas_solve_plan(ctx, S, D.BF16)
    assert res and n > 1
    k = sms // n + 2                       # more resident CTAs than SMs
    made = [synth.random_psd_system(rng, S) for _ in range(k)]
    systems, solo = [], []
    for A64, b64 in made:
        A = padded(A64, torch.bfloat16)
        b = torch.as_tensor(b64.astype(np.float32), device="cuda")
        systems.append(D.System(A, b, torch.zeros(S, device="cuda"), 100))
        solo.append(D.System(A, b, torch.zeros(S, device="cuda"), 100))
    D.damas_solve(ctx, systems)
    for s_ in solo:
        D.damas_solve(ctx, s_)
    for (A64, b64), a, s_ in zip(made, systems, solo):
        assert torch.equal(a.x, s_.x)
    assert rel_l2(systems[0].x.cpu().numpy(), _oracle_fp32_inputs(*made[0], 100, bf16=True)) <= 1e-4


def test_equal_teams_one_cluster_each(ctx):
    """Systems whose teams have the same size run as one thread-block cluster per
    team: each result equals the same system solved alone (cooperative or one
    cluster) and under a forced cooperative-sized team of another size, bit for bit,
    and matches the oracle iteration."""
    rng = np.random.default_rng(12)
    made = [synth.random_psd_system(rng, S) for S in (300, 290, 310, 257, 280, 300)]
    for ctas in (2, 3, 5):
        systems, solo = [], []
        for A64, b64 in made:
            A = padded(A64)
            b = torch.as_tensor(b64.astype(np.float32), device="cuda")
            systems.append(D.System(A, b, torch.zeros(len(b64), device="cuda"), 120, ctas=ctas))
            solo.append(D.System(A, b, torch.zeros(len(b64), device="cuda"), 120))
        sizes = {D.damas_solve_plan(ctx, s.b.numel(), ctas=ctas)[0] for s in systems}
        assert len(sizes) == 1 and min(sizes) >= 2   # one team size: the clustered launch
        D.damas_solve(ctx, systems)
        for s in solo:
            D.damas_solve(ctx, s)
        for (A64, b64), a, s in zip(made, systems, solo):
            assert torch.equal(a.x, s.x)
            assert rel_l2(a.x.cpu().numpy(), _oracle_fp32_inputs(A64, b64, 120)) <= 1e-4


def test_sweep_wait_timeout_reports_status_and_context_survives(ctx):
    """A withheld block flag makes the other CTAs' bounded waits run out: the
    call reports DAMAS_ETIMEDOUT, no GPU fault, and the next solve is correct."""
    A64, b64 = synth.random_psd_system(np.random.default_rng(5), 200)
    with pytest.raises(D.DamasError) as ei:
        _solve_gpu(ctx, A64, b64, 20, ctas_per_system=3, timeout_ms=200, withhold_block=1)
    assert ei.value.code == D._lib.DAMAS_ETIMEDOUT
    x = _solve_gpu(ctx, A64, b64, 20, ctas_per_system=3)
    assert rel_l2(x, _oracle_fp32_inputs(A64, b64, 20)) <= 1e-4
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    _solve_gpu(ctx, A64, b64, 5, ctas_per_system=3, timeout_ms=100, withhold_block=2, status=st)
    torch.cuda.synchronize()
    assert st.item() == D._lib.DAMAS_ETIMEDOUT


def test_invalid_arguments_are_rejected(ctx):
    A, b = synth.random_psd_system(np.random.default_rng(0), 40)
    At = padded(A)
    bt = torch.as_tensor(b.astype(np.float32), device="cuda")
    x = torch.zeros(40, device="cuda")
    with pytest.raises(D.DamasError):
        D.damas_solve(ctx, D.System(At[:, :40].contiguous(), bt, x, 5))   # lda not a multiple of 32
    with pytest.raises(D.DamasError):
        D.damas_solve(ctx, D.System(At, bt, x, 5, init=D.INIT_STATE))     # no state buffer
    with pytest.raises(D.DamasError):
        D.wavelet_compress_grid(ctx, bt, 5, 8, 0)                         # levels 0
