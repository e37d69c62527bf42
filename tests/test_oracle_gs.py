"""Pins for the oracle's DAMAS Gauss-Seidel iteration (§3, Eq. (13)-(14)).

Hand-derived iterates on 2x2 and 3x3 systems (they separate Gauss-Seidel from
Jacobi and catch index slips), the unconstrained limit (a library linear solve),
the fixed-point (KKT) conditions, monotone descent of the quadratic for symmetric
PSD A, exhaustive brute force over supports on tiny grids, the unique NNLS
optimum (a library active-set solver) on 5x5 grids, and the recovery of an
on-grid monopole (§5 Case 1).
"""
import itertools

import numpy as np
import pytest

import oracle as O
import synth


def test_two_by_two_hand_iterates():
    """A = [[1, 1/2], [1/2, 1]], b = (1, 4/5), x^0 = 0.
    sweep 1: x1 = 1, x2 = 4/5 - 1/2 = 3/10;
    sweep 2: x1 = 1 - 3/20 = 17/20, x2 = 4/5 - 17/40 = 3/8.
    (Jacobi would give x2 = 4/5 in sweep 1.)"""
    A = np.array([[1.0, 0.5], [0.5, 1.0]])
    b = np.array([1.0, 0.8])
    assert np.allclose(O.gauss_seidel(A, b, 1), [1.0, 0.3], atol=1e-15)
    assert np.allclose(O.gauss_seidel(A, b, 2), [0.85, 0.375], atol=1e-15)
    # clamp: b2 small => x2 stays at 0
    assert np.allclose(O.gauss_seidel(A, np.array([1.0, 0.2]), 5), [1.0, 0.0], atol=1e-15)


def test_three_by_three_nonsymmetric_hand_iterate():
    """Non-symmetric A with unit diagonal (formulation P shape), one sweep from x^0 = (1, 1, 1):
    r1 = 1 + 0.2 + 0.1 - 1 = 0.3           -> x1 = 0.7
    r2 = 0.4*0.7 + 1 + 0.3 - 2 = -0.42      -> x2 = 1.42
    r3 = 0.5*0.7 + 0.6*1.42 + 1 - 0.1 = 2.102 -> x3 = max(1 - 2.102, 0) = 0."""
    A = np.array([[1.0, 0.2, 0.1], [0.4, 1.0, 0.3], [0.5, 0.6, 1.0]])
    b = np.array([1.0, 2.0, 0.1])
    x = O.gauss_seidel(A, b, 1, x0=np.ones(3))
    assert np.allclose(x, [0.7, 1.42, 0.0], atol=1e-14)


def test_non_unit_diagonal_division():
    """Eq. (14) divides the residual by A_ii."""
    A = np.array([[2.0, 0.0], [0.0, 4.0]])
    x = O.gauss_seidel(A, np.array([1.0, 2.0]), 1)
    assert np.allclose(x, [0.5, 0.5])


def test_unconstrained_limit_is_linear_solve():
    """With a positive solution the clamp never binds near convergence and the
    iteration converges to A^-1 b (SPD A)."""
    rng = np.random.default_rng(1)
    S = 30
    Y = rng.standard_normal((S, 2 * S))
    A = Y @ Y.T / (2 * S) + 0.5 * np.eye(S)
    d = np.sqrt(np.diag(A))
    A = A / d[:, None] / d[None, :]
    np.fill_diagonal(A, 1.0)
    xs = 1.0 + rng.random(S)
    b = A @ xs
    x = O.gauss_seidel(A, b, 3000)
    assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-10)


def _psd_case(seed, S):
    A, b = synth.random_psd_system(np.random.default_rng(seed), S)
    return A, b


def test_objective_monotone_and_kkt_at_convergence():
    A, b = _psd_case(2, 64)
    x = np.zeros(64)
    prev = O.objective(A, b, x)
    for _ in range(200):
        x = O.gauss_seidel(A, b, 1, x0=x)
        f = O.objective(A, b, x)
        assert f <= prev + 1e-12
        prev = f
    x = O.gauss_seidel(A, b, 20000, x0=x)
    assert x.min() >= 0.0
    assert O.kkt_residual(A, b, x) < 1e-7


def _brute_force_min(A, b):
    """min 0.5 x^T A x - b^T x over x >= 0 by enumerating supports: on each
    support solve the equality part, keep feasible KKT points, take the smallest
    objective (the problem is convex, so every KKT point is a minimiser)."""
    S = len(b)
    best = np.inf
    for r in range(S + 1):
        for sup in itertools.combinations(range(S), r):
            x = np.zeros(S)
            if r:
                sup = list(sup)
                xs, *_ = np.linalg.lstsq(A[np.ix_(sup, sup)], b[sup], rcond=None)
                if xs.min() < -1e-12:
                    continue
                x[sup] = xs
            g = A @ x - b
            if r and np.abs(g[sup]).max() > 1e-9:
                continue
            mask = np.ones(S, bool)
            if r:
                mask[sup] = False
            if mask.any() and g[mask].min() < -1e-9:
                continue
            best = min(best, O.objective(A, b, x))
    return best


@pytest.mark.parametrize("N,seed", [(3, 0), (3, 1), (4, 2)])
def test_brute_force_qp_on_tiny_grids(N, seed):
    """PSF systems of tiny grids (formulation E) with a two-source map: the
    Gauss-Seidel objective after many sweeps equals the exhaustive minimum."""
    rng = np.random.default_rng(seed)
    mics = synth.mic_disc(8, 0.5, rng)
    grid = synth.square_plane(N, 0.6, 1.0)
    pts = grid.points()
    src = np.array([[0.05, -0.1, 1.0], [-0.2, 0.15, 1.0]])
    C = synth.simulate_csm(mics, src, np.array([1.0, 0.6]), 2500.0, 343.0, 25.0, rng)
    A, _ = O.psf_matrix(mics, pts, 2500.0, 343.0, O.FORM_E)
    b = O.das_map(mics, pts, 2500.0, 343.0, C, O.FORM_E)
    fmin = _brute_force_min(A, b)
    x = O.gauss_seidel(A, b, 20000)
    f = O.objective(A, b, x)
    assert abs(f - fmin) <= 1e-9 * abs(fmin)


def test_on_grid_monopole_recovered():
    """§5 Case 1 analogue: a noise-free unit monopole on grid point s is
    recovered at s with the integrated power within 1% of 1."""
    sc = synth.scene_monopole_small(seed=0, snr_db=None)
    pts = sc.grid.points()
    A, g2 = O.psf_matrix(sc.mics, pts, sc.freq, sc.c, O.FORM_E)
    b = O.das_map(sc.mics, pts, sc.freq, sc.c, sc.C, O.FORM_E)
    x = O.gauss_seidel(A, b, sc.extra["iters"])
    p = O.to_power(x, g2)
    assert int(np.argmax(p)) == sc.extra["src_index"]
    assert abs(p.sum() - 1.0) < 0.01


def test_warm_start_resume_is_exact():
    """x is the whole state of the iteration: T1 sweeps then T2 more from that
    point equal T1 + T2 sweeps bit for bit."""
    A, b = _psd_case(5, 40)
    x1 = O.gauss_seidel(A, b, 70)
    x2 = O.gauss_seidel(A, b, 30, x0=x1)
    assert np.array_equal(x2, O.gauss_seidel(A, b, 100))


def test_compressed_pipeline_end_to_end():
    """§5 procedure on the 81x81 spiral scene: compressed grid of about 10% of
    the points, Gauss-Seidel on it, integrated power close to the scene's."""
    sc = synth.scene_spiral_81()
    out = O.solve_bin(sc.mics, sc.grid, sc.freq, sc.c, sc.C, 300, compressed=True, levels=2,
                      predictor=O.PRED_HAAR, eps_mode=O.EPS_KEEP_FRAC, eps=0.10)
    assert 0.095 * 6561 <= len(out["idx"]) <= 0.12 * 6561
    assert abs(out["x"].sum() - sc.powers.sum()) < 0.15 * sc.powers.sum()
    assert out["x"].min() >= 0


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_nnls_optimum_on_5x5_grids(seed):
    """5x5 grids (25 unknowns, too many supports to enumerate): with 8
    microphones the PSF matrix is positive definite, so min 0.5 x^T A x - b^T x
    over x >= 0 is the non-negative least-squares problem min |L x - y| with
    A = L^T L and L^T y = b, whose minimiser is unique.  The Lawson-Hanson NNLS
    of scipy gives it; the Gauss-Seidel iteration with the clamp must reach the
    same x after many sweeps."""
    so = pytest.importorskip("scipy.optimize")
    rng = np.random.default_rng(seed)
    mics = synth.mic_disc(8, 0.5, rng)
    grid = synth.square_plane(5, 0.6, 1.0)
    pts = grid.points()
    src = np.array([[0.05, -0.1, 1.0], [-0.2, 0.15, 1.0]])
    C = synth.simulate_csm(mics, src, np.array([1.0, 0.6]), 2500.0, 343.0, 25.0, rng)
    A, _ = O.psf_matrix(mics, pts, 2500.0, 343.0, O.FORM_E)
    b = O.das_map(mics, pts, 2500.0, 343.0, C, O.FORM_E)
    assert np.linalg.eigvalsh(A).min() > 1e-3
    L = np.linalg.cholesky(A).T
    x_nnls, _ = so.nnls(L, np.linalg.solve(L.T, b), maxiter=10000)
    x = O.gauss_seidel(A, b, 20000)
    assert np.allclose(x, x_nnls, rtol=1e-9, atol=1e-12)
    assert abs(O.objective(A, b, x) - O.objective(A, b, x_nnls)) <= 1e-12 * abs(O.objective(A, b, x_nnls))
