"""Oracle pins for neighbour padding of the compressed grid (an extension aimed at
the aliasing §5 reports on the compressed grid): closed forms for isolated
points, clipping at edges and corners, composition of dilations, and agreement
with scipy's binary dilation by a square structuring element."""
import numpy as np
import pytest

import oracle as O


def test_radius_zero_is_the_sorted_set_without_repeats():
    idx = np.array([17, 3, 3, 40, 0, 17], np.int32)
    assert O.pad_grid(idx, 9, 5, 0).tolist() == [0, 3, 17, 40]


@pytest.mark.parametrize("r", [1, 2, 3])
def test_isolated_interior_point_gives_its_square(r):
    nx, ny, ix, iy = 13, 11, 6, 5
    got = O.pad_grid([iy * nx + ix], nx, ny, r)
    want = sorted((iy + dy) * nx + ix + dx for dy in range(-r, r + 1) for dx in range(-r, r + 1))
    assert got.tolist() == want
    assert len(got) == (2 * r + 1) ** 2


@pytest.mark.parametrize("r", [1, 2])
def test_corner_and_edge_points_are_clipped(r):
    nx, ny = 10, 8
    assert len(O.pad_grid([0], nx, ny, r)) == (r + 1) ** 2
    assert len(O.pad_grid([nx * ny - 1], nx, ny, r)) == (r + 1) ** 2
    assert len(O.pad_grid([4], nx, ny, r)) == (r + 1) * (2 * r + 1)          # bottom edge, interior column
    assert len(O.pad_grid([3 * nx], nx, ny, r)) == (r + 1) * (2 * r + 1)     # left edge, interior row


def test_out_of_range_entries_are_ignored():
    assert O.pad_grid([-1, 12, 99], 4, 3, 0).tolist() == []
    assert O.pad_grid([-5, 5, 1000], 4, 3, 0).tolist() == [5]


def test_dilations_compose():
    rng = np.random.default_rng(3)
    nx, ny = 23, 17
    idx = rng.choice(nx * ny, 12, replace=False)
    for r1, r2 in [(1, 1), (1, 2), (2, 3)]:
        two = O.pad_grid(O.pad_grid(idx, nx, ny, r1), nx, ny, r2)
        assert two.tolist() == O.pad_grid(idx, nx, ny, r1 + r2).tolist()


@pytest.mark.parametrize("r", [0, 1, 2, 4])
def test_matches_binary_dilation_by_a_square(r):
    ndi = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(10 + r)
    nx, ny = 31, 19
    idx = rng.choice(nx * ny, 25, replace=False)
    mask = np.zeros((ny, nx), bool)
    mask.flat[idx] = True
    want = mask if r == 0 else ndi.binary_dilation(mask, structure=np.ones((2 * r + 1, 2 * r + 1), bool))
    assert O.pad_grid(idx, nx, ny, r).tolist() == np.flatnonzero(want).tolist()


def test_padding_contains_the_input_and_is_bounded():
    rng = np.random.default_rng(5)
    nx, ny, r = 40, 40, 2
    idx = np.unique(rng.choice(nx * ny, 60, replace=False)).astype(np.int32)
    out = O.pad_grid(idx, nx, ny, r)
    assert set(idx.tolist()) <= set(out.tolist())
    assert len(idx) <= len(out) <= len(idx) * (2 * r + 1) ** 2
    assert np.all(np.diff(out) > 0)
