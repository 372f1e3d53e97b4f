"""Pins of the oracle's shape functions, binning and sparsity (CPU only).

Each check is fixed by the mathematics, not by the oracle itself:
partition of unity, linear-field reproduction, brute-force midpoint integration
of the GIMP integral (Eq. gimp-basis), GIMP == FE basis when a domain touches
cell faces only (Sec. 5, first example), the constant basis S0 summing to one
(Sec. 4.4), and brute-force enumeration of the coupling pattern.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1905_00671_gb300 import inputs as I


def brute_gimp(dx, lp, h, ncell, node, nsamp=200000):
    """Midpoint rule over the (grid-clipped) particle domain, many samples."""
    lo, hi = max(dx - lp, 0.0), min(dx + lp, ncell * h)
    t = lo + (np.arange(nsamp) + 0.5) / nsamp * (hi - lo)
    xi = t / h - node
    N = np.clip(1.0 - np.abs(xi), 0.0, None)
    dN = np.where(np.abs(xi) < 1.0, -np.sign(xi) / h, 0.0)
    return N.mean(), dN.mean()


@pytest.mark.parametrize("seed", range(5))
def test_gimp_1d_matches_brute_force(seed):
    rng = np.random.default_rng(seed)
    h, ncell = 0.3, 10
    for _ in range(20):
        lp = rng.uniform(0.05, 0.49) * h
        dx = rng.uniform(0.0, ncell * h)
        dx = min(max(dx, 1e-9), ncell * h - 1e-9)
        first, S, dS, S0 = O.shape_1d(I.GIMP, dx, lp, h, ncell)
        for s in range(len(S)):
            bN, bdN = brute_gimp(dx, lp, h, ncell, first + s)
            assert abs(S[s] - bN) < 2e-6
            assert abs(dS[s] - bdN) < 2e-6 / h * 10


@pytest.mark.parametrize("shape", [I.ORIG, I.GIMP])
def test_partition_of_unity_and_linear_reproduction(shape):
    rng = np.random.default_rng(1)
    h, ncell = 0.25, 12
    for _ in range(200):
        lp = rng.uniform(0.05, 0.49) * h
        dx = rng.uniform(lp, ncell * h - lp)   # domain inside the grid
        first, S, dS, S0 = O.shape_1d(shape, dx, lp, h, ncell)
        xs = (first + np.arange(len(S))) * h
        assert abs(S.sum() - 1.0) < 1e-14
        assert abs(dS.sum()) < 1e-12 / h
        assert abs(S0.sum() - 1.0) < 1e-14
        assert abs((S * xs).sum() - dx) < 1e-13 * ncell * h    # sum S_i x_i = x_p
        assert abs((dS * xs).sum() - 1.0) < 1e-12               # gradient of x is 1
        assert np.all(S >= 0.0)


def test_gimp_clipped_at_grid_wall_still_sums_to_one():
    h, ncell = 0.25, 8
    lp = 0.3 * h
    for dx in [1e-6, 0.1 * h, ncell * h - 0.1 * h]:
        first, S, dS, S0 = O.shape_1d(I.GIMP, dx, lp, h, ncell)
        assert first >= 0 and first + len(S) - 1 <= ncell
        assert abs(S.sum() - 1.0) < 1e-14 and abs(S0.sum() - 1.0) < 1e-14


def test_gimp_equals_fe_basis_when_domains_touch_faces_only():
    # points at 1/4 and 3/4 of a cell with lp = h/4: domains cover half cells
    h, ncell = 0.25, 6
    for c in range(ncell):
        for frac in (0.25, 0.75):
            dx = (c + frac) * h
            fg, Sg, dSg, S0g = O.shape_1d(I.GIMP, dx, 0.25 * h, h, ncell)
            fo, So, dSo, S0o = O.shape_1d(I.ORIG, dx, 0.25 * h, h, ncell)
            assert fg == fo and len(Sg) == len(So) == 2
            np.testing.assert_allclose(Sg, So, rtol=0, atol=1e-15)
            np.testing.assert_allclose(dSg, dSo, rtol=1e-14)
            np.testing.assert_allclose(S0g, S0o, rtol=0, atol=1e-15)


def test_original_mpm_constant_basis_is_cell_average_weight():
    # R5: for a point domain S0 = 1/2 per node and axis -> 1/4 on the 4 cell nodes
    first, S, dS, S0 = O.shape_1d(I.ORIG, 0.37, 0.01, 0.25, 4)
    np.testing.assert_array_equal(S0, [0.5, 0.5])


def test_out_of_grid_is_rejected():
    with pytest.raises(O.OracleError):
        O.shape_1d(I.ORIG, -1e-12, 0.1, 0.25, 4)
    with pytest.raises(O.OracleError):
        O.shape_1d(I.GIMP, 4 * 0.25, 0.05, 0.25, 4)


def test_binning_order_is_cell_then_index():
    w = I.small_footing(seed=3)
    g = O.grid_struct(w.dim, w.shape, w.ncell, w.origin, w.h)
    cell, order = O.binning(g, w.x)
    cx = np.floor(w.x[:, 0] / w.h).astype(int)
    cy = np.floor(w.x[:, 1] / w.h).astype(int)
    np.testing.assert_array_equal(cell, cx + w.ncell[0] * cy)
    key = cell[order].astype(np.int64) * w.n + order
    assert np.all(np.diff(key) > 0)
    assert sorted(order.tolist()) == list(range(w.n))


@pytest.mark.parametrize("shape", [I.ORIG, I.GIMP])
def test_pattern_matches_brute_force(shape):
    w = I.small_footing(seed=5, shape=shape, body=(6, 4), pad=1)
    g = O.grid_struct(w.dim, w.shape, w.ncell, w.origin, w.h)
    first, count, S, dS, S0 = O.shape(g, w.x, w.lp)
    row_ptr, col = O.pattern(g, first, count)
    nn0 = w.ncell[0] + 1
    nn = w.nnodes
    dense = np.eye(nn, dtype=bool)
    for p in range(w.n):
        nodes = [(first[p, 0] + i) + nn0 * (first[p, 1] + j)
                 for j in range(count[p, 1]) for i in range(count[p, 0])]
        for a in nodes:
            for b in nodes:
                dense[a, b] = True
    rows = np.repeat(np.arange(nn), np.diff(row_ptr))
    got = np.zeros_like(dense)
    got[rows, col] = True
    np.testing.assert_array_equal(got, dense)
    for a in range(nn):   # ascending columns within each row
        assert np.all(np.diff(col[row_ptr[a]:row_ptr[a + 1]]) > 0)
    np.testing.assert_array_equal(dense, dense.T)
