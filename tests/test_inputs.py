"""The seeded workload recipes (no GPU): the sizes the measurements are quoted
on, GIMP domains inside the grid (the padding rule of the support reading), the
3D slope's geometry, pore pressure and boundary data, the volume of the filled
cells, and reproducibility from the seed."""
import numpy as np
import pytest

from paper_1905_00671_gb300 import inputs as I

SIZES = {
    "terzaghi-4x40": (lambda: I.terzaghi_column(), 640),
    "footing-200x100": (lambda: I.strip_footing(), 80_000),
    "block3d-64x64x32": (lambda: I.consolidation_block(), 1_048_576),
    "slope-128x128x64": (lambda: I.slope_3d(), 4_208_640),
    "harmonic-footing-40x40": (lambda: I.harmonic_footing(), 6_400),
}


@pytest.fixture(scope="module")
def built():
    return {name: make() for name, (make, _) in SIZES.items()}


@pytest.mark.parametrize("name", list(SIZES))
def test_sizes_and_domains(built, name):
    w = built[name]
    assert w.n == SIZES[name][1]
    d = w.dim
    lo = np.asarray(w.origin[:d])
    hi = lo + np.asarray(w.ncell[:d]) * w.h
    # each point's GIMP domain (x -+ lp) stays inside the grid; original MPM points strictly inside
    assert np.all(w.x - w.lp >= lo - 1e-12) and np.all(w.x + w.lp <= hi + 1e-12)
    if w.shape == I.ORIG:
        assert np.all(w.x > lo) and np.all(w.x < hi)
    assert np.all(w.vol > 0) and np.all(w.lp > 0)
    assert w.u_fixed.shape == (w.nnodes, d) and w.p_fixed.shape == (w.nnodes,)


def test_filled_volume(built):
    # points tile their cells exactly: the volumes sum to the filled cells' volume
    for name, w in built.items():
        cells = w.n / 2 ** w.dim if name != "terzaghi-4x40" else w.n / 4
        np.testing.assert_allclose(w.vol.sum(), cells * w.h ** w.dim, rtol=1e-12, err_msg=name)


def test_slope_geometry_pressure_and_boundaries(built):
    w = built["slope-128x128x64"]
    h, nc = w.h, w.ncell
    tan30 = np.tan(np.deg2rad(30.0))
    # the points fill the cells whose centre is below the clipped ground line
    xc = (np.floor(w.x[:, 0] / h) + 0.5) * h
    zs = np.clip(1.2 + tan30 * (xc - 2.9), 1.2, 5.2)
    top = (np.floor(w.x[:, 2] / h) + 1) * h           # top face of the point's cell
    assert np.all(top <= np.floor(zs / h + 0.5) * h + 1e-9)
    # hydrostatic pore pressure below the water table at mid-height, none above
    zw = 0.5 * nc[2] * h
    np.testing.assert_allclose(w.p0, np.maximum(1000.0 * 9.81 * (zw - w.x[:, 2]), 0.0), rtol=1e-14)
    assert w.g == (0.0, 0.0, -9.81) and not w.dynamic
    nco = I.node_coords(3, nc)
    assert np.all(w.u_fixed[nco[:, 2] == 0] == 1)                       # fixed bottom
    side_x = (nco[:, 0] == 0) | (nco[:, 0] == nc[0])
    side_y = (nco[:, 1] == 0) | (nco[:, 1] == nc[1])
    assert np.all(w.u_fixed[side_x, 0] == 1) and np.all(w.u_fixed[side_y, 1] == 1)   # rollers
    inner = (~side_x) & (~side_y) & (nco[:, 2] > 0)
    assert not w.u_fixed[inner].any()
    # drained ground surface at the water table's pressure
    pf = w.p_fixed.astype(bool)
    assert pf.any()
    np.testing.assert_allclose(w.p_value[pf], np.maximum(1000.0 * 9.81 * (zw - nco[pf, 2] * h), 0.0), rtol=1e-14)


def test_batch_sizes_and_kinds():
    ws = I.batch_instances(256)
    assert len(ws) == 256 and sum(w.n for w in ws) == 3_572_300
    for i, w in enumerate(ws):
        if i % 2 == 0:
            assert w.shape == I.ORIG and not w.dynamic and w.dt == 1.0
        else:
            assert w.shape == I.GIMP and w.dynamic and w.dt == 1e-3
        assert 16 <= w.ncell[0] <= 128 and 32 <= w.ncell[1] - (0 if i % 2 == 0 else 2) <= 64


def test_recipes_are_reproducible():
    a, b = I.small_footing(seed=9), I.small_footing(seed=9)
    for f in ("x", "vol", "lp", "p0", "E", "k"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f))
    c = I.small_footing(seed=10)
    assert not np.array_equal(a.x, c.x)
