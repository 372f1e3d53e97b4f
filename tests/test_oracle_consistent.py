"""The consistent-mass Stage-1 mapping (Eq. map-from-particles-to-nodes-
consistent) in the oracle, pinned to two exact properties: a point field
interpolated from nodal values by the basis is mapped back to exactly those
values (the lumped mapping of Eq. map-from-particles-to-nodes smooths it), and
the mapped field keeps sum_i M_i f_i = sum_mp m f (the lumped masses are the
row sums of the consistent mass)."""
from dataclasses import replace

import numpy as np

from oracle import oracle as O
from paper_1905_00671_gb300 import inputs as I


def _column(n=6):
    # original MPM, the body filling the grid: every node active
    return I.self_weight_consolidation(ncell=(n, n), h=2.0 / n, ppc_axis=2, K=1.5e6, k0=1e-10,
                                       g=0.0, shape=I.ORIG)


def _bilinear(w, gnode, x):
    """Original MPM basis (bilinear FE functions on the cells) at x, applied to
    the nodal values gnode (x index fastest)."""
    nx = w.ncell[0] + 1
    cx = np.minimum((x[:, 0] / w.h).astype(int), w.ncell[0] - 1)
    cy = np.minimum((x[:, 1] / w.h).astype(int), w.ncell[1] - 1)
    xi, eta = x[:, 0] / w.h - cx, x[:, 1] / w.h - cy
    n00, n10 = cy * nx + cx, cy * nx + cx + 1
    n01, n11 = n00 + nx, n10 + nx
    return ((1 - xi) * (1 - eta) * gnode[n00] + xi * (1 - eta) * gnode[n10]
            + (1 - xi) * eta * gnode[n01] + xi * eta * gnode[n11])


def test_consistent_mapping_reproduces_interpolated_fields():
    w = _column()
    rng = np.random.default_rng(0)
    g = 1e4 * rng.standard_normal(w.nnodes)
    w = replace(w, p0=_bilinear(w, g, w.x))
    prep_c = O.Oracle(replace(w, p2g_mass=I.P2G_CONSISTENT)).prepare(w.dt)
    prep_l = O.Oracle(w).prepare(w.dt)
    assert np.all(prep_c["active"])
    np.testing.assert_allclose(prep_c["nodal"]["P"], g, rtol=0, atol=1e-9 * np.abs(g).max())
    assert np.abs(prep_l["nodal"]["P"] - g).max() > 0.05 * np.abs(g).max()


def test_consistent_mapping_conserves_the_mass_weighted_sum():
    w = _column()
    rng = np.random.default_rng(1)
    w = replace(w, p0=1e3 * rng.standard_normal(w.n), p2g_mass=I.P2G_CONSISTENT)
    o = O.Oracle(w)
    prep = o.prepare(w.dt)
    total = np.sum(prep["m"] * w.p0)
    np.testing.assert_allclose(np.sum(prep["M"] * prep["nodal"]["P"]), total, rtol=1e-12)


def test_consistent_mapping_keeps_inactive_nodes_lumped():
    """Nodes outside the active set (a footing with empty cells above) keep the
    lumped values; the others change."""
    w = I.small_footing(seed=8, shape=I.ORIG, body=(20, 10), pad=2)
    prep_c = O.Oracle(replace(w, p2g_mass=I.P2G_CONSISTENT)).prepare(w.dt)
    prep_l = O.Oracle(w).prepare(w.dt)
    ina = ~prep_c["active"]
    np.testing.assert_array_equal(prep_c["nodal"]["P"][ina], prep_l["nodal"]["P"][ina])
    for k in ("v", "a"):
        np.testing.assert_array_equal(prep_c["nodal"][k][ina], prep_l["nodal"][k][ina])


def test_consistent_mapping_reproduces_interpolated_fields_3d():
    """3D, original MPM, the body filling the grid: a trilinear nodal field
    sampled at the points maps back to itself under the consistent mapping."""
    w = I.consolidation_block(body=(3, 3, 3), pad=0, h=0.5, shape=I.ORIG, logk=(-10.0, -10.0))
    rng = np.random.default_rng(2)
    g = 1e4 * rng.standard_normal(w.nnodes)
    n0, n1 = w.ncell[0] + 1, w.ncell[1] + 1
    c = [np.minimum((w.x[:, k] / w.h).astype(int), w.ncell[k] - 1) for k in range(3)]
    f = [w.x[:, k] / w.h - c[k] for k in range(3)]
    p0 = np.zeros(w.n)
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                wt = ((f[0] if dx else 1 - f[0]) * (f[1] if dy else 1 - f[1]) * (f[2] if dz else 1 - f[2]))
                p0 += wt * g[(c[0] + dx) + n0 * ((c[1] + dy) + n1 * (c[2] + dz))]
    w = replace(w, p0=p0)
    prep_c = O.Oracle(replace(w, p2g_mass=I.P2G_CONSISTENT)).prepare(w.dt)
    prep_l = O.Oracle(w).prepare(w.dt)
    assert np.all(prep_c["active"])
    np.testing.assert_allclose(prep_c["nodal"]["P"], g, rtol=0, atol=1e-9 * np.abs(g).max())
    assert np.abs(prep_l["nodal"]["P"] - g).max() > 0.05 * np.abs(g).max()
