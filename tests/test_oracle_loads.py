"""Neumann data in the oracle (reading R10: each surface point carries its
measure A and adds N_a(x_p + lp n) t A to the momentum rows, and
-N_a(x_p + lp n) q A to the mass rows, of its support nodes, N the linear hat
basis).  The hat basis sums to one and reproduces linear fields, so over all
nodes the load terms give exactly the total force sum_p t A, its first moment
sum_p t A (x_p + lp n), and the total flux -sum_p q A."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1905_00671_gb300 import inputs as I


def _load_terms(w, trac, flux):
    o = O.Oracle(w)
    prep = o.prepare(w.dt)
    X = o.initial_guess(prep)
    R1, _ = o.eval(prep, X, trac, flux, want_J=False)
    R0, _ = o.eval(prep, X, np.zeros_like(trac), np.zeros_like(flux), want_J=False)
    return o, (R1 - R0).reshape(o.nn, w.dim + 1)


@pytest.mark.parametrize("case", ["footing-2d", "block-3d"])
def test_neumann_terms_sum_to_the_applied_force_flux_and_moment(case):
    if case == "footing-2d":
        w = I.small_footing(seed=3, body=(16, 8), pad=2, h=0.25, dynamic=False, jitter=0.0)
    else:
        w = I.small_block(seed=3, body=(6, 6, 4), pad=1, h=0.25, jitter=0.0)
    d = w.dim
    rng = np.random.default_rng(4)
    trac = 1e4 * rng.standard_normal((w.n_surf, d))        # any traction per surface point
    flux = 1e-6 * rng.standard_normal(w.n_surf)
    o, dR = _load_terms(w, trac, flux)
    sid = w.surf_id
    on = sid >= 0
    A = w.surf_area[on]
    t = trac[sid[on]]
    q = flux[sid[on]]
    y = w.x[on] + w.lp[on] * w.surf_normal[on]             # where the hat basis is evaluated
    nodes = I.node_coords(d, w.ncell) * w.h
    scale = np.abs(t * A[:, None]).sum()
    np.testing.assert_allclose(dR[:, :d].sum(axis=0), (t * A[:, None]).sum(axis=0), rtol=0, atol=1e-12 * scale)
    moment = np.einsum("ai,aj->ij", dR[:, :d], nodes)
    np.testing.assert_allclose(moment, np.einsum("pi,pj->ij", t * A[:, None], y), rtol=0,
                               atol=1e-12 * scale * np.abs(nodes).max())
    np.testing.assert_allclose(dR[:, d].sum(), -(q * A).sum(), rtol=0, atol=1e-12 * np.abs(q * A).sum())
