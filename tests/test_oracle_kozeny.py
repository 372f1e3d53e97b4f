"""Permeability from porosity (Eq. kozeny-carman) and the self-weight
consolidation set-up of Sec. 5.3 in the oracle, pinned to: hand-computed values
of the Kozeny-Carman relation, the Darcy part of the mass residual scaling by
exactly k(J)/k0 at a uniform compression, the Jacobian (with dk/dJ) against
central differences at a compacted state, the undrained response to gravity
(pore pressure = overburden, checkerboard without stabilization, converging
with it on refinement), and the dissipation of the excess pressure."""
from dataclasses import replace

import numpy as np
import pytest

from oracle import oracle as O
from paper_1905_00671_gb300 import inputs as I
from tests.test_oracle_physics import dense_J, perturbed_X

H = 2.0
RHO = 0.5 * 2600.0 + 0.5 * 1000.0   # mixture density at phi0 = 0.5


def test_kozeny_carman_values():
    # phi0 = 0.5: (1 - phi0)^2 / phi0^3 = 2; phi = 1 - 0.5 / J
    assert O.kozeny_carman(1.0, 0.5, 1.0) == 1.0                           # phi = phi0
    np.testing.assert_allclose(O.kozeny_carman(1.0, 0.5, 0.8), 0.27, rtol=1e-14)   # phi = 3/8
    np.testing.assert_allclose(O.kozeny_carman(1.0, 0.5, 2.0), 13.5, rtol=1e-14)   # phi = 3/4
    assert O.kozeny_carman(1.0, 0.5, 0.5) == 0.0                           # pores closed
    assert O.kozeny_carman(1.0, 0.5, 0.4) == 0.0
    # another phi0: 0.33 at J = 1 gives k0 back
    np.testing.assert_allclose(O.kozeny_carman(3e-12, 0.33, 1.0), 3e-12, rtol=1e-14)


def _column(n=4, **kw):
    # the body fills the grid (original MPM): every node active, bases exactly linear
    return I.self_weight_consolidation(ncell=(n, n), h=H / n, ppc_axis=2, **kw)


def test_darcy_term_scales_with_kozeny_carman():
    """Uniform compression J = 0.8 and a linear pressure field, no gravity, no
    stabilization: the mass rows' Darcy part sum_p vol k(J)/mu_f grad S . grad p
    is exactly 0.27 times its value with the constant permeability."""
    out = {}
    for perm in (I.PERM_CONSTANT, I.PERM_KOZENY_CARMAN):
        w = replace(_column(K=1.5e6, k0=1e-10), g=(0.0, 0.0, 0.0), stabilize=False, permeability=perm)
        o = O.Oracle(w)
        prep = o.prepare(1.0)
        nc = I.node_coords(2, w.ncell) * w.h
        X = np.zeros((o.nn, 3))
        X[:, 1] = -0.2 * nc[:, 1]                       # dF = diag(1, 0.8)
        with_p = X.copy()
        with_p[:, 2] = 1e4 * nc[:, 0]
        Rp = o.eval(prep, with_p.reshape(-1), None, want_J=False)[0].reshape(-1, 3)[:, 2]
        R0 = o.eval(prep, X.reshape(-1), None, want_J=False)[0].reshape(-1, 3)[:, 2]
        out[perm] = Rp - R0
    scale = np.abs(out[I.PERM_CONSTANT]).max()
    assert scale > 0
    np.testing.assert_allclose(out[I.PERM_KOZENY_CARMAN], 0.27 * out[I.PERM_CONSTANT], rtol=0,
                               atol=1e-12 * scale)


def test_jacobian_matches_central_differences_kozeny():
    """dk/dJ enters the displacement columns of the mass rows; checked at a
    state compacted by 5 % with a pressure gradient and gravity."""
    w = _column(n=3, K=1.5e6, k0=1e-10)
    o = O.Oracle(w)
    prep = o.prepare(w.dt)
    nc = I.node_coords(2, w.ncell) * w.h
    X = perturbed_X(o, prep, 1).reshape(-1, 3)
    X[:, 1] -= 0.05 * nc[:, 1]
    X[:, 2] += 2e4 * (H - nc[:, 1])
    X = X.reshape(-1)
    R, Jv = o.eval(prep, X, None)
    J = dense_J(o, prep, Jv)
    Jfd = np.zeros_like(J)
    for j in range(o.nn * 3):
        hstep = 1e-5 * (1e-3 if j % 3 < 2 else 1e3)
        Xp, Xm = X.copy(), X.copy()
        Xp[j] += hstep
        Xm[j] -= hstep
        Jfd[:, j] = (o.eval(prep, Xp, None, want_J=False)[0] - o.eval(prep, Xm, None, want_J=False)[0]) / (2 * hstep)
    for r in range(3):
        for c in range(3):
            A, B = J[r::3, c::3], Jfd[r::3, c::3]
            scale = max(np.abs(A).max(), np.abs(B).max())
            assert np.abs(A - B).max() <= 1e-6 * scale, (r, c)
    # without the dk/dJ term the displacement columns of the mass rows would differ
    wc = replace(w, permeability=I.PERM_CONSTANT)
    oc = O.Oracle(wc)
    _, Jc = oc.eval(oc.prepare(w.dt), X, None)
    assert not np.allclose(dense_J(oc, prep, Jc)[2::3, 0::3], J[2::3, 0::3], rtol=1e-6, atol=0)


def _undrained(n, stabilize):
    w = _column(n=n, K=1.5e6, k0=1e-14, stabilize=stabilize)
    o = O.Oracle(w, newton_rtol=1e-10, newton_stag=1e-6)
    o.step(w.dt)
    _, X, _ = o.last
    P = X.reshape(-1, 3)[:, 2].reshape(n + 1, n + 1)          # [row y][column x]
    y = np.arange(n + 1) * H / n
    exact = RHO * 9.81 * (H - y)                               # the overburden carried by the fluid
    dev = (P[1:-1, : n // 2] - exact[1:-1, None]) / (RHO * 9.81 * H)   # interior rows, left half
    return np.abs(dev).max()


def test_self_weight_undrained_response():
    """Sec. 5.3: gravity applied at t = 0 on a nearly undrained deposit. The
    pore pressure carries the overburden; equal-order MPM without
    stabilization oscillates; the stabilized solution is free of it and
    converges on refinement."""
    d8_u, d8_s, d16_s = _undrained(8, False), _undrained(8, True), _undrained(16, True)
    assert d8_u > 0.3
    assert d8_s < 0.03 and d16_s < 0.02
    assert d16_s < d8_s


def test_self_weight_consolidation_dissipates():
    """Growing steps (dt x 1.2): the excess pore pressure over the hydrostatic
    state decays and the top settles, both monotonically."""
    w = _column(n=8, K=1.5e6, k0=1e-10)
    o = O.Oracle(w, newton_rtol=1e-10, newton_stag=1e-6)
    mid = (np.abs(w.x[:, 0] - 0.625) < 0.07) & (np.abs(w.x[:, 1] - 0.875) < 0.07)
    exc, settle = [], []
    for dt in w.step_sizes(10):
        info = o.step(dt)
        assert info.newton_iters <= 5
        st = o.state()
        exc.append((st["p"][mid] - 1000.0 * 9.81 * (H - w.x[mid, 1])).mean())
        settle.append(-st["u"][w.x[:, 1] > H - 0.2, 1].mean())
    exc, settle = np.array(exc), np.array(settle)
    assert np.all(np.diff(exc[1:]) < 0) and exc[-1] < 0.5 * exc[0]
    assert np.all(np.diff(settle) > 0)


@pytest.mark.parametrize("model", [I.MODEL_NEOHOOKE, I.MODEL_HENCKY])
def test_self_weight_paper_setup_consolidates(model):
    """The paper's own set-up and grid (Sec. 5.3: K = 15 kPa, Kozeny-Carman,
    h = 0.125 m with 25 points per cell, dt = 0.1 s x 1.2), ten steps: Newton
    converges in every step; at t = 0.1 s the pore fluid carries the submerged
    weight (rho - rho_f) g (H - y) at mid-depth (nearly undrained); then the
    excess pressure dissipates and the top settles, step after step."""
    w = replace(I.self_weight_consolidation(), model=model)
    assert w.ncell[:2] == (16, 16) and w.n == 6400
    o = O.Oracle(w, newton_rtol=1e-8, newton_max=25)
    mid = (np.abs(w.x[:, 0] - 1.0) < 0.07) & (np.abs(w.x[:, 1] - 1.0) < 0.07)
    top = w.x[:, 1] > H - 0.1
    submerged = (RHO - 1000.0) * 9.81 * (H - w.x[mid, 1])
    exc, settle = [], []
    for dt in w.step_sizes(10):
        info = o.step(dt)
        assert info.newton_iters <= 6
        st = o.state()
        exc.append((st["p"][mid] - 1000.0 * 9.81 * (H - w.x[mid, 1])).mean())
        settle.append(-st["u"][top, 1].mean())
    assert abs(exc[0] / submerged.mean() - 1.0) < 0.05
    assert exc[-1] < 0.85 * exc[0]
    assert np.all(np.diff(settle) > 0) and settle[0] > 0


def test_self_weight_first_step_on_both_paper_grids():
    """Sec. 5.3 names two discretisations: h = 0.125 m with 25 points per cell
    (6,400 points) and h = 0.0625 m with 16 (16,384).  After the first 0.1 s
    the mid-depth excess pressure is within 2% of the submerged weight on both,
    and closer on the finer grid."""
    gaps = []
    for ncell, h, ppc, n in (((16, 16), 0.125, 5, 6400), ((32, 32), 0.0625, 4, 16384)):
        w = replace(I.self_weight_consolidation(ncell=ncell, h=h, ppc_axis=ppc), model=I.MODEL_HENCKY)
        assert w.n == n
        o = O.Oracle(w, newton_rtol=1e-8, newton_max=25)
        info = o.step(w.dt)
        assert info.newton_iters <= 6
        mid = (np.abs(w.x[:, 0] - 1.0) < 0.07) & (np.abs(w.x[:, 1] - 1.0) < 0.07)
        exc = (o.state()["p"][mid] - 1000.0 * 9.81 * (H - w.x[mid, 1])).mean()
        gaps.append(abs(exc / ((RHO - 1000.0) * 9.81 * (H - w.x[mid, 1])).mean() - 1.0))
    assert max(gaps) < 0.02 and gaps[1] < gaps[0]
