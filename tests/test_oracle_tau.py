"""The three expressions of the PPP stabilization parameter (Sec. 4.3) in the
oracle, pinned to what the paper fixes: the values of Eqs. tau-white, tau-sun
and tau-monforte at their special points, the Sec. 5.1 checkerboard study with
tau_S (the oscillation removed, the same solution as tau_W away from the
drainage boundary layer), and tau_M against tau_W on a dynamic footing
(Sec. 5.2: both give about the same pressures)."""
import math
from dataclasses import replace
from types import SimpleNamespace

import numpy as np
import pytest

from oracle import oracle as O
from paper_1905_00671_gb300 import inputs as I


def _w(kind, dynamic=True, stabilize=True, scale=1.0, h=0.1):
    return SimpleNamespace(stabilize=stabilize, tau_kind=kind, tau_scale=scale, h=h, beta=0.3025,
                           gamma=0.6, dynamic=dynamic)


LAM, G = np.array([1.5e7, 4.0e6]), np.array([1.0e7, 2.5e6])
M = LAM + 2.0 * G


def test_tau_white_is_half_inverse_shear_modulus_for_any_step():
    for dt in (1e-4, 1.0, 1e3):
        tau = O.stabilization_parameter(_w(I.TAU_WHITE), LAM, G, np.array([1e-9, 1e-12]), dt)
        np.testing.assert_array_equal(tau, 1.0 / (2.0 * G))
    tau = O.stabilization_parameter(_w(I.TAU_WHITE, scale=10.0), LAM, G, np.zeros(2), 1.0)
    np.testing.assert_allclose(tau, 10.0 / (2.0 * G), rtol=1e-15)


def test_unstabilized_is_zero_for_every_kind():
    for kind in (I.TAU_WHITE, I.TAU_SUN, I.TAU_MONFORTE):
        tau = O.stabilization_parameter(_w(kind, stabilize=False), LAM, G, np.ones(2), 1.0)
        np.testing.assert_array_equal(tau, 0.0)


def test_tau_sun_special_points():
    kap = np.array([1e-9, 1e-12])
    # dt -> 0: (1 + tanh 2) / M, the P-wave modulus M = K + 4G/3 = lambda + 2G
    tau0 = O.stabilization_parameter(_w(I.TAU_SUN), LAM, G, kap, 0.0)
    np.testing.assert_allclose(tau0, (1.0 + math.tanh(2.0)) / M, rtol=1e-15)
    # c_v dt / h^2 = 1/3: the first factor vanishes
    h = 0.1
    dt = h * h / (3.0 * M * kap)
    for i in range(2):
        k1 = np.full(2, kap[i])
        t = O.stabilization_parameter(_w(I.TAU_SUN, h=h), LAM, G, k1, dt[i])
        assert abs(t[i]) * M[i] < 1e-12
    # large c_v dt / h^2: tanh(2 - 12 r) -> -1, tau_S -> 0
    t = O.stabilization_parameter(_w(I.TAU_SUN, h=h), LAM, G, kap, 1e6)
    assert np.all(np.abs(t) * M < 1e-12)
    # it depends on h only through c_v dt / h^2
    t1 = O.stabilization_parameter(_w(I.TAU_SUN, h=0.1), LAM, G, kap, 2.0)
    t2 = O.stabilization_parameter(_w(I.TAU_SUN, h=0.2), LAM, G, kap, 8.0)
    np.testing.assert_allclose(t1, t2, rtol=1e-14)


def test_tau_monforte_special_points():
    kap = np.array([1e-9, 0.0])
    # dt -> 0 (or kappa = 0): 2 kappa / c_v = 2 / M
    np.testing.assert_allclose(O.stabilization_parameter(_w(I.TAU_MONFORTE), LAM, G, kap, 0.0), 2.0 / M,
                               rtol=1e-15)
    np.testing.assert_allclose(O.stabilization_parameter(_w(I.TAU_MONFORTE), LAM, G, kap, 5.0)[1],
                               2.0 / M[1], rtol=1e-15)
    # zero exactly where 2/M = (beta/gamma) 12 kappa dt / h^2, and clamped to 0 beyond
    w = _w(I.TAU_MONFORTE)
    dt0 = (2.0 / M[0]) / ((w.beta / w.gamma) * 12.0 * kap[0] / (w.h * w.h))
    assert abs(O.stabilization_parameter(w, LAM, G, kap, dt0)[0]) * M[0] < 1e-12
    assert O.stabilization_parameter(w, LAM, G, kap, 10 * dt0)[0] == 0.0
    # linear in dt below the clamp, slope -(beta/gamma) 12 kappa / h^2
    a, b = (O.stabilization_parameter(w, LAM, G, kap, t)[0] for t in (0.1 * dt0, 0.2 * dt0))
    np.testing.assert_allclose(b - a, -(w.beta / w.gamma) * 12.0 * kap[0] / (w.h * w.h) * 0.1 * dt0,
                               rtol=1e-9)


def test_tau_monforte_is_for_dynamic_steps_only():
    with pytest.raises(ValueError):
        O.stabilization_parameter(_w(I.TAU_MONFORTE, dynamic=False), LAM, G, np.ones(2), 1.0)


def _terzaghi(n, kind, stabilize=True):
    w = replace(I.paper_terzaghi(n, stabilize=stabilize), tau_kind=kind)
    o = O.Oracle(w, newton_rtol=1e-10, newton_stag=1e-6)
    o.step()
    _, X, _ = o.last
    P = X.reshape(-1, 3)[:, 2].reshape(n + 1, 2)[:, 0] / 1e3   # nodal p / load, bottom to top
    interior = P[:-3]
    amp = np.abs(interior[1:-1] - 0.5 * (interior[:-2] + interior[2:])).max()
    return P, amp


@pytest.mark.parametrize("n", [40, 80])
def test_tau_sun_removes_the_checkerboard_like_tau_white(n):
    """Sec. 5.1, two discretisations: tau_S and tau_W give more or less the same
    solution; they differ only in the boundary layer under the drained top."""
    _, amp_u = _terzaghi(n, I.TAU_WHITE, stabilize=False)
    P_w, amp_w = _terzaghi(n, I.TAU_WHITE)
    P_s, amp_s = _terzaghi(n, I.TAU_SUN)
    assert amp_u > 0.3
    assert amp_s < 0.05 * amp_u and amp_w < 0.05 * amp_u
    assert np.abs(P_s - P_w)[:-5].max() < 1e-3      # below the 4 cells of the boundary layer
    assert np.abs(P_s - P_w).max() < 0.1


def test_tau_monforte_close_to_tau_white_on_a_dynamic_footing():
    """Sec. 5.2: tau_M and tau_W give about the same pressures; without
    stabilization the pressure field is far from both."""
    w0 = I.small_footing(seed=7, body=(24, 12), pad=2, h=0.25)
    p = {}
    for key, w in (("W", w0), ("M", replace(w0, tau_kind=I.TAU_MONFORTE)), ("u", replace(w0, stabilize=False))):
        o = O.Oracle(w, newton_rtol=1e-10, newton_stag=1e-6)
        for _ in range(4):
            o.step()
        p[key] = o.state()["p"]
    scale = np.abs(p["W"]).max()
    assert np.abs(p["M"] - p["W"]).max() < 0.05 * scale
    assert np.abs(p["u"] - p["W"]).max() > 0.3 * scale
