"""The dynamic (Newmark) terms of the residual in the oracle that the paper
leaves out of the linearization (Sec. 3.3), pinned by closed forms:

* the Kelvin viscous stress alpha (lambda tr D 1 + 2 (G - lambda ln J) D) of an
  affine motion from rest, by virtual work (a uniform D for a plane-strain
  uniaxial stretch and for a simple shear, the Newmark velocity being
  gamma / (beta dt) times the displacement increment);
* the fluid acceleration inside Darcy's law, q = -kappa (grad p - rho_f (g - a)),
  for a rigid translation: a = c / (beta dt^2) everywhere, and the mass rows
  change by exactly rho_f kappa V a by virtual work;
* the Jacobian at rest with the Kelvin stress against central differences: D
  vanishes at rest, so the geometric dependence the Jacobian omits does too and
  the viscous tangent gamma / (beta dt) alpha c is all that remains;
* away from rest (Kelvin stress and fluid density on, velocities and
  accelerations nonzero), the Jacobian against central differences of the
  residual with exactly the unlinearized terms frozen at the iterate (the
  Kelvin stress's geometry, Darcy's acceleration): every other term of the
  Jacobian is the exact derivative, and what it leaves out is only those terms.
"""
from dataclasses import replace

import numpy as np
import pytest

from oracle import oracle as O
from paper_1905_00671_gb300 import inputs as I
from tests.test_oracle_physics import dense_J, perturbed_X

E, NU = 12e6, 0.3
LAM = E * NU / ((1 + NU) * (1 - 2 * NU))
G = E / (2 * (1 + NU))
ALPHA = 0.05
DT = 1e-3


def _column(alpha=ALPHA, rho_f=1000.0):
    # original MPM, the body filling the grid: every node active, bases exactly linear
    w = I.terzaghi_column(ncell_y=6, ncell_x=3, h=0.25, E=E, nu=NU, k=1e-10)
    return replace(w, dynamic=True, alpha_vis=alpha, rho_f=rho_f, dt=DT,
                   trac_full=np.zeros_like(w.trac_full))


def _residual(w, X):
    o = O.Oracle(w)
    prep = o.prepare(w.dt)
    R, _ = o.eval(prep, X.reshape(-1), None, want_J=False)
    return o, R.reshape(-1, w.dim + 1)


def _affine_X(w, grad):
    """Nodal unknowns of the displacement increment x -> grad x (pressure 0)."""
    nc = I.node_coords(2, w.ncell) * w.h
    X = np.zeros((nc.shape[0], 3))
    X[:, :2] = nc @ np.asarray(grad).T
    return X, nc + X[:, :2]


def _viscous_virtual_work(grad):
    """-sum_a dR_a (x) x_a / V0 of the Kelvin term (alpha on minus alpha off)."""
    w1, w0 = _column(), _column(alpha=0.0)
    X, xcur = _affine_X(w1, grad)
    _, R1 = _residual(w1, X)
    _, R0 = _residual(w0, X)
    dR = R1[:, :2] - R0[:, :2]
    return -np.einsum("ai,aj->ij", dR, xcur) / w1.vol.sum()


@pytest.mark.parametrize("s", [0.9, 1.1])
def test_kelvin_stress_of_a_uniaxial_stretch(s):
    w = _column()
    k = w.gamma * (s - 1.0) / (w.beta * w.dt)     # grad_X v_yy of the Newmark velocity
    D = k / s                                       # grad_x v_yy = grad_X v_yy / s
    mu_p = G - LAM * np.log(s)
    sig = _viscous_virtual_work([[0.0, 0.0], [0.0, s - 1.0]])
    scale = ALPHA * (LAM + 2 * G) * abs(D)
    np.testing.assert_allclose(sig[1, 1], ALPHA * (LAM + 2 * mu_p) * D, rtol=1e-10)
    np.testing.assert_allclose(sig[0, 0], ALPHA * LAM * D, rtol=1e-10)
    assert abs(sig[0, 1]) < 1e-10 * scale and abs(sig[1, 0]) < 1e-10 * scale


def test_kelvin_stress_of_a_simple_shear():
    """dF = [[1, g], [0, 1]]: J = 1, grad_x v = k e_x (x) e_y with k = gamma g /
    (beta dt), D its symmetric part, tr D = 0: sigma_xy = alpha G k."""
    w = _column()
    gs = 0.02
    k = w.gamma * gs / (w.beta * w.dt)
    sig = _viscous_virtual_work([[0.0, gs], [0.0, 0.0]])
    scale = ALPHA * G * k
    np.testing.assert_allclose(sig[0, 1], scale, rtol=1e-10)
    np.testing.assert_allclose(sig[1, 0], scale, rtol=1e-10)
    assert abs(sig[0, 0]) < 1e-10 * scale and abs(sig[1, 1]) < 1e-10 * scale


def test_darcy_acceleration_of_a_rigid_translation():
    w = _column(alpha=0.0)
    c = np.array([2e-6, -3e-6])
    nc = I.node_coords(2, w.ncell) * w.h
    X = np.zeros((nc.shape[0], 3))
    X[:, :2] = c
    o, R1 = _residual(w, X)
    _, R0 = _residual(w, np.zeros_like(X))
    dm = R1[:, 2] - R0[:, 2]
    a = c / (w.beta * w.dt ** 2)
    kappa = w.k[0] / w.mu_f
    got = np.einsum("a,aj->j", dm, nc + c)
    np.testing.assert_allclose(got, w.rho_f * kappa * w.vol.sum() * a, rtol=1e-9)
    # no fluid density: the translation leaves the mass rows alone
    w0 = _column(alpha=0.0, rho_f=0.0)
    _, S1 = _residual(w0, X)
    _, S0 = _residual(w0, np.zeros_like(X))
    assert np.abs(S1[:, 2] - S0[:, 2]).max() < 1e-9 * np.abs(dm).max()


def test_jacobian_with_kelvin_stress_at_rest_matches_central_differences():
    w = I.small_footing(seed=4, body=(4, 3), pad=1, h=0.25, dynamic=True)
    w = replace(w, alpha_vis=0.2, rho_f=0.0, v0=None)
    o = O.Oracle(w)
    prep = o.prepare(w.dt)
    X = o.initial_guess(prep)
    trac = w.traction(w.dt)
    _, Jv = o.eval(prep, X, trac)
    J = dense_J(o, prep, Jv)
    nb = o.d + 1
    Jfd = np.zeros_like(J)
    for j in range(o.nn * nb):
        hstep = 1e-5 * (1e-3 if j % nb < o.d else 1e3)
        Xp, Xm = X.copy(), X.copy()
        Xp[j] += hstep
        Xm[j] -= hstep
        Jfd[:, j] = (o.eval(prep, Xp, trac, want_J=False)[0] - o.eval(prep, Xm, trac, want_J=False)[0]) / (2 * hstep)
    for r in range(nb):
        for cc in range(nb):
            A, B = J[r::nb, cc::nb], Jfd[r::nb, cc::nb]
            scale = max(np.abs(A).max(), np.abs(B).max())
            assert np.abs(A - B).max() <= 1e-6 * scale, (r, cc)
    # the Kelvin tangent is present: without it the displacement block differs
    o0 = O.Oracle(replace(w, alpha_vis=0.0))
    _, J0 = o0.eval(o0.prepare(w.dt), X, trac)
    A0 = dense_J(o0, prep, J0)[0::nb, 0::nb]
    assert np.abs(A0 - J[0::nb, 0::nb]).max() > 1e-3 * np.abs(J[0::nb, 0::nb]).max()


def _fd_columns(o, prep, X, fn):
    nb = o.d + 1
    Jfd = np.zeros((o.nn * nb, o.nn * nb))
    for j in range(o.nn * nb):
        hstep = 1e-5 * (1e-3 if j % nb < o.d else 1e3)
        Xp, Xm = X.copy(), X.copy()
        Xp[j] += hstep
        Xm[j] -= hstep
        Jfd[:, j] = (fn(Xp) - fn(Xm)) / (2 * hstep)
    return Jfd


# a permeable soil (k = 1e-9 m^2), so that the Darcy terms weigh in the mass
# rows as much as the Newmark divergence does
def _permeable(w):
    return replace(w, k=np.full_like(w.k, 1e-9))


FROZEN_CASES = {
    "footing2d-neohookean": lambda: _permeable(replace(
        I.small_footing(seed=4, body=(4, 3), pad=1, h=0.25, dynamic=True), alpha_vis=0.2, rho_f=1000.0)),
    "footing2d-hencky": lambda: _permeable(replace(
        I.small_footing(seed=5, body=(4, 3), pad=1, h=0.25, dynamic=True), alpha_vis=0.2, rho_f=1000.0,
        model=I.MODEL_HENCKY)),
    "block3d-neohookean": lambda: _permeable(replace(
        I.small_block(seed=6, body=(2, 2, 2)), dynamic=True, alpha_vis=0.2, rho_f=1000.0, dt=1e-3)),
    "block3d-hencky": lambda: _permeable(replace(
        I.small_block(seed=7, body=(2, 2, 2)), dynamic=True, alpha_vis=0.2, rho_f=1000.0, dt=1e-3,
        model=I.MODEL_HENCKY)),
    # Kozeny-Carman: the mobility follows the iterate's porosity (Eq. kozeny-carman)
    "footing2d-kozeny": lambda: _permeable(replace(
        I.small_footing(seed=8, body=(4, 3), pad=1, h=0.25, dynamic=True), alpha_vis=0.2, rho_f=1000.0,
        permeability=I.PERM_KOZENY_CARMAN, phi0=0.4)),
}


@pytest.mark.parametrize("name", list(FROZEN_CASES))
def test_jacobian_away_from_rest_is_the_derivative_of_the_frozen_residual(name):
    w = FROZEN_CASES[name]()
    o = O.Oracle(w)
    prep = o.prepare(w.dt)
    X0 = perturbed_X(o, prep, seed=3, amp_u=2e-4, amp_p=1e3)
    trac = w.traction(w.dt)
    R0, Jv = o.eval(prep, X0, trac)
    # frozen at the iterate itself, the variant is the residual
    np.testing.assert_array_equal(o.eval_frozen(prep, X0, X0, trac), R0)
    J = dense_J(o, prep, Jv)
    nb = o.d + 1
    Jfz = _fd_columns(o, prep, X0, lambda X: o.eval_frozen(prep, X, X0, trac))
    Jfull = _fd_columns(o, prep, X0, lambda X: o.eval(prep, X, trac, want_J=False)[0])
    # displacement columns to 1e-9 of each block type's largest entry (the
    # central differences reach about 1e-11 there, so that terms a thousandth
    # of the dominant inertia and stiffness still count); the pressure
    # columns, differenced with steps of 10 Pa, to 1e-6
    left_out = 0.0
    for r in range(nb):
        for cc in range(nb):
            A, B, Cf = J[r::nb, cc::nb], Jfz[r::nb, cc::nb], Jfull[r::nb, cc::nb]
            scale = max(np.abs(A).max(), np.abs(B).max())
            tol = 1e-9 if cc < o.d else 1e-6
            assert np.abs(A - B).max() <= tol * scale, (name, r, cc, np.abs(A - B).max() / scale)
            left_out = max(left_out, np.abs(A - Cf).max() / scale)
    # the frozen terms matter at this iterate: the full residual's differences
    # are not the Jacobian
    assert left_out > 1e-4, left_out
