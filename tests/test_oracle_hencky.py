"""Hencky elasticity (Sec. 2.2: Psi = lambda/2 (ln J)^2 + G tr((1/2 ln b)^2)) in
the oracle, pinned to: the exact Kirchhoff stress of a finite plane-strain
uniaxial stretch, tau'_yy = (lambda + 2G) ln s and tau'_xx = lambda ln s (the
neo-Hookean law gives G (s^2 - 1) + lambda ln s), a stress-free rigid rotation,
the zero-strain tangent (all stretches equal: the Hencky and neo-Hookean
Jacobians agree there), and the Jacobian against central differences in 2D
(quasi-static and Newmark) and 3D."""
from dataclasses import replace

import numpy as np
import pytest

from oracle import oracle as O
from paper_1905_00671_gb300 import inputs as I
from tests.test_oracle_physics import dense_J, perturbed_X

E, NU = 12e6, 0.3
LAM = E * NU / ((1 + NU) * (1 - 2 * NU))
G = E / (2 * (1 + NU))


def _column(shape, model=I.MODEL_HENCKY):
    w = I.terzaghi_column(ncell_y=6, ncell_x=3, h=0.25, E=E, nu=NU, shape=shape)
    return replace(w, model=model)


def _virtual_work_stress(w, s, shear=0.0):
    o = O.Oracle(w)
    prep = o.prepare(1.0)
    nc = I.node_coords(2, w.ncell) * w.h
    X = np.zeros((o.nn, 3))
    X[:, 1] = (s - 1.0) * nc[:, 1]                 # dF = diag(1, s) (+ shear)
    X[:, 0] = shear * nc[:, 1]
    R, _ = o.eval(prep, X.reshape(-1), None, want_J=False)
    Rn = R.reshape(-1, 3)
    xcur = nc + X[:, :2]
    V0 = w.vol.sum()
    # -sum_a R_a,i x_a,j = tau_ij V0 for an affine motion (sum_a x_a grad S_a = 1)
    return np.array([[-np.sum(Rn[:, i] * xcur[:, j]) / V0 for j in range(2)] for i in range(2)])


@pytest.mark.parametrize("shape", [I.ORIG, I.GIMP])
@pytest.mark.parametrize("s", [0.8, 1.25])
def test_hencky_stress_of_a_finite_uniaxial_stretch(shape, s):
    tau = _virtual_work_stress(_column(shape), s)
    scale = (LAM + 2 * G) * abs(np.log(s))
    np.testing.assert_allclose(tau[1, 1], (LAM + 2 * G) * np.log(s), rtol=1e-10)
    np.testing.assert_allclose(tau[0, 0], LAM * np.log(s), rtol=1e-10)
    assert abs(tau[0, 1]) < 1e-10 * scale and abs(tau[1, 0]) < 1e-10 * scale
    # the neo-Hookean law differs at this strain
    tn = _virtual_work_stress(_column(shape, I.MODEL_NEOHOOKE), s)
    np.testing.assert_allclose(tn[1, 1], G * (s * s - 1.0) + LAM * np.log(s), rtol=1e-10)
    assert abs(tn[1, 1] - tau[1, 1]) > 1e-2 * scale


def test_hencky_simple_shear_is_symmetric_and_isochoric():
    """dF = [[1, g], [0, 1]]: J = 1, so tr tau' = 2G tr eps = 0 and tau' is
    symmetric; its shear part is G ln b of the simple shear."""
    gam = 0.4
    tau = _virtual_work_stress(_column(I.ORIG), 1.0, shear=gam)
    scale = G * gam
    assert abs(tau[0, 1] - tau[1, 0]) < 1e-10 * scale
    assert abs(tau[0, 0] + tau[1, 1]) < 1e-10 * scale
    b = np.array([[1 + gam * gam, gam], [gam, 1.0]])
    wv, Q = np.linalg.eigh(b)
    lnb = Q @ np.diag(np.log(wv)) @ Q.T
    np.testing.assert_allclose(tau, G * lnb, rtol=0, atol=1e-10 * scale)


def test_hencky_rigid_rotation_is_stress_free():
    w = _column(I.ORIG)
    w = replace(w, trac_full=np.zeros_like(w.trac_full))
    o = O.Oracle(w)
    prep = o.prepare(1.0)
    nc = I.node_coords(2, w.ncell) * w.h
    th = np.deg2rad(30.0)
    Rm = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    X = np.zeros((o.nn, 3))
    X[:, :2] = nc @ Rm.T - nc
    R, _ = o.eval(prep, X.reshape(-1), None, want_J=False)
    assert np.abs(R.reshape(-1, 3)[:, :2]).max() < 1e-6 * G * w.h    # vs G h ~ force of a unit strain


def test_hencky_tangent_at_zero_strain_is_the_linear_one():
    """All stretches equal (the degenerate limit of theta_AB): the Hencky
    Jacobian equals the neo-Hookean one, both lambda 1 (x) 1 + 2 G I there."""
    w = I.small_footing(seed=4, body=(4, 3), pad=1, h=0.25, dynamic=False)
    Js = []
    for model in (I.MODEL_NEOHOOKE, I.MODEL_HENCKY):
        o = O.Oracle(replace(w, model=model))
        prep = o.prepare(w.dt)
        X = o.initial_guess(prep)
        Js.append(o.eval(prep, X, w.traction(w.dt))[1])
    np.testing.assert_allclose(Js[1], Js[0], rtol=0, atol=1e-10 * np.abs(Js[0]).max())


def _fd_check(w, seed):
    o = O.Oracle(w)
    prep = o.prepare(w.dt)
    X = perturbed_X(o, prep, seed, amp_u=3e-2)         # strains of a few per cent
    trac = w.traction(w.dt)
    R, Jv = o.eval(prep, X, trac)
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
        for c in range(nb):
            A, B = J[r::nb, c::nb], Jfd[r::nb, c::nb]
            scale = max(np.abs(A).max(), np.abs(B).max())
            assert np.abs(A - B).max() <= 1e-6 * scale, (r, c)


@pytest.mark.parametrize("dynamic", [False, True])
def test_hencky_jacobian_matches_central_differences(dynamic):
    w = I.small_footing(seed=4, body=(4, 3), pad=1, h=0.25, dynamic=dynamic)
    w = replace(w, model=I.MODEL_HENCKY)
    if dynamic:
        w = replace(w, alpha_vis=0.0, rho_f=0.0)
    _fd_check(w, 0)


def test_hencky_jacobian_3d_matches_central_differences():
    w = replace(I.small_block(seed=3, body=(2, 2, 2), pad=1, h=0.25), model=I.MODEL_HENCKY)
    _fd_check(w, 1)


def _column_3d(model=I.MODEL_HENCKY):
    # original MPM, the body filling the grid laterally: bases exactly linear
    w = I.consolidation_block(body=(3, 3, 4), pad=0, h=0.25, E=E, nu=NU, shape=I.ORIG,
                              logk=(-10.0, -10.0))
    return replace(w, model=model, trac_full=np.zeros_like(w.trac_full))


def _virtual_work_stress_3d(w, grad):
    """-sum_a R_a (x) x_a / V0 for the affine increment x -> x + grad x."""
    o = O.Oracle(w)
    prep = o.prepare(1.0)
    nc = I.node_coords(3, w.ncell) * w.h
    X = np.zeros((o.nn, 4))
    X[:, :3] = nc @ np.asarray(grad).T
    R, _ = o.eval(prep, X.reshape(-1), None, want_J=False)
    Rn = R.reshape(-1, 4)
    return -np.einsum("ai,aj->ij", Rn[:, :3], nc + X[:, :3]) / w.vol.sum()


@pytest.mark.parametrize("s", [0.8, 1.25])
def test_hencky_3d_uniaxial_stretch(s):
    tau = _virtual_work_stress_3d(_column_3d(), np.diag([0.0, 0.0, s - 1.0]))
    scale = (LAM + 2 * G) * abs(np.log(s))
    expect = np.diag([LAM * np.log(s), LAM * np.log(s), (LAM + 2 * G) * np.log(s)])
    np.testing.assert_allclose(tau, expect, rtol=0, atol=1e-10 * scale)


def test_hencky_3d_simple_shear_is_G_ln_b():
    """dF = 1 + g e_x (x) e_z + g2 e_y (x) e_x (two shears, J = 1): tau' = G ln b
    with b = dF dF^T, its logarithm from numpy's symmetric eigensolver."""
    g1, g2 = 0.3, -0.2
    grad = np.zeros((3, 3))
    grad[0, 2], grad[1, 0] = g1, g2
    tau = _virtual_work_stress_3d(_column_3d(), grad)
    F = np.eye(3) + grad
    b = F @ F.T
    wv, Q = np.linalg.eigh(b)
    expect = G * (Q @ np.diag(np.log(wv)) @ Q.T)      # lambda ln J = 0: J = 1
    assert abs(np.linalg.det(F) - 1.0) < 1e-14
    np.testing.assert_allclose(tau, expect, rtol=0, atol=1e-10 * G * abs(g1))


def test_hencky_3d_rigid_rotation_is_stress_free():
    ax = np.array([1.0, 2.0, 2.0]) / 3.0
    th = np.deg2rad(40.0)
    K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
    Rm = np.eye(3) + np.sin(th) * K + (1 - np.cos(th)) * K @ K
    tau = _virtual_work_stress_3d(_column_3d(), Rm - np.eye(3))
    assert np.abs(tau).max() < 1e-8 * G
