"""Stage 3 of the oracle (Sec. 3.5: G2P, convection and the GIMP domain
update) under an affine nodal increment x -> x + grad x, where everything it
computes has a plain definition: every point moves by grad x_p, the incremental
deformation gradient is 1 + grad at every point, the volume scales by its
determinant, and each GIMP half length scales by the matching diagonal entry
of the right stretch U = (dF^T dF)^(1/2) (reading R9), taken here from numpy's
symmetric eigensolver rather than the oracle's Jacobi rotations."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1905_00671_gb300 import inputs as I


def _right_stretch(F):
    wv, Q = np.linalg.eigh(F.T @ F)
    return Q @ np.diag(np.sqrt(wv)) @ Q.T


def _check_affine_update(w, grad):
    d = w.dim
    o = O.Oracle(w)
    prep = o.prepare(w.dt)
    assert np.all(prep["active"])                    # the body fills the grid: exact linear bases
    nc = I.node_coords(d, w.ncell) * w.h
    X = np.zeros((o.nn, d + 1))
    X[:, :d] = nc @ grad.T
    x0, V0, lp0 = o.x.copy(), o.V.copy(), o.lp.copy()
    o.update(prep, X.reshape(-1))
    dF = np.eye(d) + grad
    np.testing.assert_allclose(o.x, x0 + x0 @ grad.T, rtol=0, atol=1e-14 * np.abs(x0).max())
    np.testing.assert_allclose(o.u, x0 @ grad.T, rtol=0, atol=1e-14 * np.abs(x0).max())
    np.testing.assert_allclose(o.F.reshape(-1, d, d), np.broadcast_to(dF, (o.n, d, d)), rtol=0, atol=1e-13)
    np.testing.assert_allclose(o.V, np.linalg.det(dF) * V0, rtol=1e-13)
    Ud = np.diag(_right_stretch(dF))
    np.testing.assert_allclose(o.lp, lp0 * Ud, rtol=1e-12)


GRADS_2D = {
    "stretch": np.diag([0.1, -0.2]),
    "rotation": np.array([[np.cos(0.5) - 1, -np.sin(0.5)], [np.sin(0.5), np.cos(0.5) - 1]]),
    "simple-shear": np.array([[0.0, 0.3], [0.0, 0.0]]),
    "general": np.array([[0.05, 0.2], [-0.1, 0.15]]),
}


@pytest.mark.parametrize("name", list(GRADS_2D))
def test_g2p_affine_update_2d(name):
    w = I.terzaghi_column(ncell_y=6, ncell_x=3, h=0.25, shape=I.GIMP)
    _check_affine_update(w, GRADS_2D[name])


def test_g2p_affine_update_3d():
    w = I.consolidation_block(body=(3, 3, 3), pad=0, h=0.25, shape=I.GIMP, logk=(-10.0, -10.0))
    grad = np.array([[0.04, 0.2, -0.05], [-0.1, 0.02, 0.15], [0.03, -0.12, -0.06]])
    _check_affine_update(w, grad)
    # a rigid rotation leaves every half length unchanged
    th, ax = 0.7, np.array([2.0, -1.0, 2.0]) / 3.0
    K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
    R = np.eye(3) + np.sin(th) * K + (1 - np.cos(th)) * K @ K
    _check_affine_update(w, R - np.eye(3))


def test_g2p_newmark_from_rest_with_affine_fields():
    """Newmark step from rest (v_n = a_n = 0, p_n = 0): for an affine increment
    the nodal acceleration a = dU / (beta dt^2) is affine, so every point gets
    a_p = grad x_p / (beta dt^2) (PIC) and v_p = gamma dt a_p (FLIP,
    v = v_n + dt sum S ((1 - gamma) a_n + gamma a)); a linear nodal pressure
    gives p_p at the point (PIC) and its Newmark rate gamma / (beta dt) p_p."""
    from dataclasses import replace

    w = I.terzaghi_column(ncell_y=6, ncell_x=3, h=0.25, shape=I.GIMP)
    w = replace(w, dynamic=True, dt=2e-3, v0=np.zeros((w.n, 2)))
    o = O.Oracle(w)
    prep = o.prepare(w.dt)
    assert np.all(prep["active"])
    grad = np.array([[0.002, -0.001], [0.0015, 0.003]])
    cp = np.array([3e3, -5e3])
    nc = I.node_coords(2, w.ncell) * w.h
    X = np.zeros((o.nn, 3))
    X[:, :2] = nc @ grad.T
    X[:, 2] = nc @ cp
    x0 = o.x.copy()
    o.update(prep, X.reshape(-1))
    b, gm, dt = w.beta, w.gamma, w.dt
    a = (x0 @ grad.T) / (b * dt * dt)
    scale = np.abs(a).max()
    np.testing.assert_allclose(o.a, a, rtol=0, atol=1e-11 * scale)
    np.testing.assert_allclose(o.v, gm * dt * a, rtol=0, atol=1e-11 * gm * dt * scale)
    p = x0 @ cp
    np.testing.assert_allclose(o.p, p, rtol=0, atol=1e-12 * np.abs(p).max())
    np.testing.assert_allclose(o.pd, gm / (b * dt) * p, rtol=0, atol=1e-11 * gm / (b * dt) * np.abs(p).max())
