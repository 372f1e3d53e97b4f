"""The 3D quasi-static path of the oracle against Terzaghi's series (Eq.
terzaghi-exact): a 2 x 2 x 20-cell column (H = 10 m) with rollers on its four
sides, a fixed impermeable bottom, and a drained top loaded by a uniform 10 kPa
is a one-dimensional consolidation problem, so the nodal pressure must be
uniform across each horizontal layer and follow the series in depth and time,
as the 2D column does."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1905_00671_gb300 import inputs as I
from tests.test_oracle_physics import terzaghi_series


@pytest.mark.parametrize("shape", [I.ORIG, I.GIMP])
def test_terzaghi_3d_column_against_series(shape):
    nz, h, load, k = 20, 0.5, 10e3, 1e-10
    w = I.consolidation_block(body=(2, 2, nz), pad=1, h=h, logk=(np.log10(k), np.log10(k)),
                              load=load, patch_half=100.0, dt=1.0, nsteps=10, shape=shape)
    assert np.allclose(w.k, k)
    o = O.Oracle(w, newton_rtol=1e-10, newton_stag=1e-6)
    lam, G = O.lame(10e6, 0.3)
    cv = (lam + 2 * G) * k / w.mu_f
    H = nz * h
    nn = [c + 1 for c in w.ncell]
    z = H - np.arange(nz + 1) * h
    for s in range(w.nsteps):
        info = o.step()
        assert info.newton_iters <= 5
        _, X, _ = o.last
        P = X.reshape(-1, 4)[:, 3].reshape(nn[2], nn[1], nn[0])[:nz + 1]   # [z][y][x], body layers
        assert np.abs(P - P[:, :1, :1]).max() <= 1e-8 * load                 # uniform per layer
        err = np.abs(P[:, 0, 0] / load - terzaghi_series(z / H, cv * o.t / H ** 2))
        worst = err[:-2].max()                                               # 2 layers at the drain
        assert worst <= 0.15 / (s + 1), (s, worst)
    assert worst <= 0.02


def test_jacobian_3d_newmark_matches_central_differences():
    """Newmark in 3D (GIMP, jittered), with the Kelvin stress and the fluid
    density off so that the omitted terms of the linearization vanish (R8):
    every sampled column of the analytic Jacobian against central differences."""
    from dataclasses import replace

    from tests.test_oracle_physics import dense_J, perturbed_X

    w = I.small_block(seed=3, body=(2, 2, 2), pad=1, h=0.25)
    w = replace(w, dynamic=True, dt=2e-3, alpha_vis=0.0, rho_f=0.0,
                v0=0.01 * np.random.default_rng(5).standard_normal((w.n, 3)))
    o = O.Oracle(w)
    prep = o.prepare(w.dt)
    X = perturbed_X(o, prep, 2)
    trac = w.traction(w.dt)
    _, Jv = o.eval(prep, X, trac)
    J = dense_J(o, prep, Jv)
    nb = 4
    rng = np.random.default_rng(1)
    for j in rng.choice(o.nn * nb, 48, replace=False):
        hstep = 1e-5 * (1e-3 if j % nb < 3 else 1e3)
        Xp, Xm = X.copy(), X.copy()
        Xp[j] += hstep
        Xm[j] -= hstep
        col = (o.eval(prep, Xp, trac, want_J=False)[0] - o.eval(prep, Xm, trac, want_J=False)[0]) / (2 * hstep)
        for r in range(nb):
            scale = max(np.abs(J[r::nb, j % nb::nb]).max(), 1e-300)
            assert np.abs(J[r::nb, j] - col[r::nb]).max() <= 1e-6 * scale, (j, r)


def test_free_fall_3d_matches_newmark_closed_form():
    """A 2 x 2 x 2-cell block with no support in a larger grid falls under
    gravity: every point follows the Newmark recursion of a rigid body exactly
    (u, v, a), without deformation, with GIMP bases."""
    from dataclasses import replace

    w = I.small_block(seed=3, body=(2, 2, 2), pad=1, h=0.25, jitter=0.0)
    ncell = (6, 6, 8)
    uf, uv, pf, pv = I.empty_bcs(3, ncell)
    w = replace(w, x=w.x + np.array([0.5, 0.5, 1.25]), ncell=ncell, g=(0.0, 0.0, -9.81),
                dynamic=True, dt=2e-3, v0=np.zeros((w.n, 3)), trac_full=np.zeros_like(w.trac_full),
                u_fixed=uf, u_value=uv, p_fixed=pf, p_value=pv)
    o = O.Oracle(w, newton_rtol=1e-12, newton_stag=1e-6)
    x0 = o.x.copy()
    b, gm, dt = w.beta, w.gamma, w.dt
    u = v = a = 0.0
    for _ in range(4):
        o.step()
        u += dt * v + dt * dt * ((0.5 - b) * a + b * (-9.81))
        v += dt * ((1 - gm) * a + gm * (-9.81))
        a = -9.81
        np.testing.assert_allclose(o.v[:, 2], v, rtol=1e-9)
        np.testing.assert_allclose(o.x[:, 2] - x0[:, 2], u, rtol=1e-9)
        # the acceleration is the increment over beta dt^2: it carries the residual's round-off floor
        np.testing.assert_allclose(o.a[:, 2], a, rtol=1e-8)
        assert np.abs(o.x[:, :2] - x0[:, :2]).max() < 1e-13        # round-off of 3D sums, x ~ 1 m
        assert np.abs(o.F - np.eye(3).reshape(-1)).max() < 1e-12
