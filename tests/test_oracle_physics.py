"""Pins of the oracle's discrete equations (CPU only).

What fixes each expected value:
  * Terzaghi's consolidation series (Eq. terzaghi-exact) and first-order
    convergence of implicit Euler (Eq. implicit-euler);
  * textbook small-strain oedometric modulus E(1-nu)/((1+nu)(1-2nu));
  * central finite differences of the residual (Eq. jacobian-system);
  * the PPP block (Eq. stab-term-ppp): symmetric PSD, cellwise constants in
    its null space, and a zero lower block when undrained and unstabilized
    (Eq. jacobian-system-undrained);
  * lumped P2G conserving mass (Eq. map-from-particles-to-nodes);
  * Newmark's exact integration of constant acceleration (free fall);
  * the checkerboard study of Sec. 5.1 (unstabilized oscillates, tau_W does not,
    0.1 tau_W still oscillates, 10 tau_W over-smooths).
"""
from dataclasses import replace

import numpy as np
import pytest
import scipy.sparse as sps

from oracle import oracle as O
from paper_1905_00671_gb300 import inputs as I


def terzaghi_series(Z, T, terms=400):
    P = np.zeros_like(Z)
    for m in range(terms):
        M = np.pi * (2 * m + 1) / 2
        P += 2.0 / M * np.sin(M * Z) * np.exp(-M * M * T)
    return P


def dense_J(o, prep, Jv):
    nb = o.d + 1
    nnzb = int(prep["row_ptr"][-1])
    return sps.bsr_matrix((Jv.reshape(nnzb, nb, nb), prep["col"], prep["row_ptr"]),
                          shape=(o.nn * nb, o.nn * nb)).toarray()


def perturbed_X(o, prep, seed, amp_u=1e-3, amp_p=1e3):
    rng = np.random.default_rng(seed)
    nb = o.d + 1
    X = o.initial_guess(prep).reshape(-1, nb)
    X[:, :o.d] += amp_u * rng.standard_normal((o.nn, o.d))
    X[:, o.d] += amp_p * rng.standard_normal(o.nn)
    return X.reshape(-1)


# ---------------------------------------------------------------- Stage 1
def test_p2g_conserves_mass():
    w = I.small_footing(seed=2)
    o = O.Oracle(w)
    prep = o.prepare(w.dt)
    assert abs(prep["M"].sum() - prep["m"].sum()) <= 1e-13 * prep["m"].sum()
    # a constant field maps to itself on every active node
    M, out = O.p2g(o.g, prep["first"], prep["count"], prep["S"], prep["m"], np.full(w.n, 3.5))
    np.testing.assert_allclose(out[M > 0, 0], 3.5, rtol=1e-14)


# ---------------------------------------------------------------- residual
def test_zero_residual_at_rest():
    w = I.small_footing(seed=2, jitter=0.15)
    w = replace(w, p0=np.zeros(w.n), trac_full=np.zeros_like(w.trac_full), dynamic=False)
    o = O.Oracle(w)
    prep = o.prepare(w.dt)
    R, _ = o.eval(prep, np.zeros(o.nn * 3), w.traction(w.dt), want_J=False)
    assert np.abs(R).max() == 0.0


@pytest.mark.parametrize("shape", [I.ORIG, I.GIMP])
def test_small_strain_oedometric_modulus(shape):
    E, nu = 12e6, 0.3
    w = I.terzaghi_column(ncell_y=6, ncell_x=3, h=0.25, E=E, nu=nu, shape=shape)
    o = O.Oracle(w)
    prep = o.prepare(1.0)
    nn0 = w.ncell[0] + 1
    ynode = (np.arange(o.nn) // nn0) * w.h
    M_text = E * (1 - nu) / ((1 + nu) * (1 - 2 * nu))
    errs = []
    for eps in (-1e-4, -1e-5):
        X = np.zeros((o.nn, 3))
        X[:, 1] = eps * ynode                       # affine uniaxial strain
        R, _ = o.eval(prep, X.reshape(-1), None, want_J=False)
        Rn = R.reshape(-1, 3)
        # virtual work with the current nodal coordinates: -sum R_y y = tau_yy V0
        tau_yy = -np.sum(Rn[:, 1] * (ynode + X[:, 1])) / w.vol.sum()
        errs.append(abs(tau_yy / (M_text * eps) - 1.0))
    assert errs[0] < 5e-4 and errs[1] < 5e-5      # O(eps) deviation from linear elasticity


# ---------------------------------------------------------------- Jacobian
FD_CASES = [
    ("qs-orig", dict(shape=I.ORIG, dynamic=False), {}),
    ("qs-gimp", dict(shape=I.GIMP, dynamic=False), {}),
    ("dyn-gimp", dict(shape=I.GIMP, dynamic=True), dict(alpha_vis=0.0, rho_f=0.0)),
    ("dyn-orig", dict(shape=I.ORIG, dynamic=True), dict(alpha_vis=0.0, rho_f=0.0)),
]


@pytest.mark.parametrize("name,kw,over", FD_CASES, ids=[c[0] for c in FD_CASES])
def test_jacobian_matches_central_differences(name, kw, over):
    w = I.small_footing(seed=4, body=(4, 3), pad=1, h=0.25, **kw)
    w = replace(w, **over)
    o = O.Oracle(w)
    prep = o.prepare(w.dt)
    X = perturbed_X(o, prep, 0)
    trac = w.traction(w.dt)
    R, Jv = o.eval(prep, X, trac)
    J = dense_J(o, prep, Jv)
    nb = 3
    Jfd = np.zeros_like(J)
    for j in range(o.nn * nb):
        hstep = 1e-5 * (1e-3 if j % nb < 2 else 1e3)
        Xp, Xm = X.copy(), X.copy()
        Xp[j] += hstep
        Xm[j] -= hstep
        Jfd[:, j] = (o.eval(prep, Xp, trac, want_J=False)[0]
                     - o.eval(prep, Xm, trac, want_J=False)[0]) / (2 * hstep)
    for r in range(nb):
        for c in range(nb):
            A, B = J[r::nb, c::nb], Jfd[r::nb, c::nb]
            scale = max(np.abs(A).max(), np.abs(B).max())
            assert np.abs(A - B).max() <= 1e-6 * scale, (name, r, c)


def test_jacobian_3d_matches_central_differences():
    w = I.small_block(seed=3, body=(2, 2, 2), pad=1, h=0.25)
    o = O.Oracle(w)
    prep = o.prepare(w.dt)
    X = perturbed_X(o, prep, 1)
    trac = w.traction(w.dt)
    R, Jv = o.eval(prep, X, trac)
    J = dense_J(o, prep, Jv)
    nb = 4
    rng = np.random.default_rng(0)
    for j in rng.choice(o.nn * nb, 40, replace=False):
        hstep = 1e-5 * (1e-3 if j % nb < 3 else 1e3)
        Xp, Xm = X.copy(), X.copy()
        Xp[j] += hstep
        Xm[j] -= hstep
        col = (o.eval(prep, Xp, trac, want_J=False)[0]
               - o.eval(prep, Xm, trac, want_J=False)[0]) / (2 * hstep)
        for r in range(nb):
            A, B = J[r::nb, j], col[r::nb]
            scale = max(np.abs(J[r::nb, j % nb::nb]).max(), 1e-300)
            assert np.abs(A - B).max() <= 1e-6 * scale


# ---------------------------------------------------------------- PPP block
@pytest.mark.parametrize("shape", [I.ORIG, I.GIMP])
def test_stabilization_block_is_symmetric_psd_with_constant_null_space(shape):
    w = I.small_footing(seed=6, shape=shape, dynamic=False, body=(6, 4), pad=1)
    w = replace(w, k=np.zeros(w.n))          # C = 0, so the p-p block is C_stab alone
    o = O.Oracle(w)
    prep = o.prepare(w.dt)
    _, Jv = o.eval(prep, perturbed_X(o, prep, 2), None)
    Cs = dense_J(o, prep, Jv)[2::3, 2::3]
    scale = np.abs(Cs).max()
    assert scale > 0
    np.testing.assert_allclose(Cs, Cs.T, rtol=0, atol=1e-15 * scale)
    assert np.linalg.eigvalsh(0.5 * (Cs + Cs.T)).min() >= -1e-13 * scale
    assert np.abs(Cs.sum(axis=1)).max() <= 1e-13 * scale


def test_stabilization_per_element_null_space_original_mpm():
    # all points in one cell: the element block annihilates the cell constant
    w = I.small_footing(seed=8, shape=I.ORIG, dynamic=False, body=(3, 3), pad=0, jitter=0.0)
    keep = np.nonzero((np.floor(w.x[:, 0] / w.h) == 1) & (np.floor(w.x[:, 1] / w.h) == 1))[0]
    sub = lambda a: None if a is None else np.ascontiguousarray(a[keep])
    w = replace(w, x=sub(w.x), vol=sub(w.vol), lp=sub(w.lp), p0=sub(w.p0), v0=sub(w.v0), E=sub(w.E),
                nu=sub(w.nu), k=np.zeros(len(keep)), surf_id=np.full(len(keep), -1, np.int32),
                surf_normal=sub(w.surf_normal), surf_area=sub(w.surf_area))
    o = O.Oracle(w)
    prep = o.prepare(w.dt)
    _, Jv = o.eval(prep, o.initial_guess(prep), None)
    Cs = dense_J(o, prep, Jv)[2::3, 2::3]
    nodes = [1 + 4 * 1, 2 + 4 * 1, 1 + 4 * 2, 2 + 4 * 2]
    Ce = Cs[np.ix_(nodes, nodes)]
    assert np.abs(Ce).max() > 0
    assert np.abs(Ce @ np.ones(4)).max() <= 1e-13 * np.abs(Ce).max()


def test_undrained_unstabilized_lower_block_vanishes():
    w = I.small_footing(seed=6, dynamic=False, body=(5, 4), pad=1)
    w = replace(w, k=np.zeros(w.n), stabilize=False)
    o = O.Oracle(w)
    prep = o.prepare(w.dt)
    _, Jv = o.eval(prep, perturbed_X(o, prep, 3), None)
    assert np.abs(dense_J(o, prep, Jv)[2::3, 2::3]).max() == 0.0


# ---------------------------------------------------------------- whole steps
def test_terzaghi_column_against_series():
    """4 x 40 column, E = 10 MPa, nu = 0.3, k = 1e-10, 10 kPa, dt = 1 s, 10 steps."""
    w = I.terzaghi_column()
    o = O.Oracle(w, newton_rtol=1e-10, newton_stag=1e-6)
    lam, G = O.lame(10e6, 0.3)
    cv = (lam + 2 * G) * 1e-10 / 1e-3
    H = 10.0
    z = H - np.arange(41) * w.h
    worst = 0.0
    # implicit Euler from the undrained state has an initial-layer error that
    # decays like dt / t: the bound is err_n <= 0.15 / n, and <= 0.02 at the end
    for s in range(w.nsteps):
        info = o.step()
        assert info.newton_iters <= 5
        _, X, _ = o.last
        Pn = X.reshape(-1, 3)[:, 2].reshape(41, 5)
        assert np.abs(Pn - Pn[:, :1]).max() <= 1e-8 * 10e3   # 1D: uniform across the width
        err = np.abs(Pn[:, 2] / 10e3 - terzaghi_series(z / H, cv * o.t / H ** 2))
        worst = err[:-2].max()                                # exclude the 2 rows at the drain
        assert worst <= 0.15 / (s + 1)
        # point pressures (PIC from the nodes) away from the drained boundary layer
        zp = H - o.x[:, 1]
        far = zp > 2 * w.h
        perr = np.abs(o.p / 10e3 - terzaghi_series(zp / H, cv * o.t / H ** 2))[far]
        assert perr.max() <= 0.15 / (s + 1)
    assert worst <= 0.02


def test_terzaghi_first_order_in_time():
    lam, G = O.lame(10e6, 0.3)
    cv = (lam + 2 * G) * 1e-10 / 1e-3
    errs = []
    for dt, n in ((2.0, 5), (1.0, 10), (0.5, 20)):
        w = I.terzaghi_column(dt=dt, nsteps=n)
        o = O.Oracle(w, newton_rtol=1e-10, newton_stag=1e-6)
        for _ in range(n):
            o.step()
        _, X, _ = o.last
        P = X.reshape(-1, 3)[:, 2].reshape(41, 5)[:, 2] / 10e3
        z = 10.0 - np.arange(41) * w.h
        errs.append(np.abs(P - terzaghi_series(z / 10.0, cv * 10.0 / 100.0))[:-2].max())
    order = np.log2(errs[0] / errs[1]), np.log2(errs[1] / errs[2])
    assert min(order) >= 0.8, (errs, order)


def _checkerboard(stabilize, tau_scale):
    w = I.paper_terzaghi(40, stabilize=stabilize, tau_scale=tau_scale)
    o = O.Oracle(w, newton_rtol=1e-10, newton_stag=1e-6)
    o.step()
    _, X, _ = o.last
    P = X.reshape(-1, 3)[:, 2].reshape(41, 2)[:, 0] / 1e3
    interior = P[:-3]                                        # away from the drained top
    amp = np.abs(interior[1:-1] - 0.5 * (interior[:-2] + interior[2:])).max()
    return P, amp


def test_checkerboard_study_of_section_5_1():
    P_u, amp_u = _checkerboard(False, 1.0)
    P_s, amp_s = _checkerboard(True, 1.0)
    P_lo, amp_lo = _checkerboard(True, 0.1)
    P_hi, amp_hi = _checkerboard(True, 10.0)
    assert amp_u > 0.3                  # unstabilized equal order: checkerboard
    assert amp_s < 0.05 * amp_u         # tau_W removes it
    assert amp_lo > 4 * amp_s           # 0.1 tau_W: insufficient
    assert np.all(np.diff(P_hi[:-1]) <= 1e-9)                 # 10 tau_W: monotone ...
    # ... but over-smoothed: the deficit reaches 4 cells below the drain, where the
    # exact boundary layer (about 1.3 mm) and the tau_W solution are still at 1
    assert P_hi[-5] < 0.995 and abs(P_s[-5] - 1.0) < 0.005


def test_free_fall_matches_newmark_closed_form():
    w = I.small_footing(body=(6, 4), pad=1, dynamic=True, jitter=0.0)
    ncell = (8, 10, 0)
    uf, uv, pf, pv = I.empty_bcs(2, ncell)
    w = replace(w, x=w.x + np.array([0.5, 0.75]), g=(0.0, -9.81, 0.0),
                trac_full=np.zeros_like(w.trac_full), u_fixed=uf, u_value=uv, p_fixed=pf,
                p_value=pv, ncell=ncell)
    o = O.Oracle(w, newton_rtol=1e-12, newton_stag=1e-6)
    x0 = o.x.copy()
    b, gm, dt = w.beta, w.gamma, w.dt
    u = v = a = 0.0
    for _ in range(4):
        o.step()
        u += dt * v + dt * dt * ((0.5 - b) * a + b * (-9.81))
        v += dt * ((1 - gm) * a + gm * (-9.81))
        a = -9.81
        np.testing.assert_allclose(o.v[:, 1], v, rtol=1e-9)
        np.testing.assert_allclose(o.x[:, 1] - x0[:, 1], u, rtol=1e-9)
        np.testing.assert_allclose(o.a[:, 1], a, rtol=1e-9)
        assert np.abs(o.x[:, 0] - x0[:, 0]).max() < 1e-14
        assert np.abs(o.F - np.array([1.0, 0.0, 0.0, 1.0])).max() < 1e-12


def _footing_volume_change(k, stabilize):
    w = I.small_footing(seed=9, dynamic=False, body=(20, 8), pad=1, jitter=0.0)
    w = replace(w, k=np.full(w.n, k), dt=1.0, stabilize=stabilize)
    o = O.Oracle(w, newton_rtol=1e-10, newton_stag=1e-6)
    V0 = o.V.sum()
    o.step()
    F = o.F.reshape(-1, 2, 2)
    shear = np.abs(F - np.eye(2)).max()
    dJ = np.abs(np.linalg.det(F) - 1.0).max()
    return (o.V.sum() - V0) / V0, shear, dJ


def test_undrained_loading_conserves_volume():
    # mass balance with q -> 0 and incompressible constituents: no net volume change
    dv_u, shear_u, dJ_u = _footing_volume_change(1e-22, False)
    assert shear_u > 1e-3
    assert abs(dv_u) <= 10.0 * dJ_u ** 2          # only the second-order ln J vs J - 1 gap
    dv_s, shear_s, _ = _footing_volume_change(1e-22, True)
    dv_d, _, _ = _footing_volume_change(1e-12, True)
    assert abs(dv_s) <= 2e-3 * shear_s            # PPP allows only local fluctuation
    assert abs(dv_d) > 2e-3 * shear_s             # drainage does compact the block


def test_newton_converges_quadratically_on_terzaghi():
    w = I.terzaghi_column()
    o = O.Oracle(w, newton_rtol=1e-8)
    info = o.step()
    h = info.res_hist
    assert info.newton_iters <= 4
    assert h[2] / h[0] < (h[1] / h[0]) ** 1.5


def test_p2g_conserves_momentum_and_maps_constants_exactly():
    """Lumped Stage-1 mapping (Eq. map-from-particles-to-nodes): sum_i M_i v_i =
    sum_p m_p v_p, and a field constant over the points is mapped to that
    constant at every node with mass."""
    w = I.small_footing(seed=2)
    o = O.Oracle(w)
    prep = o.prepare(w.dt)
    first, count, S, m = prep["first"], prep["count"], prep["S"], prep["m"]
    rng = np.random.default_rng(0)
    v = rng.standard_normal((w.n, 2))
    M, out = O.p2g(o.g, first, count, S, m, np.concatenate([v, np.full((w.n, 1), 7.25)], axis=1))
    np.testing.assert_allclose((M[:, None] * out[:, :2]).sum(axis=0), (m[:, None] * v).sum(axis=0),
                               rtol=1e-12)
    has = M > 0
    np.testing.assert_allclose(out[has, 2], 7.25, rtol=1e-13)


def test_mixture_mass_keeps_the_solid_mass():
    """Reading R11 (incompressible constituents, phi = 1 - (1 - phi0) / J): after
    any volume change the solid mass of a point is still (1 - phi0) rho_s V0 and
    the fluid mass is rho_f (J - 1 + phi0) V0."""
    w = I.small_footing(seed=2)
    o = O.Oracle(w)
    rng = np.random.default_rng(1)
    Fs = np.eye(2) + 0.1 * rng.standard_normal((w.n, 2, 2))
    J = np.linalg.det(Fs)
    assert J.min() > 0.5
    V0 = o.V.copy()
    o.F = Fs.reshape(w.n, 4).copy()
    o.V = J * V0
    m = o.mixture_mass()
    np.testing.assert_allclose(m, (1 - w.phi0) * w.rho_s * V0 + w.rho_f * (J - 1 + w.phi0) * V0, rtol=1e-13)
