"""Pins of the numpy preconditioner reference (no GPU)."""
import pytest

from oracle import oracle as O
from paper_1905_00671_gb300 import inputs as I
from tests.precond_reference import fixed_stress_diag


def test_fixed_stress_reference_term_is_the_bulk_mass():
    """With uniform E, nu the lumped fixed-stress term sums (partition of unity
    over the active support nodes) to the total volume / (dt K), K = lambda +
    2 G / dim the drained bulk modulus."""
    for w in (I.terzaghi_column(), I.small_block(seed=11, body=(4, 3, 3), jitter=0.0)):
        orc = O.Oracle(w)
        prep = orc.prepare(w.dt)
        fs = fixed_stress_diag(w, prep)
        E, nu, d = w.E[0], w.nu[0], w.dim
        K = E * nu / ((1 + nu) * (1 - 2 * nu)) + 2 * E / (2 * (1 + nu)) / d
        assert abs(fs.sum() - w.vol.sum() / (w.dt * K)) <= 1e-12 * fs.sum()
        assert (fs >= 0).all()


def _a_block_rate(w, omega, sweeps=None):
    """Asymptotic error reduction per V-cycle of the A-block multigrid used as a
    stationary iteration, x <- x + V(b - A x), on the Jacobian the oracle
    assembles at the start of the first step."""
    import numpy as np

    from tests import precond_reference as PR

    orc = O.Oracle(w)
    prep = orc.prepare(w.dt)
    X = orc.initial_guess(prep)
    fixed = orc.fixed_dofs(prep)
    _, Jv = orc.eval(prep, X, None)
    J = orc.jacobian_matrix(prep, Jv, fixed).tocsr()
    d, nb = w.dim, w.dim + 1
    iu = np.array([a * nb + k for a in range(orc.nn) for k in range(d)])
    A = J[iu][:, iu].tocsr()
    nn = [c + 1 for c in w.ncell[:d]]
    levels = PR.hierarchy(A, nn, d, d, ~fixed[iu], sweeps=sweeps)
    for lev in levels:
        lev["omega"] = omega
    rng = np.random.default_rng(0)
    b = A @ rng.standard_normal(A.shape[0])
    x = np.zeros_like(b)
    res = []
    for _ in range(20):
        x = x + PR.vcycle(levels, b - A @ x)
        res.append(np.linalg.norm(b - A @ x))
    return np.median([res[i + 1] / res[i] for i in range(10, 19)])


@pytest.mark.parametrize("sweeps,bound", [(1, 0.7), (2, 0.6)])
def test_3d_smoother_damping_keeps_the_slope_vcycle_contracting(sweeps, bound):
    """Block Jacobi is stable only while omega lambda_max(Dinv A) < 2; next to
    the inclined free face of the 3D slope lambda_max is about 3.5, so the 3D
    damping (0.5) contracts there, with the default V(1,1) cycle and with
    V(2,2), while 0.6 makes either cycle grow the error."""
    from tests.precond_reference import OMEGA

    w = I.slope_3d(ncell=(16, 16, 8), h=0.8)
    assert OMEGA[3] == 0.5
    assert _a_block_rate(w, OMEGA[3], sweeps) < bound
    assert _a_block_rate(w, 0.6, sweeps) > 1.0
