"""The library's Newton-system preconditioner (Schur complement + geometric
multigrid) against its numpy restatement in tests/precond_reference.py, on the
Jacobian the oracle assembles at the same iterate."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1905_00671_gb300 import inputs as I
from tests.precond_reference import SchurMG, fixed_stress_diag

pytestmark = pytest.mark.gpu

CASES = {
    "footing2d-gimp-newmark": lambda: I.small_footing(seed=7, body=(24, 12), pad=2, h=0.25),
    "footing2d-orig-newmark": lambda: I.small_footing(seed=8, shape=I.ORIG, body=(20, 10), pad=2),
    "footing2d-gimp-qs": lambda: I.small_footing(seed=9, dynamic=False, body=(20, 10), pad=2, dt=1.0),
    "terzaghi-4x40": lambda: I.terzaghi_column(),
    "block3d-gimp-qs": lambda: I.small_block(seed=11, body=(6, 5, 4)),
}


@pytest.fixture(scope="module")
def mpm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_00671_gb300 import mpm as m

    m.load()
    return m


# solver options of the preconditioner: (mpm_options, restatement keywords)
VARIANTS = {
    "default": ({}, {}),
    "upper-v22": (dict(schur_order=1, mg_sweeps=2), dict(lower=False, sweeps=2)),
    "v22-omega06": (dict(mg_sweeps=2, mg_omega=0.6), dict(sweeps=2, omega=0.6)),
    "v33-upper": (dict(mg_sweeps=3, schur_order=1), dict(sweeps=3, lower=False)),
}
VARIANT_CASES = [(n, "default") for n in CASES] + [
    ("footing2d-gimp-newmark", "upper-v22"), ("block3d-gimp-qs", "upper-v22"),
    ("footing2d-gimp-newmark", "v22-omega06"), ("terzaghi-4x40", "v22-omega06"),
    ("block3d-gimp-qs", "v33-upper")]


@pytest.mark.parametrize("name,variant", VARIANT_CASES)
def test_preconditioner_matches_reference(mpm, name, variant):
    w = CASES[name]()
    opts, ref_kw = VARIANTS[variant]
    sim = mpm.Simulation(w, **opts)
    sim.debug_prepare()
    orc = O.Oracle(w)
    prep = orc.prepare(w.dt)
    rng = np.random.default_rng(1)
    nb = w.dim + 1
    X = orc.initial_guess(prep).reshape(-1, nb)
    # quasi-static steps use the fixed-stress Schur approximation, whose
    # reference term is taken at the start of the step (X = initial guess)
    fs = None if w.dynamic else fixed_stress_diag(w, prep)
    if w.dynamic:
        X[:, :w.dim] += 1e-5 * rng.standard_normal((orc.nn, w.dim))
    X = X.reshape(-1)
    _, Jv = orc.eval(prep, X, w.traction(w.dt))
    fixed = orc.fixed_dofs(prep)
    J = orc.jacobian_matrix(prep, Jv, fixed)
    nn = [w.ncell[k] + 1 for k in range(w.dim)] + [1]
    ref = SchurMG(J, prep["row_ptr"], prep["col"], fixed, nn, w.dim, fs=fs, **ref_kw)
    for trial in range(2):
        v = rng.standard_normal(orc.nn * nb)
        v[fixed] = 0.0
        z = sim.debug_precond(X, v)
        zr = ref.apply(v)
        err = np.abs(z - zr).max() / np.abs(zr).max()
        assert err <= 1e-7, (name, variant, trial, err)
    sim.close()

