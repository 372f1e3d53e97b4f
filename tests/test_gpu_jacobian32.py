"""The FP32 Jacobian of the mixed mode (Eq. jacobian-system-stabilized-ppp in
FP32) by every kernel configuration the autotuner chooses from (per-term and
staged; 64, 128, 256 threads; Hencky elasticity staged only),
against the oracle's FP64 Jacobian at a perturbed iterate and against one
another.

Bars: each block type entry-wise within 2e-5 of that type's largest entry
(FP32 records and FP32 sums of a few hundred terms at most), and the
configurations within 2e-6 of one another (the same FP32 products summed in
different orders).  Sparsity, Dirichlet rows and columns exact.
"""

from dataclasses import replace

import numpy as np
import pytest

from oracle import oracle as O
from paper_1905_00671_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FORMS = (0, 1)
TPBS = (64, 128, 256)


@pytest.fixture(scope="module")
def mpm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_00671_gb300 import mpm as m

    m.load()
    return m


def rel(a, b):
    scale = max(np.abs(b).max(), 1e-300)
    return np.abs(np.asarray(a, dtype=np.float64) - np.asarray(b, dtype=np.float64)).max() / scale


CASES = {
    "footing2d-gimp-newmark": lambda: I.small_footing(seed=7, body=(24, 12), pad=2, h=0.25),
    "footing2d-orig-newmark": lambda: I.small_footing(seed=8, shape=I.ORIG, body=(20, 10), pad=2),
    "footing2d-gimp-qs": lambda: I.small_footing(seed=9, dynamic=False, body=(20, 10), pad=2, dt=1.0),
    "block3d-gimp-qs": lambda: I.small_block(seed=11, body=(6, 5, 4)),
    "block3d-orig-qs": lambda: I.small_block(seed=12, shape=I.ORIG, body=(5, 4, 4)),
    "block3d-gimp-lattice": lambda: I.small_block(seed=13, body=(6, 6, 4), jitter=0.0),
    # Hencky (Sec. 2.2) with the Kelvin stress of Sec. 5.2
    "footing2d-gimp-newmark-hencky": lambda: replace(I.small_footing(seed=7, body=(24, 12), pad=2, h=0.25),
                                                     model=I.MODEL_HENCKY, alpha_vis=0.04),
    "block3d-gimp-qs-hencky": lambda: replace(I.small_block(seed=11, body=(6, 5, 4)), model=I.MODEL_HENCKY),
}


def forms_of(w):
    return (1,) if w.model == I.MODEL_HENCKY else FORMS


@pytest.mark.parametrize("name", list(CASES))
def test_fp32_jacobian_every_configuration(mpm, name):
    w = CASES[name]()
    sim = mpm.Simulation(w, precision=mpm.MPM_MIXED)
    sim.debug_prepare()
    orc = O.Oracle(w)
    prep = orc.prepare(w.dt)
    row_ptr, col = sim.debug_pattern()
    np.testing.assert_array_equal(col, prep["col"])
    rng = np.random.default_rng(1)
    nb = w.dim + 1
    X = orc.initial_guess(prep).reshape(-1, nb)
    X[:, :w.dim] += 1e-4 * rng.standard_normal((orc.nn, w.dim))
    X[:, w.dim] += 1e3 * rng.standard_normal(orc.nn)
    X = X.reshape(-1)
    _, Jo = orc.eval(prep, X, w.traction(w.dt))
    Jo = Jo.reshape(-1, nb, nb)
    first = None
    for form in forms_of(w):
        for tpb in TPBS:
            Jg = sim.debug_jacobian32(X, len(col), form, tpb, apply_bc=False).reshape(-1, nb, nb)
            for r in range(nb):
                for c in range(nb):
                    assert rel(Jg[:, r, c], Jo[:, r, c]) <= 2e-5, (form, tpb, "J", r, c)
            if first is None:
                first = Jg
            else:
                for r in range(nb):
                    for c in range(nb):
                        assert rel(Jg[:, r, c], first[:, r, c]) <= 2e-6, (form, tpb, "vs form 0", r, c)
    # Dirichlet elimination: identity on fixed diagonal entries, zero elsewhere in
    # fixed rows and columns, by every form
    fixed = np.asarray(orc.fixed_dofs(prep), dtype=bool).reshape(-1, nb)
    rows = np.repeat(np.arange(len(row_ptr) - 1), np.diff(row_ptr))
    for form in forms_of(w):
        Jb = sim.debug_jacobian32(X, len(col), form, 128, apply_bc=True).reshape(-1, nb, nb)
        fr = fixed[rows][:, :, None] | fixed[col][:, None, :]
        eye = (rows == col)[:, None, None] & np.eye(nb, dtype=bool)[None]
        np.testing.assert_array_equal(Jb[fr & eye], 1.0)
        np.testing.assert_array_equal(Jb[fr & ~eye], 0.0)
        if form == forms_of(w)[0]:  # the same form and kernel: the free entries bit for bit
            np.testing.assert_array_equal(Jb[~fr], first[~fr])
    sim.close()


def test_fp32_jacobian_rejects_a_fp64_context_and_bad_configurations(mpm):
    w = CASES["footing2d-gimp-qs"]()
    sim = mpm.Simulation(w)
    sim.debug_prepare()
    _, col = sim.debug_pattern()
    X = np.zeros(w.nnodes * (w.dim + 1))
    with pytest.raises(mpm.MPMError):
        sim.debug_jacobian32(X, len(col), 0)
    sim.close()
    sim = mpm.Simulation(w, precision=mpm.MPM_MIXED)
    sim.debug_prepare()
    for form, tpb in ((2, 128), (-1, 128), (0, 96)):
        with pytest.raises(mpm.MPMError):
            sim.debug_jacobian32(X, len(col), form, tpb)
    sim.close()
    # the per-term form has no Hencky tangent
    sim = mpm.Simulation(replace(w, model=I.MODEL_HENCKY), precision=mpm.MPM_MIXED)
    sim.debug_prepare()
    with pytest.raises(mpm.MPMError) as e:
        sim.debug_jacobian32(X, len(col), 0)
    assert e.value.code == -1
    sim.close()


@pytest.mark.parametrize("autotune", [0, 1])
def test_hencky_mixed_step_uses_the_staged_form(mpm, autotune):
    """A mixed-precision Hencky context assembles by the staged form, fixed or
    tuned: the autotuner times only the staged candidates (the per-term
    candidates' times stay 0)."""
    w = CASES["footing2d-gimp-newmark-hencky"]()
    sim = mpm.Simulation(w, precision=mpm.MPM_MIXED, autotune=autotune, newton_max=40)
    sim.step()
    st = sim.stats()
    assert st["jac_config"][1] // 1000 == 1, st["jac_config"]
    assert st["jac_tuned"][1] == autotune
    assert all(t == 0.0 for t in st["jac_tune_ms"][1][:3])
    if autotune:
        assert all(t > 0.0 for t in st["jac_tune_ms"][1][3:])
    sim.close()
