"""GPU parity of the configurations the other parity files leave out, and the
host-made failures of a step.

  * the unstabilized switch (Eq. stab-term-ppp off) on a consolidation column
    and on GIMP footings;
  * the strip footing under harmonic loading as the paper sets it up (Sec.
    5.2: Hencky, consistent mass, w = 3 - 3 cos(100 t) MPa) at full size, step
    by step against the oracle, and at the paper's tolerances through the
    steps of its Newton-Krylov table;
  * batched instances against the oracle directly (not only against the
    GPU's own one-by-one runs);
  * MPM_ERR_NEGATIVE_J and MPM_ERR_NONFINITE from bad inputs made on the host
    (an absurd load, a NaN initial pressure, a NaN traction), with the state
    kept at the last completed step and the context usable afterwards.
Parity bar as in test_gpu_parity: 1e-10 relative per field and step with both
sides at their round-off floor.
"""
from dataclasses import replace

import numpy as np
import pytest

from oracle import oracle as O
from paper_1905_00671_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TIGHT = dict(newton_rtol=1e-13, newton_stag=1e-6, newton_max=12)
GPU_TIGHT = dict(TIGHT, krylov_rtol=1e-13, krylov_max=20000)


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
    return np.abs(np.asarray(a) - np.asarray(b)).max() / scale


def _compare(w, got, ref, fields, where):
    """1e-10 of each field's largest magnitude; for the fields stored as totals
    (x, F, V, lp) 1e-10 of the largest change over the run, plus the rounding
    of the stored totals themselves (8 ulp of their largest value): a change
    smaller than that cannot be resolved in a stored total."""
    eps = np.finfo(np.float64).eps
    for k in fields:
        r = ref[k].reshape(got[k].shape)
        if k in ("x", "F", "V", "lp"):       # the change over the run, not the offset
            base = {"x": w.x, "F": np.tile(np.eye(w.dim).reshape(-1), (w.n, 1)),
                    "V": w.vol, "lp": w.lp}[k].reshape(got[k].shape)
            bound = 1e-10 * np.abs(r - base).max() + 8 * eps * np.abs(base).max()
            diff = np.abs(got[k] - r).max()
            assert diff <= bound, (where, k, diff, bound)
        else:
            assert rel(got[k], r) <= 1e-10, (where, k, rel(got[k], r))


def _fields(w):
    return ("x", "u", "p", "F", "V", "lp") + (("v", "a", "pd", "pdd") if w.dynamic else ())


UNSTAB = {
    # the 4 x 40 consolidation column (k = 1e-10 m^2, dt = 1 s): drained enough
    # that the unstabilized equal-order system stays well posed.  (The Sec. 5.1
    # column in its undrained first step is not a parity case: without the
    # stabilization its checkerboard pressure mode is singular to round-off,
    # which is the paper's point, so two correct solvers differ there by more
    # than 1e-10.)
    "terzaghi-4x40-unstabilized": (lambda: I.terzaghi_column(stabilize=False), 3),
    "footing2d-gimp-qs-unstabilized": (
        lambda: replace(I.small_footing(seed=9, dynamic=False, body=(20, 10), pad=2, dt=1.0),
                        stabilize=False), 2),
    "footing2d-gimp-newmark-unstabilized": (
        lambda: replace(I.small_footing(seed=7, body=(24, 12), pad=2, h=0.25), stabilize=False), 2),
}


@pytest.mark.parametrize("name", list(UNSTAB))
def test_unstabilized_step_parity(mpm, name):
    make, nsteps = UNSTAB[name]
    w = make()
    assert not w.stabilize
    sim = mpm.Simulation(w, **GPU_TIGHT)
    orc = O.Oracle(w, **TIGHT)
    for s in range(nsteps):
        sim.step()
        orc.step()
        _compare(w, sim.read(_fields(w)), orc.state(), _fields(w), (name, s))
    sim.close()


def test_harmonic_footing_step_parity(mpm):
    """The Sec. 5.2 set-up at full size (6,400 points, 40 x 44 cells of
    0.25 m): Hencky, consistent-mass Stage 1, Newmark, the harmonic load."""
    w = I.harmonic_footing()
    sim = mpm.Simulation(w, **GPU_TIGHT)
    orc = O.Oracle(w, **TIGHT)
    for s in range(3):
        sim.step()
        orc.step()
        _compare(w, sim.read(_fields(w)), orc.state(), _fields(w), ("harmonic", s))
    sim.close()


def test_harmonic_footing_newton_history_at_paper_tolerances(mpm):
    """At the paper's tolerances (Newton 1e-8, Krylov 1e-8 of the current
    residual) the GPU steps the harmonic footing to its 100th step (t =
    0.1 s, the first row of the paper's Newton-Krylov table), every step
    converging; at step 100 it takes three Newton iterations, as the table
    reports, each reducing the residual."""
    w = I.harmonic_footing()
    sim = mpm.Simulation(w, newton_rtol=1e-8, krylov_rtol=1e-8)
    for s in range(1, 101):
        st = sim.step()
        assert st["res_norm"][-1] <= 1e-8 * st["res_norm"][0]
    assert 2 <= st["newton_iters"] <= 4, st
    r = st["res_norm"]
    assert all(r[i + 1] < r[i] for i in range(len(r) - 1)), r
    assert all(k >= 1 for k in st["krylov_iters"]), st
    sim.close()


def _terzaghi_set():
    return [I.terzaghi_column(ncell_y=12, ncell_x=3, h=0.25, k=1e-10, load=10e3),
            I.terzaghi_column(ncell_y=8, ncell_x=5, h=0.25, k=1e-11, load=50e3)]


def _footing_set():
    return [I.small_footing(seed=21, body=(24, 12), pad=2, k=1e-12),
            I.small_footing(seed=23, body=(28, 8), pad=2, k=3e-12)]


@pytest.mark.parametrize("maker", [_terzaghi_set, _footing_set])
def test_batch_instances_against_the_oracle(mpm, maker):
    """Each instance of a batched context against the oracle stepping that
    instance alone (Sec. 3.1 per instance; batching changes no equation)."""
    ws = maker()
    batch = mpm.Batch(ws, **GPU_TIGHT)
    orcs = [O.Oracle(w, **TIGHT) for w in ws]
    for s in range(2):
        batch.step()
        for o in orcs:
            o.step()
        got = batch.read(("x", "u", "p"))
        for i, (w, o) in enumerate(zip(ws, orcs)):
            _compare(w, got[i], o.state(), ("x", "u", "p"), (w.name, s))
    batch.close()


# ---------------------------------------------------------------- host-made failures
def test_negative_jacobian_is_reported_state_kept_and_context_usable(mpm):
    """A load a thousand times the footing's crushes the first Newton iterate
    (det F <= 0 at some point): MPM_ERR_NEGATIVE_J, the state of the last
    completed step kept, and the next step with the regular load matches the
    oracle's first step."""
    w = I.small_footing(seed=3, body=(8, 4), pad=1, dynamic=False, dt=1.0)
    with pytest.raises(O.OracleError, match="non-positive Jacobian"):
        O.Oracle(w).step(traction=w.traction(w.dt) * 1000.0)
    sim = mpm.Simulation(w, **GPU_TIGHT)
    before = sim.read(("x", "u", "p", "F"))
    with pytest.raises(mpm.MPMError) as e:
        sim.step(traction=w.traction(w.dt) * 1000.0)
    assert e.value.code == -3
    after = sim.read(("x", "u", "p", "F"))
    for k in before:
        np.testing.assert_array_equal(before[k], after[k])
    assert sim.stats()["steps"] == 0
    sim.step(traction=w.traction(w.dt))
    orc = O.Oracle(w, **TIGHT)
    orc.step()
    _compare(w, sim.read(("x", "u", "p")), orc.state(), ("x", "u", "p"), "after NEGATIVE_J")
    sim.close()


def test_nan_initial_pressure_is_nonfinite(mpm):
    w = I.small_footing(seed=3, body=(8, 4), pad=1, dynamic=False, dt=1.0)
    p0 = w.p0.copy()
    p0[7] = np.nan
    sim = mpm.Simulation(replace(w, p0=p0))
    before = sim.read(("x", "u"))
    with pytest.raises(mpm.MPMError) as e:
        sim.step()
    assert e.value.code == -4
    after = sim.read(("x", "u"))
    for k in before:
        np.testing.assert_array_equal(before[k], after[k])
    sim.close()


def test_nan_traction_is_nonfinite_and_the_state_stays_at_the_last_step(mpm):
    w = I.small_footing(seed=3, body=(8, 4), pad=1)              # Newmark
    sim = mpm.Simulation(w, **GPU_TIGHT)
    orc = O.Oracle(w, **TIGHT)
    sim.step()
    orc.step()
    keep = sim.read(_fields(w))
    bad = w.traction(sim.t + w.dt).copy()
    bad[0, 1] = np.nan
    with pytest.raises(mpm.MPMError) as e:
        sim.step(traction=bad)
    assert e.value.code == -4
    now = sim.read(_fields(w))
    for k in keep:
        np.testing.assert_array_equal(keep[k], now[k])
    sim.step(traction=w.traction(sim.t + w.dt))
    orc.step()
    _compare(w, sim.read(_fields(w)), orc.state(), _fields(w), "after NONFINITE")
    sim.close()


def test_coarse_levels_kept_over_steps_leave_the_steps_unchanged(mpm):
    """mpm_options.precond_reuse keeps the multigrid coarse levels of one
    Galerkin product for several steps (the finest levels refreshed): the
    preconditioner changes, the solution does not (steps against the oracle at
    the parity bar, on a Newmark footing and a quasi-static 3D block)."""
    for w, nsteps in ((I.small_footing(seed=7, body=(24, 12), pad=2, h=0.25), 4),
                      (I.small_block(seed=11, body=(6, 5, 4)), 3)):
        sim = mpm.Simulation(w, precond_reuse=3, **GPU_TIGHT)
        orc = O.Oracle(w, **TIGHT)
        for s in range(nsteps):
            sim.step()
            orc.step()
            _compare(w, sim.read(_fields(w)), orc.state(), _fields(w), ("reuse", w.name, s))
        sim.close()


WIDE = {
    # GIMP domains of 0.7 h (two points per cell and axis overlap): supports of
    # four nodes along an axis, the widest the first-node bins (and the
    # candidate cells) handle
    "footing2d-gimp-qs-wide": lambda: I.small_footing(seed=9, dynamic=False, body=(20, 10), pad=2, dt=1.0),
    "footing2d-gimp-newmark-wide": lambda: I.small_footing(seed=7, body=(24, 12), pad=2, h=0.25),
    "block3d-gimp-qs-wide": lambda: I.small_block(seed=11, body=(6, 5, 4)),
}


@pytest.mark.parametrize("name", list(WIDE))
def test_four_node_supports(mpm, name):
    """Pattern bit-exact, residual and Jacobian entry-wise (FP64 and every FP32
    configuration) and two steps against the oracle on GIMP domains wide enough
    that supports span four nodes along an axis."""
    w = WIDE[name]()
    w = replace(w, lp=np.ascontiguousarray(w.lp * 2.8), name=w.name + "-wide")
    orc = O.Oracle(w, **TIGHT)
    prep = orc.prepare(w.dt)
    assert (prep["count"] == 4).any()
    nb = w.dim + 1
    rng = np.random.default_rng(3)
    X = orc.initial_guess(prep).reshape(-1, nb)
    X[:, :w.dim] += 1e-4 * rng.standard_normal((orc.nn, w.dim))
    X[:, w.dim] += 1e3 * rng.standard_normal(orc.nn)
    X = X.reshape(-1)
    Ro, Jo = orc.eval(prep, X, w.traction(w.dt))
    Jo = Jo.reshape(-1, nb, nb)
    for precision in (mpm.MPM_FP64, mpm.MPM_MIXED):
        sim = mpm.Simulation(w, precision=precision)
        sim.debug_prepare()
        row_ptr, col = sim.debug_pattern()
        np.testing.assert_array_equal(row_ptr, prep["row_ptr"])
        np.testing.assert_array_equal(col, prep["col"])
        Rg, Jg = sim.debug_eval(X, nnzb=len(col), apply_bc=False)
        for r in range(nb):
            assert rel(Rg[r::nb], Ro[r::nb]) <= 1e-11, ("R", r)
        Jg = Jg.reshape(-1, nb, nb)
        for r in range(nb):
            for c in range(nb):
                assert rel(Jg[:, r, c], Jo[:, r, c]) <= 1e-11, ("J", r, c)
        if precision == mpm.MPM_MIXED:
            for form in (0, 1):
                J32 = sim.debug_jacobian32(X, len(col), form, 128).reshape(-1, nb, nb)
                for r in range(nb):
                    for c in range(nb):
                        assert rel(J32[:, r, c], Jo[:, r, c]) <= 2e-5, ("J32", form, r, c)
        sim.close()
    sim = mpm.Simulation(w, **GPU_TIGHT)
    orc = O.Oracle(w, **TIGHT)
    for s in range(2):
        sim.step()
        orc.step()
        _compare(w, sim.read(_fields(w)), orc.state(), _fields(w), (name, s))
    sim.close()
