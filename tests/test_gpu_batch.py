"""Batched stepping (mpm_create_batch / mpm_step_batch) against the same
instances stepped one at a time: the instances never couple through the
discrete equations, so at the round-off floor of both solves the per-instance
states must agree."""
import numpy as np
import pytest

from paper_1905_00671_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TIGHT = dict(newton_rtol=1e-13, newton_stag=1e-6, newton_max=12, krylov_rtol=1e-13, krylov_max=20000)


@pytest.fixture(scope="module")
def mpm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_00671_gb300 import mpm as m

    m.load()
    return m


def footing_set():
    # jittered, shuffled points whose GIMP domains straddle faces (and the grid
    # walls, where each instance's own grid must clip them), uneven sizes
    return [I.small_footing(seed=21, body=(24, 12), pad=2, k=1e-12),
            I.small_footing(seed=22, body=(20, 10), pad=2, k=1e-11),
            I.small_footing(seed=23, body=(28, 8), pad=2, k=3e-12)]


def terzaghi_set():
    return [I.terzaghi_column(ncell_y=12, ncell_x=3, h=0.25, k=1e-10, load=10e3),
            I.terzaghi_column(ncell_y=8, ncell_x=5, h=0.25, k=1e-11, load=50e3),
            I.terzaghi_column(ncell_y=10, ncell_x=2, h=0.25, k=3e-10, load=20e3)]


@pytest.mark.parametrize("maker,precision", [(footing_set, 0), (terzaghi_set, 0), (footing_set, 1)])
def test_batch_matches_one_by_one(mpm, maker, precision):
    """FP64 batch vs FP64 one by one, both at the round-off floor: <= 1e-9.
    Mixed batch vs FP64 one by one, both to a Newton tolerance of 1e-11 (at
    1e-8 the FP64 reference itself is only as close as the conditioning of
    the smaller instances allows): <= 1e-7."""
    ws = maker()
    if precision == mpm.MPM_MIXED:
        opts = dict(precision=precision, newton_rtol=1e-11, newton_max=60)
        ref_opts = dict(newton_rtol=1e-11, newton_max=60)
        tol = 1e-7
    else:
        opts = ref_opts = dict(TIGHT)
        tol = 1e-9
    batch = mpm.Batch(ws, **opts)
    singles = [mpm.Simulation(w, **ref_opts) for w in ws]
    for _ in range(2):
        st = batch.step()
        assert st["newton_iters"] >= 1
        for s in singles:
            s.step()
    got = batch.read(("x", "u", "p"))
    for i, s in enumerate(singles):
        ref = s.read(("x", "u", "p"))
        for f in ("u", "p"):
            err = np.abs(got[i][f] - ref[f]).max() / max(np.abs(ref[f]).max(), 1e-300)
            assert err <= tol, (ws[i].name, f, err)
        # positions stay in each instance's own coordinates (x = X + u)
        xerr = np.abs(got[i]["x"] - ref["x"]).max()
        assert xerr <= 1e-12 * np.abs(ref["x"]).max() + tol * np.abs(ref["u"]).max(), (ws[i].name, xerr)
        s.close()
    batch.close()


def test_batch_instance_leaving_its_grid_is_an_error(mpm):
    ws = footing_set()
    w = ws[1]
    x = w.x.copy()
    x[0, 0] = w.origin[0] + w.ncell[0] * w.h + 0.5 * w.h     # beyond its own grid
    from dataclasses import replace
    bad = [ws[0], replace(w, x=x), ws[2]]
    batch = mpm.Batch(bad)
    with pytest.raises(mpm.MPMError):
        batch.step()
    batch.close()
