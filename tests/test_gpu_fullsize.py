"""The 3D consolidation block at its full size (64 x 64 x 32 cells, 1,048,576
GIMP points, quasi-static) in the launch configuration the bench times, and
the 3D slope at its full size (128 x 128 x 64 cells, 4,208,640 points).  The
oracle cannot take a step of this size, so the checks are properties that hold
at any size: Newton reaches the tolerance of Eq. newton-tolerance; the mixed
precision path agrees with FP64 within its stated bound; det F stays positive;
the loaded patch moves down with a positive excess pore pressure below it; the
state at rest is reproduced exactly by a zero-load step; and on the slope no
Krylov solve stops at its cap (the multigrid smoother stays stable next to the
inclined free face)."""
import numpy as np
import pytest

from paper_1905_00671_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mpm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_00671_gb300 import mpm as m

    m.load()
    return m


def test_block3d_full_size_step(mpm):
    w = I.consolidation_block()
    assert w.n == 1048576
    fp64 = mpm.Simulation(w, newton_rtol=1e-8)
    st = fp64.step()
    r = st["res_norm"]
    assert r[-1] <= 1e-8 * r[0], r
    got = fp64.read(("x", "u", "p", "F"))
    mixed = mpm.Simulation(w, precision=mpm.MPM_MIXED, newton_rtol=1e-8, newton_max=60)
    mixed.step()
    gm = mixed.read(("u", "p"))
    for f in ("u", "p"):
        err = np.abs(gm[f] - got[f]).max() / np.abs(got[f]).max()
        assert err <= 1e-6, (f, err)
    F = got["F"].reshape(-1, 3, 3)
    assert (np.linalg.det(F) > 0).all()
    # the loaded patch (top, |x - 3.2|, |y - 3.2| <= 1 m) settles and the pore
    # pressure below it rises (positive in compression)
    top = w.surf_id >= 0
    assert got["u"][top, 2].mean() < 0.0
    below = (np.abs(w.x[:, 0] - 3.2) < 0.8) & (np.abs(w.x[:, 1] - 3.2) < 0.8) & (w.x[:, 2] > 2.0)
    assert got["p"][below].mean() > 0.0
    fp64.close()
    mixed.close()


def test_block3d_full_size_zero_load_keeps_rest(mpm):
    from dataclasses import replace

    w = I.consolidation_block()
    w = replace(w, trac_full=np.zeros_like(w.trac_full))
    sim = mpm.Simulation(w)
    sim.step()
    got = sim.read(("u", "p"))
    assert np.abs(got["u"]).max() == 0.0 and np.abs(got["p"]).max() == 0.0
    sim.close()


def test_slope_full_size_mixed_step(mpm):
    """One mixed-precision step of the slope under gravity (water table at
    3.2 m): Newton converges with every FGMRES solve below its cap, the ground
    settles, and the nearly undrained response lifts the pore pressure above
    the hydrostatic value at the base."""
    w = I.slope_3d()
    assert w.n == 4208640
    sim = mpm.Simulation(w, precision=mpm.MPM_MIXED, newton_rtol=1e-8, newton_max=8, krylov_max=400)
    st = sim.step()
    r = st["res_norm"]
    assert 1 <= st["newton_iters"] <= 6 and r[-1] <= 1e-8 * r[0], r
    assert max(st["krylov_iters"]) < 400, st["krylov_iters"]
    got = sim.read(("u", "p"))
    assert np.isfinite(got["u"]).all() and np.isfinite(got["p"]).all()
    crest = w.x[:, 2] > 5.0
    assert got["u"][crest, 2].mean() < 0.0
    assert np.abs(got["u"]).max() < 0.2
    assert got["p"].max() > 1.5 * 1000.0 * 9.81 * 3.2
    sim.close()
