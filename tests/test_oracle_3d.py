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
