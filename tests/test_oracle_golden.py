"""The oracle still reproduces its committed Terzaghi trajectory (guards the
oracle's arithmetic against unintended change)."""

import numpy as np

from tests.golden.make_golden import OUT, generate


def test_terzaghi_golden_trajectory():
    ref = np.loadtxt(OUT)
    got = np.array(generate())
    np.testing.assert_array_equal(ref[:, :2], got[:, :2])
    np.testing.assert_allclose(got[:, 2], ref[:, 2], rtol=0, atol=1e-9 * 10e3)
