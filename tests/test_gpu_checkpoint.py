"""Checkpoint / resume: the full point state read after a few steps and
written into a fresh context of the same workload repeats the run exactly."""
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


@pytest.mark.parametrize("make", [lambda: I.small_footing(seed=31, body=(12, 6), pad=2),
                                  lambda: I.small_block(seed=32, body=(5, 4, 3))])
def test_resumed_trajectory_is_bit_exact(mpm, make):
    w = make()
    a = mpm.Simulation(w)
    for _ in range(2):
        a.step()
    ck = a.checkpoint()
    for _ in range(2):
        a.step()
    ra = a.read()
    b = mpm.Simulation(w)
    b.restore(ck)
    assert b.t == ck["t"]
    for _ in range(2):
        b.step()
    rb = b.read()
    for f in ra:
        assert np.array_equal(ra[f], rb[f]), f
    assert b.stats()["steps"] == a.stats()["steps"]
    a.close()
    b.close()
