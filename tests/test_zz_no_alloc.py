"""mpm_bin_noalloc, the allocation-free binning entry point, against the
binning of the regular path (mpm_debug_bin).

It exists for callers that cannot allocate device memory where they bin points
(a solver inside a host application that owns all device memory through its
own pool, or a latency-critical loop that cannot afford cudaMalloc's implicit
synchronisation).  Binning is integer work, so the two must agree exactly, on
two calls in a row (the second on a different grid, so that counters left over
from the first call would show).  This file is collected last on purpose.
"""
import ctypes as C
from dataclasses import replace

import numpy as np
import pytest

from paper_1905_00671_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_00671_gb300 import mpm

    lib = mpm.load()
    lib.mpm_bin_noalloc.argtypes = [C.POINTER(mpm.mpm_grid), C.c_int64, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_void_p]
    lib.mpm_bin_noalloc.restype = C.c_int
    return torch, mpm, lib


def noalloc_bin(torch, mpm, lib, w):
    g = mpm.mpm_grid()
    g.dim = w.dim
    for k in range(3):
        g.ncell[k] = int(w.ncell[k]) if k < w.dim else 0
        g.origin[k] = float(w.origin[k]) if k < w.dim else 0.0
    g.h = float(w.h)
    x = torch.from_numpy(np.ascontiguousarray(w.x)).cuda()
    cell = torch.full((w.n,), -7, dtype=torch.int32, device="cuda")
    order = torch.full((w.n,), -7, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.mpm_bin_noalloc(C.byref(g), w.n, x.data_ptr(), cell.data_ptr(), order.data_ptr(),
                             stream)
    return rc, cell.cpu().numpy(), order.cpu().numpy()


def test_noalloc_binning_matches_regular_path_twice(env):
    torch, mpm, lib = env
    for w in (I.small_footing(seed=7, body=(24, 12), pad=2, h=0.25),
              I.small_block(seed=11, body=(6, 5, 4))):
        sim = mpm.Simulation(w)
        ref_cell, ref_order = sim.debug_bin()
        sim.close()
        rc, cell, order = noalloc_bin(torch, mpm, lib, w)
        assert rc == 0
        np.testing.assert_array_equal(cell, ref_cell)
        np.testing.assert_array_equal(order, ref_order)


def test_noalloc_rejects_grids_beyond_its_scratch(env):
    torch, mpm, lib = env
    w = I.small_footing(seed=7, body=(24, 12), pad=2, h=0.25)
    g = mpm.mpm_grid()
    g.dim = 2
    g.ncell[0], g.ncell[1] = 1024, 1024          # 1,048,576 cells > 262,144
    g.h = 0.01
    x = torch.zeros((4, 2), dtype=torch.float64, device="cuda")
    out_c = torch.zeros(4, dtype=torch.int32, device="cuda")
    out_o = torch.zeros(4, dtype=torch.int64, device="cuda")
    rc = lib.mpm_bin_noalloc(C.byref(g), 4, x.data_ptr(), out_c.data_ptr(), out_o.data_ptr(), None)
    assert rc == -10


def test_noalloc_rejects_cell_counts_that_would_overflow(env):
    """Per-axis counts whose product wraps (2^21 x 2^21 x 2^22 = 2^64) are
    rejected before any kernel runs; with n = 0 nothing touches the array."""
    torch, mpm, lib = env
    g = mpm.mpm_grid()
    g.dim = 3
    g.ncell[0], g.ncell[1], g.ncell[2] = 1 << 21, 1 << 21, 1 << 22
    g.h = 1.0
    assert lib.mpm_bin_noalloc(C.byref(g), 0, None, None, None, None) == -10


def test_noalloc_point_outside_grid_then_valid_call(env):
    """A point outside the grid: MPM_ERR_OUT_OF_GRID and cell -1 for it; the
    next valid call starts from a cleared error word and matches the regular
    path exactly."""
    torch, mpm, lib = env
    w = I.small_footing(seed=7, body=(24, 12), pad=2, h=0.25)
    bad = replace(w, x=w.x.copy())
    j = 5
    bad.x[j, 0] = -0.3                     # left of the grid's origin
    rc, cell, _ = noalloc_bin(torch, mpm, lib, bad)
    assert rc == -2
    assert cell[j] == -1
    sim = mpm.Simulation(w)
    ref_cell, ref_order = sim.debug_bin()
    sim.close()
    rc, cell, order = noalloc_bin(torch, mpm, lib, w)
    assert rc == 0
    np.testing.assert_array_equal(cell, ref_cell)
    np.testing.assert_array_equal(order, ref_order)
