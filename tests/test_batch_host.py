"""Host-side layout of batched instances (mpm_batch_pack): no GPU needed."""
import numpy as np
import pytest

from paper_1905_00671_gb300 import inputs as I
from paper_1905_00671_gb300 import mpm

GAP = 2  # MPM_BATCH_GAP in include/mpm.h


def _boxes(ws, offs):
    return [(offs[i, 0], offs[i, 1], offs[i, 0] + w.ncell[0], offs[i, 1] + w.ncell[1])
            for i, w in enumerate(ws)]


@pytest.mark.parametrize("count,seed", [(1, 1), (7, 2), (64, 5)])
def test_layout_is_disjoint_and_inside(count, seed):
    ws = I.batch_instances(count=count, seed=seed)
    offs, nc = mpm.batch_pack(ws)
    boxes = _boxes(ws, offs)
    for (x0, y0, x1, y1) in boxes:
        assert x0 >= 0 and y0 >= 0 and x1 <= nc[0] and y1 <= nc[1]
    # node boxes [x0, x1] x [y0, y1] of two instances are at least GAP cells apart
    for i in range(count):
        for j in range(i + 1, count):
            a, b = boxes[i], boxes[j]
            sep_x = max(b[0] - a[2], a[0] - b[2])
            sep_y = max(b[1] - a[3], a[1] - b[3])
            assert max(sep_x, sep_y) >= GAP, (i, j, a, b)
    assert nc[2] == 1


def test_layout_is_compact_and_deterministic():
    ws = I.batch_instances(count=64, seed=5)
    offs, nc = mpm.batch_pack(ws)
    offs2, nc2 = mpm.batch_pack(ws)
    assert np.array_equal(offs, offs2) and np.array_equal(nc, nc2)
    used = sum((w.ncell[0] + GAP) * (w.ncell[1] + GAP) for w in ws)
    assert nc[0] * nc[1] <= 2.0 * used        # shelf packing wastes at most half


def test_layout_rejects_mixed_grids():
    ws = I.batch_instances(count=3, seed=1)
    from dataclasses import replace
    bad = [ws[0], replace(ws[1], h=ws[1].h * 2.0), ws[2]]
    with pytest.raises(mpm.MPMError):
        mpm.batch_pack(bad)
