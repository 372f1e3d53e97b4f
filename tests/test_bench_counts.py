"""The bench's roofline arithmetic (no GPU): the Jacobian's flop counts follow
their stated formulas, the per-assembly total combines pairs and diagonal
terms as stated, the SpMV's algorithmic bytes, and the lookup of committed ncu
traffic by kernel source hash and workload."""
import pytest

import bench


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("dynamic", [False, True])
def test_jacobian_flop_counts_follow_their_formulas(dim, dynamic):
    d = dim
    f_diag = 2 * (2 * d * d + 6 * d + 1) + 1 + (2 * (d + 1) if dynamic else 0)
    f_pair = 2 * (2 * d * d + 6 * d + 1) + 1 + 6 * d + (2 * (2 * d + 1) if dynamic else 0)
    fp, fd, _ = bench.JAC_FLOPS[(dim, dynamic)]
    assert (fp, fd) == (f_pair, f_diag)


def test_jacobian_flops_per_assembly():
    # T ordered terms over points, P point-node pairs: (T - P) / 2 unordered
    # pairs a != b and P diagonal terms, plus the staging G per point-node pair
    fp, fd, g = bench.JAC_FLOPS[(3, False)]
    T, P = 1000, 40
    assert bench.jacobian_flops(3, False, False, T, P) == fp * (T - P) / 2 + (fd + g) * P
    h, gh = bench.JAC_FLOPS_HENCKY[3]
    assert bench.jacobian_flops(3, False, True, T, P) == (fp + h) * (T - P) / 2 + (fd + h + g + gh) * P


def test_spmv_bytes():
    # values + column indices + row pointers, x read once, y written once
    nnodes, nnzb, nb = 10, 37, 4
    assert bench.spmv_bytes(nnodes, nnzb, nb) == nnzb * (16 * 8 + 4) + 11 * 4 + 2 * 10 * 4 * 8
    assert bench.spmv_bytes(nnodes, nnzb, nb, word=4) == nnzb * (16 * 4 + 4) + 11 * 4 + 2 * 10 * 4 * 4


def test_traffic_lookup_by_hash_and_workload(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    h = bench.kernel_source_hash("k_bsr_spmv")  # read from the real tree
    (prof / "dram_traffic.txt").write_text(
        "# comment\n"
        f"k_bsr_spmv {h} slope-128x128x64 1 123456\n"
        "k_bsr_spmv 0000000000000000 footing-200x100 1 99\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda k: h)
    assert bench.ncu_traffic("k_bsr_spmv", "slope-128x128x64") == 123456.0
    assert bench.ncu_traffic("k_bsr_spmv", "footing-200x100") is None   # another source
    assert bench.ncu_traffic("k_jacobian", "slope-128x128x64") is None  # no line
    assert bench.ncu_traffic("k_bsr_spmv", "slope-64x64x32") is None    # another workload


def test_fp32_jacobian_bytes():
    # 3D quasi-static: 2 d^2 + 2 d + 9 + 12 d words per point; Hencky adds
    # the principal directions (d^2), kappa_A (d) and theta_AB (d (d - 1) / 2)
    n, nnzb, nnodes = 100, 2000, 50
    base = 4 * (18 + 6 + 9 + 36) * n + nnzb * (16 * 4 + 4) + nnodes * 52
    assert bench.jacobian32_bytes(n, nnzb, nnodes, 3, False) == base
    assert bench.jacobian32_bytes(n, nnzb, nnodes, 3, False, True) == base + 4 * (9 + 3 + 3) * n
    assert bench.jacobian32_bytes(n, nnzb, nnodes, 2, True, True) - bench.jacobian32_bytes(
        n, nnzb, nnodes, 2, True) == 4 * (4 + 2 + 1) * n
