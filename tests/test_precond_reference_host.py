"""Pins of the numpy preconditioner reference (no GPU)."""
from oracle import oracle as O
from paper_1905_00671_gb300 import inputs as I
from tests.precond_reference import fixed_stress_diag


def test_fixed_stress_reference_term_is_the_bulk_mass():
    """With uniform E, nu the lumped fixed-stress term sums (partition of unity
    over the active support nodes) to the total volume / (dt K), K = lambda +
    2 G / dim the drained bulk modulus."""
    for w in (I.terzaghi_column(), I.small_block(seed=11, body=(4, 3, 3), jitter=0.0)):
        orc = O.Oracle(w)
        prep = orc.prepare(w.dt)
        fs = fixed_stress_diag(w, prep)
        E, nu, d = w.E[0], w.nu[0], w.dim
        K = E * nu / ((1 + nu) * (1 - 2 * nu)) + 2 * E / (2 * (1 + nu)) / d
        assert abs(fs.sum() - w.vol.sum() / (w.dt * K)) <= 1e-12 * fs.sum()
        assert (fs >= 0).all()
