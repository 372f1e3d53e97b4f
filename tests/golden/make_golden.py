"""Writes tests/golden/terzaghi_4x40_oracle.txt from the CPU oracle alone.

Column 4 x 40 (h = 0.25 m), E = 10 MPa, nu = 0.3, k = 1e-10 m^2,
mu_f = 1e-3 Pa s, 10 kPa top load, dt = 1 s, 10 steps, original MPM + PPP
(Sec. 5.1 set-up with these parameters).  Each line: step, depth z of the
centre-column node, nodal pressure P (Pa) after the step's Newton solve.
Regenerate with `python tests/golden/make_golden.py` only when a change to the
oracle's arithmetic is justified by the paper.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O  # noqa: E402
from paper_1905_00671_gb300 import inputs as I  # noqa: E402

OUT = os.path.join(HERE, "terzaghi_4x40_oracle.txt")


def generate():
    w = I.terzaghi_column()
    o = O.Oracle(w, newton_rtol=1e-12, newton_stag=1e-6)
    rows = []
    for s in range(w.nsteps):
        o.step()
        _, X, _ = o.last
        P = X.reshape(-1, 3)[:, 2].reshape(41, 5)[:, 2]
        for j in range(41):
            rows.append((s + 1, 10.0 - 0.25 * j, P[j]))
    return rows


if __name__ == "__main__":
    with open(OUT, "w") as f:
        f.write("# oracle Terzaghi 4x40 column: step depth_m P_Pa (written by make_golden.py)\n")
        for s, z, p in generate():
            f.write(f"{s} {z:.4f} {p:.12e}\n")
    print("wrote", OUT)
