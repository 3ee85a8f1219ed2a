"""Writes the regression fixtures of this directory from the FP64 oracle alone.

The paper prints no worked numerical example of the residual (its tables are
timings, grid bandwidths and code sizes), so these fixtures hold no paper
values.  They freeze what the oracle computes for small seeded inputs -- the
oracle itself is pinned by closed forms and invariants in the -m "not gpu"
tests -- so that a later change of the oracle's arithmetic shows up as a
diff of a committed file, and the GPU path can be checked against stored
numbers.

    python tests/golden/make_golden.py      # rewrites residual_*.txt

Inputs come from the seeded generators (paper_2209_01877_gb300/inputs.py);
values only from oracle/.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle.dg import Problem  # noqa: E402
from paper_2209_01877_gb300 import inputs as I  # noqa: E402

# name -> (cube cells per side, jitter, order, flux, field); the fixtures keep the residual of
# the first NKEEP elements (caller order) of the full periodic mesh
CASES = {
    "residual_p1_cube3_rusanov_vortex": (3, 0.10, 1, "rusanov", "vortex"),
    "residual_p2_cube3_roe_entropywave": (3, 0.15, 2, "roe", "entropy_wave"),
}
NKEEP = 24


def field_of(name):
    if name == "vortex":
        return lambda x: I.isentropic_vortex(x, radius=0.2)
    return lambda x: I.entropy_wave(x)


def inputs(case):
    """mesh, projected state and oracle of a case (the state is input data, not a fixture)"""
    n, jitter, p, flux, field = CASES[case]
    m = I.make_periodic_cube(n, jitter=jitter)
    P = Problem(m.tet_vid, m.tet_xyz, None, p=p, flux=flux)
    return m, P, P.project(field_of(field))


def compute(case):
    m, P, U = inputs(case)
    return U, P.residual(U, np.arange(NKEEP))


def write(case):
    U, R = compute(case)
    n, jitter, p, flux, field = CASES[case]
    with open(os.path.join(HERE, case + ".txt"), "w") as f:
        f.write(f"# oracle residual of elements 0..{NKEEP - 1}, periodic {n}^3 x 6 cube, jitter {jitter}, P{p}, "
                f"{flux} flux, {field} projected by the oracle (conical rule); shape {R.shape}; "
                f"written by make_golden.py\n")
        for x in R.ravel():
            f.write(f"{x:.17e}\n")


def read(case):
    return np.loadtxt(os.path.join(HERE, case + ".txt"))


if __name__ == "__main__":
    for c in CASES:
        write(c)
        print("wrote", c)
