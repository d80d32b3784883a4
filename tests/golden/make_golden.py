"""Writes the golden fixtures of this folder from the CPU oracle alone (no CUDA code).

rt_16x32_3steps.txt: a 16 x 32 Rayleigh-Taylor state (seed 9, tau 0.8, g = 1e-4 in -y,
walls at 1.15 and 0.85) after 3 oracle steps.  Per population i: the sum of f_i over the
lattice, and f_i at sites (0, 0), (7, 15) and (15, 31) (a wall corner, the interior and
the opposite corner), as float64 hex strings.  The fixture guards the oracle against
unintended change (its pins are the closed-form tests in tests/test_oracle_*.py) and gives
the GPU path a stored reference.

    python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import lbm as OL  # noqa: E402
from paper_1703_04594_gb300 import inputs as I  # noqa: E402

LX, LY, SEED, STEPS = 16, 32, 9, 3
SITES = ((0, 0), (7, 15), (15, 31))


def compute():
    fields = I.rt_state(LX, LY, SEED)
    f = OL.run(OL.init_equilibrium(*fields), OL.Params(LX, LY), STEPS)
    rows = []
    for i in range(37):
        vals = [float(f[i].sum())] + [float(f[i, x, y]) for x, y in SITES]
        rows.append(vals)
    return rows


def main():
    path = os.path.join(HERE, "rt_16x32_3steps.txt")
    with open(path, "w") as out:
        out.write(f"# oracle: {LX}x{LY} RT seed {SEED}, {STEPS} steps; per population: sum, f at {SITES}\n")
        for i, vals in enumerate(compute()):
            out.write(" ".join([str(i)] + [v.hex() for v in vals]) + "\n")
    print("wrote", path)


if __name__ == "__main__":
    main()
