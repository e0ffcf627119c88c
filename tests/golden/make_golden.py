"""Write the oracle regression fixture (calls only oracle/ and the seeded input generators)."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1710_09995_gb300 import cases  # noqa: E402


def fixture():
    c = cases.smooth_random(12, 10, 8, seed=21, amp=0.1, viscous=True, mu=5e-3)
    M = oracle.metrics(cases.warped_nodes(12, 10, 8, 0.05))
    R = oracle.residual(oracle.params(mu=5e-3, viscous=True), oracle.pad(c.state), M)
    rng = np.random.Generator(np.random.PCG64(5))
    cells = [(int(rng.integers(8)), int(rng.integers(10)), int(rng.integers(12))) for _ in range(24)]
    return cells, R


def main():
    cells, R = fixture()
    with open(os.path.join(HERE, "oracle_residual_warped.txt"), "w") as f:
        f.write("# k j i R_rho R_rhou R_rhov R_rhow R_rhoE  (oracle, seeded 12x10x8 warped NS case, mu 5e-3)\n")
        for k, j, i in cells:
            f.write(f"{k} {j} {i} " + " ".join(f"{R[m, k, j, i]:.17e}" for m in range(5)) + "\n")


if __name__ == "__main__":
    main()
