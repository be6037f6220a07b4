"""Writes the stored expected values under tests/golden/ by calling only oracle/.

The paper prints no entry of Theta and no wavelet coefficient (its only numbers are
timings), so these fixtures are regression values of the FP64 oracle on the seeded
1-D workload c1 (n=256, db2, L=5, m=4 Gaussian blurs, 4 hat windows): a fixed set of
entries Theta[mu, lambda], with the trace.  Run: python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import pc_inputs as P  # noqa: E402


def main():
    op = P.workload("c1")
    cols = np.arange(op.N)
    T = oracle.theta_columns(op, cols).T
    rng = np.random.default_rng(20050987)
    pairs = rng.integers(0, op.N, size=(64, 2))
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c1_theta_entries.txt")
    with open(path, "w") as f:
        f.write("# workload c1 (pc_inputs.workload('c1')): mu lambda Theta[mu,lambda] (FP64 oracle)\n")
        f.write(f"# trace {np.trace(T):.17e}\n")
        for mu, lam in pairs:
            f.write(f"{mu} {lam} {T[mu, lam]:.17e}\n")
        for i in range(0, op.N, 17):
            f.write(f"{i} {i} {T[i, i]:.17e}\n")
    print("wrote", path)


if __name__ == "__main__":
    main()
