"""Writes the stored expected values under tests/golden/ from the CPU oracle only.

    python tests/golden/make_golden.py

quadrature_refined.txt: the oracle's refinement of the printed Sec. 2.3
quadrature onto the exact solutions of Eq. orthonormal (17 significant digits).
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import quadrature  # noqa: E402


def main():
    q = quadrature.quadrature()
    with open(os.path.join(HERE, "quadrature_refined.txt"), "w") as f:
        f.write("# Oracle refinement (minimum-norm Gauss-Newton onto Eq. orthonormal) of the\n")
        f.write("# quadrature printed in Sec. 2.3; written by tests/golden/make_golden.py.\n")
        f.write("# columns: shell j, w_1j, w_2j, p0_j\n")
        for j in range(4):
            f.write(f"{j + 1} {q['w1'][j]:.17e} {q['w2'][j]:.17e} {q['p0'][j]:.17e}\n")


if __name__ == "__main__":
    main()
