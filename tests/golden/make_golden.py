"""Writes the stored expected values under tests/golden/ from the oracle only.

lattice_d2q{9,17,37}.txt: scale r, then one line "ex ey w" per velocity, derived by the
oracle's Gauss-Hermite solve (Sec. 2, "Velocity stencils"). The CUDA library derives its own
constants with different code; the CPU tests compare the two.

Run: python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.stencil import lattice  # noqa: E402


def main():
    for q in (9, 17, 37):
        L = lattice(q)
        with open(os.path.join(HERE, f"lattice_d2q{q}.txt"), "w") as fh:
            fh.write(f"# D2Q{q} Gauss-Hermite rule from oracle/stencil.py (Sec. 2)\n")
            fh.write(f"r {L.r!r}\n")
            for (ex, ey), w in zip(L.e.tolist(), L.w.tolist()):
                fh.write(f"{ex} {ey} {w!r}\n")


if __name__ == "__main__":
    main()
