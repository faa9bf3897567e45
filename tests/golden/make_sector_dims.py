"""Writes sector_dims.txt: sizes of a few (M, N, P) sectors counted by the CPU
oracle's brute-force enumeration (special Hilbert spaces, Sec. III B and App. A).
Calls only oracle/.  Run from the repository root:  python tests/golden/make_sector_dims.py
"""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
import oracle as orc  # noqa: E402

CASES = [(5, 6, 0), (5, 6, 2), (7, 12, 0), (7, 16, 3), (9, 10, 0), (5, 30, 1), (11, 20, 0), (11, 8, 5)]

if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "sector_dims.txt")
    with open(out, "w") as f:
        f.write("# M N P dim -- momentum labels i-(M-1)/2, conserved mod M; written by make_sector_dims.py\n")
        for M, N, P in CASES:
            f.write(f"{M} {N} {P} {orc.sector_dim(M, N, P)}\n")
    print(open(out).read())
