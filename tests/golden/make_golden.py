"""Writes the frozen oracle outputs of this folder.  Calls only oracle/ (and workloads.py
for the seeded inputs)."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
import oracle  # noqa: E402
import workloads  # noqa: E402


def write(name, arrays):
    with open(os.path.join(HERE, name), "w") as f:
        for key, a in arrays.items():
            a = np.atleast_2d(np.asarray(a, dtype=np.float64))
            f.write(f"# {key} {a.shape[0]} {a.shape[1]}\n")
            for row in a:
                f.write(" ".join(repr(float(x)) for x in row) + "\n")


def main():
    A = workloads.sym_gaussian(12, seed=5)
    Aout, tau = oracle.sy2sb(A, 3)
    write("sy2sb_n12_w3.txt", {"A": A, "Aout_lower": np.tril(Aout), "tau": tau})
    G = workloads.gen_gaussian(10, 8, seed=6)
    Gout, tq, tp = oracle.ge2gb(G, 2)
    write("ge2gb_m10_n8_w2.txt", {"A": G, "Aout": Gout, "tauq": tq, "taup": tp})
    # the second stage: a symmetric band -> tridiagonal, an upper band -> bidiagonal
    S = workloads.sym_gaussian(14, seed=7)
    i, j = np.indices(S.shape)
    S[np.abs(i - j) > 3] = 0.0
    d, e = oracle.sb2st(np.tril(S), 3)
    write("sb2st_n14_w3.txt", {"A_lower": np.tril(S), "d": d, "e": e})
    U = np.triu(workloads.gen_gaussian(14, 14, seed=8))
    U = U - np.triu(U, 4)
    d, e = oracle.gb2bd(U, 3)
    write("gb2bd_n14_w3.txt", {"A_upper": U, "d": d, "e": e})


if __name__ == "__main__":
    main()
