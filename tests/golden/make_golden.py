"""Writes the stored expected values under tests/golden/ from the oracle alone.

c1_tiny.txt holds, for the tiny workload (10 target and 20 continuum orbitals,
N = 6 + 1, 40 target determinants, 3 states, 50 L2 functions; dimension 110):
* the excitation record (degree, two holes, two particles, phase; Section 2.1)
  of 200 seeded determinant pairs, from the oracle's bitstring rules;
* every diagonal element and 400 seeded off-diagonal elements of the
  Hamiltonian of Eq. 1 in the close-coupling basis (classes 1-8, Section 2.2),
  from the oracle's structured build (Eq. 5, 7, 8);
* all 110 eigenvalues of that matrix (numpy's eigh of the oracle's matrix).
Values are printed with 17 significant digits, so they read back bit for bit.

Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import coracle  # noqa: E402
from paper_1709_03005_gb300 import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c1_tiny.txt")


def sample_pairs(P, rng, n):
    dets = np.concatenate([g.dets for g in P.groups])
    i = rng.integers(0, dets.shape[0], n)
    j = rng.integers(0, dets.shape[0], n)
    return dets, i, j


def main():
    P = synth.make_config("c1")
    o = coracle.Oracle(P)
    H = o.dense()
    rng = np.random.default_rng(2024)
    dets, pi, pj = sample_pairs(P, rng, 200)
    lines = ["# c1_tiny: oracle values (see make_golden.py); dimension %d, contracted %d" % (o.dim, o.Dc)]
    lines.append("# excitation i j degree h1 h2 p1 p2 phase  (determinants of the target groups, in group order)")
    for a, b in zip(pi, pj):
        r = coracle.Oracle.excitation(P.n_words, dets[a], dets[b])
        lines.append("x %d %d %s" % (a, b, " ".join(str(int(v)) for v in r)))
    lines.append("# element row col value")
    for i in range(o.dim):
        lines.append("e %d %d %.17g" % (i, i, H[i, i]))
    r, c = rng.integers(0, o.dim, 400), rng.integers(0, o.dim, 400)
    for i, j in zip(r, c):
        lines.append("e %d %d %.17g" % (i, j, H[i, j]))
    lines.append("# eigenvalue index value")
    for k, w in enumerate(np.linalg.eigvalsh(H)):
        lines.append("w %d %.17g" % (k, w))
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
