"""The oracle against the stored values of tests/golden/c1_tiny.txt.

The file was written by tests/golden/make_golden.py from the oracle; the oracle
is built without fused multiply-adds and sums in a fixed order, so it must
reproduce every stored element and excitation record bit for bit on any
host (a change to its arithmetic shows up here first).  The stored records also
satisfy what the bitstring rules fix (Section 2.1): the degree is half the
number of differing spin orbitals, records of degree 1 and 2 carry distinct
holes and particles and a phase of +1 or -1, and the matrix is symmetric."""
import numpy as np

from golden_io import read
from oracle import coracle
from paper_1709_03005_gb300 import synth


def test_oracle_reproduces_golden():
    exc, elem, evals = read()
    P = synth.make_config("c1")
    o = coracle.Oracle(P)
    H = o.dense()
    dets = np.concatenate([g.dets for g in P.groups])
    for rec in exc:
        i, j = rec[0], rec[1]
        got = coracle.Oracle.excitation(P.n_words, dets[i], dets[j])
        assert np.array_equal(got, rec[2:]), (i, j, got, rec[2:])
    for i, j, v in elem:
        assert H[i, j] == v, (i, j, H[i, j], v)
    np.testing.assert_allclose(np.linalg.eigvalsh(H), evals, rtol=0, atol=1e-10 * np.abs(evals).max())


def test_golden_records_are_consistent():
    exc, elem, evals = read()
    P = synth.make_config("c1")
    dets = np.concatenate([g.dets for g in P.groups])
    for rec in exc:
        i, j, deg, h1, h2, p1, p2, ph = rec
        nd = sum(bin(int(a) ^ int(b)).count("1") for a, b in zip(dets[i], dets[j]))
        assert deg == nd // 2
        if 1 <= deg <= 2:
            assert ph in (-1, 1)
            holes, parts = [h for h in (h1, h2) if h >= 0], [p for p in (p1, p2) if p >= 0]
            assert len(holes) == deg and len(parts) == deg
            assert not set(holes) & set(parts)
    table = {(i, j): v for i, j, v in elem}
    for (i, j), v in table.items():
        if (j, i) in table:
            assert table[(j, i)] == v
    assert len(evals) == 110 and np.all(np.diff(evals) >= 0)
