"""Spin-adapted target groups (configuration state functions, Eq. 2 with the
eta_im of the paper being CSFs): pins of the generator and of the oracle.

* every CSF the generator makes is an eigenfunction of S^2 (oracle/fock.py
  applies S^2 by its operator definition) with its stated spin, and the CSFs
  of a group are orthonormal;
* the structured build of a problem whose singlet and triplet target groups
  share their determinants and their continuum range equals the brute-force
  T^T H T with the CI vectors expanded over determinants;
* the singlet-triplet block is not zero: the target states couple through the
  exchange of the continuum electron (the classes 5 and 6 of Section 2.2
  between target spins), while their overlap and their H^N element vanish."""
import numpy as np
import pytest

from oracle import brute, coracle, fock
from paper_1709_03005_gb300 import synth


def _csf_vectors(g):
    n = g.dets.shape[0]
    out = []
    for i in range(len(g.csf_ptr) - 1):
        v = np.zeros(n)
        for k in range(g.csf_ptr[i], g.csf_ptr[i + 1]):
            v[g.csf_det[k]] += g.csf_coef[k]
        out.append(v)
    return np.array(out)


@pytest.mark.parametrize("seed,n_elec", [(12, 4), (13, 6)])
def test_csfs_are_spin_eigenfunctions(seed, n_elec):
    P = synth.make_csf_problem(seed=seed, n_to=8, n_elec=n_elec, n_config=12)
    for g in P.groups:
        tuples = [fock.words_to_tuple(d, P.n_words, P.n_to) for d in g.dets]
        index = {t: i for i, t in enumerate(tuples)}
        S2 = np.zeros((len(tuples), len(tuples)))
        for j, t in enumerate(tuples):
            for t2, c in fock.apply_s2(t, P.n_to).items():
                assert t2 in index          # every configuration carries all its determinants
                S2[index[t2], j] += c
        B = _csf_vectors(g)
        np.testing.assert_allclose(B @ B.T, np.eye(len(B)), atol=1e-12)
        s = g.spin
        np.testing.assert_allclose(B @ S2, s * (s + 1) * B, atol=1e-12)


def test_csf_groups_structured_equals_brute():
    P = synth.make_csf_problem(seed=14, n_to=7, n_co=4, n_elec=4, n_config=8, n_state=(2, 2), n_l2=6)
    Hb = brute.contracted_hamiltonian(P)
    o = coracle.Oracle(P)
    Ho = o.dense()
    np.testing.assert_allclose(Ho, Hb, rtol=0, atol=1e-12 * np.abs(Hb).max())
    # singlet (group 0) x triplet (group 1) block of the continuum part
    r0, r1, r2 = o.offsets[0], o.offsets[1], o.offsets[2]
    blk = Ho[r1:r2, r0:r1]
    assert np.abs(blk).max() > 1e-3, np.abs(blk).max()
    # their target parts vanish: overlap and H^N between spin states
    C0, C1 = brute.det_ci(P.groups[0]), brute.det_ci(P.groups[1])
    np.testing.assert_allclose(C1.T @ C0, 0.0, atol=1e-13)
    nd = P.groups[0].dets.shape[0]
    HN = np.array([[o.hij(P.groups[0].dets[a], P.groups[0].dets[b]) for b in range(nd)] for a in range(nd)])
    np.testing.assert_allclose(C1.T @ HN @ C0, 0.0, atol=1e-12)
