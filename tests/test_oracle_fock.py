"""Pins of the definition-level Hamiltonian (oracle/fock.py) against closed forms,
textbook results and invariances that do not use it to check itself."""
import itertools

import numpy as np
import pytest

from oracle import fock


def _rand_ints(rng, n, rank=6):
    h = rng.normal(0, 0.3, (n, n)); h = h + h.T
    L = rng.normal(0, 0.4, (n, n, rank)); L = L + L.transpose(1, 0, 2)
    eri = np.einsum("pqk,rsk->pqrs", L, L)
    return h, eri


def _all_dets(n, na, nb):
    out = []
    for a in itertools.combinations(range(n), na):
        for b in itertools.combinations(range(n), nb):
            out.append(tuple(sorted(list(a) + [n + x for x in b])))
    return out


def test_integral_eightfold_symmetry_generator():
    from paper_1709_03005_gb300 import synth
    P = synth.make_tiny(7)
    g = P.full_eri()
    for perm in ["qprs", "pqsr", "rspq", "srqp", "qpsr", "rsqp", "srpq"]:
        np.testing.assert_allclose(np.einsum(f"pqrs->{perm}", g), g, atol=1e-14)


def test_class_arrays_match_full_tensor():
    from paper_1709_03005_gb300 import synth
    P = synth.make_tiny(8, n_to=4, n_co=3)
    g = P.full_eri()
    nt, nc = P.n_to, P.n_co
    pi = lambda p, q: synth.pair_index(p, q)
    for p, q, r, s in itertools.product(range(nt), repeat=4):
        assert P.eri_tttt[pi(p, q), pi(r, s)] == pytest.approx(g[p, q, r, s], abs=1e-13)
    for p, q, r, j in itertools.product(range(nt), range(nt), range(nt), range(nc)):
        assert P.eri_tttc[pi(p, q), r * nc + j] == pytest.approx(g[p, q, r, nt + j], abs=1e-13)
    for p, q, j, k in itertools.product(range(nt), range(nt), range(nc), range(nc)):
        assert P.eri_ttcc[pi(p, q), j * nc + k] == pytest.approx(g[p, q, nt + j, nt + k], abs=1e-13)
    for r, j, s, k in itertools.product(range(nt), range(nc), range(nt), range(nc)):
        assert P.eri_tctc[r * nc + j, s * nc + k] == pytest.approx(g[r, nt + j, s, nt + k], abs=1e-13)


def test_single_determinant_energy_textbook():
    """<D|H|D> = sum_i h_ii + 1/2 sum_ij [(ii|jj) - delta_spin (ij|ji)] (Szabo-Ostlund Table 2.4)."""
    rng = np.random.default_rng(0)
    n = 5
    h, eri = _rand_ints(rng, n)
    for det in [(0, 2, 5, 6), (1, 3, 4, 7, 9), (0, 1, 2)]:
        occ = [(so // n, so % n) for so in det]
        e = sum(h[p, p] for _, p in occ)
        for (s1, p), (s2, q) in itertools.product(occ, occ):
            e += 0.5 * eri[p, p, q, q]
            if s1 == s2:
                e -= 0.5 * eri[p, q, q, p]
        Hm = fock.hamiltonian_matrix([det], h, eri, n)
        assert Hm[0, 0] == pytest.approx(e, abs=1e-12)


def test_one_electron_spectrum_closed_form():
    """No two-electron integrals, complete determinant space: the eigenvalues are
    sums of orbital energies (eigenvalues of h) over occupied alpha and beta sets."""
    rng = np.random.default_rng(1)
    n, na, nb = 5, 2, 1
    h = rng.normal(0, 0.5, (n, n)); h = h + h.T
    eri = np.zeros((n, n, n, n))
    dets = _all_dets(n, na, nb)
    H = fock.hamiltonian_matrix(dets, h, eri, n)
    eps = np.linalg.eigvalsh(h)
    ref = sorted(sum(eps[list(a)]) + sum(eps[list(b)])
                 for a in itertools.combinations(range(n), na)
                 for b in itertools.combinations(range(n), nb))
    np.testing.assert_allclose(np.linalg.eigvalsh(H), ref, atol=1e-12)


def test_two_electrons_two_orbitals_textbook():
    """Minimal-basis two-electron problem: the Ms=1 triplet energy is
    h11 + h22 + J12 - K12, and the singlet block is the textbook 3x3 CI."""
    rng = np.random.default_rng(2)
    n = 2
    h, eri = _rand_ints(rng, n)
    trip = fock.hamiltonian_matrix([(0, 1)], h, eri, n)[0, 0]
    assert trip == pytest.approx(h[0, 0] + h[1, 1] + eri[0, 0, 1, 1] - eri[0, 1, 1, 0], abs=1e-12)
    # Ms = 0 space: |1a1b>, |1a2b>, |2a1b>, |2a2b>; the triplet Ms=0 component
    # (1a2b + 2a1b)/sqrt2 up to sign is degenerate with the Ms=1 triplet.
    dets = [(0, 2), (0, 3), (1, 2), (1, 3)]
    H = fock.hamiltonian_matrix(dets, h, eri, n)
    ev = np.linalg.eigvalsh(H)
    assert np.min(np.abs(ev - trip)) < 1e-12
    # closed-shell diagonal: 2 h11 + J11
    assert H[0, 0] == pytest.approx(2 * h[0, 0] + eri[0, 0, 0, 0], abs=1e-12)


def test_hermitian_and_conserving():
    rng = np.random.default_rng(3)
    n = 4
    h, eri = _rand_ints(rng, n)
    dets = _all_dets(n, 2, 1)
    H = fock.hamiltonian_matrix(dets, h, eri, n)
    np.testing.assert_allclose(H, H.T, atol=1e-13)
    # H never leaves the (N_alpha, N_beta) sector
    for d in dets[:5]:
        for d2 in fock.apply_hamiltonian(d, h, eri, n):
            assert sum(1 for so in d2 if so < n) == 2 and len(d2) == 3


def test_full_ci_invariant_under_orbital_rotation():
    """The full-CI spectrum does not depend on the orbital basis: rotating h and
    (pq|rs) by an orthogonal U leaves every eigenvalue unchanged.  A wrong sign
    or index anywhere in the operator application breaks this."""
    rng = np.random.default_rng(4)
    n = 4
    h, eri = _rand_ints(rng, n)
    U, _ = np.linalg.qr(rng.standard_normal((n, n)))
    h2 = U.T @ h @ U
    eri2 = np.einsum("pqrs,pa,qb,rc,sd->abcd", eri, U, U, U, U)
    dets = _all_dets(n, 2, 2)
    e1 = np.linalg.eigvalsh(fock.hamiltonian_matrix(dets, h, eri, n))
    e2 = np.linalg.eigvalsh(fock.hamiltonian_matrix(dets, h2, eri2, n))
    np.testing.assert_allclose(e1, e2, atol=1e-11)
