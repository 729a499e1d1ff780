"""Pins of the C oracle (oracle/hb_oracle.c): bitstring Slater-Condon rules
(Section 2.1) against the operator definition, and the structured prototype /
contract / expand build (Eq. 6-8) against the brute-force T^T H T (Eq. 3-5)
plus invariances and special cases that reduce to library routines."""
import itertools

import numpy as np
import pytest

from oracle import brute, coracle, fock
from paper_1709_03005_gb300 import synth


def _words(alpha, beta, W):
    return synth.occ_to_words(sorted(alpha), sorted(beta), W)


def _op_phase(I, J, W, holes, parts):
    """<I| a+_p1 a+_p2 a_h2 a_h1 |J> by applying operators (fock)."""
    n = 64 * W
    d = fock.words_to_tuple(J, W, n)
    sign = 1
    for so in holes:            # a_h1 first, then a_h2
        s, d = fock.annihilate(d, so)
        sign *= s
    for so in reversed(parts):  # a+_p2 first, then a+_p1
        s, d = fock.create(d, so)
        sign *= s
    assert d == fock.words_to_tuple(I, W, n)
    return sign


@pytest.mark.parametrize("W,orbs", [
    (1, list(range(12))),
    (2, [0, 1, 2, 61, 62, 63, 64, 65, 66, 127]),
    (3, [0, 5, 62, 63, 64, 65, 126, 127, 128, 129, 190, 191]),
])
def test_excitation_phase_against_operators(W, orbs):
    """Degree, holes, particles and phase, including orbitals at indices
    63/64/127/128 where the paper reports a mask bug at multiples of 64."""
    rng = np.random.default_rng(W)
    bra, ket = synth.random_det_pairs(rng, 64 * W, 3, 3, W, 400, max_exc=3, orbitals=orbs)
    seen = set()
    for I, J in zip(bra, ket):
        out = coracle.Oracle.excitation(W, I, J)
        deg = int(out[0])
        xor = sum(bin(int(a) ^ int(b)).count("1") for a, b in zip(I, J))
        assert deg == xor // 2
        seen.add(deg)
        if deg == 0 or deg > 2:
            continue
        holes = [int(h) for h in out[1:1 + deg]]
        parts = [int(p) for p in out[3:3 + deg]]
        bitsI = {64 * w + b for w in range(2 * W) for b in range(64) if (int(I[w]) >> b) & 1}
        bitsJ = {64 * w + b for w in range(2 * W) for b in range(64) if (int(J[w]) >> b) & 1}
        assert holes == sorted(bitsJ - bitsI) and parts == sorted(bitsI - bitsJ)
        assert int(out[5]) == _op_phase(I, J, W, holes, parts)
    assert {1, 2} <= seen


def _tiny_problem_and_eri(seed, **kw):
    P = synth.make_tiny(seed, **kw)
    return P, P.full_eri()


def test_slater_condon_elements_against_operators():
    """Numeric <I|H|J> of the bitstring rules == operator definition."""
    P, eri = _tiny_problem_and_eri(21, n_to=7, n_co=2, n_elec=4)
    o = coracle.Oracle(P)
    rng = np.random.default_rng(5)
    bra, ket = synth.random_det_pairs(rng, P.n_to, 3, 2, P.n_words, 300, max_exc=3)
    n = P.n_orb
    for I, J in zip(bra, ket):
        dI = fock.words_to_tuple(I, P.n_words, n)
        dJ = fock.words_to_tuple(J, P.n_words, n)
        ref = fock.apply_hamiltonian(dJ, P.h, eri, n).get(dI, 0.0)
        assert o.hij(I, J) == pytest.approx(ref, abs=1e-12)


CASES = [
    dict(),
    dict(n_to=6, n_elec=4, n_det=8, n_state=3, n_l2=7),
    dict(n_groups=2, n_state=[2, 3], cont_ranges=[(0, 3), (1, 2)]),
    dict(cont_spin=1),
    dict(n_groups=3, n_det=4, n_state=[1, 2, 2], cont_ranges=[(0, 2), (0, 3), (2, 1)], cont_spin=1),
    dict(n_to=6, n_co=4, n_elec=6, n_det=10, n_state=4, n_l2=9),
    dict(n_l2=0),
    dict(n_groups=2, n_co=4, n_det=5, n_state=[2, 2], cont_ranges=[(0, 2), (2, 2)], n_l2=3),
    dict(n_groups=2, n_state=[2, 2], cont_ranges=[(0, 3), (0, 2)], e_core=-4.75),
]


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("seed", [101, 202, 303])
def test_structured_equals_brute_force(case, seed):
    P = synth.make_tiny(seed + case, **CASES[case])
    Hb = brute.contracted_hamiltonian(P)
    Ho = coracle.Oracle(P).dense()
    scale = max(1.0, np.abs(Hb).max())
    np.testing.assert_allclose(Ho, Hb, rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(Ho, Ho.T, rtol=0, atol=0)


def test_identity_ci_reproduces_uncontracted():
    """C = I: the contracted matrix is the uncontracted determinant matrix."""
    P = synth.make_tiny(31, n_det=5, n_state=2)
    g = P.groups[0]
    g.ci = np.eye(g.dets.shape[0])
    Ho = coracle.Oracle(P).dense()
    Hb, Hu, T, _ = brute.contracted_hamiltonian(P, return_parts=True)
    # T is a permutation here
    assert np.allclose(np.sort(T.sum(0)), 1) and np.allclose(T @ T.T, np.eye(T.shape[0]))
    np.testing.assert_allclose(Ho, T.T @ Hu @ T, atol=1e-12)


def test_target_energy_identity():
    """With every integral that touches a continuum orbital set to zero, the
    continuum-continuum block is delta_jj' <phi_n|H^N|phi_n'>; with CI vectors
    that are eigenvectors of the target Hamiltonian (numpy eigh) it is
    diag(E_n), the target-energy substitution of Section 3.1."""
    P = synth.make_tiny(41, n_to=5, n_co=3, n_elec=4, n_det=12, n_state=3, n_l2=0)
    nt = P.n_to
    P.h[nt:, :] = 0.0; P.h[:, nt:] = 0.0
    P.eri_tttc[:] = 0.0; P.eri_ttcc[:] = 0.0; P.eri_tctc[:] = 0.0
    o = coracle.Oracle(P)
    g = P.groups[0]
    HN = np.array([[o.hij(a, b) for b in g.dets] for a in g.dets])
    E, V = np.linalg.eigh(HN)
    g.ci = np.ascontiguousarray(V[:, :3])
    H = coracle.Oracle(P).dense()
    nco = P.n_co
    ref = np.kron(np.diag(E[:3]), np.eye(nco))
    np.testing.assert_allclose(H, ref, atol=1e-12)


def test_state_rotation_and_sign_invariance():
    P = synth.make_tiny(51, n_det=8, n_state=3)
    ev0 = np.linalg.eigvalsh(coracle.Oracle(P).dense())
    rng = np.random.default_rng(0)
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    P.groups[0].ci = np.ascontiguousarray(P.groups[0].ci @ Q * np.array([1, -1, 1]))
    ev1 = np.linalg.eigvalsh(coracle.Oracle(P).dense())
    np.testing.assert_allclose(ev0, ev1, atol=1e-11)


def _permute_target_orbitals(P, perm):
    """New problem with target orbital p renamed perm[p] (integrals and bits)."""
    import copy
    Q = copy.deepcopy(P)
    nt, nc = P.n_to, P.n_co
    full = np.arange(P.n_orb)
    full[:nt] = perm
    inv = np.argsort(full)
    Q.h = P.h[np.ix_(inv, inv)]
    pi = synth.pair_index
    ip = np.array([pi(inv[p], inv[q]) for p in range(nt) for q in range(p + 1)])
    Q.eri_tttt = P.eri_tttt[np.ix_(ip, ip)]
    tc = np.array([inv[r] * nc + j for r in range(nt) for j in range(nc)])
    Q.eri_tttc = P.eri_tttc[np.ix_(ip, tc)]
    Q.eri_ttcc = P.eri_ttcc[ip]
    Q.eri_tctc = P.eri_tctc[np.ix_(tc, tc)]

    def parity(seq):
        # sign of the permutation that sorts seq (count inversions)
        inv_count = sum(1 for i in range(len(seq)) for k in range(i + 1, len(seq)) if seq[i] > seq[k])
        return -1.0 if inv_count % 2 else 1.0

    def remap(D):
        out = np.zeros_like(D)
        sign = np.ones(D.shape[0])
        W = P.n_words
        for i, w in enumerate(D):
            a = [perm[p] for p in range(nt) if (int(w[p // 64]) >> (p % 64)) & 1]
            b = [perm[p] for p in range(nt) if (int(w[W + p // 64]) >> (p % 64)) & 1]
            out[i] = synth.occ_to_words(a, b, W)
            sign[i] = parity(a) * parity(b)
        return out, sign
    # the renamed determinant a+_{perm p1} a+_{perm p2}... equals the canonically
    # ordered one times the parity of the sort, so the CI coefficients take
    # that sign to describe the same target state
    for g in Q.groups:
        g.dets, sgn = remap(g.dets)
        g.ci = np.ascontiguousarray(g.ci * sgn[:, None])
    Q.l2_dets, _ = remap(P.l2_dets)
    Q.chol = None
    return Q


def test_target_orbital_relabelling_invariance():
    """Renaming target orbitals changes every phase but not the spectrum."""
    P = synth.make_tiny(61, n_to=6, n_elec=4, n_det=9, n_state=3, n_l2=8)
    ev0 = np.linalg.eigvalsh(coracle.Oracle(P).dense())
    perm = np.array([3, 0, 5, 1, 4, 2])
    Q = _permute_target_orbitals(P, perm)
    ev1 = np.linalg.eigvalsh(coracle.Oracle(Q).dense())
    np.testing.assert_allclose(ev0, ev1, atol=1e-11)


def test_beyond_double_excitations_vanish():
    """L2-L2 elements between determinants more than doubly excited are exactly 0,
    and C = I class-4 elements vanish unless the pair is within a double."""
    P = synth.make_tiny(71, n_to=7, n_elec=4, n_det=10, n_state=2, n_l2=30)
    o = coracle.Oracle(P)
    H = o.dense()
    Dc = o.Dc
    L2 = P.l2_dets
    for a in range(P.n_l2):
        for b in range(P.n_l2):
            nd = sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(L2[a], L2[b]))
            if nd > 4:
                assert H[Dc + a, Dc + b] == 0.0
    P.groups[0].ci = np.eye(10)
    o = coracle.Oracle(P)
    H = o.dense()
    nco = P.n_co
    for m in range(10):
        D = P.groups[0].dets[m]
        for l in range(P.n_l2):
            d = sum(bin(int(x) & ~int(y)).count("1") for x, y in zip(D, L2[l]))
            if d > 1:
                assert np.all(H[o.Dc + l, m * nco:(m + 1) * nco] == 0.0)


def test_contraction_interlacing():
    """Contracted eigenvalues lie above the uncontracted ones (Cauchy interlacing
    for an orthonormal contraction T), so contraction never lowers a root."""
    P = synth.make_tiny(81, n_det=8, n_state=2, n_l2=6)
    Hb, Hu, T, _ = brute.contracted_hamiltonian(P, return_parts=True)
    a = np.linalg.eigvalsh(coracle.Oracle(P).dense())
    b = np.linalg.eigvalsh(Hu)
    assert np.all(a >= b[: len(a)] - 1e-11)


def test_tl2_classification_record():
    """T x L2 records: degree of the (N+1)-electron pair and its phase against the
    operator definition, with the continuum electron appended above every target
    orbital of its spin."""
    for spin in (0, 1):
        P = synth.make_tiny(91 + spin, n_to=7, n_elec=4, n_det=20, n_l2=40, cont_spin=spin)
        o = coracle.Oracle(P)
        W, n = P.n_words, 64 * P.n_words + 1
        cnt = 0
        for D in P.groups[0].dets:
            for chi in P.l2_dets:
                out = o.excitation_tl2(D, chi)
                d = sum(bin(int(x) & ~int(y)).count("1") for x, y in zip(D, chi))
                assert out[0] == d + 1
                if d > 1:
                    continue
                cnt += 1
                # operator check in an orbital space of 64W+1 orbitals per spin
                # where orbital 64W is the continuum orbital
                def tup(words, extra):
                    occ = [s * n + 64 * w + b for s in (0, 1) for w in range(W) for b in range(64)
                           if (int(words[s * W + w]) >> b) & 1]
                    return tuple(sorted(occ + extra))
                I = tup(D, [spin * n + 64 * W])
                J = tup(chi, [])
                holes = sorted(set(J) - set(I)); parts = sorted(set(I) - set(J))
                d_ = J
                sign = 1
                for so in holes:
                    s, d_ = fock.annihilate(d_, so); sign *= s
                for so in reversed(parts):
                    s, d_ = fock.create(d_, so); sign *= s
                assert d_ == I
                assert out[4] == sign
                tgt_h = [(so // n) * 64 * W + so % n for so in holes]
                assert list(out[1:1 + len(holes)]) == tgt_h
        assert cnt > 0


@pytest.mark.parametrize("key", ["c1", "mid"])
def test_l2_block_is_symmetric(key):
    """Classes 2 and 8 (Section 2.2): the oracle evaluates every L2 x L2 entry
    from its own pair, and the block comes out symmetric, pattern exactly and
    values to rounding, with every diagonal entry present.  The GPU build
    evaluates the upper triangle and copies each lower entry from its mirror on
    the strength of this (nnz - n entries off the diagonal, half below it)."""
    import scipy.sparse as sp
    P = synth.make_config(key)
    rp, cols, vals = coracle.Oracle(P).l2_csr()
    n = P.n_l2
    for r in range(n):
        row = cols[rp[r]:rp[r + 1]]
        assert np.all(np.diff(row) > 0) and r in row
    assert (rp[-1] - n) % 2 == 0
    A = sp.csr_matrix((vals, cols, rp), shape=(n, n))
    S = sp.csr_matrix((np.ones_like(vals), cols, rp), shape=(n, n))
    assert (S != S.T).nnz == 0
    assert abs(A - A.T).max() <= 1e-14 * np.abs(vals).max()


def _target_hamiltonian(P, g):
    """H^N + e_core over group g's determinants, by the oracle's Slater-Condon
    evaluation of the L2-L2 elements (which takes any electron count)."""
    import copy
    Q = copy.copy(P)
    Q.l2_dets = P.groups[g].dets
    Q.groups = []
    return coracle.Oracle(Q).l2_rows(0, Q.n_l2)


@pytest.mark.parametrize("e_core", [0.0, -2.5])
def test_target_energy_substitution_identity(e_core):
    """Section 3.1: with CI vectors that are eigenvectors of H^N + e_core
    (numpy eigh) the target-only part of every continuum element is
    delta_nn' E_n, so the build with the target energies substituted equals the
    plain build, whatever the integrals touching the continuum."""
    P = synth.make_tiny(45, n_to=6, n_co=3, n_elec=4, n_det=14, n_state=3, n_l2=6, e_core=e_core)
    HN = _target_hamiltonian(P, 0)
    np.testing.assert_allclose(HN, HN.T, atol=1e-14)
    E, V = np.linalg.eigh(HN)
    P.groups[0].ci = np.ascontiguousarray(V[:, :3])
    R = coracle.Oracle(P).dense()
    P.groups[0].energy = E[:3].copy()
    Rs = coracle.Oracle(P).dense()
    np.testing.assert_allclose(Rs, R, rtol=0, atol=1e-12 * np.abs(R).max())
    # with other energies only the delta_jj' delta_nn' diagonal of the continuum block moves
    P.groups[0].energy = E[:3] + np.array([1.0, 2.0, 3.0])
    Rt = coracle.Oracle(P).dense()
    D = Rt - Rs
    nco = P.n_co
    expect = np.zeros_like(D)
    for n in range(3):
        for j in range(nco):
            expect[n * nco + j, n * nco + j] = n + 1.0
    np.testing.assert_allclose(D, expect, rtol=0, atol=1e-12 * np.abs(R).max())
