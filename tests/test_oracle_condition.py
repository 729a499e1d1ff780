"""Pins of the oracle's sampled-element path and of its condition scales.

The GPU parity tests of the continuum block at full size compare sampled
elements with `orc_cc_element` (Eq. 7 for one element after the Eq. 8
contraction), and every GPU parity test measures the errors of elements that
cancel against condition scales: sum_b |D^b X(I^b)| over the contracted
coefficients (`orc_cc_element_abs`, `cc_condition()`), the full scale
sum_b |X(I^b)| sum_{mm'} |c c C^b| over every term of Eq. 8 and Eq. 7
(`orc_cc_element_cond`, `cc_condition(full=True)`), and the class-4 and L2
scales.  These are separate code
paths from the dense build, so they are pinned here on their own:

* against the brute-force operator build resolved by integral
  (oracle/brute.symbolic_blocks, from oracle/fock.apply_hamiltonian_terms),
  which shares nothing with the C oracle's Slater-Condon case analysis,
  prototypes or placeholders;
* against the dense build at every continuum element of c1, mid and
  multi-group problems, within the rounding bound of two summation orders;
* by closed forms: a scale is at least the magnitude of its value, equals it
  where a single integral contributes (no two-electron integrals, identity CI),
  and is linear in the integrals (exactly so for a factor of 2).
"""
import numpy as np
import pytest

from oracle import brute, coracle
from paper_1709_03005_gb300 import synth

U = np.finfo(np.float64).eps / 2


def _gamma(k):
    """Higham's gamma_k = k u / (1 - k u): the relative bound of a k-term sum."""
    return k * U / (1 - k * U)


TINY = [
    ("one_group", dict(seed=301)),
    ("groups_overlap", dict(seed=302, n_groups=2, n_state=[2, 3], cont_ranges=[(0, 3), (1, 2)])),
    ("beta_three", dict(seed=303, n_groups=3, n_det=4, n_state=[1, 2, 2], cont_ranges=[(0, 2), (0, 3), (2, 1)],
                        cont_spin=1)),
    ("e_core", dict(seed=304, n_groups=2, n_det=5, n_state=[2, 2], cont_ranges=[(0, 3), (0, 3)], e_core=-7.25)),
    ("wide_W2", dict(seed=305, n_to=70, n_co=2, n_elec=4, n_det=5, n_state=2, n_l2=4, rank=3)),
]


def _cc_elements(o, P, fn):
    """fn(cc, n, j, n', j') over every continuum element, as a Dc x Dc matrix."""
    out = np.zeros((o.Dc, o.Dc))
    for g, G in enumerate(P.groups):
        for gp, Gp in enumerate(P.groups):
            cc = o.contract(g, gp) if gp <= g else None
            for n in range(G.ci.shape[1]):
                for jj in range(G.cont_count):
                    r = o.offsets[g] + n * G.cont_count + jj
                    for n_ in range(Gp.ci.shape[1]):
                        for jjp in range(Gp.cont_count):
                            c = o.offsets[gp] + n_ * Gp.cont_count + jjp
                            if cc is None:
                                continue
                            v = fn(cc, n, G.cont_first + jj, n_, Gp.cont_first + jjp)
                            out[r, c] = out[c, r] = v
    return out


@pytest.mark.parametrize("name,kw", TINY, ids=[t[0] for t in TINY])
def test_symbolic_brute_is_the_operator_matrix(name, kw):
    """The label-resolved operator build sums to the plain operator build."""
    kw = dict(kw)
    P = synth.make_tiny(kw.pop("seed"), **kw)
    V, S, F = brute.symbolic_blocks(P)
    Hb = brute.contracted_hamiltonian(P)
    np.testing.assert_allclose(V, Hb, rtol=0, atol=1e-13 * max(1.0, np.abs(Hb).max()))
    assert np.all(S >= np.abs(V) * (1 - 1e-13))
    assert np.all(F >= S * (1 - 1e-13))


@pytest.mark.parametrize("name,kw", TINY, ids=[t[0] for t in TINY])
def test_element_and_condition_against_brute(name, kw):
    """orc_cc_element at every continuum element equals the brute-force
    contracted matrix; the oracle's condition scales of all three classes
    (continuum, class 4, L2), with contracted coefficients and in full, equal
    the brute-force sums of term magnitudes."""
    kw = dict(kw)
    P = synth.make_tiny(kw.pop("seed"), **kw)
    o = coracle.Oracle(P)
    V, S, F = brute.symbolic_blocks(P)
    Dc = o.Dc
    E = _cc_elements(o, P, lambda cc, *a: cc.element(*a))
    Ea = _cc_elements(o, P, lambda cc, *a: cc.element_abs(*a))
    Ec = _cc_elements(o, P, lambda cc, *a: cc.element_cond(*a))
    scale = max(1.0, np.abs(V).max())
    np.testing.assert_allclose(E, V[:Dc, :Dc], rtol=0, atol=1e-13 * scale)
    np.testing.assert_allclose(Ea, S[:Dc, :Dc], rtol=1e-13, atol=1e-15 * scale)
    np.testing.assert_allclose(Ec, F[:Dc, :Dc], rtol=1e-13, atol=1e-15 * scale)
    np.testing.assert_allclose(o.condition(full=False), S, rtol=1e-13, atol=1e-15 * scale)
    Sc = o.condition()
    np.testing.assert_allclose(Sc, F, rtol=1e-13, atol=1e-15 * scale)
    # the dense scales of the continuum block are the element functions'
    np.testing.assert_array_equal(Sc[:Dc, :Dc], Ec)
    np.testing.assert_array_equal(o.cc_condition(), Ea)


@pytest.mark.parametrize("key,kw", [("c1", {}), ("mid", {}),
                                    ("mid", dict(n_co=9, n_det=40, n_l2=20, seed=77))])
def test_element_equals_dense(key, kw):
    """The sampled-element path (orc_cc_element) against the dense build at
    every continuum element, within the rounding bound of two orders of the
    same K-term sum: |a - b| <= 2 gamma_K sum|terms|."""
    P = synth.make_config(key, **kw)
    o = coracle.Oracle(P)
    R = o.dense()
    cond = o.cc_condition()
    cc = o.contract(0, 0)
    K = cc.nlabels(0) + cc.nlabels(1) + 1
    E = _cc_elements(o, P, lambda c, *a: c.element(*a))
    d = np.abs(E - R[: o.Dc, : o.Dc])
    assert np.all(d <= 2 * _gamma(K) * cond), (d / np.maximum(cond, 1e-300)).max()
    # a scale bounds the magnitude of its value
    assert np.all(cond >= np.abs(R[: o.Dc, : o.Dc]) * (1 - 2 * _gamma(K)))


def test_multigroup_element_equals_dense():
    P = synth.make_tiny(311, n_to=6, n_co=5, n_elec=4, n_det=6, n_groups=3, n_state=[2, 3, 1],
                        cont_ranges=[(0, 5), (1, 3), (2, 2)], n_l2=0)
    o = coracle.Oracle(P)
    R = o.dense()
    E = _cc_elements(o, P, lambda c, *a: c.element(*a))
    cond = o.cc_condition()
    assert np.all(np.abs(E - R) <= 2 * _gamma(400) * cond)


def test_single_label_elements_have_condition_equal_to_value():
    """No two-electron integrals and identity CI vectors: every element with
    j != j' holds the single label h_jj' (delta_mm'), every element between
    different target determinants with j == j' the single label h_kl of the
    target excitation, every class-4 element of a single excitation a single h
    label; there the scale is exactly |value|."""
    P = synth.make_tiny(321, n_to=5, n_co=3, n_elec=4, n_det=6, n_state=2, n_l2=6)
    for a in ("eri_tttt", "eri_tttc", "eri_ttcc", "eri_tctc"):
        setattr(P, a, np.zeros_like(getattr(P, a)))
    P.chol = np.zeros_like(P.chol)
    g = P.groups[0]
    g.ci = np.eye(g.dets.shape[0])
    o = coracle.Oracle(P)
    R = o.dense()
    S = o.condition()
    nco = P.n_co
    Dc = o.Dc
    nd = g.dets.shape[0]
    checked = 0
    for m in range(nd):
        for mp in range(nd):
            for j in range(nco):
                for jp in range(nco):
                    if j == jp and m == mp:
                        continue
                    r, c = m * nco + j, mp * nco + jp
                    assert S[r, c] == abs(R[r, c]), (m, mp, j, jp)
                    checked += R[r, c] != 0.0
    assert checked > 0
    # with identity CI vectors the contraction adds single terms, so the full
    # scale is the contracted one; class 4 against the brute-force scales
    np.testing.assert_array_equal(o.condition(full=False)[:Dc, :Dc], S[:Dc, :Dc])
    V, Sb, F = brute.symbolic_blocks(P)
    np.testing.assert_allclose(S[Dc:, :Dc], Sb[Dc:, :Dc], rtol=1e-14, atol=0)


@pytest.mark.parametrize("factor", [2.0, 3.0])
def test_condition_is_linear_in_the_integrals(factor):
    """Scaling h, every ERI and e_core by f scales every element and every
    condition scale by f (exactly for f = 2, a change of exponent only)."""
    P = synth.make_tiny(331, n_groups=2, n_state=[2, 2], cont_ranges=[(0, 3), (1, 2)], e_core=1.5)
    o = coracle.Oracle(P)
    R, S = o.dense(), o.condition()
    Q = synth.make_tiny(331, n_groups=2, n_state=[2, 2], cont_ranges=[(0, 3), (1, 2)], e_core=1.5)
    Q.h = Q.h * factor
    for a in ("eri_tttt", "eri_tttc", "eri_ttcc", "eri_tctc"):
        setattr(Q, a, getattr(Q, a) * factor)
    Q.e_core *= factor
    oq = coracle.Oracle(Q)
    Rq, Sq = oq.dense(), oq.condition()
    if factor == 2.0:
        np.testing.assert_array_equal(Rq, factor * R)
        np.testing.assert_array_equal(Sq, factor * S)
    else:
        np.testing.assert_allclose(Rq, factor * R, rtol=0, atol=1e-14 * np.abs(R).max() * factor)
        np.testing.assert_allclose(Sq, factor * S, rtol=1e-14, atol=0)
