"""Brute-force contracted Hamiltonian: build every uncontracted (N+1)-electron
determinant, evaluate H on it by the operator definition, then contract.

ORACLE / TEST INFRASTRUCTURE ONLY.

This is the plain definition the structured algorithm reaches exactly (up to
rounding order):

* basis (Eq. 1): target-times-continuum functions A phi_in u_ij and L2
  functions chi_l;
* target states (Eq. 2): phi_in = sum_m c_imn eta_im (here eta are determinants);
* uncontracted elements (Eq. 3) <eta_im u_ij | H | eta_i'm' u_i'j'> between the
  (N+1)-electron determinants |D_m + {j, continuum spin}>;
* contraction (Eq. 4 and Eq. 5): H~ = T^T H T with
  T = blockdiag_g(C_g (x) I_{n_co(g)}, I_{n_L2}).

Phase convention (the paper's "phase mask" issue, Section 3.1): the
target-times-continuum function is *defined* as the canonically ordered
(N+1)-electron determinant built from D_m plus the continuum spin orbital,
summed with the CI coefficients.  Continuum spin orbitals sit above every target
orbital of the same spin, so this sign convention is the same for every j.

Basis order of the result: for each group g, for each state n, for each
continuum orbital j of the group (n-major), then the L2 functions.
"""
from __future__ import annotations

import numpy as np

from . import fock


def det_ci(group) -> np.ndarray:
    """CI vectors of a target group over its determinants: ci itself, or, for a
    group given over configuration state functions, C_det[d, n] =
    sum_i csf_coef(i, d) ci[i, n] (one more contraction level)."""
    if getattr(group, "csf_ptr", None) is None:
        return np.asarray(group.ci, np.float64)
    ptr, det, coef = group.csf_ptr, group.csf_det, group.csf_coef
    B = np.zeros((len(ptr) - 1, group.dets.shape[0]))
    for i in range(len(ptr) - 1):
        for k in range(ptr[i], ptr[i + 1]):
            B[i, det[k]] += coef[k]
    return B.T @ np.asarray(group.ci, np.float64)


def uncontracted(problem):
    """(list of determinant tuples, T matrix) for a synth.Problem."""
    P = problem
    n_orb, W, sc = P.n_orb, P.n_words, P.cont_spin
    dets, index = [], {}

    def add(d):
        if d not in index:
            index[d] = len(dets)
            dets.append(d)
        return index[d]

    cols = []
    for g in P.groups:
        ci = det_ci(g)
        for n in range(ci.shape[1]):
            for j in range(g.cont_first, g.cont_first + g.cont_count):
                col = {}
                for m in range(g.dets.shape[0]):
                    d = fock.words_to_tuple(g.dets[m], W, n_orb, extra=[(sc, P.n_to + j)])
                    col[add(d)] = col.get(add(d), 0.0) + ci[m, n]
                cols.append(col)
    for l in range(P.n_l2):
        d = fock.words_to_tuple(P.l2_dets[l], W, n_orb)
        cols.append({add(d): 1.0})
    T = np.zeros((len(dets), len(cols)))
    for c, col in enumerate(cols):
        for r, v in col.items():
            T[r, c] += v
    return dets, T


def contracted_hamiltonian(problem, return_parts=False):
    P = problem
    eri = P.full_eri()
    dets, T = uncontracted(P)
    H = fock.hamiltonian_matrix(dets, P.h, eri, P.n_orb, P.e_core)
    Ht = T.T @ H @ T
    if return_parts:
        return Ht, H, T, dets
    return Ht


def _is_target_only(label, n_to):
    """Labels with no continuum index (and the constant e_core)."""
    return label[0] == "core" or all(i < n_to for i in label[1:])


def symbolic_blocks(problem):
    """Values and condition scales of every element of the contracted matrix,
    from the operator definition resolved by integral (fock.apply_hamiltonian_terms).

    For a continuum-continuum element (Eq. 7 after Eq. 8) the symbolic
    coefficient of label b is D^b = sum_{m m'} c_mn c_m'n' C^b(m j, m' j');
    the value is sum_b D^b X(b) and the condition scale is
        |sum_{b without continuum index} D^b X(b)| + sum_{other b} |D^b X(b)|
    (the labels without a continuum index, and e_core, form one term because a
    prototype holds them as one number that does not depend on j), and its full
    scale, every term of the contraction included, is
        sum_b |X(b)| sum_{m m'} |c_mn c_m'n' C^b(m j, m' j')|.
    For a class-4 element (Eq. 5) both scales are
    sum_m sum_b |c_mn C^b(m j, l) X(b)|, for an L2-L2 element sum_b |C^b X(b)|:
    the sums of the magnitudes of the terms any evaluation order adds.
    Returns (value, scale, full scale), each dim x dim.  Tiny problems only."""
    P = problem
    n_orb, W, sc, nt = P.n_orb, P.n_words, P.cont_spin, P.n_to
    eri = P.full_eri()

    def X(label):
        return fock.label_value(label, P.h, eri, P.e_core)

    rows = []          # (kind, payload) per basis function in the contracted order
    for gi, g in enumerate(P.groups):
        for n in range(g.ci.shape[1]):
            for jj in range(g.cont_count):
                rows.append(("c", gi, n, g.cont_first + jj))
    for l in range(P.n_l2):
        rows.append(("l", l))
    dim = len(rows)

    def det_cj(g, m, j):
        return fock.words_to_tuple(g.dets[m], W, n_orb, extra=[(sc, nt + j)])

    terms = {}

    def terms_of(ket):
        if ket not in terms:
            terms[ket] = fock.apply_hamiltonian_terms(ket, n_orb, P.e_core)
        return terms[ket]

    V = np.zeros((dim, dim))
    S = np.zeros((dim, dim))
    F = np.zeros((dim, dim))
    for a, ra in enumerate(rows):
        for b, rb in enumerate(rows):
            if ra[0] == "c" and rb[0] == "c":
                g, gp = P.groups[ra[1]], P.groups[rb[1]]
                cg, cgp = det_ci(g), det_ci(gp)
                n, j, n_, jp = ra[2], ra[3], rb[2], rb[3]
                D = {}
                f = 0.0
                for mp in range(gp.dets.shape[0]):
                    tk = terms_of(det_cj(gp, mp, jp))
                    for m in range(g.dets.shape[0]):
                        for lab, c in tk.get(det_cj(g, m, j), {}).items():
                            D[lab] = D.get(lab, 0.0) + cg[m, n] * cgp[mp, n_] * c
                            f += abs(cg[m, n] * cgp[mp, n_] * c * X(lab))
                F[a, b] = f
                tgt = sum(d * X(lab) for lab, d in D.items() if _is_target_only(lab, nt))
                oth = [d * X(lab) for lab, d in D.items() if not _is_target_only(lab, nt)]
                V[a, b] = tgt + sum(oth)
                S[a, b] = abs(tgt) + sum(abs(x) for x in oth)
            elif ra[0] == "l" and rb[0] == "l":
                tk = terms_of(fock.words_to_tuple(P.l2_dets[rb[1]], W, n_orb))
                t = tk.get(fock.words_to_tuple(P.l2_dets[ra[1]], W, n_orb), {})
                V[a, b] = sum(c * X(lab) for lab, c in t.items())
                S[a, b] = F[a, b] = sum(abs(c * X(lab)) for lab, c in t.items())
            else:
                (cr, lr) = (ra, rb) if ra[0] == "c" else (rb, ra)
                g, n, j = P.groups[cr[1]], cr[2], cr[3]
                cg = det_ci(g)
                tk = terms_of(fock.words_to_tuple(P.l2_dets[lr[1]], W, n_orb))
                v = s = 0.0
                for m in range(g.dets.shape[0]):
                    for lab, c in tk.get(det_cj(g, m, j), {}).items():
                        x = cg[m, n] * c * X(lab)
                        v += x
                        s += abs(x)
                V[a, b], S[a, b], F[a, b] = v, s, s
    return V, S, F
