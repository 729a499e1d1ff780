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
        for n in range(g.ci.shape[1]):
            for j in range(g.cont_first, g.cont_first + g.cont_count):
                col = {}
                for m in range(g.dets.shape[0]):
                    d = fock.words_to_tuple(g.dets[m], W, n_orb, extra=[(sc, P.n_to + j)])
                    col[add(d)] = col.get(add(d), 0.0) + g.ci[m, n]
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
