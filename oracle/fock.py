"""Second-quantised electronic Hamiltonian applied term by term (tiny systems).

ORACLE / TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this.

This is the plain definition that every matrix element in the close-coupling
Hamiltonian (Eq. 3, the uncontracted elements <eta u|H|eta' u'>) rests on:

    H = sum_{pq,s} h_pq a+_{p s} a_{q s}
        + 1/2 sum_{pqrs} sum_{s,t} (pq|rs) a+_{p s} a+_{r t} a_{s t} a_{q s}

with chemists'-notation integrals over real orthonormal spin orbitals (Section 2 of
the paper: "an orthogonal set of spin-orbitals").  No Slater-Condon rule is
used: each creation/annihilation operator is applied to an ordered occupation
tuple and the sign is the parity of the number of occupied spin orbitals it
passes.  Because it is independent of any case analysis (diagonal / single /
double), it pins the bitstring Slater-Condon rules of Section 2.1.

Spin-orbital index:  so = spin * n_orb + p  (all alpha orbitals first, then all
beta; within a spin, ascending spatial index).  A determinant is the sorted tuple
of its occupied spin orbitals, i.e. a+_{so_1} a+_{so_2} ... |0> with
so_1 < so_2 < ...
"""
from __future__ import annotations

import bisect
from collections import defaultdict

import numpy as np


def annihilate(det: tuple, so: int):
    """a_so |det> -> (sign, det') or (0, None)."""
    i = bisect.bisect_left(det, so)
    if i == len(det) or det[i] != so:
        return 0, None
    return (-1) ** i, det[:i] + det[i + 1:]


def create(det: tuple, so: int):
    """a+_so |det> -> (sign, det') or (0, None)."""
    i = bisect.bisect_left(det, so)
    if i < len(det) and det[i] == so:
        return 0, None
    return (-1) ** i, det[:i] + (so,) + det[i:]


def apply_hamiltonian(det: tuple, h: np.ndarray, eri: np.ndarray, n_orb: int,
                      e_core: float = 0.0) -> dict:
    """H|det> as {det': coefficient}."""
    out = defaultdict(float)
    if e_core:
        out[det] += e_core
    # one-electron part
    for Q in det:
        s, q = divmod(Q, n_orb)
        sq, d1 = annihilate(det, Q)
        for p in range(n_orb):
            sp, d2 = create(d1, s * n_orb + p)
            if sp:
                out[d2] += sq * sp * h[p, q]
    # two-electron part: 1/2 (pq|rs) a+_{p s} a+_{r t} a_{s t} a_{q s}
    for Q in det:
        s, q = divmod(Q, n_orb)
        sq, d1 = annihilate(det, Q)
        for S in d1:
            t, ss = divmod(S, n_orb)
            s_s, d2 = annihilate(d1, S)
            for r in range(n_orb):
                sr, d3 = create(d2, t * n_orb + r)
                if not sr:
                    continue
                for p in range(n_orb):
                    sp, d4 = create(d3, s * n_orb + p)
                    if not sp:
                        continue
                    v = eri[p, q, r, ss]
                    if v != 0.0:
                        out[d4] += 0.5 * sq * s_s * sr * sp * v
    return out


def hamiltonian_matrix(dets, h, eri, n_orb, e_core=0.0) -> np.ndarray:
    """<D_i|H|D_j> over a list of determinants (sorted spin-orbital tuples)."""
    index = {d: i for i, d in enumerate(dets)}
    if len(index) != len(dets):
        raise ValueError("duplicate determinants")
    H = np.zeros((len(dets), len(dets)))
    for j, d in enumerate(dets):
        for d2, c in apply_hamiltonian(d, h, eri, n_orb, e_core).items():
            i = index.get(d2)
            if i is not None:
                H[i, j] += c
    return H


def words_to_tuple(words, W: int, n_orb: int, extra=()) -> tuple:
    """Target bitstring (alpha words, beta words) -> sorted spin-orbital tuple.

    `extra` adds further spin orbitals given as (spin, spatial index) pairs,
    e.g. the continuum electron.
    """
    occ = []
    for spin in (0, 1):
        for w in range(W):
            x = int(words[spin * W + w])
            b = 0
            while x:
                if x & 1:
                    occ.append(spin * n_orb + 64 * w + b)
                x >>= 1
                b += 1
    for spin, p in extra:
        occ.append(spin * n_orb + p)
    occ = sorted(occ)
    if len(set(occ)) != len(occ):
        raise ValueError("doubly occupied spin orbital")
    return tuple(occ)


def canonical_label(p: int, q: int, r: int | None = None, s: int | None = None) -> tuple:
    """Canonical name of an integral under its permutational symmetry.

    One-electron h_pq (real, symmetric): ('h', max, min).  Two-electron (pq|rs)
    (real orbitals, 8-fold symmetric): ('g', P, Q) with P = (max(p,q), min(p,q)),
    Q likewise for (r, s), and P >= Q.  Two index tuples name the same integral
    exactly when their canonical labels are equal."""
    if r is None:
        return ("h", max(p, q), min(p, q))
    a, b = (max(p, q), min(p, q)), (max(r, s), min(r, s))
    return ("g",) + (a + b if a >= b else b + a)


def apply_hamiltonian_terms(det: tuple, n_orb: int, e_core: float = 0.0) -> dict:
    """H|det> resolved by integral: {det': {label: coefficient}}.

    The same operator walk as apply_hamiltonian, but every contribution is
    filed under the canonical label of the integral it multiplies (the
    constant e_core under ('core',)), so <det'|H|det> = sum over labels of
    coefficient * integral.  This is the symbolic form of a matrix element
    (the paper's Eq. 6, C^a X(I^a)) reached by the definition of the
    operators, with no Slater-Condon case analysis."""
    out = defaultdict(lambda: defaultdict(float))
    if e_core:
        out[det][("core",)] += 1.0
    for Q in det:
        s, q = divmod(Q, n_orb)
        sq, d1 = annihilate(det, Q)
        for p in range(n_orb):
            sp, d2 = create(d1, s * n_orb + p)
            if sp:
                out[d2][canonical_label(p, q)] += sq * sp
    for Q in det:
        s, q = divmod(Q, n_orb)
        sq, d1 = annihilate(det, Q)
        for S in d1:
            t, ss = divmod(S, n_orb)
            s_s, d2 = annihilate(d1, S)
            for r in range(n_orb):
                sr, d3 = create(d2, t * n_orb + r)
                if not sr:
                    continue
                for p in range(n_orb):
                    sp, d4 = create(d3, s * n_orb + p)
                    if sp:
                        out[d4][canonical_label(p, q, r, ss)] += 0.5 * sq * s_s * sr * sp
    return out


def label_value(label: tuple, h: np.ndarray, eri: np.ndarray, e_core: float = 0.0) -> float:
    """The integral a canonical label names."""
    if label[0] == "core":
        return e_core
    if label[0] == "h":
        return h[label[1], label[2]]
    return eri[label[1], label[2], label[3], label[4]]


def apply_s2(det: tuple, n_orb: int) -> dict:
    """S^2 |det> as {det': coefficient}, by S^2 = S- S+ + Sz (Sz + 1) with
    S+ = sum_p a+_{p alpha} a_{p beta} (spin orbital s * n_orb + p)."""
    out = defaultdict(float)
    na = sum(1 for so in det if so < n_orb)
    sz = 0.5 * (na - (len(det) - na))
    out[det] += sz * (sz + 1.0)
    for p in range(n_orb):
        s1, d1 = annihilate(det, n_orb + p)
        if not s1:
            continue
        s2, d2 = create(d1, p)
        if not s2:
            continue
        for q in range(n_orb):
            s3, d3 = annihilate(d2, q)
            if not s3:
                continue
            s4, d4 = create(d3, n_orb + q)
            if s4:
                out[d4] += s1 * s2 * s3 * s4
    return out
