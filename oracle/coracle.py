"""ctypes front end of the C oracle (hb_oracle.c).

ORACLE / TEST INFRASTRUCTURE ONLY.

`build()` compiles hb_oracle.c with plain gcc (-O2, OpenMP) into
oracle/_build/libhb_oracle.so; `load()` builds it on first use.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hb_oracle.c")
_OUT = os.path.join(_HERE, "_build", "libhb_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".tmp{os.getpid()}"
        # no contraction of a*b + c into fused multiply-adds: with the fixed
        # summation order the results are then the same bits on every host
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


class _Problem(C.Structure):
    _fields_ = [("n_to", C.c_int32), ("n_co", C.c_int32), ("n_elec", C.c_int32),
                ("W", C.c_int32), ("cont_spin", C.c_int32),
                ("h", C.c_void_p), ("tttt", C.c_void_p), ("tttc", C.c_void_p),
                ("ttcc", C.c_void_p), ("tctc", C.c_void_p),
                ("n_groups", C.c_int32),
                ("g_ndet", C.c_void_p), ("g_nstate", C.c_void_p),
                ("g_cfirst", C.c_void_p), ("g_ccount", C.c_void_p),
                ("g_dets", C.c_void_p), ("g_ci", C.c_void_p),
                ("n_l2", C.c_int32), ("l2", C.c_void_p), ("e_core", C.c_double),
                ("g_energy", C.c_void_p)]


def load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
        lib.orc_hij.restype = dbl
        lib.orc_hij.argtypes = [vp, vp, vp]
        lib.orc_excitation_api.restype = C.c_int
        lib.orc_excitation_api.argtypes = [C.c_int, vp, vp, vp]
        lib.orc_excitation_tl2.restype = C.c_int
        lib.orc_excitation_tl2.argtypes = [vp, vp, vp, vp]
        lib.orc_cc_contract.restype = vp
        lib.orc_cc_contract.argtypes = [vp, C.c_int, C.c_int]
        lib.orc_cc_contract_ex.restype = vp
        lib.orc_cc_contract_ex.argtypes = [vp, C.c_int, C.c_int, C.c_int]
        lib.orc_cc_free.argtypes = [vp]
        lib.orc_cc_nlabels.restype = i64
        lib.orc_cc_nlabels.argtypes = [vp, C.c_int]
        lib.orc_cc_element.restype = dbl
        lib.orc_cc_element.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int]
        lib.orc_cc_expand.argtypes = [vp, vp, i64, i64, i64]
        lib.orc_class4_row.argtypes = [vp, C.c_int, vp]
        lib.orc_l2_element.restype = dbl
        lib.orc_l2_element.argtypes = [vp, C.c_int, C.c_int]
        lib.orc_contracted_dim.restype = i64
        lib.orc_contracted_dim.argtypes = [vp]
        lib.orc_build_dense.argtypes = [vp, vp]
        lib.orc_l2_csr.argtypes = [vp, vp, vp, vp]
        lib.orc_l2_rows.argtypes = [vp, C.c_int, C.c_int, vp]
        lib.orc_cc_element_abs.restype = dbl
        lib.orc_cc_element_abs.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int]
        lib.orc_cc_expand_abs.argtypes = [vp, vp, i64, i64, i64]
        lib.orc_cc_element_cond.restype = dbl
        lib.orc_cc_element_cond.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int]
        lib.orc_cc_expand_cond.argtypes = [vp, vp, i64, i64, i64]
        lib.orc_cc_expand_rows.argtypes = [vp, vp, C.c_int, C.c_int]
        lib.orc_class4_rows.argtypes = [vp, C.c_int, C.c_int, vp]
        lib.orc_class4_rows_abs.argtypes = [vp, C.c_int, C.c_int, vp]
        lib.orc_l2_rows_abs.argtypes = [vp, C.c_int, C.c_int, vp]
        lib.orc_l2_element_abs.restype = dbl
        lib.orc_l2_element_abs.argtypes = [vp, C.c_int, C.c_int]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _det_ci(group) -> np.ndarray:
    """The group's CI vectors over its determinants (CSF groups expanded)."""
    from .brute import det_ci
    return det_ci(group)


class Oracle:
    """Holds a synth.Problem in the C oracle's layout (keeps arrays alive)."""

    def __init__(self, problem):
        self.lib = load()
        P = problem
        self.problem = P
        keep = []

        def arr(x, dt):
            a = np.ascontiguousarray(x, dtype=dt)
            keep.append(a)
            return a

        gs = P.groups
        self.g_ndet = arr([g.dets.shape[0] for g in gs], np.int32)
        self.g_nstate = arr([g.ci.shape[1] for g in gs], np.int32)
        self.g_cfirst = arr([g.cont_first for g in gs], np.int32)
        self.g_ccount = arr([g.cont_count for g in gs], np.int32)
        dets = [arr(g.dets, np.uint64) for g in gs]
        cis = [arr(_det_ci(g), np.float64) for g in gs]
        self.g_dets = arr([_ptr(d) for d in dets], np.uint64)
        self.g_ci = arr([_ptr(c) for c in cis], np.uint64)
        h = arr(P.h, np.float64)
        t4 = arr(P.eri_tttt, np.float64)
        t3 = arr(P.eri_tttc, np.float64)
        t2 = arr(P.eri_ttcc, np.float64)
        tc = arr(P.eri_tctc, np.float64)
        l2 = arr(P.l2_dets, np.uint64) if P.n_l2 else arr(np.zeros((1, 2 * P.n_words)), np.uint64)
        ens = [getattr(g, "energy", None) for g in gs]
        if any(e is not None for e in ens):
            if any(e is None for e in ens):
                raise ValueError("target energies must be given for every group or for none")
            ens = [arr(e, np.float64) for e in ens]
            g_energy = _ptr(arr([_ptr(e) for e in ens], np.uint64))
        else:
            g_energy = None
        self._keep = keep
        self.s = _Problem(P.n_to, P.n_co, P.n_elec, P.n_words, P.cont_spin,
                          _ptr(h), _ptr(t4), _ptr(t3), _ptr(t2), _ptr(tc),
                          len(gs), _ptr(self.g_ndet), _ptr(self.g_nstate),
                          _ptr(self.g_cfirst), _ptr(self.g_ccount),
                          _ptr(self.g_dets), _ptr(self.g_ci),
                          P.n_l2, _ptr(l2), float(P.e_core), g_energy)
        self.sp = C.addressof(self.s)
        self.offsets = np.concatenate([[0], np.cumsum(self.g_nstate.astype(np.int64) *
                                                      self.g_ccount.astype(np.int64))])
        self.Dc = int(self.offsets[-1])
        self.dim = self.Dc + P.n_l2

    # -- Slater-Condon --------------------------------------------------------
    def hij(self, I: np.ndarray, J: np.ndarray) -> float:
        I = np.ascontiguousarray(I, np.uint64); J = np.ascontiguousarray(J, np.uint64)
        return self.lib.orc_hij(self.sp, _ptr(I), _ptr(J))

    @staticmethod
    def excitation(W, I, J):
        lib = load()
        I = np.ascontiguousarray(I, np.uint64); J = np.ascontiguousarray(J, np.uint64)
        out = np.zeros(6, np.int32)
        lib.orc_excitation_api(W, _ptr(I), _ptr(J), _ptr(out))
        return out

    def excitation_tl2(self, D, chi):
        D = np.ascontiguousarray(D, np.uint64); chi = np.ascontiguousarray(chi, np.uint64)
        out = np.zeros(5, np.int32)
        self.lib.orc_excitation_tl2(self.sp, _ptr(D), _ptr(chi), _ptr(out))
        return out

    # -- structured build -----------------------------------------------------
    def dense(self) -> np.ndarray:
        H = np.zeros((self.dim, self.dim))
        self.lib.orc_build_dense(self.sp, _ptr(H))
        return H

    def contract(self, g, gp, cond=True):
        """Eq. 8 for the group pair (g, gp); cond=False skips the magnitude
        sums that element_cond needs."""
        return _CC(self, g, gp, cond)

    def class4_row(self, l) -> np.ndarray:
        out = np.zeros(max(self.Dc, 1))
        self.lib.orc_class4_row(self.sp, int(l), _ptr(out))
        return out[: self.Dc]

    def l2_element(self, a, b) -> float:
        return self.lib.orc_l2_element(self.sp, int(a), int(b))

    def l2_rows(self, a0, a1) -> np.ndarray:
        out = np.zeros((max(a1 - a0, 1), max(self.problem.n_l2, 1)))
        self.lib.orc_l2_rows(self.sp, int(a0), int(a1), _ptr(out))
        return out[: a1 - a0, : self.problem.n_l2]

    def class4_rows(self, l0, l1) -> np.ndarray:
        out = np.zeros((max(l1 - l0, 1), max(self.Dc, 1)))
        self.lib.orc_class4_rows(self.sp, int(l0), int(l1), _ptr(out))
        return out[: l1 - l0, : self.Dc]

    def class4_rows_abs(self, l0, l1) -> np.ndarray:
        """Condition scales of the class-4 rows [l0, l1): sum of the magnitudes
        of the Eq. 5 terms of every element."""
        out = np.zeros((max(l1 - l0, 1), max(self.Dc, 1)))
        self.lib.orc_class4_rows_abs(self.sp, int(l0), int(l1), _ptr(out))
        return out[: l1 - l0, : self.Dc]

    def l2_rows_abs(self, a0, a1) -> np.ndarray:
        """Condition scales of the L2 x L2 rows [a0, a1)."""
        out = np.zeros((max(a1 - a0, 1), max(self.problem.n_l2, 1)))
        self.lib.orc_l2_rows_abs(self.sp, int(a0), int(a1), _ptr(out))
        return out[: a1 - a0, : self.problem.n_l2]

    def condition(self, full=True) -> np.ndarray:
        """dim x dim condition scales of every element, symmetric: the sums of
        the magnitudes of the terms of each element (continuum block from
        cc_condition(full), class 4 and L2 rows from their own sums)."""
        S = np.zeros((self.dim, self.dim))
        Dc = self.Dc
        S[:Dc, :Dc] = self.cc_condition(full)
        if self.problem.n_l2:
            c4 = self.class4_rows_abs(0, self.problem.n_l2)
            S[Dc:, :Dc] = c4
            S[:Dc, Dc:] = c4.T
            S[Dc:, Dc:] = self.l2_rows_abs(0, self.problem.n_l2)
        return S

    def cc_condition(self, full=False) -> np.ndarray:
        """Dc x Dc matrix of sum_b |D^b X(I^b)| for every continuum element
        (full=True: sum_b |X(I^b)| sum_{m m'} |c c C^b|, the contraction's
        terms included)."""
        H = np.zeros((self.Dc, self.Dc))
        fn = self.lib.orc_cc_expand_cond if full else self.lib.orc_cc_expand_abs
        for g in range(len(self.problem.groups)):
            for gp in range(g + 1):
                cc = self.lib.orc_cc_contract(self.sp, g, gp)
                fn(cc, _ptr(H), self.Dc, int(self.offsets[g]), int(self.offsets[gp]))
                self.lib.orc_cc_free(cc)
        return H

    def cc_block(self, g, gp) -> np.ndarray:
        """Contract and expand one group-pair block (Eq. 8 then Eq. 7)."""
        rows = int(self.g_nstate[g] * self.g_ccount[g])
        cols = int(self.g_nstate[gp] * self.g_ccount[gp])
        n = rows + cols
        H = np.zeros((n, n))
        cc = self.lib.orc_cc_contract(self.sp, int(g), int(gp))
        self.lib.orc_cc_expand(cc, _ptr(H), n, 0, rows if g != gp else 0)
        self.lib.orc_cc_free(cc)
        return H[:rows, rows:] if g != gp else H[:rows, :rows]

    def l2_csr(self):
        nl = self.problem.n_l2
        rp = np.zeros(nl + 1, np.int64)
        self.lib.orc_l2_csr(self.sp, _ptr(rp), None, None)
        cols = np.zeros(max(int(rp[-1]), 1), np.int32)
        vals = np.zeros(max(int(rp[-1]), 1), np.float64)
        self.lib.orc_l2_csr(self.sp, _ptr(rp), _ptr(cols), _ptr(vals))
        return rp, cols[: rp[-1]], vals[: rp[-1]]


class _CC:
    def __init__(self, orc: Oracle, g, gp, cond=True):
        self.orc, self.g, self.gp = orc, g, gp
        self.h = orc.lib.orc_cc_contract_ex(orc.sp, g, gp, 1 if cond else 0)

    def element(self, n, j, np_, jp) -> float:
        """Continuum indices j, jp are 0-based within the continuum."""
        return self.orc.lib.orc_cc_element(self.h, n, j, np_, jp)

    def element_abs(self, n, j, np_, jp) -> float:
        """sum_b |D^b X(I^b)| (contracted coefficients)."""
        return self.orc.lib.orc_cc_element_abs(self.h, n, j, np_, jp)

    def element_cond(self, n, j, np_, jp) -> float:
        """sum_b |X(I^b)| sum_{m m'} |c_mn c_m'n' C^b| (every term of Eq. 8 and Eq. 7)."""
        return self.orc.lib.orc_cc_element_cond(self.h, n, j, np_, jp)

    def expand_rows(self, jj0, jj1):
        """Elements [(jj, jj', n, n')] for rows jj0 <= jj < jj1 of this block."""
        P = self.orc.problem
        cnp = P.groups[self.gp].cont_count
        ns, nsp = P.groups[self.g].ci.shape[1], P.groups[self.gp].ci.shape[1]
        out = np.zeros((jj1 - jj0, cnp, ns, nsp))
        self.orc.lib.orc_cc_expand_rows(self.h, _ptr(out), int(jj0), int(jj1))
        return out

    def nlabels(self, which=0):
        return self.orc.lib.orc_cc_nlabels(self.h, which)

    def __del__(self):
        if getattr(self, "h", None):
            self.orc.lib.orc_cc_free(self.h)
            self.h = None
