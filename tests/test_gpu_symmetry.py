"""Orbital symmetry (hb_problem.orb_irrep): the expansion panel keeps, for each
continuum pair, only the labels whose target pair has the pair's symmetry.

* Small symmetry-blocked Hamiltonians (D2h-like: 8 irreps, XOR product, as
  the batched workload) built with the symmetry against the oracle's dense
  matrix (which ignores it), on both paths, with the element criterion of
  tests/gpu_util.py.
* The same problems built without it: the FP64 path is bit-identical (the
  dropped labels are exact zeros in every sum, and the kept ones are summed in
  the same order); the mixed path agrees to within its rounding (only the
  chunking of the K sums changes).
* Inputs the symmetry cannot hold for are refused: a group whose continuum
  range spans two irreps, integrals that break the declared symmetry,
  irreps outside 0..7, and a shared context whose base has no symmetry."""
import copy

import numpy as np
import pytest

from oracle import coracle
from paper_1709_03005_gb300 import synth

from gpu_util import assert_blocks_close, gpu_dense

pytestmark = pytest.mark.gpu


def _family():
    return synth.make_batched_family(seed=9, n_hams=4, n_to=16, cont_per_irrep=(2, 5), n_elec=4, rank=12,
                                     dim_range=(40, 160), max_det=24, max_states=3)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1709_03005_gb300 import build_ext
    build_ext.build()


@pytest.mark.parametrize("precision", [0, 1])
def test_symmetric_panel_against_oracle(precision):
    for P in _family():
        assert P.orb_irrep is not None
        o = coracle.Oracle(P)
        R = o.dense()
        G, _, _ = gpu_dense(P, precision=precision)
        assert_blocks_close(G, R, o, 1e-10 if precision else 1e-12, P.name, mixed=precision == 1)
        Q = copy.copy(P)
        Q.orb_irrep = None
        G0, _, _ = gpu_dense(Q, precision=precision)
        if precision == 0:
            assert np.array_equal(G, G0), P.name
        else:
            S = o.condition()
            assert np.all(np.abs(G - G0) <= 1e-11 * np.maximum(S, 1e-300) + 1e-14 * np.abs(R).max()), P.name


def test_symmetry_inputs_checked():
    from paper_1709_03005_gb300 import hb
    P = _family()[1]
    # a continuum range across two irreps
    Q = copy.copy(P)
    Q.groups = [copy.copy(g) for g in P.groups]
    g = Q.groups[0]
    g.cont_count = g.cont_count + 1 if g.cont_first + g.cont_count < P.n_co else g.cont_count
    g.cont_first = max(0, g.cont_first - 1) if g.cont_first + g.cont_count > P.n_co else g.cont_first
    with pytest.raises(hb.HBError):
        hb.Hamiltonian(Q)
    # an integral of the continuum classes that breaks the symmetry
    Q = copy.copy(P)
    ttcc = P.eri_ttcc.copy()
    ir = np.asarray(P.orb_irrep)
    t_ir, c_ir = ir[:P.n_to], ir[P.n_to:]
    # pair (0, 0) of target irrep 0 against continuum orbitals of different irreps
    j = 0
    jp = int(np.nonzero(c_ir != c_ir[0])[0][0])
    ttcc[0, j * P.n_co + jp] = 1e-3
    ttcc[0, jp * P.n_co + j] = 1e-3
    Q.eri_ttcc = ttcc
    with pytest.raises(hb.HBError) as e:
        hb.Hamiltonian(Q)
    assert e.value.code == hb.HB_ERR_INVALID_ARG
    # irreps out of range
    Q = copy.copy(P)
    Q.orb_irrep = np.asarray(P.orb_irrep).copy()
    Q.orb_irrep[0] = 8
    with pytest.raises(hb.HBError):
        hb.Hamiltonian(Q)
    # a context sharing the integrals of a base without the symmetry
    B0 = copy.copy(P)
    B0.orb_irrep = None
    base = hb.Hamiltonian(B0)
    with pytest.raises(hb.HBError):
        hb.Hamiltonian(P, validate=False, base=base)
    base.close()
