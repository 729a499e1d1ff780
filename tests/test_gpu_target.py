"""Target states from the library's own solve and the target-energy
substitution of Section 3.1, on the GPU through the C ABI.

hb_target_diag builds the N-electron target Hamiltonian H^N + e_core over a
group's determinants with the L2-L2 Slater-Condon kernels and solves it with
the block Davidson of hb_diag; its energies and CI vectors are checked
against numpy's eigh of the oracle's H^N.  Builds that substitute those
energies for the target-only integrals are checked against the oracle's
substituted build (element criterion of tests/gpu_util.py), and against the
plain build, which they equal to the accuracy of the eigenvectors."""
import copy

import numpy as np
import pytest

from oracle import coracle
from paper_1709_03005_gb300 import synth

from gpu_util import assert_blocks_close, gpu_dense

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1709_03005_gb300 import build_ext
    build_ext.build()


def _target_hamiltonian(P, g):
    Q = copy.copy(P)
    Q.l2_dets = P.groups[g].dets
    Q.groups = []
    return coracle.Oracle(Q).l2_rows(0, Q.n_l2)


CASES = [
    ("tiny", lambda: synth.make_tiny(46, n_to=6, n_co=3, n_elec=4, n_det=14, n_state=3, n_l2=6, e_core=-1.25), 0, 3),
    ("tiny_beta_two_groups", lambda: synth.make_tiny(47, n_to=7, n_co=4, n_elec=4, n_det=12, n_groups=2,
                                                     n_state=[2, 3], cont_ranges=[(0, 4), (1, 3)], cont_spin=1), 1, 3),
    ("mid", lambda: synth.make_config("mid"), 0, 7),
    ("c2", lambda: synth.make_config("c2"), 0, 20),
]


@pytest.mark.parametrize("name,make,g,k", CASES, ids=[c[0] for c in CASES])
def test_target_diag_against_eigh(name, make, g, k):
    from paper_1709_03005_gb300 import hb
    P = make()
    E, C, st = hb.target_diag(P, g, k, tol=1e-10)
    HN = _target_hamiltonian(P, g)
    w, V = np.linalg.eigh(HN)
    np.testing.assert_allclose(E, w[:k], rtol=0, atol=1e-9 * max(1.0, np.abs(w).max()))
    R = HN @ C - C * E
    assert np.linalg.norm(R, axis=0).max() <= 1e-9, np.linalg.norm(R, axis=0).max()
    np.testing.assert_allclose(C.T @ C, np.eye(k), atol=1e-12)
    # each column's largest-magnitude entry is positive
    assert np.all(C[np.argmax(np.abs(C), axis=0), np.arange(k)] > 0)
    print(f"{name}: {k} target states of {C.shape[0]} determinants in {st.iterations} iterations, "
          f"max residual {st.max_residual:.2e}")


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name,make,g,k", CASES[:3], ids=[c[0] for c in CASES[:3]])
def test_substituted_build(name, make, g, k, precision):
    """Every group's CI vectors and energies from hb_target_diag, then the
    build with the energies substituted: against the oracle's substituted
    build, and against the plain build of the same CI vectors."""
    from paper_1709_03005_gb300 import hb
    P = make()
    for gi, G in enumerate(P.groups):
        ns = G.ci.shape[1]
        E, C, _ = hb.target_diag(P, gi, ns, tol=1e-10)
        G.ci, G.energy = C, E
    o = coracle.Oracle(P)
    R = o.dense()
    G, _, _ = gpu_dense(P, precision=precision)
    assert_blocks_close(G, R, o, 1e-10 if precision else 1e-12, f"{name} substituted", mixed=precision == 1)
    if len(P.groups) == 1:
        plain = copy.deepcopy(P)
        for Gr in plain.groups:
            Gr.energy = None
        Gp, _, _ = gpu_dense(plain, precision=precision)
        assert np.abs(G - Gp).max() <= 1e-9 * np.abs(Gp).max(), np.abs(G - Gp).max()


def test_substitution_inputs_validated():
    from paper_1709_03005_gb300 import hb
    P = synth.make_tiny(48, n_groups=2, n_state=[2, 2], cont_ranges=[(0, 3), (0, 3)])
    P.groups[0].energy = np.array([-1.0, -0.5])
    with pytest.raises(hb.HBError) as e:
        hb.Hamiltonian(P)
    assert e.value.code == hb.HB_ERR_INVALID_ARG
    P.groups[1].energy = np.array([np.nan, 0.0])
    with pytest.raises(hb.HBError):
        hb.Hamiltonian(P)
    with pytest.raises(hb.HBError):
        hb.target_diag(P, 2, 1)
    with pytest.raises(hb.HBError):
        hb.target_diag(P, 0, P.groups[0].dets.shape[0] + 1)
