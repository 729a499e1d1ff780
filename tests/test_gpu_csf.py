"""Spin-adapted target groups on the GPU through the C ABI: CI vectors over
configuration state functions, expanded over determinants by the library, and
a singlet and a triplet group over the same determinants coupled to the same
continuum (built as one group).  Every element against the oracle, both
build paths, with the element criterion of tests/gpu_util.py."""
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


CASES = [
    ("tiny_singlet_triplet", dict(seed=14, n_to=7, n_co=4, n_elec=4, n_config=8, n_state=(2, 2), n_l2=6)),
    ("mid_singlet_triplet", dict(seed=15, n_to=12, n_co=23, n_elec=6, n_config=70, n_state=(5, 4), n_l2=150,
                                 rank=12, keep_chol=False)),
]


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name,kw", CASES, ids=[c[0] for c in CASES])
def test_csf_build(name, kw, precision):
    from paper_1709_03005_gb300 import hb
    P = synth.make_csf_problem(**kw)
    o = coracle.Oracle(P)
    R = o.dense()
    G, st, _ = gpu_dense(P, precision=precision)
    assert G.shape == R.shape
    assert_blocks_close(G, R, o, 1e-10 if precision else 1e-12, name, mixed=precision == 1)
    H = hb.Hamiltonian(P)
    assert H.group_offsets == [int(x) for x in o.offsets]
    # the singlet-triplet block couples (exchange with the continuum electron)
    r0, r1, r2 = o.offsets[:3]
    assert np.abs(G[r1:r2, r0:r1]).max() > 1e-3
    H.close()


def test_csf_group_beside_determinant_groups():
    """A CSF group between two determinant groups of disjoint determinants
    (the merged-group path with single members)."""
    P = synth.make_csf_problem(seed=16, n_to=7, n_co=5, n_elec=4, n_config=8, n_state=(2, 2), spins=(0.0,), n_l2=5)
    Q = synth.make_tiny(17, n_to=7, n_co=5, n_elec=4, n_det=6, n_groups=2, n_state=[2, 1], n_l2=0)
    used = {tuple(d) for d in P.groups[0].dets}
    for g in Q.groups:
        keep = [i for i, d in enumerate(g.dets) if tuple(d) not in used]
        g.dets, g.ci = g.dets[keep], np.linalg.qr(g.ci[keep])[0]
    P.groups = [Q.groups[0], P.groups[0], Q.groups[1]]
    P.groups[1].cont_first, P.groups[1].cont_count = 1, 3
    o = coracle.Oracle(P)
    R = o.dense()
    G, _, _ = gpu_dense(P)
    assert_blocks_close(G, R, o, 1e-12, "mixed groups")


def test_shared_determinants_must_match():
    from paper_1709_03005_gb300 import hb
    P = synth.make_csf_problem(seed=14, n_to=7, n_co=4, n_elec=4, n_config=8, n_state=(2, 2), n_l2=6)
    P.groups[1].cont_first, P.groups[1].cont_count = 1, 3     # same determinants, other continuum
    with pytest.raises(hb.HBError) as e:
        hb.Hamiltonian(P)
    assert e.value.code == hb.HB_ERR_INVALID_ARG
    P = synth.make_csf_problem(seed=14, n_to=7, n_co=4, n_elec=4, n_config=8, n_state=(2, 2), n_l2=6)
    P.groups[0].csf_det = P.groups[0].csf_det.copy()
    P.groups[0].csf_det[0] = P.groups[0].dets.shape[0]           # index out of range
    with pytest.raises(hb.HBError):
        hb.Hamiltonian(P)
