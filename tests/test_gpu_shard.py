"""Sharded build (Section 3.1: the prototype contraction split over ranks and
the reduction of the contracted coefficients, Eq. 11; Section 3.2: the
distributed matrix) through the C ABI.  R ranks run one after the other on
one GPU (their kernels never wait on each other: the exchange is the sum of
the partial coefficient rows, done here by torch in rank order, by NCCL under
torchrun).  Checked: the ranks' outputs add up to the whole matrix, which
matches the oracle with the element criterion of tests/gpu_util.py and the
one-rank build; every element the one-rank build writes is written by exactly
one rank, and no rank writes anything else."""
import numpy as np
import pytest

from oracle import coracle
from paper_1709_03005_gb300 import synth

from gpu_util import assert_blocks_close

pytestmark = pytest.mark.gpu
KEYS = ("Hcc", "Hlc", "row_ptr", "col", "val")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1709_03005_gb300 import build_ext
    build_ext.build()


def _filled(H):
    """Output blocks with every entry marked unwritten (NaN, -1)."""
    b = H.allocate()
    for k in ("Hcc", "Hlc", "val"):
        b[k].fill_(float("nan"))
    for k in ("row_ptr", "col"):
        b[k].fill_(-1)
    return b


def _written(b):
    return {k: (~b[k].isnan()) if k in ("Hcc", "Hlc", "val") else (b[k] != -1) for k in KEYS}


def _energies(P):
    """Eigenvector CI and energies of every group (numpy eigh of the oracle's H^N)."""
    import copy
    for g in P.groups:
        Q = copy.copy(P)
        Q.l2_dets, Q.groups = g.dets, []
        E, V = np.linalg.eigh(coracle.Oracle(Q).l2_rows(0, g.dets.shape[0]))
        ns = g.ci.shape[1]
        g.ci, g.energy = np.ascontiguousarray(V[:, :ns]), E[:ns].copy()
    return P


CASES = [
    ("c1", lambda: synth.make_config("c1")),
    ("mid", lambda: synth.make_config("mid")),
    ("groups_beta", lambda: synth.make_tiny(403, n_to=7, n_co=5, n_elec=4, n_det=9, n_groups=3, n_state=[2, 3, 1],
                                            cont_ranges=[(0, 5), (1, 3), (0, 5)], n_l2=12, cont_spin=1, e_core=-3.5)),
    ("substituted", lambda: _energies(synth.make_tiny(404, n_to=6, n_co=4, n_elec=4, n_det=14, n_state=3,
                                                      n_l2=9))),
    ("class4_tensor", lambda: synth.make_config("mid", n_co=48, n_state=36, n_l2=200, seed=405)),
]


@pytest.mark.parametrize("nranks", [2, 3])
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_sharded_build(name, make, precision, nranks):
    import torch
    from paper_1709_03005_gb300 import hb
    P = make()
    H = hb.Hamiltonian(P)
    one = _filled(H)
    H.build(precision, one)
    torch.cuda.synchronize()
    want = _written(one)
    # 1. every rank's partial coefficient rows; 2. their sum in rank order
    partials = [H.build_contract(precision, r, nranks)[0].clone() for r in range(nranks)]
    reduced = partials[0].clone()
    for p in partials[1:]:
        reduced += p
    # 3. every rank's share, into blocks marked unwritten
    outs = [H.build_expand(precision, r, nranks, reduced, _filled(H))[0] for r in range(nranks)]
    torch.cuda.synchronize()
    merged = {}
    count = {k: torch.zeros_like(want[k], dtype=torch.int32) for k in KEYS}
    for b in outs:
        w = _written(b)
        for k in KEYS:
            count[k] += w[k].to(torch.int32)
            merged[k] = torch.where(w[k], b[k], merged[k]) if k in merged else b[k].clone()
    for k in KEYS:
        assert torch.equal(count[k], want[k].to(torch.int32)), f"{k}: written by other than exactly one rank"
    # the merged matrix against the oracle, and against the one-rank build
    o = coracle.Oracle(P)
    G = hb.dense_from_blocks({k: torch.nan_to_num(v) for k, v in merged.items()}).cpu().numpy()
    assert_blocks_close(G, o.dense(), o, 1e-10 if precision else 1e-12, f"{name} x{nranks}", mixed=precision == 1)
    for k in ("row_ptr", "col"):
        assert torch.equal(merged[k], one[k]), k
    G1 = hb.dense_from_blocks({k: torch.nan_to_num(v) for k, v in one.items()}).cpu().numpy()
    tol = (1e-11 if precision else 1e-13) * np.abs(G1).max()
    assert np.abs(G - G1).max() <= tol, np.abs(G - G1).max()
    H.close()


def test_shard_arguments_checked():
    from paper_1709_03005_gb300 import hb
    H = hb.Hamiltonian(synth.make_config("c1"))
    with pytest.raises(hb.HBError):
        H.build_contract(0, 2, 2)
    with pytest.raises(hb.HBError):
        H.build_contract(2, 0, 1)
    H.close()
