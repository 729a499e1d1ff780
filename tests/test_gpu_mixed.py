"""GPU parity of the mixed-precision build (split bf16 tensor-core expansion).

Continuum-continuum elements: |G - R| <= 1e-10 * sum_b |D^b X(I^b)|, the
condition scale of the Eq. 7 sum computed by the oracle.  For elements without
cancellation this is the relative bound 1e-10; for elements that cancel far
below the size of their terms no finite-precision evaluation (an FP64 sum in
another order included) is closer than a small multiple of the unit roundoff of
that scale.  Class 4 (double-float or split-bf16 tensor cores) and classes 2, 8
(FP64) are held to 1e-12 of their block scale.
"""
import numpy as np
import pytest

from oracle import coracle
from paper_1709_03005_gb300 import synth

from gpu_util import gpu_dense

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1709_03005_gb300 import build_ext
    build_ext.build()


def _check_mixed(P, slices=0, what=""):
    o = coracle.Oracle(P)
    R = o.dense()
    cond = o.cc_condition()
    G, st, _ = gpu_dense(P, precision=1, split_slices=slices)
    Dc = o.Dc
    d = np.abs(G[:Dc, :Dc] - R[:Dc, :Dc])
    bad = d > TOL * cond
    assert not bad.any(), f"{what}: {bad.sum()} elements beyond 1e-10 of their condition scale; " \
                          f"worst ratio {(d / np.maximum(cond, 1e-300)).max():.3e}"
    np.testing.assert_array_equal(G, G.T)
    # class 4 (double-float or tensor cores), classes 2 and 8 (FP64)
    for blk in (np.s_[Dc:, :Dc], np.s_[Dc:, Dc:]):
        g, r = G[blk], R[blk]
        if r.size:
            assert np.all(np.abs(g - r) <= 1e-12 * np.maximum(np.abs(r), np.abs(r).max())), what
    rel = d / np.maximum(np.abs(R[:Dc, :Dc]), 1e-300)
    return float((rel <= TOL).mean()), float((d / np.maximum(cond, 1e-300)).max())


CASES = [
    ("tiny_groups", dict(seed=3, n_groups=2, n_state=[2, 3], cont_ranges=[(0, 3), (1, 2)])),
    ("tiny_beta", dict(seed=4, cont_spin=1)),
    ("tiny_three", dict(seed=5, n_groups=3, n_det=4, n_state=[1, 2, 2], cont_ranges=[(0, 2), (0, 3), (2, 1)],
                        cont_spin=1)),
    ("tiny_no_l2", dict(seed=6, n_l2=0)),
]


@pytest.mark.parametrize("name,kw", CASES, ids=[c[0] for c in CASES])
def test_mixed_small(name, kw):
    kw = dict(kw)
    P = synth.make_tiny(kw.pop("seed"), **kw)
    _check_mixed(P, what=name)


@pytest.mark.parametrize("key", ["c1", "mid"])
def test_mixed_configs(key):
    frac, worst = _check_mixed(synth.make_config(key), what=key)
    print(f"{key}: {100 * frac:.1f} % of elements within 1e-10 relative, worst condition ratio {worst:.2e}")


def test_mixed_six_slices():
    _check_mixed(synth.make_config("mid"), slices=6, what="mid S=6")


def test_mixed_medium_sampled():
    import torch
    from paper_1709_03005_gb300 import hb
    P = synth.make_config("c2")
    o = coracle.Oracle(P)
    H = hb.Hamiltonian(P)
    b, st = H.build(hb.HB_MIXED)
    torch.cuda.synchronize()
    Hcc = b["Hcc"].cpu().numpy()
    cc = o.contract(0, 0)
    rng = np.random.default_rng(1)
    ns, nco = P.groups[0].ci.shape[1], P.n_co
    for _ in range(400):
        n, np_ = rng.integers(0, ns, 2)
        j, jp = rng.integers(0, nco, 2)
        if rng.random() < 0.1:
            jp = j
        ref = cc.element(int(n), int(j), int(np_), int(jp))
        cond = cc.element_abs(int(n), int(j), int(np_), int(jp))
        got = Hcc[n * nco + j, np_ * nco + jp]
        assert abs(got - ref) <= TOL * cond, (n, j, np_, jp, got, ref, cond)
    # class 4 and L2 are the FP64 kernels
    rp, cols, vals = o.l2_csr()
    np.testing.assert_array_equal(b["col"][: rp[-1]].cpu().numpy(), cols)
    H.close()


def test_mixed_deterministic():
    import torch
    from paper_1709_03005_gb300 import hb
    H = hb.Hamiltonian(synth.make_config("mid"))
    b1, _ = H.build(hb.HB_MIXED)
    x = b1["Hcc"].clone()
    b2, _ = H.build(hb.HB_MIXED)
    torch.cuda.synchronize()
    assert torch.equal(x, b2["Hcc"])
    H.close()


@pytest.mark.parametrize("n_state", [7, 20, 50])
def test_class4_wide_continuum(n_state):
    """Class 4 (Eq. 5) of the mixed build (double-float) for 80 continuum
    orbitals and 7, 20 or 50 states (one pass over the states): the FP64
    tolerance against the oracle, per row scale."""
    from paper_1709_03005_gb300 import hb
    import torch
    P = synth.make_config("mid", n_co=80, n_state=n_state, n_l2=300, seed=21 + n_state)
    o = coracle.Oracle(P)
    H = hb.Hamiltonian(P)
    b, _ = H.build(hb.HB_MIXED)
    torch.cuda.synchronize()
    Hlc = b["Hlc"].cpu().numpy()
    H.close()
    rows = o.class4_rows(0, P.n_l2)
    scale = np.maximum(np.abs(rows), np.abs(rows).max(axis=1, keepdims=True))
    worst = float((np.abs(Hlc - rows) / np.maximum(scale, 1e-300)).max())
    assert np.all(np.abs(Hlc - rows) <= 1e-12 * scale), worst
    print(f"class 4, {n_state} states: worst |d| / row scale {worst:.2e}")


@pytest.mark.parametrize("name,kw", CASES[:3] + [("mid", None)], ids=[c[0] for c in CASES[:3]] + ["mid"])
def test_class4_tensor_cores(name, kw):
    """Class 4 on the tensor cores for every group (class4_path=2; by default
    only groups of 32..64 states take it): the Eq. 5 block against the oracle
    at 1e-12 of the block scale, against the double-float kernel
    (class4_path=1) likewise, and every other block identical to that build."""
    import torch
    from paper_1709_03005_gb300 import hb
    if kw is None:
        P = synth.make_config("mid")
    else:
        kw = dict(kw)
        P = synth.make_tiny(kw.pop("seed"), **kw)
    o = coracle.Oracle(P)
    R = o.dense()
    Dc = o.Dc
    Ht = hb.Hamiltonian(P, class4_path=2)
    Hd = hb.Hamiltonian(P, class4_path=1)
    bt, _ = Ht.build(hb.HB_MIXED)
    bd, _ = Hd.build(hb.HB_MIXED)
    torch.cuda.synchronize()
    assert "class4 tensor cores" in Ht.tuning_report() or P.n_l2 == 0
    for key in ("Hcc", "row_ptr", "col", "val"):
        assert torch.equal(bt[key], bd[key]), key
    G = hb.dense_from_blocks(bt).cpu().numpy()
    D = hb.dense_from_blocks(bd).cpu().numpy()
    blk = np.s_[Dc:, :Dc]
    r = R[blk]
    if r.size:
        scale = np.abs(r).max()
        assert np.all(np.abs(G[blk] - r) <= 1e-12 * np.maximum(np.abs(r), scale))
        assert np.all(np.abs(G[blk] - D[blk]) <= 1e-12 * np.maximum(np.abs(r), scale))
    Ht.close()
    Hd.close()
