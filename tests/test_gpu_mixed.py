"""GPU parity of the mixed-precision build (split bf16 tensor-core expansion).

Every element is held to the criterion of tests/gpu_util.py: the floored
relative bound 1e-10 max(|ref|, 1e-6 max|block|) on the continuum block and on
class 4 (double-float or split-bf16 tensor cores), 1e-12 on the FP64 L2 block,
or, for an element whose value cancels far below the magnitude of its terms, a
fixed fraction of its condition scale from the oracle (the sum of the
magnitudes of every term of Eq. 8 and Eq. 7, or of Eq. 5).  The tests print the fraction of continuum elements within 1e-10 of
their own magnitude and the number of elements that pass only by the
cancellation clause.
"""
import numpy as np
import pytest

from oracle import coracle
from paper_1709_03005_gb300 import synth

from gpu_util import (FP64_FALLBACK, MIXED_C4_FALLBACK, MIXED_C4_TC_ABS, MIXED_CC_FALLBACK, assert_blocks_close,
                      check_elements, gpu_dense, l2_csr_cond)

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1709_03005_gb300 import build_ext
    build_ext.build()


def _check_mixed(P, slices=0, what=""):
    o = coracle.Oracle(P)
    R = o.dense()
    S = o.condition()
    G, st, _ = gpu_dense(P, precision=1, split_slices=slices)
    np.testing.assert_array_equal(G, G.T)
    res = assert_blocks_close(G, R, o, TOL, what, S=S, mixed=True)
    strict, floored, n_canc, worst = res["cc"]
    print(f"{what}: {100 * strict:.2f} % of continuum elements within 1e-10 relative, {100 * floored:.2f} % within "
          f"the floored bound, {n_canc} by the cancellation clause, worst |d|/cond {worst:.2e}")
    return strict, worst


CASES = [
    ("tiny_groups", dict(seed=3, n_groups=2, n_state=[2, 3], cont_ranges=[(0, 3), (1, 2)])),
    ("tiny_beta", dict(seed=4, cont_spin=1)),
    ("tiny_three", dict(seed=5, n_groups=3, n_det=4, n_state=[1, 2, 2], cont_ranges=[(0, 2), (0, 3), (2, 1)],
                        cont_spin=1)),
    ("tiny_no_l2", dict(seed=6, n_l2=0)),
    ("tiny_wide_W2", dict(seed=7, n_to=70, n_co=3, n_elec=4, n_det=12, n_state=2, n_l2=10, rank=4)),
    ("tiny_single_state", dict(seed=8, n_state=1, n_det=3, n_l2=1)),
    ("tiny_e_core", dict(seed=10, n_groups=2, n_state=[2, 2], cont_ranges=[(0, 3), (0, 2)], e_core=-4.75)),
]


@pytest.mark.parametrize("name,kw", CASES, ids=[c[0] for c in CASES])
def test_mixed_small(name, kw):
    kw = dict(kw)
    P = synth.make_tiny(kw.pop("seed"), **kw)
    _check_mixed(P, what=name)


@pytest.mark.parametrize("key", ["c1", "mid"])
def test_mixed_configs(key):
    _check_mixed(synth.make_config(key), what=key)


def test_mixed_six_slices():
    _check_mixed(synth.make_config("mid"), slices=6, what="mid S=6")


def test_mixed_medium_sampled():
    """The 8000-dimensional workload: sampled continuum elements, 40 whole
    class-4 rows and the whole L2 block against the oracle."""
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
    idx = [(int(n), int(j), int(n_), int(j if rng.random() < 0.1 else jp))
           for n, n_, j, jp in zip(*[rng.integers(0, m, 600) for m in (ns, ns, nco, nco)])]
    ref = np.array([cc.element(*t) for t in idx])
    cond = np.array([cc.element_cond(*t) for t in idx])
    got = np.array([Hcc[n * nco + j, n_ * nco + jp] for n, j, n_, jp in idx])
    strict, floored, n_canc, worst = check_elements(got, ref, cond, TOL, MIXED_CC_FALLBACK, "c2 cc sampled",
                                                    blockmax=np.abs(Hcc).max())
    print(f"c2 mixed: {100 * strict:.2f} % of sampled continuum elements within 1e-10 relative, {n_canc} by the "
          f"cancellation clause, worst |d|/cond {worst:.2e}")
    Hlc = b["Hlc"].cpu().numpy()
    rows = np.sort(rng.choice(P.n_l2, 40, replace=False))
    ref4 = np.stack([o.class4_row(int(l)) for l in rows])
    cond4 = np.stack([o.class4_rows_abs(int(l), int(l) + 1)[0] for l in rows])
    check_elements(Hlc[rows], ref4, cond4, TOL, MIXED_C4_FALLBACK, "c2 class 4 rows", blockmax=np.abs(Hlc).max(),
                   abs_frac=MIXED_C4_TC_ABS)
    rp, cols, vals = o.l2_csr()
    np.testing.assert_array_equal(b["row_ptr"].cpu().numpy(), rp)
    np.testing.assert_array_equal(b["col"][: rp[-1]].cpu().numpy(), cols)
    check_elements(b["val"][: rp[-1]].cpu().numpy(), vals, l2_csr_cond(o, rp, cols), 1e-12, FP64_FALLBACK, "c2 L2")
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
    cond = o.class4_rows_abs(0, P.n_l2)
    _, _, n_canc, worst = check_elements(Hlc, rows, cond, TOL, MIXED_C4_FALLBACK, f"class 4, {n_state} states",
                                         abs_frac=MIXED_C4_TC_ABS)
    print(f"class 4, {n_state} states: worst |d| / cond {worst:.2e}, {n_canc} by the cancellation clause")


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
        S = o.condition()[blk]
        check_elements(G[blk], r, S, TOL, MIXED_C4_FALLBACK, f"{name} tensor cores", abs_frac=MIXED_C4_TC_ABS)
        check_elements(G[blk], D[blk], S, TOL, 2 * MIXED_C4_FALLBACK, f"{name} tensor cores vs double-float",
                       abs_frac=2 * MIXED_C4_TC_ABS,
                       zeros=False)
    Ht.close()
    Hd.close()


def test_class4_tensor_cores_ragged_tiles():
    """Class 4 on the tensor cores by default (a group of 40 states) over 300
    continuum orbitals, that is two whole 128-orbital tiles and a ragged tail of
    44: every element of the block against the oracle, and against the
    double-float kernel."""
    import torch
    from paper_1709_03005_gb300 import hb
    P = synth.make_config("mid", n_co=300, n_state=40, n_l2=240, seed=33)
    o = coracle.Oracle(P)
    Ht = hb.Hamiltonian(P)
    bt, _ = Ht.build(hb.HB_MIXED)
    torch.cuda.synchronize()
    assert "class4 tensor cores" in Ht.tuning_report(), Ht.tuning_report()
    Hlc = bt["Hlc"].cpu().numpy()
    Ht.close()
    Hd = hb.Hamiltonian(P, class4_path=1)
    bd, _ = Hd.build(hb.HB_MIXED)
    torch.cuda.synchronize()
    Hld = bd["Hlc"].cpu().numpy()
    Hd.close()
    rows = o.class4_rows(0, P.n_l2)
    cond = o.class4_rows_abs(0, P.n_l2)
    _, _, n_canc, worst = check_elements(Hlc, rows, cond, TOL, MIXED_C4_FALLBACK, "300 orbitals, tensor cores",
                                         abs_frac=MIXED_C4_TC_ABS)
    check_elements(Hld, rows, cond, TOL, MIXED_C4_FALLBACK, "300 orbitals, double-float")
    print(f"class 4 tensor cores, 300 orbitals: worst |d|/cond {worst:.2e}, {n_canc} by the cancellation clause")
