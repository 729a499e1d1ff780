"""GPU parity of the FP64 build through the C ABI against the oracle.

Excitation classes, phases and sparsity pattern are compared bit-exactly.
Matrix elements: |d| <= 1e-12 max(|ref|, 1e-6 max|block|) per element, or, for
an element that cancels below 7.1e-3 of its condition scale (the sum of the
magnitudes of its terms, from the oracle), |d| <= 64 u times that scale: the
rounding of two summation orders of the same terms (tests/gpu_util.py)."""
import numpy as np
import pytest

from oracle import coracle
from paper_1709_03005_gb300 import synth

from gpu_util import FP64_FALLBACK, assert_blocks_close, check_elements, gpu_dense, l2_csr_cond

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1709_03005_gb300 import build_ext
    build_ext.build()


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, np.uint64).view(np.int64)).cuda()


def _oracle_records(W, A, B, mode, cont_spin, o=None, lower=False):
    """Oracle classification of every pair within a double excitation, in (a, b) order."""
    out = []
    for ia, a in enumerate(A):
        for ib, b in enumerate(B):
            if lower and ib > ia:
                continue
            if mode == 0:
                r = coracle.Oracle.excitation(W, a, b)
                if r[0] > 2:
                    continue
                out.append((ia, ib, int(r[0]), tuple(int(x) for x in r[1:3]), tuple(int(x) for x in r[3:5]),
                            int(r[5])))
            else:
                r = o.excitation_tl2(b, a)
                if r[0] > 2:
                    continue
                out.append((ia, ib, int(r[0]), (int(r[1]), int(r[2])), (int(r[3]), -1), int(r[4])))
    return out


def _gpu_records(rec, deg0_phase=True):
    return [(int(r["row"]), int(r["col"]), int(r["degree"]), tuple(int(x) for x in r["hole"]),
             tuple(int(x) for x in r["part"]), int(r["phase"])) for r in rec]


def _norm(recs):
    # degree-0 records carry no holes/particles; the oracle reports -1 and phase +1
    out = []
    for r in recs:
        if r[2] == 0:
            out.append((r[0], r[1], 0, (-1, -1), (-1, -1), 1))
        else:
            out.append(r)
    return out


@pytest.mark.parametrize("W,orbs", [(1, None), (2, [0, 1, 2, 62, 63, 64, 65, 66, 127]),
                                    (3, [0, 5, 62, 63, 64, 65, 126, 127, 128, 129, 190, 191])])
def test_classify_same_count_bit_exact(W, orbs):
    from paper_1709_03005_gb300 import hb
    rng = np.random.default_rng(100 + W)
    n_orb = 64 * W if orbs else 14
    A, B = synth.random_det_pairs(rng, n_orb, 3, 3, W, 150, max_exc=3, orbitals=orbs)
    B = np.concatenate([B, A[:20]])
    for lower in (False, True):
        rp, rec = hb.classify(_dev(A), _dev(B), W, 0, 0, 2, lower)
        ref = _oracle_records(W, A, B, 0, 0, lower=lower)
        assert _norm(_gpu_records(rec)) == _norm(ref)
        counts = np.diff(rp.cpu().numpy())
        assert counts.sum() == len(ref)


@pytest.mark.parametrize("spin", [0, 1])
def test_classify_target_l2_bit_exact(spin):
    from paper_1709_03005_gb300 import hb
    P = synth.make_tiny(500 + spin, n_to=9, n_elec=6, n_det=60, n_l2=80, cont_spin=spin)
    o = coracle.Oracle(P)
    A, B = P.l2_dets, P.groups[0].dets
    rp, rec = hb.classify(_dev(A), _dev(B), P.n_words, 1, spin, 2)
    ref = _oracle_records(P.n_words, A, B, 1, spin, o=o)
    got = [(r[0], r[1], r[2], r[3], (r[4][0], -1), r[5]) for r in _gpu_records(rec)]
    assert got == ref
    assert len(ref) > 10


CASES = [
    ("tiny_a", dict(seed=1)),
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
def test_build_fp64_small(name, kw):
    kw = dict(kw)
    seed = kw.pop("seed")
    P = synth.make_tiny(seed, **kw)
    o = coracle.Oracle(P)
    R = o.dense()
    G, st, _ = gpu_dense(P)
    assert G.shape == R.shape
    assert_blocks_close(G, R, o, 1e-12, name)
    np.testing.assert_array_equal(G, G.T)


@pytest.mark.parametrize("key", ["c1", "mid"])
def test_build_fp64_configs(key):
    """Several GPU tiles with ragged tails in every kernel; full element compare."""
    P = synth.make_config(key)
    o = coracle.Oracle(P)
    R = o.dense()
    G, st, blocks = gpu_dense(P)
    assert_blocks_close(G, R, o, 1e-12, key)
    # the L2 sparsity pattern is exactly the pairs within a double excitation
    rp, cols, vals = o.l2_csr()
    np.testing.assert_array_equal(blocks["row_ptr"].cpu().numpy(), rp)
    np.testing.assert_array_equal(blocks["col"][: rp[-1]].cpu().numpy(), cols)


def test_build_fp64_medium_sampled():
    """The 8000-dimensional medium workload at full size: the whole L2 block and
    sampled continuum-continuum and class-4 elements against the oracle."""
    import torch
    from paper_1709_03005_gb300 import hb
    P = synth.make_config("c2")
    o = coracle.Oracle(P)
    H = hb.Hamiltonian(P)
    b, st = H.build(hb.HB_FP64)
    torch.cuda.synchronize()
    rp, cols, vals = o.l2_csr()
    np.testing.assert_array_equal(b["row_ptr"].cpu().numpy(), rp)
    np.testing.assert_array_equal(b["col"][: rp[-1]].cpu().numpy(), cols)
    gv = b["val"][: rp[-1]].cpu().numpy()
    check_elements(gv, vals, l2_csr_cond(o, rp, cols), 1e-12, FP64_FALLBACK, "c2 L2")
    Hcc = b["Hcc"].cpu().numpy()
    cc = o.contract(0, 0)
    rng = np.random.default_rng(0)
    ns, nco = P.groups[0].ci.shape[1], P.n_co
    idx = [(int(n), int(j), int(n_), int(j if rng.random() < 0.2 else jp))
           for n, n_, j, jp in zip(*[rng.integers(0, m, 600) for m in (ns, ns, nco, nco)])]
    ref = np.array([cc.element(*t) for t in idx])
    cond = np.array([cc.element_cond(*t) for t in idx])
    got = np.array([Hcc[n * nco + j, n_ * nco + jp] for n, j, n_, jp in idx])
    check_elements(got, ref, cond, 1e-12, FP64_FALLBACK, "c2 cc sampled", blockmax=np.abs(Hcc).max())
    Hlc = b["Hlc"].cpu().numpy()
    rows = np.sort(rng.choice(P.n_l2, 40, replace=False))
    ref4 = np.stack([o.class4_row(int(l)) for l in rows])
    cond4 = np.stack([o.class4_rows_abs(int(l), int(l) + 1)[0] for l in rows])
    check_elements(Hlc[rows], ref4, cond4, 1e-12, FP64_FALLBACK, "c2 class 4 rows", blockmax=np.abs(Hlc).max())
    H.close()


@pytest.mark.parametrize("key,precision", [("mid", 0), ("mid", 1), ("c1", 1)])
def test_l2_block_every_entry_written(key, precision):
    """Classes 2 and 8 evaluate the upper triangle of the symmetric L2 x L2
    block and copy each lower entry from its mirror.  With the output filled
    with NaN and -1 beforehand, every entry is written, the block is exactly
    symmetric, and it matches the oracle's CSR."""
    import scipy.sparse as sp
    from paper_1709_03005_gb300 import hb
    P = synth.make_config(key)
    o = coracle.Oracle(P)
    rp, cols, vals = o.l2_csr()
    H = hb.Hamiltonian(P)
    b = H.allocate()
    b["val"].fill_(float("nan"))
    b["col"].fill_(-1)
    H.build(precision, blocks=b)
    n = P.n_l2
    g_rp = b["row_ptr"].cpu().numpy()
    g_col = b["col"][: rp[-1]].cpu().numpy()
    g_val = b["val"][: rp[-1]].cpu().numpy()
    np.testing.assert_array_equal(g_rp, rp)
    np.testing.assert_array_equal(g_col, cols)
    assert np.isfinite(g_val).all()
    A = sp.csr_matrix((g_val, g_col, g_rp), shape=(n, n))
    assert abs(A - A.T).max() == 0.0
    check_elements(g_val, vals, l2_csr_cond(o, rp, cols), 1e-12, FP64_FALLBACK, f"{key} L2")
    H.close()


def test_build_is_deterministic():
    import torch
    from paper_1709_03005_gb300 import hb
    P = synth.make_config("mid")
    H = hb.Hamiltonian(P)
    b1, _ = H.build()
    c1 = {k: v.clone() for k, v in b1.items()}
    b2, _ = H.build()
    torch.cuda.synchronize()
    for k in c1:
        assert torch.equal(c1[k], b2[k]), k
    H.close()


def test_invalid_inputs_rejected():
    from paper_1709_03005_gb300 import hb
    P = synth.make_tiny(9)
    P.groups[0].dets = P.groups[0].dets.copy()
    P.groups[0].dets[1] = P.groups[0].dets[0]
    with pytest.raises(hb.HBError) as e:
        hb.Hamiltonian(P)
    assert e.value.code == hb.HB_ERR_INVALID_ARG
    P = synth.make_tiny(9)
    P.h = P.h.copy(); P.h[0, 1] += 1.0
    with pytest.raises(hb.HBError):
        hb.Hamiltonian(P)
    P = synth.make_tiny(9)
    P.groups[0].cont_count = P.n_co + 1
    with pytest.raises(hb.HBError):
        hb.Hamiltonian(P)
