"""The precision workload at full size (40 target + 400 continuum orbitals,
20000 target determinants, 50 states, 30000 L2 functions, dimension 50000):
sampled elements of every class against the oracle, and the per-element error
of the mixed continuum block against the FP64 GPU build."""
import numpy as np
import pytest

from oracle import coracle
from paper_1709_03005_gb300 import synth

pytestmark = pytest.mark.gpu


def test_precision_workload_sampled():
    import torch
    from paper_1709_03005_gb300 import build_ext, hb
    build_ext.build()
    P = synth.make_config("c3")
    o = coracle.Oracle(P)
    H = hb.Hamiltonian(P, validate=False)
    bm, stm = H.build(hb.HB_MIXED)
    mixed_cc = bm["Hcc"].clone()
    b64, st64 = H.build(hb.HB_FP64)
    torch.cuda.synchronize()
    # whole-block comparison of the two GPU paths
    d = (mixed_cc - b64["Hcc"]).abs()
    ref = b64["Hcc"].abs()
    scale = float(ref.max())
    rel = d / ref.clamp_min(1e-300)
    frac_rel = float((rel <= 1e-10).double().mean())
    print(f"c3 mixed vs FP64: max |d| {float(d.max()):.3e} (scale {scale:.2e}), "
          f"{100 * frac_rel:.2f} % of elements within 1e-10 relative; "
          f"build {stm.ms_total:.1f} ms mixed vs {st64.ms_total:.1f} ms FP64")
    Hcc = mixed_cc.cpu().numpy()
    del mixed_cc, d, rel, ref
    cc = o.contract(0, 0)
    rng = np.random.default_rng(3)
    ns, nco = 50, 400
    worst = 0.0
    for _ in range(300):
        n, np_ = rng.integers(0, ns, 2)
        j, jp = rng.integers(0, nco, 2)
        if rng.random() < 0.1:
            jp = j
        r = cc.element(int(n), int(j), int(np_), int(jp))
        cond = cc.element_abs(int(n), int(j), int(np_), int(jp))
        g = Hcc[n * nco + j, np_ * nco + jp]
        worst = max(worst, abs(g - r) / cond)
        assert abs(g - r) <= 1e-10 * cond, (n, j, np_, jp, g, r, cond)
    print(f"c3 sampled continuum elements: worst |d| / condition scale {worst:.2e}")
    Hlc = bm["Hlc"]
    for l in rng.choice(P.n_l2, 12, replace=False):
        r = o.class4_row(int(l))
        g = Hlc[int(l)].cpu().numpy()
        assert np.all(np.abs(g - r) <= 1e-12 * np.maximum(np.abs(r), np.abs(r).max())), l
    rp = bm["row_ptr"].cpu().numpy()
    for a in rng.choice(P.n_l2, 12, replace=False):
        row = o.l2_rows(int(a), int(a) + 1)[0]
        cols = bm["col"][rp[a]:rp[a + 1]].cpu().numpy()
        vals = bm["val"][rp[a]:rp[a + 1]].cpu().numpy()
        dense = np.zeros(P.n_l2)
        dense[cols] = vals
        assert np.all(np.abs(dense - row) <= 1e-12 * np.maximum(np.abs(row), np.abs(row).max())), a
        assert set(cols.tolist()) >= set(np.nonzero(row)[0].tolist())
    H.close()
