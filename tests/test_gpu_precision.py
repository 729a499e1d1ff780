"""The precision workload at full size (40 target + 400 continuum orbitals,
20000 target determinants, 50 states, 30000 L2 functions, dimension 50000)
and the learned-preconditioner workload (the same family with 40000 L2
functions, dimension 60000): sampled elements of every class against the
oracle with the element criterion of tests/gpu_util.py, on both build paths,
and the per-element difference of the mixed continuum block from the FP64 GPU
build."""
import numpy as np
import pytest

from oracle import coracle
from paper_1709_03005_gb300 import synth

from gpu_util import FP64_FALLBACK, MIXED_C4_FALLBACK, MIXED_C4_TC_ABS, MIXED_CC_FALLBACK, check_elements

pytestmark = pytest.mark.gpu


def sampled_checks(P, o, cc, b, rng, precision, n_cc=400, n_rows=12, what=""):
    """Sampled continuum elements, whole class-4 rows and whole L2 rows of the
    built blocks b against the oracle.  Returns the fraction of sampled
    continuum elements within 1e-10 of their own magnitude."""
    mixed = precision == 1
    rel = 1e-10 if mixed else 1e-12
    ns, nco = P.groups[0].ci.shape[1], P.n_co
    idx = [(int(n), int(j), int(n_), int(j if rng.random() < 0.1 else jp))
           for n, n_, j, jp in zip(*[rng.integers(0, m, n_cc) for m in (ns, ns, nco, nco)])]
    ref = np.array([cc.element(*t) for t in idx])
    cond = np.array([cc.element_cond(*t) for t in idx])
    Hcc = b["Hcc"]
    got = np.array([float(Hcc[n * nco + j, n_ * nco + jp]) for n, j, n_, jp in idx])
    bm = float(Hcc.abs().max())
    _, _, n_canc, worst = check_elements(got, ref, cond, rel, MIXED_CC_FALLBACK if mixed else FP64_FALLBACK,
                                         f"{what} cc sampled", blockmax=bm)
    strict10 = float(np.mean(np.abs(got - ref) <= 1e-10 * np.abs(ref)))
    print(f"{what}: {100 * strict10:.2f} % of sampled continuum elements within 1e-10 of their magnitude, "
          f"{n_canc} by the cancellation clause, worst |d|/cond {worst:.2e}")
    rows = np.sort(rng.choice(P.n_l2, n_rows, replace=False))
    ref4 = np.stack([o.class4_row(int(l)) for l in rows])
    cond4 = np.stack([o.class4_rows_abs(int(l), int(l) + 1)[0] for l in rows])
    g4 = b["Hlc"][rows].cpu().numpy()
    check_elements(g4, ref4, cond4, rel, MIXED_C4_FALLBACK if mixed else FP64_FALLBACK, f"{what} class 4 rows",
                   blockmax=float(b["Hlc"].abs().max()), abs_frac=MIXED_C4_TC_ABS if mixed else None)
    rp = b["row_ptr"].cpu().numpy()
    for a in rng.choice(P.n_l2, n_rows, replace=False):
        row = o.l2_rows(int(a), int(a) + 1)[0]
        rcond = o.l2_rows_abs(int(a), int(a) + 1)[0]
        cols = b["col"][rp[a]:rp[a + 1]].cpu().numpy()
        vals = b["val"][rp[a]:rp[a + 1]].cpu().numpy()
        dense = np.zeros(P.n_l2)
        dense[cols] = vals
        check_elements(dense, row, rcond, 1e-12, FP64_FALLBACK, f"{what} L2 row {a}")
        assert set(cols.tolist()) >= set(np.nonzero(row)[0].tolist())
    return strict10


def test_precision_workload_sampled():
    import torch
    from paper_1709_03005_gb300 import build_ext, hb
    build_ext.build()
    P = synth.make_config("c3")
    o = coracle.Oracle(P)
    cc = o.contract(0, 0)
    H = hb.Hamiltonian(P, validate=False)
    bm, stm = H.build(hb.HB_MIXED)
    torch.cuda.synchronize()
    rng = np.random.default_rng(3)
    sampled_checks(P, o, cc, bm, rng, 1, what="c3 mixed")
    mixed_cc = bm["Hcc"]
    b64, st64 = H.build(hb.HB_FP64)
    torch.cuda.synchronize()
    sampled_checks(P, o, cc, b64, np.random.default_rng(3), 0, what="c3 FP64")
    # whole-block comparison of the two GPU paths
    d = (mixed_cc - b64["Hcc"]).abs()
    ref = b64["Hcc"].abs()
    frac_rel = float((d <= 1e-10 * ref).double().mean())
    print(f"c3 mixed vs FP64 GPU: max |d| {float(d.max()):.3e} (scale {float(ref.max()):.2e}), "
          f"{100 * frac_rel:.2f} % of elements within 1e-10 relative; "
          f"build {stm.ms_total:.1f} ms mixed vs {st64.ms_total:.1f} ms FP64")
    H.close()


def test_learned_workload_sampled():
    """The 60000-dimensional workload of the learned preconditioner, mixed
    build: sampled elements of every class against the oracle."""
    import torch
    from paper_1709_03005_gb300 import build_ext, hb
    build_ext.build()
    P = synth.make_config("c5")
    o = coracle.Oracle(P)
    cc = o.contract(0, 0)
    H = hb.Hamiltonian(P, validate=False)
    b, st = H.build(hb.HB_MIXED)
    torch.cuda.synchronize()
    assert H.dim == 60000
    sampled_checks(P, o, cc, b, np.random.default_rng(5), 1, n_cc=300, n_rows=8, what="c5 mixed")
    H.close()
