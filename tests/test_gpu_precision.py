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

from gpu_util import sampled_checks

pytestmark = pytest.mark.gpu


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
    sampled_checks(P, o, cc, bm, rng, 1, n_cc=2000, what="c3 mixed")
    mixed_cc = bm["Hcc"]
    b64, st64 = H.build(hb.HB_FP64)
    torch.cuda.synchronize()
    sampled_checks(P, o, cc, b64, np.random.default_rng(3), 0, n_cc=2000, what="c3 FP64")
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
    sampled_checks(P, o, cc, b, np.random.default_rng(5), 1, n_cc=1000, n_rows=8, what="c5 mixed")
    H.close()
