"""Batched build of the 16 symmetry / spin-coupling Hamiltonians of one
molecule (shared integrals, one CUDA-graph launch): identical to building each
context on its own, and the smallest members match the oracle."""
import numpy as np
import pytest

from oracle import coracle
from paper_1709_03005_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def family():
    from paper_1709_03005_gb300 import build_ext
    build_ext.build()
    return synth.make_batched_family()


def test_batch_equals_individual_builds(family):
    import torch
    from paper_1709_03005_gb300 import hb
    B = hb.Batch(family, hb.HB_MIXED)
    st = B.launch()
    torch.cuda.synchronize()
    assert B.nodes > len(family)
    for h, b in zip(B.hams, B.blocks):
        ref, _ = h.build(hb.HB_MIXED)
        torch.cuda.synchronize()
        for key in ("Hcc", "Hlc", "row_ptr", "col", "val"):
            assert torch.equal(ref[key], b[key]), key
    print(f"batched build: {len(family)} Hamiltonians, {B.positions:.3e} positions, {st.ms_total:.2f} ms, "
          f"{B.nodes} graph nodes")
    B.close()


def test_batch_members_match_oracle(family):
    import torch
    from paper_1709_03005_gb300 import hb
    order = np.argsort([P.dim for P in family])[:2]
    members = [family[i] for i in order]
    B = hb.Batch(members, hb.HB_MIXED)
    B.launch()
    torch.cuda.synchronize()
    for P, b in zip(members, B.blocks):
        o = coracle.Oracle(P)
        R = o.dense()
        cond = o.cc_condition()
        G = hb.dense_from_blocks(b).cpu().numpy()
        Dc = o.Dc
        d = np.abs(G[:Dc, :Dc] - R[:Dc, :Dc])
        assert np.all(d <= 1e-10 * cond), (P.name, (d / np.maximum(cond, 1e-300)).max())
        for blk in (np.s_[Dc:, :Dc], np.s_[Dc:, Dc:]):
            g, r = G[blk], R[blk]
            if r.size:
                assert np.all(np.abs(g - r) <= 1e-12 * np.maximum(np.abs(r), np.abs(r).max())), P.name
        # classes 5 and 6: two groups of the same irrep share a continuum range
        ranges = [(g.cont_first, g.cont_count) for g in P.groups]
        assert len(set(ranges)) < len(ranges)
    B.close()


def test_batch_class4_tensor_cores(family):
    """Class 4 of every group on the tensor cores (class4_path=2) in one
    grouped launch over several Hamiltonians, whose contexts borrow the first
    one's integral slices: identical to building each context on its own, and
    the smallest member within 1e-12 of the oracle's class-4 block."""
    import torch
    from paper_1709_03005_gb300 import hb
    order = np.argsort([P.dim for P in family])
    members = [family[i] for i in order[:4]]
    B = hb.Batch(members, hb.HB_MIXED, class4_path=2)
    B.launch()
    torch.cuda.synchronize()
    assert "class4 tensor cores" in B.report(), B.report()
    for h, b in zip(B.hams, B.blocks):
        ref, _ = h.build(hb.HB_MIXED)
        torch.cuda.synchronize()
        for key in ("Hcc", "Hlc", "row_ptr", "col", "val"):
            assert torch.equal(ref[key], b[key]), key
    P = members[0]
    o = coracle.Oracle(P)
    R = o.dense()
    G = hb.dense_from_blocks(B.blocks[0]).cpu().numpy()
    blk = np.s_[o.Dc:, :o.Dc]
    r = R[blk]
    if r.size:
        assert np.all(np.abs(G[blk] - r) <= 1e-12 * np.maximum(np.abs(r), np.abs(r).max()))
    B.close()
