"""Batched build of the 16 symmetry / spin-coupling Hamiltonians of one
molecule (shared integrals, orbital symmetry, one CUDA-graph launch):
identical to building each context on its own, the two smallest members
against the oracle's whole matrix, and every member on sampled elements.
The full workload (50-400 continuum orbitals per irrep, 2513 in all: 121 GB
of dense integrals) is staged once for the module; the class-4 tensor-core
variant runs on the same family with 20-60 continuum orbitals per irrep."""
import numpy as np
import pytest

from oracle import coracle
from paper_1709_03005_gb300 import synth

from gpu_util import FP64_FALLBACK, MIXED_C4_FALLBACK, MIXED_C4_TC_ABS, MIXED_CC_FALLBACK, check_elements

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def family():
    from paper_1709_03005_gb300 import build_ext
    build_ext.build()
    return synth.make_batched_family()


@pytest.fixture(scope="module")
def batch(family):
    """The mixed batch of the whole family, launched once."""
    import torch
    from paper_1709_03005_gb300 import hb
    B = hb.Batch(family, hb.HB_MIXED)
    st = B.launch()
    torch.cuda.synchronize()
    yield B, st
    B.close()


def test_batch_equals_individual_builds(batch):
    import torch
    from paper_1709_03005_gb300 import hb
    B, st = batch
    assert B.nodes > len(B.hams)
    for h, b in zip(B.hams, B.blocks):
        ref, _ = h.build(hb.HB_MIXED)
        torch.cuda.synchronize()
        for key in ("Hcc", "Hlc", "row_ptr", "col", "val"):
            assert torch.equal(ref[key], b[key]), key
    print(f"batched build: {len(B.hams)} Hamiltonians, {B.positions:.3e} positions, {st.ms_total:.2f} ms, "
          f"{B.nodes} graph nodes")


def test_batch_members_match_oracle(family, batch):
    from paper_1709_03005_gb300 import hb
    B, _ = batch
    order = np.argsort([P.dim for P in family])[:2]
    from gpu_util import assert_blocks_close
    for i in order:
        P, b = family[i], B.blocks[i]
        o = coracle.Oracle(P)
        R = o.dense()
        G = hb.dense_from_blocks(b).cpu().numpy()
        assert_blocks_close(G, R, o, 1e-10, P.name, mixed=True)
        # classes 5 and 6: two groups of the same irrep share a continuum range
        ranges = [(g.cont_first, g.cont_count) for g in P.groups]
        assert len(set(ranges)) < len(ranges)


def test_batch_class4_tensor_cores():
    """Class 4 of every group on the tensor cores (class4_path=2) in one
    grouped launch over several Hamiltonians, whose contexts borrow the first
    one's integral slices: identical to building each context on its own, and
    the smallest member within 1e-12 of the oracle's class-4 block."""
    import torch
    from paper_1709_03005_gb300 import hb
    small = synth.make_batched_family(cont_per_irrep=(20, 60))
    order = np.argsort([P.dim for P in small])
    members = [small[i] for i in order[:4]]
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
    if R[blk].size:
        check_elements(G[blk], R[blk], o.condition()[blk], 1e-10, MIXED_C4_FALLBACK, "class 4 tensor cores",
                       abs_frac=MIXED_C4_TC_ABS)
    B.close()


def test_batch_every_member_sampled(family, batch):
    """Every one of the 16 Hamiltonians of the batched build against the
    oracle: sampled continuum elements over random group pairs, whole class-4
    rows and whole L2 rows."""
    from paper_1709_03005_gb300 import hb
    B, _ = batch
    rng = np.random.default_rng(44)
    for P, H, b in zip(family, B.hams, B.blocks):
        o = coracle.Oracle(P)
        Hcc = b["Hcc"].cpu().numpy()
        ng = len(P.groups)
        ref, cond, got = [], [], []
        for _ in range(10):
            g, gp = sorted(rng.integers(0, ng, 2).tolist(), reverse=True)
            cc = o.contract(g, gp)
            G, Gp = P.groups[g], P.groups[gp]
            for _ in range(20):
                n, n_ = int(rng.integers(G.ci.shape[1])), int(rng.integers(Gp.ci.shape[1]))
                jj, jjp = int(rng.integers(G.cont_count)), int(rng.integers(Gp.cont_count))
                t = (n, G.cont_first + jj, n_, Gp.cont_first + jjp)
                ref.append(cc.element(*t))
                cond.append(cc.element_cond(*t))
                got.append(Hcc[H.group_offsets[g] + n * G.cont_count + jj, H.group_offsets[gp] + n_ * Gp.cont_count + jjp])
            del cc
        check_elements(np.array(got), np.array(ref), np.array(cond), 1e-10, MIXED_CC_FALLBACK, f"{P.name} cc",
                       blockmax=np.abs(Hcc).max())
        if P.n_l2:
            rows = np.sort(rng.choice(P.n_l2, min(4, P.n_l2), replace=False))
            Hlc = b["Hlc"].cpu().numpy()
            for l in rows:
                check_elements(Hlc[l], o.class4_row(int(l)), o.class4_rows_abs(int(l), int(l) + 1)[0], 1e-10,
                               MIXED_C4_FALLBACK, f"{P.name} class 4 row {l}", blockmax=np.abs(Hlc).max(),
                               abs_frac=MIXED_C4_TC_ABS)
            rp = b["row_ptr"].cpu().numpy()
            for a in rows:
                row = o.l2_rows(int(a), int(a) + 1)[0]
                dense = np.zeros(P.n_l2)
                dense[b["col"][rp[a]:rp[a + 1]].cpu().numpy()] = b["val"][rp[a]:rp[a + 1]].cpu().numpy()
                check_elements(dense, row, o.l2_rows_abs(int(a), int(a) + 1)[0], 1e-12, FP64_FALLBACK,
                               f"{P.name} L2 row {a}")
