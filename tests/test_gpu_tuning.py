"""Launch shapes of the build plan: every tensor-core tile arrangement and width
and every class-4 shape gives the same bits, each matches the oracle, and the
autotuner (which only chooses among these) never changes the output.  The K
stage of the tensor-core expansion (32 or 64) orders the slice products
differently, which rounds their one inexact accumulator (slice pairs
i + l >= 3) differently: the two agree within the continuum tolerance of the
mixed path (3e-11 of each element's condition scale), and to the bit outside
the continuum block."""
import numpy as np
import pytest

from oracle import coracle
from paper_1709_03005_gb300 import synth

from gpu_util import gpu_dense

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1709_03005_gb300 import build_ext
    build_ext.build()


def _problems():
    # uneven continuum rectangles and tiny state counts, as in
    # the symmetry-blocked workloads, plus the ragged medium case
    return [
        synth.make_tiny(11, n_to=6, n_co=14, n_det=12, n_l2=20, n_groups=3, n_state=[1, 3, 2],
                        cont_ranges=[(0, 7), (3, 9), (5, 4)]),
        synth.make_config("mid"),
        # merged blocks of 78, 63 and 45 columns: several column tiles at width 32
        synth.make_tiny(12, n_to=6, n_co=16, n_det=14, n_l2=10, n_groups=3, n_state=[12, 7, 9],
                        cont_ranges=[(0, 16), (2, 11), (0, 9)]),
    ]


SHAPES = [dict(split_tile=3, split_cols=32, class4_states=8, class4_threads=32),
          dict(split_tile=4, split_cols=64, class4_states=16, class4_threads=64),
          dict(split_tile=5, split_cols=128, class4_states=32, class4_threads=128),
          dict(split_tile=4, split_cols=32, class4_states=4, class4_threads=32),
          dict(split_tile=3, split_cols=64, class4_states=20, class4_threads=64),
          dict(split_tile=5, split_cols=32),
          dict(split_tile=3, split_kstage=32)]
KSTAGE_SHAPES = [dict(split_tile=4, split_cols=128, split_kstage=64), dict(split_kstage=64)]


@pytest.mark.parametrize("idx", [0, 1, 2])
def test_forced_shapes_identical_and_match_oracle(idx):
    P = _problems()[idx]
    ref, _, _ = gpu_dense(P, precision=1)
    o = coracle.Oracle(P)
    R = o.dense()
    cond = o.cc_condition()
    Dc = o.Dc
    for kw in SHAPES + KSTAGE_SHAPES:
        G, _, _ = gpu_dense(P, precision=1, **kw)
        if kw in SHAPES:
            assert np.array_equal(G, ref), kw
        else:
            assert np.array_equal(G[Dc:, :], ref[Dc:, :]) and np.array_equal(G[:, Dc:], ref[:, Dc:]), kw
            assert np.all(np.abs(G[:Dc, :Dc] - ref[:Dc, :Dc]) <= 3e-11 * cond), kw
        d = np.abs(G[:Dc, :Dc] - R[:Dc, :Dc])
        assert np.all(d <= 1e-10 * cond), kw
        for blk in (np.s_[Dc:, :Dc], np.s_[Dc:, Dc:]):
            g, r = G[blk], R[blk]
            if r.size:
                assert np.all(np.abs(g - r) <= 1e-12 * np.maximum(np.abs(r), np.abs(r).max())), kw


def test_autotune_is_bit_identical():
    import torch
    from paper_1709_03005_gb300 import hb
    for P in _problems():
        a = hb.Hamiltonian(P)
        ba, _ = a.build(hb.HB_MIXED)
        t = hb.Hamiltonian(P, autotune=True)
        bt, _ = t.build(hb.HB_MIXED)
        torch.cuda.synchronize()
        for key in ("Hcc", "Hlc", "row_ptr", "col", "val"):
            assert torch.equal(ba[key], bt[key]), (P.name, key)
        rep = t.tuning_report()
        assert rep.startswith("tuned=1"), rep
        assert a.tuning_report().startswith("tuned=0")
        a.close()
        t.close()


def test_invalid_shape_options_rejected():
    from paper_1709_03005_gb300 import hb
    P = _problems()[0]
    for kw in (dict(split_tile=6), dict(split_cols=48), dict(split_cols=256), dict(split_kstage=16),
               dict(class4_states=14), dict(class4_states=36), dict(class4_threads=96),
               dict(class4_path=3),
               dict(class4_path=-1)):
        with pytest.raises(hb.HBError):
            hb.Hamiltonian(P, **kw)


def test_batch_reports_its_choices():
    from paper_1709_03005_gb300 import hb
    fam = synth.make_batched_family(cont_per_irrep=(20, 60))
    members = [fam[i] for i in np.argsort([P.dim for P in fam])[:3]]
    B = hb.Batch(members, hb.HB_MIXED)
    rep = B.report()
    assert rep.startswith("tuned=1") and "split" in rep and "class4" in rep, rep
    B.close()


def test_dump_describes_the_context(tmp_path):
    from paper_1709_03005_gb300 import hb
    P = _problems()[0]
    H = hb.Hamiltonian(P)
    path = tmp_path / "ctx.txt"
    H.dump(path)
    text = path.read_text()
    assert f"dimension {P.dim}" in text and "no build yet" in text
    assert text.count("\ngroup ") == 3
    H.build(hb.HB_MIXED)
    H.dump(path)
    assert "build plan: tuned=0" in path.read_text()
    with pytest.raises(hb.HBError):
        H.dump(tmp_path / "missing" / "ctx.txt")
    H.close()
