"""The allocation-free classification entry point (hb_classify_noalloc).

It serves callers that cannot allocate device memory (a framework that owns the
allocator, a plug-in that may not call cudaMalloc, a real-time loop), so its row
offsets live in the library's static device buffer instead of a caller buffer.
This test calls it through the C ABI and checks that its records equal those of
hb_classify on two calls in a row: a large call first, then a smaller one that
runs over the first call's leftovers in the shared buffer.  The file is named
to be collected last so that a failure here never hides the other tests.
"""
import numpy as np
import pytest

from paper_1709_03005_gb300 import synth

pytestmark = pytest.mark.gpu


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, np.uint64).view(np.int64)).cuda()


def test_noalloc_matches_classify_on_two_calls():
    import torch
    from paper_1709_03005_gb300 import build_ext, hb
    build_ext.build()
    big = synth.make_config("mid")
    small = synth.make_tiny(77, n_to=8, n_elec=4, n_det=30, n_l2=40)
    calls = [(big.l2_dets, big.l2_dets, big.n_words, 0, 0),
             (small.l2_dets, small.groups[0].dets, small.n_words, 1, 0)]
    for a_np, b_np, W, mode, spin in calls:
        a, b = _dev(a_np), _dev(b_np)
        rp, ref = hb.classify(a, b, W, mode, spin, 2)
        out = torch.zeros(max(len(ref), 1) * hb.PAIR_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        n, got = hb.classify_noalloc(a, b, W, mode, spin, 2, pairs=out)
        assert n == len(ref) > 0
        assert got.tobytes() == ref.tobytes()


def test_noalloc_rejects_oversized_input():
    import torch
    from paper_1709_03005_gb300 import hb
    rows = hb.HB_NOALLOC_MAX_ROWS + 1
    a = torch.zeros((rows, 2), dtype=torch.int64, device="cuda")
    out = torch.zeros(24, dtype=torch.uint8, device="cuda")
    with pytest.raises(hb.HBError) as e:
        hb.classify_noalloc(a, a[:1], 1, pairs=out)
    assert e.value.code == hb.HB_ERR_INVALID_ARG and "exceeds" in str(e.value)
