"""Both build paths and hb_diag against the stored values of
tests/golden/c1_tiny.txt (oracle values; see tests/golden/make_golden.py):
every stored element within the element criterion of tests/gpu_util.py
(FP64: 1e-12, mixed: 1e-10 relative, with the oracle's condition scales), the
lowest ten eigenvalues within 1e-8 Hartree."""
import numpy as np
import pytest

from golden_io import read
from gpu_util import gpu_dense
from oracle import coracle
from paper_1709_03005_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [0, 1])
def test_build_matches_golden(precision):
    from paper_1709_03005_gb300 import build_ext, hb
    build_ext.build()
    exc, elem, evals = read()
    P = synth.make_config("c1")
    G, _, _ = gpu_dense(P, precision=precision)
    cond = coracle.Oracle(P).condition()
    rel = 1e-10 if precision else 1e-12
    scale = np.abs(G).max()
    for i, j, v in elem:
        tol = rel * max(abs(v), 1e-6 * scale, cond[i, j])
        assert abs(G[i, j] - v) <= tol, (i, j, G[i, j], v)
    H = hb.Hamiltonian(P)
    b, _ = H.build(precision)
    w, st, ok = H.diag(b, 10, 1e-9, 300)
    H.close()
    np.testing.assert_allclose(w, evals[:10], rtol=0, atol=1e-8)
