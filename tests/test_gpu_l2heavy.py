"""The L2-heavy regime: the shape of the paper's H3PO4 run (Section 4.1),
contracted dimension 712 (8 target states x 89 continuum orbitals) and 122103
L2 functions, dimension 122815, with about 3.8e8 entries in the L2 x L2 CSR
block.  The mixed build is checked on sampled elements of every class against
the oracle; the lowest 20 eigenpairs come from hb_diag with both product paths
(the L2 block is a CSR product in FP64 on both), and every returned pair's
residual is recomputed on the CPU with the oracle's own matrix: its L2 CSR,
its class-4 rows and its continuum block."""
import numpy as np
import pytest

from oracle import coracle
from paper_1709_03005_gb300 import synth

from gpu_util import sampled_checks

pytestmark = pytest.mark.gpu


def test_l2_heavy_build_and_davidson():
    import scipy.sparse as sp
    import torch
    from paper_1709_03005_gb300 import build_ext, hb
    build_ext.build()
    P = synth.make_config("h3po4")
    o = coracle.Oracle(P)
    cc = o.contract(0, 0)
    H = hb.Hamiltonian(P, validate=False)
    assert H.dim == 122815 and H.contracted_dim == 712
    b, st = H.build(hb.HB_MIXED)
    torch.cuda.synchronize()
    print(f"h3po4 shape: L2 nnz {H.layout.l2_nnz:.3e}, mixed build {st.ms_total:.2f} ms")
    sampled_checks(P, o, cc, b, np.random.default_rng(7), 1, n_cc=1000, n_rows=8, what="h3po4 mixed")

    # the oracle's matrix, block by block (its dense form would be 15e9 entries)
    nl, Dc = P.n_l2, o.Dc
    rp, cols, vals = o.l2_csr()
    np.testing.assert_array_equal(b["row_ptr"].cpu().numpy(), rp)
    L = sp.csr_matrix((vals, cols, rp), shape=(nl, nl))
    C4 = o.class4_rows(0, nl)
    Hcc = o.cc_block(0, 0)

    def apply(X):
        Xc, Xl = X[:Dc], X[Dc:]
        return np.vstack([Hcc @ Xc + C4.T @ Xl, C4 @ Xc + L @ Xl])

    k = 20
    import time
    out = {}
    for flags, name in ((hb.HB_DIAG_TENSOR, "tensor-core products"), (0, "FP64 products")):
        X = torch.zeros((H.dim, k), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ev, dst, ok = H.diag(b, k, 1e-8, 400, precond=hb.HB_PRECOND_DIAG | flags, evecs=X)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        Xh = X.cpu().numpy()
        res = np.linalg.norm(apply(Xh) - Xh * ev, axis=0)
        out[name] = (ev, ok, Xh, res)
        print(f"h3po4 Davidson ({name}): converged {ok}, {dst.iterations} iterations ({dst.fp64_iterations} with FP64 products after the check), {dt:.2f} s, products "
              f"{dst.ms_matvec:.0f} ms, reported residual {dst.max_residual:.2e}, residual against the oracle's "
              f"matrix {res.max():.2e}")
    for name, (ev, ok, Xh, res) in out.items():
        assert ok, name
        np.testing.assert_allclose(Xh.T @ Xh, np.eye(k), atol=1e-10)
        # the residual bound holds with the oracle's matrix too, up to the
        # difference between the two matrices (about 1e-12 of each element)
        assert res.max() <= 1.5e-8, (name, res.max())
        assert np.all(np.diff(ev) >= -1e-12)
    np.testing.assert_allclose(out["FP64 products"][0], out["tensor-core products"][0], rtol=0, atol=1e-8)
    H.close()
