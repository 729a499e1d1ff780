"""Helpers shared by the GPU parity tests (build through the C ABI, compare with
the oracle)."""
import numpy as np

from oracle import coracle


def gpu_dense(problem, precision=0, **kw):
    import torch
    from paper_1709_03005_gb300 import hb
    H = hb.Hamiltonian(problem, **kw)
    blocks, st = H.build(precision)
    torch.cuda.synchronize()
    D = hb.dense_from_blocks(blocks).cpu().numpy()
    H.close()
    return D, st, blocks


def block_slices(o: coracle.Oracle):
    """(name, row slice, col slice) of the class blocks of the dense matrix."""
    Dc, dim = o.Dc, o.dim
    out = [("cc", slice(0, Dc), slice(0, Dc)), ("l2c", slice(Dc, dim), slice(0, Dc)),
           ("l2", slice(Dc, dim), slice(Dc, dim))]
    return [b for b in out if b[1].stop > b[1].start and b[2].stop > b[2].start]


def assert_blocks_close(G, R, o, rel=1e-12, what=""):
    """|G - R| <= rel * max(|R_ij|, max|R_block|) per element, structural zeros exact."""
    for name, rs, cs in block_slices(o):
        g, r = G[rs, cs], R[rs, cs]
        scale = max(np.abs(r).max(), 1e-300)
        tol = rel * np.maximum(np.abs(r), scale)
        bad = np.abs(g - r) > tol
        assert not bad.any(), (f"{what} block {name}: {bad.sum()} elements off, max |d| "
                               f"{np.abs(g - r).max():.3e} scale {scale:.3e}")
        # exact zeros stay exact zeros
        assert np.all(g[r == 0.0] == 0.0) or name == "cc", f"{what} block {name}: zero pattern differs"
