"""The sharded build's host orchestration over two processes on CPU (gloo).

hb.sharded_build runs, on every rank, the contraction over the rank's bra
determinants, an all-reduce (sum) of the partial coefficient rows, and the
rank's share of the expansion.  Here the device calls are replaced by a CPU
stand-in with the same contract (the GPU kernels are checked rank by rank in
test_gpu_shard.py), and the all-reduce is torch.distributed over gloo: every
rank must receive the same reduced rows, bit for bit, equal to the sum of the
partials in rank order, and the ranks' outputs must add up to the one-rank
result with every element written once."""
import os
import socket
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class _CpuShard:
    """A contraction sum_m C[m]^T W[m] split over the rows m, and an
    'expansion' out[t] = f(reduced)[t] whose tiles t go to the ranks in turn."""

    def __init__(self, seed=0, rows=103, cols=6, tiles=17):
        rng = np.random.default_rng(seed)
        self.C = rng.standard_normal((rows, cols))
        self.Wm = rng.standard_normal((rows, cols))
        self.tiles = tiles
        self.seen = None

    def build_contract(self, precision, rank, nranks, stream=None):
        import torch
        n = self.C.shape[0]
        m0, m1 = n * rank // nranks, n * (rank + 1) // nranks
        part = (self.C[m0:m1].T @ self.Wm[m0:m1]).ravel()
        return torch.from_numpy(part.copy()), None

    def build_expand(self, precision, rank, nranks, reduced, blocks=None, stream=None):
        import torch
        self.seen = reduced.numpy().copy()
        out = torch.full((self.tiles,), float("nan"), dtype=torch.float64)
        for t in range(rank, self.tiles, nranks):
            out[t] = float(np.cos(t) * reduced.numpy().sum())
        return {"out": out}, None


def _rank_main(rank, world, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1709_03005_gb300 import hb
    H = _CpuShard()
    out = hb.sharded_build(H, 0, rank, world, lambda t: dist.all_reduce(t, op=dist.ReduceOp.SUM))
    q.put((rank, H.seen, out["out"].numpy()))
    dist.destroy_process_group()


def test_sharded_build_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=120) for _ in procs], key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref = _CpuShard()
    parts = [ref.build_contract(0, r, 2)[0].numpy() for r in range(2)]
    full_order = parts[0] + parts[1]
    # every rank holds the same reduced rows, the partial sums added in rank order
    assert np.array_equal(res[0][1], res[1][1])
    assert np.array_equal(res[0][1], full_order)
    # ... which equal the one-rank contraction up to the rounding of that order
    one = (ref.C.T @ ref.Wm).ravel()
    assert np.allclose(res[0][1], one, rtol=0, atol=1e-12 * np.abs(one).max())
    # the outputs: every tile written by exactly one rank, together the whole result
    written = [~np.isnan(r[2]) for r in res]
    assert np.array_equal(written[0] ^ written[1], np.ones(ref.tiles, bool))
    merged = np.where(written[0], res[0][2], res[1][2])
    expect = np.cos(np.arange(ref.tiles)) * full_order.sum()
    assert np.array_equal(merged, expect)
