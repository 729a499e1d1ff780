"""Caller-owned workspace through the C ABI (hb_workspace_size,
hb_set_workspace): after hb_init, builds and Davidson solves take their
device memory from the caller's buffer.  Checked: the results are bit for bit
those of a context without a workspace, the device's free memory does not
move across builds and solves, a workspace too small for the set-up is
reported as HB_ERR_OOM, and the context-based training call runs in it."""
import numpy as np
import pytest

from paper_1709_03005_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1709_03005_gb300 import build_ext
    build_ext.build()


@pytest.mark.parametrize("key,precision,k", [("c2", 1, 20), ("mid", 0, 8)])
def test_workspace_build_and_solve(key, precision, k):
    import torch
    from paper_1709_03005_gb300 import hb
    P = synth.make_config(key)
    flags = hb.HB_PRECOND_DIAG | (hb.HB_DIAG_TENSOR if precision == 1 else 0)
    # the reference: the same calls on a context without a workspace (this
    # also loads every kernel the calls below launch)
    H1 = hb.Hamiltonian(P)
    ref, _ = H1.build(precision)
    X1 = torch.zeros((H1.dim, k), dtype=torch.float64, device="cuda")
    ev1, _, _ = H1.diag(ref, k, 1e-8, 400, precond=flags, evecs=X1)
    torch.cuda.synchronize()

    H2 = hb.Hamiltonian(P)
    need = H2.workspace_size(precision, k, flags)
    assert need == H2.layout.workspace_bytes > 0
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    H2.set_workspace(ws)
    out = H2.allocate()
    X2 = torch.zeros((H2.dim, k), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        H2.build(precision, out)
        ev2, _, _ = H2.diag(out, k, 1e-8, 400, precond=flags, evecs=X2)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    print(f"{key}: workspace {need / 2**20:.1f} MiB, device free memory moved by {free0 - free1} bytes")
    assert free1 == free0
    for name in ("Hcc", "Hlc", "row_ptr", "col", "val"):
        assert torch.equal(ref[name], out[name]), name
    assert np.array_equal(ev1, ev2)
    assert torch.equal(X1, X2)
    H1.close()
    H2.close()


def test_workspace_too_small():
    import torch
    from paper_1709_03005_gb300 import hb
    H = hb.Hamiltonian(synth.make_config("mid"))
    need = H.workspace_size(hb.HB_MIXED)
    ws = torch.empty(need // 8, dtype=torch.uint8, device="cuda")
    H.set_workspace(ws)
    with pytest.raises(hb.HBError) as e:
        H.build(hb.HB_MIXED)
    assert e.value.code == hb.HB_ERR_OOM
    with pytest.raises(hb.HBError):
        H.set_workspace(ws)          # one workspace per context
    H.close()


def test_mlp_training_in_the_workspace():
    """hb_mlp_train with the context's memory: its scratch fits the workspace
    measured for a solve with the learned factor, the result is that of the
    context-free loop, and the network becomes the context's."""
    import torch
    from paper_1709_03005_gb300 import hb
    P = synth.make_config("mid")
    H = hb.Hamiltonian(P)
    need = H.workspace_size(hb.HB_MIXED, 8, hb.HB_PRECOND_MLP)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    H.set_workspace(ws)
    rng = np.random.default_rng(0)
    n = 5000
    feats = torch.tensor(rng.standard_normal((n, 8)), dtype=torch.float32, device="cuda")
    a = torch.tensor(rng.standard_normal(n), dtype=torch.float32, device="cuda")
    b = (0.8 * a).contiguous()
    p0 = torch.tensor(0.05 * rng.standard_normal(hb.mlp_param_count()), dtype=torch.float32, device="cuda")
    p1, p2 = p0.clone(), p0.clone()
    st = hb.mlp_train_ctx(H, p1, feats, a, b, 1000, 20, 1e-3)
    last = hb.mlp_train(p2, feats, a, b, 1000, 20, 1e-3)
    torch.cuda.synchronize()
    assert torch.equal(p1, p2)
    assert st.mlp_loss == pytest.approx(last, rel=0, abs=0)
    blocks, _ = H.build(hb.HB_MIXED)
    ev, dst, ok = H.diag(blocks, 8, 1e-8, 400, precond=hb.HB_PRECOND_MLP, allow_not_converged=True)
    assert ok or dst.mlp_fallbacks > 0
    H.close()
