"""The preconditioner network's CUDA kernels against the FP64 reference
(forward, loss, gradient, Adam), and its use inside hb_diag."""
import numpy as np
import pytest

from oracle import mlp
from paper_1709_03005_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1709_03005_gb300 import build_ext
    build_ext.build()


def _random(seed, n=3000, scale=0.2):
    rng = np.random.default_rng(seed)
    p = rng.normal(0, scale, 4801).astype(np.float32)
    f = rng.normal(0, 1, (n, 8)).astype(np.float32)
    a = rng.normal(0, 1, n).astype(np.float32)
    b = rng.normal(0, 1, n).astype(np.float32)
    return p, f, a, b


def test_forward_and_gradient_match_reference():
    import torch
    from paper_1709_03005_gb300 import hb
    p, f, a, b = _random(0)
    t = lambda x: torch.from_numpy(x).cuda()
    loss, g = hb.mlp_loss_grad(t(p), t(f), t(a), t(b))
    w = hb.mlp_predict(t(p), t(f))
    torch.cuda.synchronize()
    ref_loss, ref_g = mlp.loss_grad(p.astype(np.float64), f.astype(np.float64), a.astype(np.float64),
                                    b.astype(np.float64))
    ref_w = mlp.factor(p.astype(np.float64), f.astype(np.float64))
    np.testing.assert_allclose(w.cpu().numpy(), ref_w, rtol=2e-5, atol=1e-6)
    assert abs(float(loss) - ref_loss) <= 1e-5 * abs(ref_loss)
    g = g.cpu().numpy()
    scale = np.abs(ref_g).max()
    np.testing.assert_allclose(g, ref_g, rtol=1e-3, atol=1e-4 * scale)


def test_adam_step():
    import torch
    from paper_1709_03005_gb300 import hb
    rng = np.random.default_rng(1)
    p = rng.normal(0, 1, 4801).astype(np.float32)
    g = rng.normal(0, 1, 4801).astype(np.float32)
    m = rng.normal(0, 0.1, 4801).astype(np.float32)
    v = np.abs(rng.normal(0, 0.1, 4801)).astype(np.float32)
    tp, tg, tm, tv = (torch.from_numpy(x.copy()).cuda() for x in (p, g, m, v))
    hb.mlp_adam(tp, tg, tm, tv, 3, 1e-2)
    torch.cuda.synchronize()
    m2 = 0.9 * m + 0.1 * g
    v2 = 0.999 * v + 0.001 * g * g
    ref = p - 1e-2 * (m2 / (1 - 0.9 ** 3)) / (np.sqrt(v2 / (1 - 0.999 ** 3)) + 1e-8)
    np.testing.assert_allclose(tp.cpu().numpy(), ref, rtol=1e-5, atol=1e-6)


def test_unit_network_reproduces_plain_davidson():
    """A network whose output is 0 gives w = 1 everywhere: HB_PRECOND_MLP must
    then take exactly the iterations of HB_PRECOND_DIAG."""
    import torch
    from paper_1709_03005_gb300 import hb
    P = synth.make_config("mid")
    H = hb.Hamiltonian(P)
    b, _ = H.build()
    w0, s0, _ = H.diag(b, 8, 1e-8, 300)
    H.set_mlp_params(np.zeros(4801, np.float32))
    w1, s1, _ = H.diag(b, 8, 1e-8, 300, precond=hb.HB_PRECOND_MLP)
    assert s0.iterations == s1.iterations
    np.testing.assert_allclose(w0, w1, atol=1e-9)
    H.close()


def test_train_loop_matches_the_separate_calls():
    """hb_mlp_train is loss-and-gradient plus Adam over consecutive windows
    (wrapping around): the same kernels called one by one give the same bits,
    and the returned loss is the oracle's loss of the last window."""
    import torch
    from paper_1709_03005_gb300 import hb
    p, f, a, b = _random(3, n=2500, scale=0.1)
    t = lambda x: torch.from_numpy(x.copy()).cuda()
    tf, ta, tb = t(f), t(a), t(b)
    pt = t(p)
    last = hb.mlp_train(pt, tf, ta, tb, 1000, 4, 1e-3)
    pr = t(p)
    m = torch.zeros_like(pr)
    v = torch.zeros_like(pr)
    windows = [(0, 1000), (1000, 2000), (2000, 2500), (0, 1000)]
    for step, (lo, hi) in enumerate(windows, 1):
        if step == 4:
            p3 = pr.cpu().numpy().astype(np.float64)
        loss, g = hb.mlp_loss_grad(pr, tf[lo:hi].contiguous(), ta[lo:hi].contiguous(), tb[lo:hi].contiguous())
        hb.mlp_adam(pr, g, m, v, step, 1e-3)
    torch.cuda.synchronize()
    assert torch.equal(pt, pr)
    assert last == float(loss)
    # the loss of the last window at the parameters it was taken at
    ref, _ = mlp.loss_grad(p3, f[:1000].astype(np.float64), a[:1000].astype(np.float64),
                           b[:1000].astype(np.float64))
    assert abs(last - ref) <= 1e-5 * abs(ref)
    assert not np.array_equal(p3, p.astype(np.float64))
    with pytest.raises(hb.HBError):
        hb.mlp_train(pt, tf, ta, tb, 0, 4, 1e-3)
    with pytest.raises(hb.HBError):
        hb.mlp_train(pt, tf, ta, tb, 100, 0, 1e-3)


def _inverse_shift_network():
    """A network whose factor undoes the preconditioning where it matters:
    o = 2 log(|H_ii - theta| + 1e-3) + 3, so w = 256^tanh(o) is below 1/100
    on the rows with |H_ii - theta| < 0.05 and above 100 on those with
    |H_ii - theta| > 0.8 (one hidden unit per layer carries
    f1 = log(|H_ii - theta| + 1e-3); FP16-exact weights)."""
    w1, b1, w2, b2, w3, b3 = (np.zeros(s, np.float32) for s in ((64, 8), (64,), (64, 64), (64,), (64,), (1,)))
    w1[0, 1], b1[0] = 1.0, 10.0          # h1_0 = relu(f1 + 10)
    w2[0, 0] = 1.0                       # h2_0 = h1_0
    w3[0], b3[0] = 2.0, -17.0            # o = 2 f1 + 3
    return np.concatenate([x.ravel() for x in (w1, b1, w2, b2, w3, b3)])


def test_harmful_network_still_converges():
    """A per-row factor cannot push Davidson off its eigenvalues: with factors
    spread over [1/256, 256] against the diagonal correction, the new
    directions are still orthogonalised against the basis, and the solve
    reaches the plain solve's eigenvalues at the same tolerance."""
    from paper_1709_03005_gb300 import hb
    P = synth.make_config("mid")
    H = hb.Hamiltonian(P)
    b, _ = H.build()
    w0, s0, _ = H.diag(b, 8, 1e-8, 400)
    H.set_mlp_params(_inverse_shift_network())
    w1, s1, ok = H.diag(b, 8, 1e-8, 400, precond=hb.HB_PRECOND_MLP)
    print(f"inverse-shift network: {s1.iterations} iterations (plain {s0.iterations}), fallbacks {s1.mlp_fallbacks}")
    assert ok
    np.testing.assert_allclose(w1, w0, atol=1e-8)
    H.close()


def test_stall_check_drops_learned_factor():
    """The stall check: when the largest wanted residual has not fallen by
    2^mlp_stall_log2 over the last mlp_stall_iters iterations, the learned
    factor is dropped for the rest of the solve (counted once in
    mlp_fallbacks).  Asking for a fall of 2^10 over 3 iterations (a plain solve
    falls by about 3 over 3) makes the check fire at the fourth iteration.  The
    network with all parameters zero has w = 256^tanh(0) = 1 exactly, so the
    learned solve and the plain solve take the same steps bit for bit, before
    and after the fallback; with the default check (halved over 10) it never
    fires on this solve."""
    from paper_1709_03005_gb300 import hb
    P = synth.make_config("mid")
    H = hb.Hamiltonian(P, mlp_stall_iters=3, mlp_stall_log2=10)
    b, _ = H.build()
    w0, s0, _ = H.diag(b, 8, 1e-8, 400)
    H.set_mlp_params(np.zeros(4801, np.float32))
    w1, s1, _ = H.diag(b, 8, 1e-8, 400, precond=hb.HB_PRECOND_MLP)
    print(f"identity network, strict stall check: {s1.iterations} iterations (plain {s0.iterations}), "
          f"fallbacks {s1.mlp_fallbacks}")
    assert s0.mlp_fallbacks == 0 and s1.mlp_fallbacks == 1
    assert s1.iterations == s0.iterations
    assert np.array_equal(w1, w0)
    H.close()
    H = hb.Hamiltonian(P)
    b, _ = H.build()
    H.set_mlp_params(np.zeros(4801, np.float32))
    w2, s2, _ = H.diag(b, 8, 1e-8, 400, precond=hb.HB_PRECOND_MLP)
    assert s2.mlp_fallbacks == 0 and s2.iterations == s0.iterations
    assert np.array_equal(w2, w0)
    H.close()
    with pytest.raises(hb.HBError):
        hb.Hamiltonian(P, mlp_stall_iters=-1)


def test_shipped_network_on_held_out_instances():
    """The network trained by precond.py (labels from hb_diag's own solves of
    200 seeded instances) on instances it never saw: the learned solve
    converges to the plain solve's eigenvalues at the same tolerance, and its
    iteration count stays within a quarter of the plain one (the stall check
    bounds the loss).  Both counts are printed: on these matrices a per-row
    factor changes the count by a few percent either way."""
    from paper_1709_03005_gb300 import hb, precond
    params = precond.load_weights()
    cases = [(synth.make_config("c5", n_det=1500, n_co=120, n_state=20, n_l2=3000, seed=55), 100),
             (precond.training_problem(1001), 20), (precond.training_problem(1002), 20)]
    for P, k in cases:
        H, b = precond.built(P)
        i0, t0, w0, _ = precond.timed_diag(H, b, k)
        i1, t1, w1, st = precond.timed_diag(H, b, k, params)
        print(f"{P.name} dim {P.dim} k {k}: plain {i0} iterations {t0:.3f} s, learned {i1} iterations {t1:.3f} s, "
              f"fallbacks {st.mlp_fallbacks}")
        assert i0 > 0 and i1 > 0
        np.testing.assert_allclose(w1, w0, atol=1e-8)
        assert i1 <= 1.25 * i0
        H.close()
