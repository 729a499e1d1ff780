"""Training data and training of the learned Davidson preconditioner.

    python -m paper_1709_03005_gb300.precond train [--instances 24] [--out FILE]
    python -m paper_1709_03005_gb300.precond evaluate
    python -m paper_1709_03005_gb300.precond large [--k 200]    # the 60000-dimensional workload

Data: plain (diagonal-preconditioned) block Davidson runs on seeded smaller
Hamiltonians of the same families as the workloads, each built by this
library.  At every iteration and for every unconverged Ritz pair j the sample
rows are the library's features f_i (hb_diag_features), a_i = the diagonal
correction r_i / (H_ii - theta_j) and b_i = the exact correction: the part of
the true eigenvector (dense eigensolver, aligned in sign) outside the current
basis.  Both are normalised per pair, so the network learns a row-wise factor
that turns the diagonal correction towards the exact one.

Training: Adam on mean_i (w(f_i) a_i - b_i)^2 with the library's forward,
backward and update kernels (hb_mlp_loss_grad, hb_mlp_adam).  The result is
saved as an .npz of the packed parameters and loaded with
hb.Hamiltonian.set_mlp.
"""
from __future__ import annotations

import argparse
import os

import numpy as np

from . import hb, synth

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "data", "precond_mlp.npz")


def training_problem(seed: int):
    """A seeded smaller instance of the medium / precision families."""
    rng = np.random.default_rng(10_000 + seed)
    n_to = int(rng.integers(12, 21))
    n_elec = int(rng.choice([6, 8]))
    n_co = int(rng.integers(30, 81))
    n_det = int(rng.integers(150, 401))
    n_state = int(rng.integers(4, 11))
    n_l2 = int(rng.integers(300, 1201))
    cont = (-3.0, -0.5) if seed % 2 == 0 else (0.0, 50.0)
    return synth.make_problem(f"train{seed}", 20_000 + seed, n_to, n_co, n_elec, n_det, n_state, n_l2,
                              rank=int(rng.integers(20, 41)), cont_diag=cont)


def davidson_samples(problem, k, max_iter=200, tol=1e-8, max_pairs_per_iter=8):
    """Run a plain block Davidson (the same method as hb_diag) in FP64 torch on
    the library-built matrix and return float32 device tensors (f, a, b)."""
    import torch
    H = hb.Hamiltonian(problem)
    blocks, _ = H.build(hb.HB_MIXED)
    D = hb.dense_from_blocks(blocks)
    n = D.shape[0]
    lam, Xs = torch.linalg.eigh(D)
    d = torch.diagonal(D).clone()
    b = min(n, k + max(4, min(16, k // 2)))
    mmax = min(n, max(5 * b, k + 4 * b))
    idx = torch.argsort(d, stable=True)[:b]
    V = torch.zeros((n, b), dtype=torch.float64, device=D.device)
    V[idx, torch.arange(b, device=D.device)] = 1.0
    AV = D @ V
    fs, As, Bs = [], [], []
    for it in range(max_iter):
        T = V.T @ AV
        T = 0.5 * (T + T.T)
        theta, S = torch.linalg.eigh(T)
        nr = min(V.shape[1], b)
        X = V @ S[:, :nr]
        R = AV @ S[:, :nr] - X * theta[:nr]
        res = torch.linalg.norm(R, dim=0)
        if bool((res[:k] <= tol).all()):
            break
        which = [j for j in range(nr) if res[j] > tol][:b]
        feats = hb.diag_features(H, blocks, theta[:nr].cpu().numpy())       # [nr, n, 8]
        for j in which[:max_pairs_per_iter]:
            den = d - theta[j]
            den = torch.where(den.abs() < 1e-4, torch.where(den < 0, -1e-4, 1e-4), den)
            a = R[:, j] / den
            xs = Xs[:, j] * torch.sign(Xs[:, j] @ X[:, j])
            e = xs - V @ (V.T @ xs)
            na, ne = torch.linalg.norm(a), torch.linalg.norm(e)
            if na < 1e-30 or ne < 1e-30:
                continue
            a, e = a / na, e / ne
            e = e * torch.sign(a @ e)
            fs.append(feats[j]); As.append(a.float()); Bs.append(e.float())
        if V.shape[1] + len(which) > mmax:
            keep = min(V.shape[1], 2 * b, mmax - len(which))
            V, AV = V @ S[:, :keep], AV @ S[:, :keep]
        den = d[:, None] - theta[which][None, :]
        den = torch.where(den.abs() < 1e-4, torch.where(den < 0, -1e-4, 1e-4), den)
        Tn = R[:, which] / den
        for _ in range(2):
            Tn = Tn - V @ (V.T @ Tn)
        Q, Rq = torch.linalg.qr(Tn)
        keep = Rq.diagonal().abs() > 1e-10 * max(1.0, float(Rq.diagonal().abs().max()))
        Q = Q[:, keep]
        Q = Q - V @ (V.T @ Q)
        Q, _ = torch.linalg.qr(Q)
        V = torch.cat([V, Q], 1)
        AV = torch.cat([AV, D @ Q], 1)
    H.close()
    if not fs:
        return None
    return torch.cat(fs), torch.cat(As), torch.cat(Bs), it + 1


def train(n_instances=24, steps=3000, lr=2e-3, batch=1 << 18, seed=0, log=print):
    import torch
    torch.manual_seed(seed)
    F, A, B = [], [], []
    for s in range(n_instances):
        P = training_problem(s)
        k = [8, 12, 20][s % 3]
        out = davidson_samples(P, k)
        if out is None:
            continue
        f, a, b, iters = out
        F.append(f); A.append(a); B.append(b)
        log(f"instance {s}: dim {P.dim}, k {k}, {iters} plain iterations, {f.shape[0]} samples")
    F, A, B = torch.cat(F).contiguous(), torch.cat(A).contiguous(), torch.cat(B).contiguous()
    n = F.shape[0]
    npar = hb.mlp_param_count()
    rng = np.random.default_rng(seed)
    # small initial weights: the network starts close to w = 1 (plain Davidson)
    p0 = rng.normal(0.0, 0.05, npar).astype(np.float32)
    p0[-1] = 0.0
    params = torch.from_numpy(p0).cuda()
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    work = torch.empty(hb._mlp_fns().hb_mlp_workspace_bytes(min(n, batch)), dtype=torch.uint8, device="cuda")
    gen = torch.Generator(device="cuda").manual_seed(seed)
    base, _ = hb.mlp_loss_grad(params, F[: min(n, batch)], A[: min(n, batch)], B[: min(n, batch)], work)
    for step in range(1, steps + 1):
        sel = torch.randint(0, n, (min(n, batch),), device="cuda", generator=gen)
        loss, g = hb.mlp_loss_grad(params, F[sel].contiguous(), A[sel].contiguous(), B[sel].contiguous(), work)
        hb.mlp_adam(params, g, m, v, step, lr)
        if step % 500 == 0 or step == 1:
            log(f"step {step}: loss {float(loss):.6e}")
    torch.cuda.synchronize()
    return params.cpu().numpy(), float(base), float(loss), n


def ab_compare(params, problems, k, tol=1e-8, max_iter=1000):
    """Plain vs learned preconditioner on the same built matrices:
    [(name, iterations_diag, seconds_diag, iterations_mlp, seconds_mlp, max |d eval|)]."""
    import time

    import torch
    out = []
    for P in problems:
        H = hb.Hamiltonian(P)
        b, _ = H.build(hb.HB_MIXED)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        w0, s0, ok0 = H.diag(b, k, tol, max_iter, allow_not_converged=True)
        t1 = time.perf_counter()
        H.set_mlp_params(params)
        w1, s1, ok1 = H.diag(b, k, tol, max_iter, precond=hb.HB_PRECOND_MLP, allow_not_converged=True)
        t2 = time.perf_counter()
        out.append((P.name, s0.iterations if ok0 else -1, t1 - t0, s1.iterations if ok1 else -1, t2 - t1,
                    float(np.abs(w0 - w1).max())))
        H.close()
    return out


def load_weights(path=DEFAULT_WEIGHTS):
    """Packed parameters of a trained network."""
    return np.load(path)["params"]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("cmd", choices=["train", "evaluate", "large"])
    ap.add_argument("--k", type=int, default=200)
    ap.add_argument("--instances", type=int, default=24)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    args = ap.parse_args()
    from . import build_ext
    build_ext.build()
    if args.cmd == "large":
        # lowest k eigenpairs of the 60000-dimensional precision-family
        # Hamiltonian, block products on the tensor cores, plain vs learned
        import time

        import torch
        P = synth.make_config("c5")
        H = hb.Hamiltonian(P, validate=False)
        b, st = H.build(hb.HB_MIXED)
        torch.cuda.synchronize()
        print(f"{P.name}: dim {P.dim}, build {st.ms_total:.1f} ms", flush=True)
        params = load_weights(args.out)
        H.set_mlp_params(params)
        for name, pc in (("diag", hb.HB_PRECOND_DIAG), ("mlp", hb.HB_PRECOND_MLP)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            w, dst, ok = H.diag(b, args.k, 1e-8, 400, precond=pc | hb.HB_DIAG_TENSOR, allow_not_converged=True)
            torch.cuda.synchronize()
            print(f"{name:5s} k={args.k}: {dst.iterations} iterations, {time.perf_counter() - t0:.1f} s, "
                  f"converged {ok}, max residual {dst.max_residual:.2e}, products {dst.ms_matvec / 1e3:.1f} s, "
                  f"small eigenproblems {dst.ms_rr / 1e3:.1f} s, projections {dst.ms_gram / 1e3:.1f} s, "
                  f"lowest {w[0]:.10f} highest wanted {w[-1]:.10f}", flush=True)
        H.close()
        return
    if args.cmd == "evaluate":
        params = load_weights(args.out)
        probs = [training_problem(1000 + s) for s in range(4)] + [synth.make_config("c2")]
        for row in ab_compare(params, probs, 20):
            print("%-14s diag %4d it %7.3f s | mlp %4d it %7.3f s | max |d eval| %.1e" % row)
        return
    p, l0, l1, n = train(args.instances, args.steps)
    os.makedirs(os.path.dirname(args.out), exist_ok=True)
    np.savez(args.out, params=p, n_samples=n, loss_start=l0, loss_end=l1, instances=args.instances,
             steps=args.steps)
    print(f"saved {args.out}: {n} samples, loss {l0:.4e} -> {l1:.4e}")


if __name__ == "__main__":
    main()
