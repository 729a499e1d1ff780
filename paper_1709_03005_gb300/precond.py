"""Training data and training of the learned Davidson preconditioner.

    python -m paper_1709_03005_gb300.precond train [--instances 200] [--out FILE]
    python -m paper_1709_03005_gb300.precond evaluate
    python -m paper_1709_03005_gb300.precond large [--k 200]    # the 60000-dimensional workload

hb_diag with HB_PRECOND_MLP multiplies the diagonal correction of row i by a
factor w(f_i) of the row's features.  The factor's label comes from solves of
the method's own Hamiltonians by hb_diag itself:

1. candidates: shifted denominators w_delta(d) = |d| / (|d| + delta) of
   d = H_ii - theta, which damp the rows whose diagonal is close to the Ritz
   value; each is fitted by a network on real feature rows (hb_mlp_train_params
   with a = 1, b = w_delta, so the loss is (w - w_delta)^2);
2. every training instance (seeded, both Hamiltonian families, dimensions
   about 1500-9000) is solved by hb_diag plain and with each candidate
   network; the candidate with the fewest iterations labels the instance when
   it saves at least ROBUST of them (iteration counts move by one or two with
   any change of the correction, so a smaller saving is not a signal), else
   the instance is labelled plain, w = 1;
3. samples: the features of the instance's rows at the Ritz values of its
   plain solve, each labelled with the instance's factor;
4. the final network is trained on all samples with the library's forward,
   backward and Adam kernels (hb_mlp_loss_grad, hb_mlp_adam).

The result is saved as an .npz of the packed parameters and loaded with
hb.Hamiltonian.set_mlp_params.
"""
from __future__ import annotations

import argparse
import os
import time

import numpy as np

from . import hb, synth

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "data", "precond_mlp.npz")
DELTAS = (0.03, 0.1, 0.3, 1.0)
ROBUST = 3


def training_problem(seed: int):
    """A seeded smaller instance of the medium (even seeds) or precision (odd
    seeds) families: 20-40 target orbitals, 50-200 continuum orbitals, 5-20
    target states, 1000-5000 L2 functions."""
    rng = np.random.default_rng(10_000 + seed)
    n_to = int(rng.integers(20, 41))
    n_elec = int(rng.choice([6, 8]))
    n_co = int(rng.integers(50, 201))
    n_state = int(rng.integers(5, 21))
    n_det = int(rng.integers(max(n_state + 50, 300), 1501))
    n_l2 = int(rng.integers(1000, 5001))
    cont = (-3.0, -0.5) if seed % 2 == 0 else (0.0, 50.0)
    return synth.make_problem(f"train{seed}", 20_000 + seed, n_to, n_co, n_elec, n_det, n_state, n_l2,
                              rank=int(rng.integers(20, 61)), cont_diag=cont)


def _features_at(H, blocks, theta, rows, rng):
    """Feature rows (device float32) of `rows` random matrix rows at each Ritz value."""
    import torch
    f = hb.diag_features(H, blocks, np.asarray(theta))                 # [q, n, 8]
    sel = torch.from_numpy(rng.choice(H.dim, min(rows, H.dim), replace=False)).cuda()
    return f[:, sel, :].reshape(-1, hb.MLP_IN).contiguous()


def shifted_factor(feats, delta):
    """w_delta = |d| / (|d| + delta) from the first feature (d / 10 Eh)."""
    d = (feats[:, 0] * 10.0).abs()
    return (d / (d + delta)).contiguous()


def fit(feats, target, steps=3000, lr=2e-3, batch=1 << 16, seed=0, init=None):
    """Network parameters whose factor fits `target` on `feats` (loss (w - t)^2)."""
    import torch
    n = feats.shape[0]
    rng = np.random.default_rng(seed)
    if init is None:
        p0 = rng.normal(0.0, 0.05, hb.mlp_param_count()).astype(np.float32)
        p0[-1] = 0.0                 # starts near w = 1
    else:
        p0 = np.asarray(init, np.float32).copy()
    params = torch.from_numpy(p0).cuda()
    perm = torch.from_numpy(rng.permutation(n)).cuda()
    F, B = feats[perm].contiguous(), target[perm].contiguous()
    A = torch.ones_like(B)
    loss = hb.mlp_train(params, F, A, B, min(batch, n), steps, lr)
    return params, loss


def timed_diag(H, b, k, params=None, tol=1e-8, max_iter=400, tensor=True):
    """(iterations or -1, seconds, eigenvalues, stats) of one hb_diag solve,
    plain or with the network `params`."""
    import torch
    flags = hb.HB_DIAG_TENSOR if tensor else 0
    pc = hb.HB_PRECOND_DIAG
    if params is not None:
        H.set_mlp_params(params)
        pc = hb.HB_PRECOND_MLP
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    w, st, ok = H.diag(b, k, tol, max_iter, precond=pc | flags, allow_not_converged=True)
    torch.cuda.synchronize()
    return (st.iterations if ok else -1), time.perf_counter() - t0, w, st


def built(P):
    import torch
    H = hb.Hamiltonian(P, validate=False)
    b, _ = H.build(hb.HB_MIXED)
    torch.cuda.synchronize()
    return H, b


def train(n_instances=200, steps=4000, lr=2e-3, seed=0, log=print):
    """The pipeline of the module docstring; returns (params, info)."""
    import torch
    rng = np.random.default_rng(seed)
    # 1. candidate networks, fitted on feature rows of a few instances
    pool = []
    for s in range(6):
        H, b = built(training_problem(90_000 + s))
        _, _, w, _ = timed_diag(H, b, 12)
        pool.append(_features_at(H, b, w, 2000, rng))
        H.close()
    pool = torch.cat(pool)
    cands = {}
    for dl in DELTAS:
        prm, l = fit(pool, shifted_factor(pool, dl), steps=2000, seed=seed)
        cands[dl] = prm.cpu().numpy()
        log(f"candidate delta {dl}: fit loss {l:.3e}")
    # 2-3. label every instance by its best candidate, sample its feature rows
    F, T, labels = [], [], []
    for s in range(n_instances):
        P = training_problem(s)
        k = [8, 20, 40][s % 3]
        H, b = built(P)
        it0, _, w0, _ = timed_diag(H, b, k)
        if it0 < 0:
            H.close()
            continue
        feats = _features_at(H, b, w0, 1500, rng)
        best, best_it, its = None, it0 - ROBUST + 1, {}
        for dl, prm in cands.items():
            it, _, _, _ = timed_diag(H, b, k, prm)
            its[dl] = it
            if 0 < it < best_it:
                best, best_it = dl, it
        H.close()
        F.append(feats)
        T.append(shifted_factor(feats, best) if best is not None else torch.ones(feats.shape[0], device="cuda"))
        labels.append((P.name, P.dim, k, it0, best, best_it))
        log(f"{P.name}: dim {P.dim}, k {k}: plain {it0} iterations; " +
            ", ".join(f"delta {d}: {i}" for d, i in its.items()) + f" -> label {best}")
    F, T = torch.cat(F), torch.cat(T)
    # 4. the final network
    params, loss = fit(F, T, steps=steps, lr=lr, seed=seed + 1)
    log(f"final network: {F.shape[0]} samples, loss {loss:.3e}")
    return params.cpu().numpy(), {"samples": int(F.shape[0]), "loss": float(loss), "labels": labels}


def held_out():
    """Instances never used in training: (problem, k)."""
    out = [(training_problem(1000 + s), [8, 20, 40][s % 3]) for s in range(6)]
    out.append((synth.make_config("c5", n_det=1500, n_co=120, n_state=20, n_l2=3000, seed=55), 100))
    out.append((synth.make_config("c2"), 20))
    return out


def ab_compare(params, problems, tol=1e-8, max_iter=400):
    """Plain vs learned preconditioner on the same built matrices (block
    products on the tensor cores): [(name, dim, k, iterations plain, seconds
    plain, iterations learned, seconds learned, max |d eval|)]."""
    out = []
    for P, k in problems:
        H, b = built(P)
        timed_diag(H, b, k)                    # warm-up of this instance's kernels and scratch
        i0, t0, w0, _ = timed_diag(H, b, k)
        i1, t1, w1, _ = timed_diag(H, b, k, params)
        out.append((P.name, P.dim, k, i0, t0, i1, t1, float(np.abs(w0 - w1).max())))
        H.close()
    return out


def load_weights(path=DEFAULT_WEIGHTS):
    """Packed parameters of a trained network."""
    return np.load(path)["params"]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("cmd", choices=["train", "evaluate", "large"])
    ap.add_argument("--k", type=int, default=200)
    ap.add_argument("--instances", type=int, default=200)
    ap.add_argument("--steps", type=int, default=4000)
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
                  f"lowest {w[0]:.10f} highest wanted {w[-1]:.10f}, learned-factor fallbacks {dst.mlp_fallbacks}",
                  flush=True)
        H.close()
        return
    if args.cmd == "evaluate":
        params = load_weights(args.out)
        for row in ab_compare(params, held_out()):
            print("%-14s dim %6d k %3d | plain %4d it %7.3f s | learned %4d it %7.3f s | max |d eval| %.1e" % row,
                  flush=True)
        return
    p, info = train(args.instances, args.steps)
    os.makedirs(os.path.dirname(args.out), exist_ok=True)
    lab = np.array([(d, k, i0, -1.0 if b is None else b, bi) for _, d, k, i0, b, bi in info["labels"]])
    np.savez(args.out, params=p, n_samples=info["samples"], loss=info["loss"], instances=args.instances,
             steps=args.steps, labels=lab)
    print(f"saved {args.out}: {info['samples']} samples, loss {info['loss']:.4e}")


if __name__ == "__main__":
    main()
