"""Eigen reference for the Davidson step (Section 3.2.2 names Davidson among
the diagonalisers; the paper gives no algorithm, so the reference is the dense
eigensolver itself plus a plain block Davidson used as the CPU baseline).

ORACLE / TEST INFRASTRUCTURE ONLY.
"""
from __future__ import annotations

import numpy as np


def lowest(H: np.ndarray, k: int):
    """The k lowest eigenpairs of a dense symmetric matrix (LAPACK via numpy)."""
    w, V = np.linalg.eigh(H)
    return w[:k], V[:, :k]


def davidson(apply, diag: np.ndarray, k: int, tol: float = 1e-8, max_iter: int = 300, block: int | None = None):
    """Plain block Davidson with the diagonal preconditioner (FP64, numpy).

    apply(X) returns H @ X for an (n, q) block.  Start: unit vectors at the
    smallest diagonal entries.  Returns (eigenvalues, vectors, iterations).
    """
    n = diag.shape[0]
    b = block or min(n, k + max(4, min(16, k // 2)))
    mmax = min(n, max(3 * b, k + 2 * b))
    idx = np.argsort(diag, kind="stable")[:b]
    V = np.zeros((n, b)); V[idx, np.arange(b)] = 1.0
    AV = apply(V)
    for it in range(1, max_iter + 1):
        T = V.T @ AV
        T = 0.5 * (T + T.T)
        theta, S = np.linalg.eigh(T)
        nr = min(V.shape[1], b)
        X = V @ S[:, :nr]
        AX = AV @ S[:, :nr]
        R = AX - X * theta[:nr]
        res = np.linalg.norm(R, axis=0)
        if np.all(res[:k] <= tol):
            return theta[:k], X[:, :k], it
        which = [j for j in range(nr) if res[j] > tol][:b]
        if V.shape[1] + len(which) > mmax:
            V, AV = X, AX
        den = diag[:, None] - theta[which][None, :]
        den = np.where(np.abs(den) < 1e-4, np.where(den < 0, -1e-4, 1e-4), den)
        Tn = R[:, which] / den
        for _ in range(2):
            Tn -= V @ (V.T @ Tn)
        Q, Rq = np.linalg.qr(Tn)
        keep = np.abs(np.diag(Rq)) > 1e-10 * max(1.0, np.abs(np.diag(Rq)).max())
        Q = Q[:, keep]
        Q -= V @ (V.T @ Q)
        Q, _ = np.linalg.qr(Q)
        V = np.hstack([V, Q])
        AV = np.hstack([AV, apply(Q)])
    return theta[:k], X[:, :k], max_iter
