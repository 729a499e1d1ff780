"""The small dense eigensolver used for the Davidson Rayleigh-Ritz step
(Householder tridiagonalisation, implicit QR for the eigenvalues, inverse
iteration for the vectors; host code of the library) against numpy's eigh."""
import ctypes

import numpy as np


def test_small_eigensolver_matches_eigh():
    """All eigenpairs (implicit QR for the eigenvalues) and the lowest quarter
    (bisection on Sturm counts), with clusters and above the size where the
    reduction runs on several threads."""
    from paper_1709_03005_gb300 import build_ext
    lib = ctypes.CDLL(build_ext.build())
    fn = lib.hb_test_symeig
    fn.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    rng = np.random.default_rng(0)
    for n in (1, 2, 7, 40, 90, 300, 700):     # above 192 rows the reduction runs on several threads
        A = rng.standard_normal((n, n)); A = A + A.T
        if n in (40, 700):
            A[:5, :5] = np.eye(5) * 3.0   # a degenerate cluster
        if n == 300:
            A[:, :] = 0.0                 # a Ritz-like spectrum: many close low values
            A[np.arange(n), np.arange(n)] = np.concatenate([np.linspace(-10, -9.99, 100), np.linspace(0, 50, 200)])
            Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
            A = Q @ A @ Q.T
            A = 0.5 * (A + A.T)
        ref = np.linalg.eigvalsh(A)
        Ac = np.ascontiguousarray(A)
        for nvec in sorted({n, max(1, n // 4)}):     # n // 4 above 256 rows: bisection
            w = np.zeros(nvec); V = np.zeros((n, nvec))
            fn(n, Ac.ctypes.data, nvec, w.ctypes.data, V.ctypes.data)
            np.testing.assert_allclose(w, ref[:nvec], atol=1e-12 * max(1, np.abs(ref).max()))
            np.testing.assert_allclose(V.T @ V, np.eye(nvec), atol=1e-12)
            np.testing.assert_allclose(A @ V, V * w, atol=1e-11 * max(1, np.abs(ref).max()))


def test_small_eigensolver_near_identity_clusters():
    """The Gram matrices of the block orthonormalisation's second pass are the
    identity plus a tiny low-rank part: hundreds of eigenvalues equal to 1
    within 1e-13.  Inverse iteration returns each vector nearly inside the span
    of the earlier ones, so one Gram-Schmidt pass left 1e-8 of
    non-orthogonality (which then floored the Davidson residuals at 4e-8);
    two passes keep the vectors orthonormal to 1e-13."""
    from paper_1709_03005_gb300 import build_ext
    lib = ctypes.CDLL(build_ext.build())
    fn = lib.hb_test_symeig
    fn.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    rng = np.random.default_rng(5)
    for n in (64, 216, 300, 432):
        for r in (1, 5, 40):
            for sc in (1e-7, 1e-5):
                B = rng.standard_normal((n, r)) * sc
                A = np.ascontiguousarray(np.eye(n) + B @ B.T)
                w = np.zeros(n); V = np.zeros((n, n))
                fn(n, A.ctypes.data, n, w.ctypes.data, V.ctypes.data)
                assert np.abs(V.T @ V - np.eye(n)).max() <= 1e-13, (n, r, sc)
                assert np.linalg.norm(A @ V - V * w, axis=0).max() <= 1e-13
