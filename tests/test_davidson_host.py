"""The small dense eigensolver used for the Davidson Rayleigh-Ritz step
(Householder tridiagonalisation, bisection, inverse iteration; host code of
the library) against numpy's eigh."""
import ctypes

import numpy as np


def test_small_eigensolver_matches_eigh():
    from paper_1709_03005_gb300 import build_ext, hb
    lib = ctypes.CDLL(build_ext.build())
    fn = lib.hb_test_symeig
    fn.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    rng = np.random.default_rng(0)
    for n in (1, 2, 7, 40, 90):
        A = rng.standard_normal((n, n)); A = A + A.T
        if n == 40:
            A[:5, :5] = np.eye(5) * 3.0   # a degenerate cluster
        w = np.zeros(n); V = np.zeros((n, n))
        Ac = np.ascontiguousarray(A)
        fn(n, Ac.ctypes.data, w.ctypes.data, V.ctypes.data)
        ref = np.linalg.eigvalsh(A)
        np.testing.assert_allclose(w, ref, atol=1e-12 * max(1, np.abs(ref).max()))
        np.testing.assert_allclose(V.T @ V, np.eye(n), atol=1e-12)
        np.testing.assert_allclose(A @ V, V * w, atol=1e-11 * max(1, np.abs(ref).max()))
