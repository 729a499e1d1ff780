"""Pins of the eigen reference: the plain Davidson reaches numpy's eigh."""
import numpy as np

from oracle import coracle, eig
from paper_1709_03005_gb300 import synth


def test_davidson_matches_eigh_random():
    rng = np.random.default_rng(3)
    n = 300
    A = rng.standard_normal((n, n)) * 0.1
    A = A + A.T + np.diag(np.linspace(-5, 20, n))
    w, V, it = eig.davidson(lambda X: A @ X, np.diag(A).copy(), 8, tol=1e-9)
    ref = np.linalg.eigvalsh(A)[:8]
    np.testing.assert_allclose(w, ref, atol=1e-9)
    assert np.linalg.norm(A @ V - V * w, axis=0).max() <= 1e-9


def test_davidson_on_contracted_hamiltonian():
    P = synth.make_config("mid")
    H = coracle.Oracle(P).dense()
    w, V, it = eig.davidson(lambda X: H @ X, np.diag(H).copy(), 10, tol=1e-8)
    ref = np.linalg.eigvalsh(H)[:10]
    np.testing.assert_allclose(w, ref, atol=1e-8)
