"""The library's host eigensolver (used by the steerable PCA fit) against numpy on CPU: eigenvalues, the
eigen-equation, unitarity, the phase convention, and degenerate spectra."""
import os

import numpy as np
import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_2105_07372_gb300 import build, mra

    if not os.path.exists(build.LIB):
        if not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("no nvcc to build libmra")
        build.build_library()
    mra.load()
    return mra


def _check(mra, A):
    w, V = mra.mra_hermitian_eig(A)
    n = A.shape[0]
    np.testing.assert_allclose(w, np.sort(np.linalg.eigvalsh(A))[::-1], atol=1e-11 * max(1.0, np.abs(w).max()))
    np.testing.assert_allclose(V.conj().T @ V, np.eye(n), atol=1e-11)
    np.testing.assert_allclose(A @ V, V * w[None, :], atol=1e-10 * max(1.0, np.abs(w).max()))
    for j in range(n):
        i = int(np.argmax(np.abs(V[:, j])))
        assert abs(V[i, j].imag) < 1e-12 and V[i, j].real > 0


@pytest.mark.parametrize("n", [1, 2, 5, 24, 64])
def test_hermitian_eig_random(lib, n):
    rng = np.random.default_rng(n)
    B = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    _check(lib, (B + B.conj().T) / 2)


def test_hermitian_eig_real_and_degenerate(lib):
    rng = np.random.default_rng(3)
    B = rng.standard_normal((10, 10))
    _check(lib, B + B.T)                      # real symmetric (all eigenvalues doubly degenerate in the embedding)
    Qm, _ = np.linalg.qr(rng.standard_normal((8, 8)) + 1j * rng.standard_normal((8, 8)))
    A = Qm @ np.diag([3.0, 3.0, 3.0, 1.0, 1.0, -2.0, 0.5, 0.5]) @ Qm.conj().T
    _check(lib, (A + A.conj().T) / 2)         # repeated eigenvalues
    _check(lib, np.eye(6, dtype=np.complex128))
