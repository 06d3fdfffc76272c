"""Steerable PCA (App. A) on the GPU against the FP64 oracle: kept counts, eigenvalues and reduced coefficients
on data with known low-rank structure, the zero padding of the reduced layout, and pixel images through the
Fourier-Bessel front end, steerable PCA and Synch-EM."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import synth
from gpu_helpers import dev_y, host, rel_err

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]


def _lowrank(N, K, Q, r, var, sigma2, seed):
    rng = np.random.default_rng(seed)
    a = np.zeros((N, K + 1, Q), dtype=np.complex128)
    for k in range(K + 1):
        Uk, _ = np.linalg.qr(rng.standard_normal((Q, r)) + 1j * rng.standard_normal((Q, r)))
        z = (rng.standard_normal((N, r)) + 1j * rng.standard_normal((N, r))) * np.sqrt(np.asarray(var) / 2)
        a[:, k, :] = z @ Uk.T
    return a + (rng.standard_normal(a.shape) + 1j * rng.standard_normal(a.shape)) * math.sqrt(sigma2 / 2)


def _gpu_spca(mra, y64, sigma2):
    N, Kp1, Q = y64.shape
    d = mra.dims(N, Kp1 - 1, Q, 360, sigma2)
    y = dev_y(y64)
    basis = torch.empty((Kp1, Q, Q), dtype=torch.complex64, device="cuda")
    ws = mra.workspace(mra.mra_spca_workspace_bytes(d))
    K2, Q2, counts, eigs = mra.mra_spca_fit(d, y, basis, ws)
    out = torch.empty((N, K2 + 1, Q2), dtype=torch.complex64, device="cuda")
    mra.mra_spca_project(d, y, K2, Q2, basis, out)
    torch.cuda.synchronize()
    return K2, Q2, counts, eigs, host(out).astype(np.complex128)


@pytest.mark.parametrize("K,Q,r,N", [(4, 10, 2, 20000), (7, 16, 3, 30000)])
def test_spca_matches_oracle(gpu_lib, K, Q, r, N):
    var = [6.0, 3.0, 1.5][:r]
    a = synth.c64_round(_lowrank(N, K, Q, r, var, 1.0, seed=9700 + K))
    K2, Q2, counts, eigs, b = _gpu_spca(gpu_lib, a, 1.0)
    f = O.spca_fit(a, 1.0)
    np.testing.assert_array_equal(counts, f.counts)
    assert (K2, Q2) == (f.K2, f.Q2)
    np.testing.assert_allclose(eigs, np.stack(f.eigs), rtol=1e-5, atol=1e-5)
    want = O.spca_project(a, f)
    assert rel_err(b, want) <= 1e-5, rel_err(b, want)


def test_spca_uneven_counts_and_padding(gpu_lib):
    """Ranks 3, 1, 0, 2 over k = 0..3 (then nothing): K2 = 3, Q2 = 3 (even (K2+1) Q2), zeros beyond each count."""
    N, K, Q = 20000, 5, 6
    rng = np.random.default_rng(9800)
    a = (rng.standard_normal((N, K + 1, Q)) + 1j * rng.standard_normal((N, K + 1, Q))) * math.sqrt(0.5)
    for k, r in enumerate([3, 1, 0, 2]):
        if r:
            Uk, _ = np.linalg.qr(rng.standard_normal((Q, r)) + 1j * rng.standard_normal((Q, r)))
            z = (rng.standard_normal((N, r)) + 1j * rng.standard_normal((N, r))) * np.sqrt(np.linspace(8, 4, r) / 2)
            a[:, k, :] += z @ Uk.T
    a = synth.c64_round(a)
    K2, Q2, counts, _, b = _gpu_spca(gpu_lib, a, 1.0)
    np.testing.assert_array_equal(counts, [3, 1, 0, 2, 0, 0])
    assert (K2, Q2) == (3, 3)
    assert np.all(b[:, 1, 1:] == 0) and np.all(b[:, 2, :] == 0) and np.all(b[:, 3, 2:] == 0)
    f = O.spca_fit(a, 1.0)
    assert rel_err(b, O.spca_project(a, f)) <= 1e-5


def test_pixels_fb_spca_synch_em(gpu_lib):
    """Pixel images (n = 65, |k| <= 10, Q = 8, L = 72, N = 6000) of a signal with a few radial components per k,
    through the Fourier-Bessel front end, steerable PCA and Synch-EM; the estimate matches the signal's reduced
    coefficients."""
    from paper_2105_07372_gb300 import pipeline

    mra = gpu_lib
    n, K, Q, L, N = 65, 10, 8, 72, 6000
    rng = np.random.default_rng(9900)
    x = synth.make_signal(K, Q, 50.0, rng)
    x[:, 3:] = 0  # three radial components carry the signal
    s = rng.integers(0, L, N)
    a = x[None] * np.exp(-2j * np.pi * np.outer(s, np.arange(K + 1)) / L)[:, :, None]
    sigma = 0.02
    img = torch.from_numpy(synth.noisy_images(a, n, sigma, seed=9901).astype(np.float32)).cuda()
    P = pipeline.fb_projection(n, K, Q)
    y = pipeline.fb_coefficients(img, P, K, Q)
    d = mra.dims(N, K, Q, L, sigma ** 2)
    basis = torch.empty((K + 1, Q, Q), dtype=torch.complex64, device="cuda")
    K2, Q2, counts, _ = mra.mra_spca_fit(d, y, basis, mra.workspace(mra.mra_spca_workspace_bytes(d)))
    assert 1 <= Q2 <= 4 and counts.max() <= 3
    yr = torch.empty((N, K2 + 1, Q2), dtype=torch.complex64, device="cuda")
    mra.mra_spca_project(d, y, K2, Q2, basis, yr)
    d2 = mra.dims(N, K2, Q2, L, sigma ** 2)
    Lw = 13
    ws = pipeline.workspaces(d2, Lw, 100, "cuda")
    lp = torch.full((Lw,), -np.log(Lw), dtype=torch.float64, device="cuda")
    res = pipeline.synch_em(yr, d2, P=100, Lw=Lw, iters=10, gamma=0.0, log_rho_bar=lp, ws=ws)
    U = host(basis).astype(np.complex128).transpose(0, 2, 1)  # block k is column-major: [k][column][row]
    xr = np.zeros((K2 + 1, Q2), dtype=np.complex128)
    for k in range(K2 + 1):
        xr[k, : counts[k]] = x[k] @ U[k][:, : counts[k]].conj()
    err = O.relerr(host(res.x), xr)
    print(f"\npixels -> FB -> sPCA ({K2 + 1} x {Q2}) -> Synch-EM: relative error {err:.3e}")
    assert err < 0.05
