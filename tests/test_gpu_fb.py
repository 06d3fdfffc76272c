"""The Fourier-Bessel front end (App. A) on the GPU: Bessel zeros against scipy, the projection of pixel images
against the oracle's least squares, steerability on the pixel grid, the TF32 option, argument checks, and pixel
images through the whole path (coefficients, synchronization, EM)."""
import numpy as np
import pytest
import torch
from scipy import special

import oracle as O
import synth
from gpu_helpers import host, rel_err

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]


def _setup(mra, n, K, Q):
    P = torch.empty((n * n, K + 1, Q), dtype=torch.complex64, device="cuda")
    R = torch.empty((K + 1, Q), dtype=torch.float64, device="cuda")
    ws = mra.workspace(mra.mra_fb_setup_workspace_bytes(n, K, Q))
    mra.mra_fb_setup(n, K, Q, P, R, ws)
    return P, host(R)


def _project(mra, images, P, K, Q, fast=False):
    img = torch.from_numpy(np.ascontiguousarray(images, dtype=np.float32)).cuda()
    n = img.shape[-1]
    op = mra.fb_operand(n, K, Q, P)
    y = torch.empty((img.shape[0], K + 1, Q), dtype=torch.complex64, device="cuda")
    mra.mra_fb_project(img.shape[0], n, K, Q, img, op, y, fast)
    torch.cuda.synchronize()
    assert mra.mra_ws_status(op) == 0  # no bounded wait of the tensor-core projection ran out
    return host(y).astype(np.complex128)


def test_fb_zeros_against_scipy(gpu_lib):
    K, Q, n = 32, 24, 129
    _, R = _setup(gpu_lib, n, K, Q)
    want = np.array([special.jn_zeros(k, Q) for k in range(K + 1)])
    np.testing.assert_allclose(R, want, rtol=1e-12, atol=0)


@pytest.mark.parametrize("n,K,Q,N", [(65, 10, 8, 300), (41, 5, 6, 200)])
def test_fb_project_matches_oracle(gpu_lib, n, K, Q, N):
    """Noisy pixel images (FP32): the GPU's coefficients against the oracle's FP64 least squares on the same pixels."""
    a = np.stack([synth.make_signal(K, Q, 20.0, np.random.default_rng(s)) for s in range(N)])
    img = synth.noisy_images(a, n, 0.02, seed=4).astype(np.float32)
    P, _ = _setup(gpu_lib, n, K, Q)
    got = _project(gpu_lib, img, P, K, Q)
    want = O.fb_project(img.astype(np.float64), K, Q)
    assert rel_err(got, want) <= 1e-5, rel_err(got, want)


def test_fb_noise_free_round_trip_and_quarter_turn(gpu_lib):
    """|k| <= 20, Q = 16 on 97 x 97 pixels: rendered coefficients come back (FP32 pixels), and images rotated by
    a quarter turn on the grid give a_k e^{-i k pi/2}."""
    n, K, Q = 97, 20, 16
    a = np.stack([synth.make_signal(K, Q, 50.0, np.random.default_rng(10 + s)) for s in range(8)])
    img = synth.render(a, n)
    P, _ = _setup(gpu_lib, n, K, Q)
    assert rel_err(_project(gpu_lib, img, P, K, Q), a) <= 1e-5
    iy, ix = np.mgrid[0:n, 0:n]
    rot = img[:, n - 1 - ix, iy]
    want = a * np.exp(-1j * np.arange(K + 1) * np.pi / 2)[None, :, None]
    assert rel_err(_project(gpu_lib, rot, P, K, Q), want) <= 1e-5
    tf = _project(gpu_lib, img, P, K, Q, fast=True)
    err = rel_err(tf, a)
    print(f"\nfast projection (three piece products): relative error {err:.1e}")
    assert err <= 1e-4


def test_fb_argument_checks(gpu_lib):
    mra = gpu_lib
    assert mra.mra_fb_setup_workspace_bytes(20, 32, 24) == 0  # beyond the sampling criterion for 20 x 20 pixels
    assert mra.mra_fb_setup_workspace_bytes(65, 2, 3) == 0    # (K+1) Q odd
    P = torch.empty((65 * 65, 4, 4), dtype=torch.complex64, device="cuda")
    ws = mra.workspace(1 << 20)
    with pytest.raises(RuntimeError):
        mra.mra_fb_setup(65, 3, 4, P, None, ws)  # workspace too small
    buf = torch.zeros(2 * 65 * 65 + 1, dtype=torch.float32, device="cuda")
    img = buf[1:].view(2, 65, 65)  # contiguous, 4 bytes off a 16-byte boundary
    y = torch.empty((2, 4, 4), dtype=torch.complex64, device="cuda")
    op = mra.workspace(mra.mra_fb_operand_bytes(65, 3, 4))
    with pytest.raises(RuntimeError):
        mra.mra_fb_project(2, 65, 3, 4, img, op, y)
    assert mra.mra_fb_operand_bytes(20, 32, 24) == 0


def test_pixel_images_through_the_whole_path(gpu_lib):
    """Pixel images of the rotated signal plus white noise (n = 65, |k| <= 10, Q = 8, L = 72, N = 4000):
    coefficients by the front end, Synchronize and Match, Synch-EM; the result is close to the signal."""
    from paper_2105_07372_gb300 import pipeline

    mra = gpu_lib
    n, K, Q, L, N = 65, 10, 8, 72, 4000
    x = synth.make_signal(K, Q, 50.0, np.random.default_rng(77))
    s = np.random.default_rng(78).integers(0, L, N)
    a = x[None] * np.exp(-2j * np.pi * np.outer(s, np.arange(K + 1)) / L)[:, :, None]
    sigma = 0.01
    img = synth.noisy_images(a, n, sigma, seed=79).astype(np.float32)
    P, _ = _setup(mra, n, K, Q)
    y = torch.from_numpy(img).cuda()
    yc = pipeline.fb_coefficients(y, mra.fb_operand(n, K, Q, P), K, Q)
    d = mra.dims(N, K, Q, L, sigma ** 2)
    Lw = 13
    ws = pipeline.workspaces(d, Lw, 100, "cuda")
    lp = torch.full((Lw,), -np.log(Lw), dtype=torch.float64, device="cuda")
    res = pipeline.synch_em(yc, d, P=100, Lw=Lw, iters=10, gamma=0.0, log_rho_bar=lp, ws=ws)
    err = pipeline.relerr(res.x, torch.from_numpy(x).cuda(), d)
    print(f"\npixels -> coefficients -> Synch-EM: relative error {err:.3e}")
    assert err < 0.05
