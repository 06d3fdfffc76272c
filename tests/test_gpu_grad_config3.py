"""The differentiable marginal log-likelihood at |k| <= 16, Q = 16, L = 180, window 36:
the GPU gradient at N = 20,000 against the FP64 oracle, against FP64 central finite
differences of the oracle on a 500-image subset, and the von Mises concentration
fitted by maximum marginal likelihood (L-BFGS through the autograd function) against
the oracle's own maximiser of the same objective."""
import numpy as np
import pytest
import torch
from scipy import optimize

import oracle as O
import synth
from gpu_helpers import TOL_LL, TOL_W, TOL_X, dev, dev_y, host, loglik_scale

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]


def _grad_gpu(mra, inst, y64, x, eta, kappa, Lw, l0, shifts):
    d = mra.dims(inst.N, inst.K, inst.Q, inst.L, inst.sigma2)
    ws = mra.workspace(mra.mra_em_workspace_bytes(d, Lw))
    ll = torch.empty(1, dtype=torch.float64, device="cuda")
    dx = torch.empty((inst.K + 1, inst.Q), dtype=torch.complex128, device="cuda")
    de = torch.empty(Lw, dtype=torch.float64, device="cuda")
    dk = torch.empty(1, dtype=torch.float64, device="cuda")
    mra.mra_loglik_grad(d, Lw, l0, dev_y(y64), dev(shifts.astype(np.int32)), dev(x), dev(eta), kappa, ll, dx, de,
                        dk, ws)
    torch.cuda.synchronize()
    return ll.item(), host(dx), host(de), dk.item()


def test_gradient_full_size_against_oracle(gpu_lib):
    c = synth.config(3)
    inst = synth.make_instance(c["K"], c["Q"], c["N"], c["L"], c["snr"], c["decay"], seed=3100)
    y64 = synth.c64_round(inst.y)
    Lw, l0 = c["Lw"], -(c["Lw"] // 2)
    eta = 0.1 * np.random.default_rng(3).standard_normal(Lw)
    x = O.align_mean(y64, inst.s, inst.L)
    ll, dx, de, dk = _grad_gpu(gpu_lib, inst, y64, x, eta, 2.0, Lw, l0, inst.s)
    llo, dxo, deo, dko = O.loglik_grad(y64, x, eta, 2.0, inst.L, inst.sigma2, l0=l0, shifts=inst.s)
    assert abs(ll - llo) <= TOL_LL * loglik_scale(y64, x, inst.sigma2)
    assert np.linalg.norm(dx - dxo) <= TOL_X * 2.0 / inst.sigma2 * inst.N * np.linalg.norm(x)
    np.testing.assert_allclose(de, deo, atol=TOL_W * inst.N)
    assert abs(dk - dko) <= TOL_W * inst.N * Lw


def test_gradient_against_fp64_finite_differences(gpu_lib):
    """Central differences (FP64, oracle log-likelihood) on the first 500 images."""
    c = synth.config(3)
    inst = synth.make_instance(c["K"], c["Q"], 500, c["L"], c["snr"], c["decay"], seed=3101)
    y64 = synth.c64_round(inst.y)
    Lw, l0 = c["Lw"], -(c["Lw"] // 2)
    rng = np.random.default_rng(5)
    eta = 0.1 * rng.standard_normal(Lw)
    kappa = 1.5
    x = O.align_mean(y64, inst.s, inst.L)
    _, dx, de, dk = _grad_gpu(gpu_lib, inst, y64, x, eta, kappa, Lw, l0, inst.s)

    def f(xx=x, ee=eta, kk=kappa):
        return O.loglik(y64, xx, ee, kk, inst.L, inst.sigma2, l0=l0, shifts=inst.s)

    h = 1e-5
    fd_k = (f(kk=kappa + h) - f(kk=kappa - h)) / (2 * h)
    assert abs(dk - fd_k) <= 1e-5 * max(1.0, abs(fd_k)) + 1e-3, (dk, fd_k)
    for l in (0, Lw // 2, Lw - 1):
        e1, e2 = eta.copy(), eta.copy()
        e1[l] += h
        e2[l] -= h
        fd = (f(ee=e1) - f(ee=e2)) / (2 * h)
        assert abs(de[l] - fd) <= 1e-5 * max(1.0, abs(fd)) + 1e-3, (l, de[l], fd)
    # x along a random complex direction v: d/dt l(x + t v) = Re <grad, v>
    v = rng.standard_normal(x.shape) + 1j * rng.standard_normal(x.shape)
    v /= np.linalg.norm(v)
    hx = 1e-6
    fd_x = (f(xx=x + hx * v) - f(xx=x - hx * v)) / (2 * hx)
    dirx = float(np.real(np.vdot(dx, v)))
    assert abs(dirx - fd_x) <= 1e-5 * abs(fd_x) + 1e-2, (dirx, fd_x)


def test_fit_kappa_by_marginal_likelihood(gpu_lib):
    """Rotations drawn from a discrete von Mises law on the window around known estimates;
    kappa maximising the GPU marginal likelihood equals the oracle's maximiser."""
    from paper_2105_07372_gb300 import pipeline

    mra = gpu_lib
    c = synth.config(3)
    K, Q, L, Lw = c["K"], c["Q"], c["L"], c["Lw"]
    l0 = -(Lw // 2)
    N, kappa_true = 4000, 40.0
    rng = np.random.default_rng(31)
    x = synth.make_signal(K, Q, c["decay"], rng)
    est = rng.integers(0, L, N)
    p = np.exp(O.vm_log_rho(np.zeros(Lw), kappa_true, L, l0))
    off = rng.choice(Lw, size=N, p=p / p.sum())
    s = (est + l0 + off) % L
    inst = synth.make_instance(K, Q, N, L, sigma2=synth.sigma2_for_snr(1 / 10, x), shifts=s, x=x, seed=32)
    y64 = synth.c64_round(inst.y)
    d = mra.dims(N, K, Q, L, inst.sigma2)
    fit = pipeline.fit_prior_ml(dev_y(y64), d, Lw, dev(x), shift=dev(est.astype(np.int32)), l0=l0, kappa0=5.0)

    def negll(k):
        return -O.loglik(y64, x, np.zeros(Lw), k, L, inst.sigma2, l0=l0, shifts=est)

    ko = optimize.minimize_scalar(negll, bounds=(1.0, 200.0), method="bounded", options={"xatol": 1e-6}).x
    assert abs(fit.kappa - ko) <= 1e-3 * ko, (fit.kappa, ko)
    # and both are close to the concentration the rotations were drawn with (Monte-Carlo error)
    assert abs(ko - kappa_true) <= 0.15 * kappa_true, (ko, kappa_true)
