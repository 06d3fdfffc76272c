"""Synch-EM (Algorithm Synch-EM) as a sequence of libmra calls on one device.

  1. Synchronize and Match      mra_sync          -> shift_hat [N]
  2. a_0 = mean of aligned y     mra_align_mean    (Eq. synch_initialization)
  3. rho_0 = rho_bar             given, or learned by mra_prior_hist + mra_fit_prior (Algorithm 1)
  4. EM loop on the window       mra_em_run        (graph-captured iterations)

Plain full-search EM (the baseline of Sec. 4) is the same loop with the whole
grid as the window, gamma = 0, a uniform rho_0 and no alignment.
"""
from __future__ import annotations

import dataclasses
import math

import torch

from . import mra


@dataclasses.dataclass
class Workspaces:
    em: torch.Tensor
    sync: torch.Tensor


def workspaces(d: mra.mra_dims, Lw: int, P: int, device="cuda") -> Workspaces:
    return Workspaces(em=mra.workspace(mra.mra_em_workspace_bytes(d, max(Lw, 1)), device),
                      sync=mra.workspace(mra.mra_sync_workspace_bytes(d, P), device))


@dataclasses.dataclass
class SynchEMResult:
    x: torch.Tensor         # complex128 [K+1, Q]
    log_rho: torch.Tensor   # float64 [Lw]
    shift: torch.Tensor     # int32 [N]
    iters: int
    stats: torch.Tensor | None


def synchronize(y, d, P, ws: Workspaces, n_power=50, n_ppm=100, stream=None) -> torch.Tensor:
    shift = torch.empty(d.N, dtype=torch.int32, device=y.device)
    mra.mra_sync(d, y, P, n_power, n_ppm, shift, ws.sync, stream)
    return shift


def fb_projection(n, K, Q, device="cuda", stream=None):
    """The Fourier-Bessel projection of App. A for n x n images onto k = 0..K, q = 1..Q, set up once
    (mra_fb_setup) and packed for the tensor-core projection (mra_fb_pack): the operand of mra_fb_project."""
    P = torch.empty((n * n, K + 1, Q), dtype=torch.complex64, device=device)
    ws = mra.workspace(mra.mra_fb_setup_workspace_bytes(n, K, Q), device)
    mra.mra_fb_setup(n, K, Q, P, None, ws, stream)
    return mra.fb_operand(n, K, Q, P, stream)


def fb_coefficients(images, op, K, Q, fast=False, stream=None) -> torch.Tensor:
    """Coefficients [N, K+1, Q] (complex64) of images [N, n, n] (float32): the observations y of Eq. MRA_Model_FB."""
    N, n = images.shape[0], images.shape[-1]
    y = torch.empty((N, K + 1, Q), dtype=torch.complex64, device=images.device)
    mra.mra_fb_project(N, n, K, Q, images.contiguous(), op, y, fast, stream)
    return y


def spca(y, d, stream=None):
    """Steerable PCA (App. A) of coefficients y [N, K+1, Q] with noise variance d.sigma2: returns
    (y_reduced [N, K2+1, Q2] complex64, dims of the reduced problem, basis [K+1, Q, Q], counts [K+1])."""
    basis = torch.empty((d.K + 1, d.Q, d.Q), dtype=torch.complex64, device=y.device)
    ws = mra.workspace(mra.mra_spca_workspace_bytes(d), y.device)
    K2, Q2, counts, _ = mra.mra_spca_fit(d, y, basis, ws, stream)
    out = torch.empty((d.N, K2 + 1, Q2), dtype=torch.complex64, device=y.device)
    mra.mra_spca_project(d, y, K2, Q2, basis, out, stream)
    return out, mra.dims(d.N, K2, Q2, d.L, d.sigma2), basis, counts


def template_match(y, d, ref, stream=None) -> torch.Tensor:
    """Template matching (Sec. 2.1.1): the shift of every image against the reference ref [K+1, Q] (complex64
    device tensor; an observation such as y[0], or a known signal)."""
    shift = torch.empty(d.N, dtype=torch.int32, device=y.device)
    mra.mra_template_match(d, y, ref.contiguous(), shift, stream)
    return shift


def learn_prior(y, d, shift_true, shift_est, x_true, Lw, l0=None, kind=0, ws: Workspaces | None = None, stream=None,
                step=1.0):
    """One Monte-Carlo trial of Algorithm 1 on a synthetic instance whose truth is known, then the window prior
    (on the window of rotations 2 pi step (l0 + i) / L)."""
    if l0 is None:
        l0 = -(Lw // 2)
    hist = torch.zeros(d.L, dtype=torch.int32, device=y.device)
    mra.mra_prior_hist(d, y, shift_true, shift_est, x_true, hist, None, ws.em, stream)
    log_prior = torch.empty(Lw, dtype=torch.float64, device=y.device)
    kappa = torch.empty(1, dtype=torch.float64, device=y.device)
    mra.mra_fit_prior(d.L, Lw, l0, hist, kind, log_prior, kappa, stream, step=step)
    return log_prior, kappa, hist


def window_for_mass(hist: torch.Tensor, L: int, mass: float) -> int:
    """Smallest window Lw (offsets -Lw//2 .. Lw-1-Lw//2 around the synchronized estimate) holding
    at least `mass` of the learned residual distribution (Sec. 3.3: BW chosen from the learned
    distribution).  Host-side choice of a parameter from the L histogram counts."""
    h = hist.detach().double().cpu()
    tot = float(h.sum())
    for Lw in range(1, L + 1):
        l0 = -(Lw // 2)
        idx = torch.arange(l0, l0 + Lw) % L
        if float(h[idx].sum()) >= mass * tot:
            return Lw
    return L


def synch_em(y, d, *, P, Lw, iters, gamma, log_rho_bar, ws: Workspaces, shift=None, tol=0.0, check_every=None,
             stats=True, x_traj=None, stream=None, l0=None, step=1.0) -> SynchEMResult:
    """Steps 1-4 given the learned window prior log_rho_bar [Lw] (float64 device tensor); step < 1 searches
    the denser window of rotations 2 pi step (l0 + i) / L."""
    if shift is None:
        shift = synchronize(y, d, P, ws, stream=stream)
    x = torch.empty((d.K + 1, d.Q), dtype=torch.complex128, device=y.device)
    mra.mra_align_mean(d, y, shift, x, ws.em, stream)
    log_rho = log_rho_bar.clone()
    prm = mra.em_params(Lw, l0=l0, gamma=gamma, log_rho_bar=log_rho_bar, update_rho=True, tol=tol, max_iters=iters,
                        check_every=check_every or iters, step=step)
    st = torch.empty((iters, 2), dtype=torch.float64, device=y.device) if stats else None
    n = mra.mra_em_run(d, prm, y, shift, x, log_rho, st, x_traj, ws.em, stream)
    return SynchEMResult(x=x, log_rho=log_rho, shift=shift, iters=n, stats=st)


def full_search_em(y, d, x0, *, iters, ws: Workspaces, tol=0.0, check_every=None, x_traj=None, stream=None):
    """Standard EM over all L rotations (uniform rho_0, rho updated without a prior)."""
    L = d.L
    x = x0.clone()
    log_rho = torch.full((L,), -math.log(L), dtype=torch.float64, device=y.device)
    prm = mra.em_params(L, l0=0, gamma=0.0, update_rho=True, tol=tol, max_iters=iters,
                        check_every=check_every or iters)
    st = torch.empty((iters, 2), dtype=torch.float64, device=y.device)
    n = mra.mra_em_run(d, prm, y, None, x, log_rho, st, x_traj, ws.em, stream)
    return SynchEMResult(x=x, log_rho=log_rho, shift=None, iters=n, stats=st)


def relerr(x_hat, x, d, stream=None) -> float:
    out = torch.empty(1, dtype=torch.float64, device=x.device)
    mra.mra_relerr(d.K, d.Q, x_hat, x, out, stream)
    return float(out.item())


@dataclasses.dataclass
class PriorFit:
    kappa: float
    logits: torch.Tensor  # float64 [Lw] (zeros unless fitted)
    loglik: float
    evals: int


def fit_prior_ml(y, d, Lw, x, shift=None, l0=None, kappa0=1.0, fit_logits=False, max_iter=50,
                 ws=None, step=1.0) -> PriorFit:
    """Von Mises prior on the window by maximum marginal likelihood at fixed x: maximise
    l(x, kappa, eta) over kappa (and the window logits eta when fit_logits) with L-BFGS, each
    evaluation one forward and one backward sweep of mra_loglik_grad through the autograd
    function (the posterior is recomputed, never stored).  The prior family is the von Mises
    extension of the learned prior of Algorithm 1; Sec. 3.2 defines the marginal likelihood."""
    from .autograd import marginal_loglik

    if l0 is None:
        l0 = -(Lw // 2)
    if ws is None:
        ws = mra.workspace(mra.mra_em_workspace_bytes(d, Lw), y.device)
    xd = x.detach()
    kappa = torch.tensor([float(kappa0)], dtype=torch.float64, device=y.device, requires_grad=True)
    eta = torch.zeros(Lw, dtype=torch.float64, device=y.device, requires_grad=fit_logits)
    params = [kappa] + ([eta] if fit_logits else [])
    opt = torch.optim.LBFGS(params, lr=1.0, max_iter=max_iter, tolerance_grad=1e-9, tolerance_change=1e-12,
                            line_search_fn="strong_wolfe")
    n = [0]
    scale = 1.0 / d.N

    def closure():
        opt.zero_grad()
        loss = -marginal_loglik(xd, eta, kappa, y, d, Lw, l0=l0, shift=shift, ws=ws, step=step) * scale
        loss.backward()
        n[0] += 1
        return loss

    opt.step(closure)
    with torch.no_grad():
        ll = float(marginal_loglik(xd, eta, kappa, y, d, Lw, l0=l0, shift=shift, ws=ws, step=step).item())
    return PriorFit(kappa=float(kappa.item()), logits=eta.detach().clone(), loglik=ll, evals=n[0])
