"""Plain FP64 CPU oracle for Synch-EM on 2-D MRA in a steerable basis.

TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct statement
of what the CUDA library computes.  Only the tests, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it; the library itself
never calls it, and it shares no code with the CUDA path.

Everything is complex128 / float64 numpy and follows the paper's formulas in
its own order and notation:

* rotation by phi multiplies a_{k,q} by exp(-i k phi)                 Eq. (fb_rotation)
* model v_i = a o exp(-i kbar theta_i) + eps_i                          Eq. (MRA_Model_FB)
* relative rotation argmin_theta sum |v^i - e^{i k theta} v^j|^2        Eq. (relative_angle_2d_dist)
* synchronization max z^* H z, projected power method z <- phase(Hz)   Eq. (cost_synchronization), Sec. 2.1.2
* align and average                                                   Eq. (synch_initialization)
* E-step weights  w ~ exp(-||a o e^{-i 2 pi l kbar/L} - v_j||^2/sigma^2) rho[l]   Eq. (weights_2d_em)
* M-step  a = (N I + sigma^2 Gamma_a^{-1})^{-1} sum_j sum_l w e^{+i..} o v_j     Eq. (coefficients_update)
* rho update (W + gamma rho_bar) / sum(W + gamma rho_bar)              Algorithm "Synch-EM", App. C
* convergence min_l ||a_{t+1} - e^{-2 pi i kbar l/L} o a_t||^2 < tol    Algorithm "Synch-EM"
* Synchronize and Match                                               Algorithm "Synchronize and Match"
* template matching: every image against one reference, O(NLM)        Sec. 2.1.1 (template matching)
* shift pmf of 1-D template matching with the true signal as reference App. B, Eq. (shift_pmf)
* Fourier-Bessel coefficients of pixel images by least squares          App. A
* steerable PCA of the coefficients (data-driven radial basis per k)   App. A (sPCA; details are the
  cited method's, restated in the readings below)
* learned rotation distribution, centred by theta_c                    Eq. (learned_distribution_formula), Algorithm 1
* relative error up to rotation                                       Sec. 2.2, relative-error equation
* likelihood with the (pi sigma^2)^{-M} factor                          Sec. 2.2, likelihood equation

Storage: coefficient arrays are [K+1, Q] (k = 0..K stored, Sec. 1 symmetry),
observations [N, K+1, Q].  Norms are over the stored entries.

Readings of the paper taken here (each also listed in the design notes):

* Window: ``Lw`` grid offsets l0, l0+1, .., l0+Lw-1 (mod L) with l0 = -floor(Lw/2)
  by default; the paper's [-BW/2, BW/2] is Lw = BW + 1 points.
* Denser-resolution window (Sec. 3.3): the window's angles are
  theta_i = 2 pi step (l0 + i) / L with 0 < step <= 1, so Lw rotations cover Lw step
  grid units.  The paper's example, the range [-pi BW/L, pi BW/L] at spacing
  pi BW/L^2, is Lw = 2 L + 1, l0 = -L, step = BW / (2 L).  Alignment shifts stay
  on the grid; the stopping rule still minimises over the L grid rotations.  The
  learned histogram gives each window angle the value of the nearest grid bin.
* Sign of the synchronization matrix: the pairwise argmin of
  Eq. (relative_angle_2d_dist) estimates theta_j - theta_i under the model's
  sign, so the matrix whose leading eigenvector has phases theta_i is
  H_ij = exp(-i theta_hat_ij) (the conjugate of the printed e^{+i theta_hat_ij}).
  With that choice arg z_i estimates theta_i up to a global rotation and the
  alignment e^{+i k theta_hat_i} v_i of Eq. (synch_initialization) undoes it.
* PPM start and stopping: z starts from the all-ones vector, ``n_power`` power
  iterations z <- Hz/||Hz||, then ``n_ppm`` projected steps z <- phase(Hz);
  phase(0) := 1; global phase fixed by theta_hat_0 = 0; angles are rounded to
  the grid: s_hat = floor(arg z * L / 2 pi + 1/2) mod L.
* Ties in every argmin / argmax go to the smallest index.
* Learned distribution: the histogram is taken over the EM's latent offset
  r_j = (s_j - s_hat_j + c) mod L, where c is the grid minimiser of
  ||R_c xbar - x||^2; r_j is the rotation for which y_j e^{+i k theta_hat_j}
  = xbar o e^{-2 pi i k r_j / L} in the noise-free case, i.e. the index that
  the EM window and rho_0 = rho_bar refer to.  This is -Delta_theta_bar of
  Algorithm 1 under the paper's rotation sign.
* rho_bar on the window is the restriction of rho_bar renormalised to sum 1.
* Steerable PCA: for every angular index k the uncentred second moment C_k = (1/N) sum_i a_ik a_ik^H
  over the Q radial entries (uncentred also at k = 0, so that the mean image's direction is kept),
  its eigenvectors kept where the eigenvalue exceeds the noise-only spectrum's upper edge
  sigma^2 (1 + sqrt(Q/N))^2 (Marchenko-Pastur); coefficients b_ik = U_k^H a_ik.  Each eigenvector's
  phase makes its largest-magnitude entry real positive; eigenvalues descend.  The output is
  [K'+1, Q'] with K' the largest k that keeps a component and Q' the largest kept count (made even
  with (K'+1) when needed), zero where a k keeps fewer.
* Relative error: the stored k > 0 entries count twice (the k < 0 half of a
  real image), the angle is continuous (fine grid then golden section).

Parity unpinned: nothing in this file.  Every function is pinned by a test in
``tests/test_oracle_pins.py`` (brute force, closed forms, library routines,
invariants); the statistical behaviour of Synchronize and Match at a given SNR
is sanity-checked only.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy import optimize, special

TWO_PI = 2.0 * math.pi


# ----------------------------------------------------------------------------
# rotations, Eq. (fb_rotation) and Eq. (MRA_Model_FB)
# ----------------------------------------------------------------------------
def kbar(K: int) -> np.ndarray:
    """Angular index of each stored row, k = 0..K."""
    return np.arange(K + 1, dtype=np.float64)


def rotate(a: np.ndarray, phi: float | np.ndarray) -> np.ndarray:
    """Rotate coefficients by angle phi: a_{k,q} -> a_{k,q} exp(-i k phi)."""
    K = a.shape[-2] - 1
    ph = np.exp(-1j * np.multiply.outer(np.asarray(phi, dtype=np.float64), kbar(K)))
    return a * ph[..., :, None]


def grid_angle(l, L: int):
    return TWO_PI * np.asarray(l, dtype=np.float64) / L


def window_offsets(L: int, Lw: int, l0: int | None = None, step: float = 1.0) -> np.ndarray:
    """Window positions in grid units (l0 + i) * step, i = 0..Lw-1 (Sec. 3.3).

    step = 1 is the grid window of the reduced search space; step < 1 is the
    denser-resolution variant (Sec. 3.3): Lw angles step grid units apart, so the
    same number of rotations covers a narrower range at a finer resolution.
    """
    if l0 is None:
        l0 = -(Lw // 2)
    o = l0 + np.arange(Lw)
    return o if step == 1.0 else o * float(step)


def align(y: np.ndarray, shifts: np.ndarray, L: int) -> np.ndarray:
    """y_i e^{+i k theta_hat_i}: undo estimated rotations (Sec. 2.1, alignment before Eq. synch_initialization)."""
    return rotate(y, -grid_angle(shifts, L))


# ----------------------------------------------------------------------------
# E-step / M-step, Eqs. (weights_2d_em), (coefficients_update), Algorithm Synch-EM
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class EMStep:
    x: np.ndarray          # a_{t+1}                       [K+1, Q]
    log_rho: np.ndarray    # log rho_{t+1} on the window   [Lw]
    w: np.ndarray          # posterior weights w_t^{l,j}   [N, Lw]
    W: np.ndarray          # W_t[l] = sum_j w              [Lw]
    loglik: float          # log p(v | a_t, rho_t) (marginal over the window)
    step: float            # min_l ||a_{t+1} - e^{-2 pi i k l/L} a_t||^2


def sq_dist_window(x: np.ndarray, y: np.ndarray, offsets: np.ndarray, L: int, chunk: int = 256) -> np.ndarray:
    """d[j, l] = || x o exp(-i 2 pi offsets[l] kbar / L) - y_j ||^2, the literal distance of Eq. (weights_2d_em)."""
    rx = rotate(x, grid_angle(offsets, L))  # [Lw, K+1, Q]
    N = y.shape[0]
    d = np.empty((N, offsets.size))
    for a in range(0, N, chunk):
        diff = rx[None, :, :, :] - y[a:a + chunk, None, :, :]
        d[a:a + chunk] = np.sum(diff.real ** 2 + diff.imag ** 2, axis=(2, 3))
    return d


def _logsumexp(v: np.ndarray, axis: int) -> np.ndarray:
    m = np.max(v, axis=axis, keepdims=True)
    m_safe = np.where(np.isfinite(m), m, 0.0)
    s = np.sum(np.exp(v - m_safe), axis=axis, keepdims=True)
    return np.squeeze(m_safe + np.log(s), axis=axis)


def posterior(x, y, log_rho, L, offsets, sigma2):
    """Normalised weights w_t^{l,j} (Algorithm Synch-EM, E-step and normalisation over the window).

    The unnormalised weight exp(-d/sigma^2) rho[l] underflows in floating point for
    realistic d/sigma^2, so it is formed as exp(log rho - d/sigma^2 - m_j) with the
    per-image maximum m_j removed; the normalised value is the same.
    Returns (w, log_terms) where log_terms[j, l] = log rho[l] - d[j, l]/sigma^2.
    """
    d = sq_dist_window(x, y, offsets, L)
    with np.errstate(invalid="ignore"):
        t = np.asarray(log_rho, dtype=np.float64)[None, :] - d / sigma2
    lse = _logsumexp(t, axis=1)
    w = np.exp(t - lse[:, None])
    return w, t, lse


def marginal_loglik(lse: np.ndarray, M: int, sigma2: float) -> float:
    """sum_j log sum_l rho[l] (pi sigma^2)^{-M} exp(-d_jl/sigma^2), Sec. 2.2 likelihood."""
    return float(np.sum(lse) - lse.size * M * math.log(math.pi * sigma2))


def step_size(x_new: np.ndarray, x_old: np.ndarray, L: int) -> float:
    """min_{l in [0, L-1]} ||a_{t+1} - e^{-2 pi i kbar l/L} o a_t||^2 (Algorithm Synch-EM, stopping rule)."""
    r = rotate(x_old, grid_angle(np.arange(L), L))  # [L, K+1, Q]
    diff = x_new[None] - r
    return float(np.min(np.sum(diff.real ** 2 + diff.imag ** 2, axis=(1, 2))))


def em_step(y, x, log_rho, L, sigma2, Lw=None, l0=None, gamma=0.0, log_rho_bar=None,
            gamma_a_inv=None, update_rho=True, shifts=None, step=1.0) -> EMStep:
    """One iteration of Algorithm Synch-EM (E-step, W_t, a-update, rho-update, step).

    y: [N, K+1, Q] observations; ``shifts`` (grid indices) align them first
    (v~_j = v_j e^{+i k theta_hat_j}); x = a_t; log_rho = log rho_t on the window.
    gamma_a_inv: diagonal of Gamma_a^{-1} as [K+1, Q] (None = flat image prior).
    step: spacing of the window's rotations in grid units (window_offsets).
    """
    y = np.asarray(y, dtype=np.complex128)
    x = np.asarray(x, dtype=np.complex128)
    N, Kp1, Q = y.shape
    M = Kp1 * Q
    if Lw is None:
        Lw = np.asarray(log_rho).size
    offs = window_offsets(L, Lw, l0, step)
    yt = y if shifts is None else align(y, np.asarray(shifts), L)
    # E-step and normalisation
    w, _, lse = posterior(x, yt, log_rho, L, offs, sigma2)
    W = w.sum(axis=0)
    # M-step for a: (N I + sigma^2 Gamma^-1)^-1 sum_j sum_l w e^{+i 2 pi l k/L} o v_j
    back = np.exp(1j * np.outer(grid_angle(offs, L), kbar(Kp1 - 1)))  # [Lw, K+1]
    num = np.zeros((Kp1, Q), dtype=np.complex128)
    for a in range(0, N, 512):
        Wk = w[a:a + 512] @ back  # [n, K+1] = sum_l w_jl e^{+i k theta_l}
        num += np.sum(Wk[:, :, None] * yt[a:a + 512], axis=0)
    den = N + (0.0 if gamma_a_inv is None else sigma2 * np.asarray(gamma_a_inv, dtype=np.float64))
    x_new = num / den
    # M-step for rho on the window (prior-weighted form of Algorithm Synch-EM)
    if update_rho:
        rb = np.zeros(Lw) if log_rho_bar is None else np.exp(np.asarray(log_rho_bar, dtype=np.float64))
        v = W + gamma * rb
        rho_new = v / np.sum(v)
        with np.errstate(divide="ignore"):
            log_rho_new = np.log(rho_new)
    else:
        log_rho_new = np.asarray(log_rho, dtype=np.float64).copy()
    return EMStep(x=x_new, log_rho=log_rho_new, w=w, W=W,
                  loglik=marginal_loglik(lse, M, sigma2), step=step_size(x_new, x, L))


def map_objective(y, x, log_rho, L, sigma2, Lw=None, l0=None, gamma=0.0, log_rho_bar=None,
                  gamma_a_inv=None, shifts=None, step=1.0) -> float:
    """log p(v|a,rho) + log p(a) + log p(rho) up to constants (Sec. 2.2, Sec. 3.2.2).

    log p(a) = -a^H Gamma_a^{-1} a, log p(rho) = -gamma D_KL(rho_bar, rho) = gamma sum rho_bar log rho + const.
    """
    y = np.asarray(y, dtype=np.complex128)
    N, Kp1, Q = y.shape
    if Lw is None:
        Lw = np.asarray(log_rho).size
    offs = window_offsets(L, Lw, l0, step)
    yt = y if shifts is None else align(y, np.asarray(shifts), L)
    _, _, lse = posterior(x, yt, log_rho, L, offs, sigma2)
    val = marginal_loglik(lse, Kp1 * Q, sigma2)
    if gamma_a_inv is not None:
        val -= float(np.sum(np.asarray(gamma_a_inv) * (x.real ** 2 + x.imag ** 2)))
    if gamma > 0 and log_rho_bar is not None:
        rb = np.exp(np.asarray(log_rho_bar, dtype=np.float64))
        lr = np.asarray(log_rho, dtype=np.float64)
        mask = rb > 0
        val += gamma * float(np.sum(rb[mask] * lr[mask]))
    return val


@dataclasses.dataclass
class EMRun:
    x: np.ndarray
    log_rho: np.ndarray
    iters: int
    loglik: np.ndarray  # loglik at the start of each iteration (a_t, rho_t)
    step: np.ndarray


def em_run(y, x0, log_rho0, L, sigma2, max_iters, tol=0.0, **kw) -> EMRun:
    """Algorithm Synch-EM, loop for t = 0..T-1 with the tolerance break."""
    x, lr = np.asarray(x0, dtype=np.complex128), np.asarray(log_rho0, dtype=np.float64)
    lls, steps = [], []
    it = 0
    for it in range(1, max_iters + 1):
        st = em_step(y, x, lr, L, sigma2, **kw)
        lls.append(st.loglik)
        steps.append(st.step)
        x, lr = st.x, st.log_rho
        if st.step < tol:
            break
    return EMRun(x=x, log_rho=lr, iters=it, loglik=np.array(lls), step=np.array(steps))


# ----------------------------------------------------------------------------
# synchronization, Sec. 2.1 and Algorithm "Synchronize and Match"
# ----------------------------------------------------------------------------
def relative_rotation(vi: np.ndarray, vj: np.ndarray, L: int) -> int:
    """argmin over the grid of sum_{k,q} |v^i - e^{i k theta} v^j|^2, Eq. (relative_angle_2d_dist)."""
    rvj = rotate(vj, -grid_angle(np.arange(L), L))  # e^{+i k theta_l} v^j, [L, K+1, Q]
    diff = vi[None] - rvj
    d = np.sum(diff.real ** 2 + diff.imag ** 2, axis=(1, 2))
    return int(np.argmin(d))


def pairwise_relative(yP: np.ndarray, L: int) -> np.ndarray:
    """rel[i, j] = grid index of theta_hat_ij for i < j; rel[j, i] = -rel[i, j] mod L; rel[i, i] = 0."""
    P = yP.shape[0]
    rel = np.zeros((P, P), dtype=np.int64)
    for i in range(P):
        for j in range(i + 1, P):
            r = relative_rotation(yP[i], yP[j], L)
            rel[i, j] = r
            rel[j, i] = (L - r) % L
    return rel


def sync_matrix(rel: np.ndarray, L: int) -> np.ndarray:
    """H_ij = exp(-i theta_hat_ij) (see the sign reading in the module docstring)."""
    return np.exp(-1j * grid_angle(rel, L))


def power_iteration(H: np.ndarray, n_power: int) -> np.ndarray:
    z = np.ones(H.shape[0], dtype=np.complex128)
    for _ in range(n_power):
        z = H @ z
        z = z / np.linalg.norm(z)
    return z


def phase(v: np.ndarray) -> np.ndarray:
    """phase(z)_i = z_i / |z_i|, with phase(0) := 1."""
    a = np.abs(v)
    out = np.ones_like(v)
    nz = a > 0
    out[nz] = v[nz] / a[nz]
    return out


def ppm_angles(rel: np.ndarray, L: int, n_power: int = 50, n_ppm: int = 100) -> np.ndarray:
    """Projected power method for max_{z in C_1^P} z^* H z; returns arg z_i - arg z_0 in (-pi, pi]."""
    H = sync_matrix(rel, L)
    z = power_iteration(H, n_power)
    for _ in range(n_ppm):
        z = phase(H @ z)
    z = z * np.conj(z[0]) / abs(z[0])
    return np.angle(z)


def ppm(rel: np.ndarray, L: int, n_power: int = 50, n_ppm: int = 100) -> np.ndarray:
    """Grid rotations phi_hat [P] from the projected power method, rounded to the nearest grid point."""
    ang = ppm_angles(rel, L, n_power, n_ppm)
    return (np.floor(ang * L / TWO_PI + 0.5).astype(np.int64)) % L


def match(y: np.ndarray, P: int, phi: np.ndarray, chunk: int = 64) -> np.ndarray:
    """Steps 3-8 of Algorithm Synchronize and Match: nearest neighbour in S_P (excluding itself)."""
    N = y.shape[0]
    yP = y[:P]
    out = np.empty(N, dtype=np.int64)
    for a in range(0, N, chunk):
        diff = y[a:a + chunk, None] - yP[None]
        d = np.sum(diff.real ** 2 + diff.imag ** 2, axis=(2, 3))  # [n, P]
        for r in range(d.shape[0]):
            i = a + r
            if i < P:
                d[r, i] = np.inf
        out[a:a + chunk] = phi[np.argmin(d, axis=1)]
    return out


def synchronize_and_match(y: np.ndarray, P: int, L: int, n_power: int = 50, n_ppm: int = 100):
    """Algorithm Synchronize and Match: returns (s_hat [N], phi_hat [P], rel [P, P])."""
    P = min(P, y.shape[0])
    rel = pairwise_relative(y[:P], L)
    phi = ppm(rel, L, n_power, n_ppm)
    return match(y, P, phi), phi, rel


def template_match(y: np.ndarray, ref: np.ndarray, L: int, chunk: int = 16) -> np.ndarray:
    """Template matching (Sec. 2.1.1): s_j = argmin over the grid of sum_{k,q} |ref - e^{i k theta} v^j|^2,
    each image against the one reference (the relative rotation of Eq. relative_angle_2d_dist)."""
    y = np.asarray(y, dtype=np.complex128)
    ref = np.asarray(ref, dtype=np.complex128)
    ph = np.exp(1j * np.outer(grid_angle(np.arange(L), L), kbar(y.shape[1] - 1)))  # e^{+i k theta_l} [L, K+1]
    out = np.empty(y.shape[0], dtype=np.int64)
    for a in range(0, y.shape[0], chunk):
        rv = y[a:a + chunk, None, :, :] * ph[None, :, :, None]  # [n, L, K+1, Q]
        diff = ref[None, None] - rv
        d = np.sum(diff.real ** 2 + diff.imag ** 2, axis=(2, 3))
        out[a:a + chunk] = np.argmin(d, axis=1)
    return out


def tm_shift_pmf(x: np.ndarray, sigma: float) -> np.ndarray:
    """App. B, Eq. (shift_pmf): the approximate pmf of the shift that 1-D template matching with the true
    signal x as reference estimates for zero-shift observations y ~ N(x, sigma^2 I):
    p[m] = int N(u; R_xx[m], sigma_c^2) prod_{l != m} Phi((u - R_xx[l]) / sigma_c) du,
    R_xx[l] = sum_n x[n] x[(n + l) mod L], sigma_c^2 = sigma^2 ||x||^2 (the correlations taken independent)."""
    from scipy import integrate, stats

    x = np.asarray(x, dtype=np.float64)
    L = x.size
    R = np.array([np.dot(x, np.roll(x, -l)) for l in range(L)])  # R[l] = sum_n x[n] x[n + l]
    sc = float(sigma) * float(np.linalg.norm(x))
    p = np.empty(L)
    for m in range(L):
        others = np.delete(R, m)

        def f(u, m=m, others=others):
            return stats.norm.pdf(u, R[m], sc) * np.prod(stats.norm.cdf((u - others) / sc))

        lo, hi = R.min() - 12 * sc, R.max() + 12 * sc
        p[m] = integrate.quad(f, lo, hi, points=sorted(set(R.tolist())), limit=400, epsabs=1e-13, epsrel=1e-11)[0]
    return p


# ----------------------------------------------------------------------------
# Fourier-Bessel front end, App. A
# ----------------------------------------------------------------------------
def fb_design(n: int, K: int, Q: int) -> np.ndarray:
    """Real least-squares design matrix [n*n, Q + 2KQ] of a real image in the Fourier-Bessel basis (App. A):
    u^{k,q} = N_{k,q} J_|k|(R_{|k|,q} r/c) e^{ik theta} on r <= c = (n-1)/2, N_{k,q} = 1/(c sqrt(pi) |J_{k+1}(R_{k,q})|),
    pixels at x = column - c, y = row - c.  With a_{-k} = conj(a_k) the image is
    sum_q a_0q u^{0q} + sum_{k>=1,q} (2 Re a_kq Re u^{kq} - 2 Im a_kq Im u^{kq}); columns k = 0 (a_0q, real), then
    per k >= 1 and q the columns of Re a_kq and Im a_kq."""
    c = (n - 1) / 2.0
    rows, colsx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    x = (colsx - c).ravel()
    y = (rows - c).ravel()
    r = np.sqrt(x * x + y * y)
    theta = np.arctan2(y, x)
    out = np.zeros((n * n, Q + 2 * K * Q))
    col = 0
    for k in range(K + 1):
        R = special.jn_zeros(k, Q)
        for q in range(Q):
            Nkq = 1.0 / (c * math.sqrt(math.pi) * abs(special.jv(k + 1, R[q])))
            f = np.where(r <= c, Nkq * special.jv(k, R[q] * r / c), 0.0)
            if k == 0:
                out[:, col] = f
                col += 1
            else:
                out[:, col] = 2.0 * f * np.cos(k * theta)
                out[:, col + 1] = -2.0 * f * np.sin(k * theta)
                col += 2
    return out


def fb_project(images: np.ndarray, K: int, Q: int) -> np.ndarray:
    """Coefficients [N, K+1, Q] (complex, k >= 0) of images [N, n, n] as the least-squares solution of App. A."""
    images = np.asarray(images, dtype=np.float64)
    n = images.shape[-1]
    A = fb_design(n, K, Q)
    beta = np.linalg.lstsq(A, images.reshape(images.shape[0], -1).T, rcond=None)[0].T  # [N, Q + 2KQ]
    a = np.zeros((images.shape[0], K + 1, Q), dtype=np.complex128)
    a[:, 0, :] = beta[:, :Q]
    ri = beta[:, Q:].reshape(images.shape[0], K, Q, 2)
    a[:, 1:, :] = ri[..., 0] + 1j * ri[..., 1]
    return a


def _phase_fix(U: np.ndarray) -> np.ndarray:
    """Columns scaled by a unit phase so that each column's largest-magnitude entry is real positive."""
    U = U.copy()
    for j in range(U.shape[1]):
        i = int(np.argmax(np.abs(U[:, j])))
        U[:, j] *= np.conj(U[i, j]) / abs(U[i, j])
    return U


@dataclasses.dataclass
class SPCA:
    bases: list          # per k: [Q, Q_k] complex, kept eigenvectors (columns)
    eigs: list           # per k: [Q] eigenvalues, descending
    counts: np.ndarray   # [K+1] kept per k
    K2: int
    Q2: int


def spca_fit(a: np.ndarray, sigma2: float) -> SPCA:
    """Steerable PCA of coefficients a [N, K+1, Q] with noise variance sigma2 per entry (readings above)."""
    a = np.asarray(a, dtype=np.complex128)
    N, Kp1, Q = a.shape
    edge = sigma2 * (1.0 + math.sqrt(Q / N)) ** 2
    bases, eigs, counts = [], [], []
    for k in range(Kp1):
        A = a[:, k, :]                      # [N, Q]
        C = A.T @ A.conj() / N              # sum_i a_ik a_ik^H / N  (entry (q, q') = mean a_q conj(a_q'))
        w, U = np.linalg.eigh(C)
        order = np.argsort(-w, kind="stable")
        w, U = w[order], _phase_fix(U[:, order])
        keep = int(np.sum(w > edge))
        bases.append(U[:, :keep])
        eigs.append(w)
        counts.append(keep)
    counts = np.array(counts)
    K2 = int(np.max(np.nonzero(counts)[0])) if np.any(counts) else 0
    Q2 = int(max(counts.max(), 1))
    if ((K2 + 1) * Q2) % 2:
        Q2 += 1
    return SPCA(bases=bases, eigs=eigs, counts=counts, K2=K2, Q2=Q2)


def spca_project(a: np.ndarray, fit: SPCA) -> np.ndarray:
    """b [N, K'+1, Q'] with b_ik = U_k^H a_ik in the first counts[k] entries of row k, zero elsewhere."""
    a = np.asarray(a, dtype=np.complex128)
    out = np.zeros((a.shape[0], fit.K2 + 1, fit.Q2), dtype=np.complex128)
    for k in range(fit.K2 + 1):
        U = fit.bases[k]
        out[:, k, :U.shape[1]] = a[:, k, :] @ U.conj()
    return out


def align_mean(y: np.ndarray, shifts: np.ndarray, L: int) -> np.ndarray:
    """a_hat = (1/N) sum_i e^{i k theta_hat_i} v^i, Eq. (synch_initialization)."""
    return np.mean(align(y, shifts, L), axis=0)


# ----------------------------------------------------------------------------
# prior on the distribution of rotations, Sec. 3.2 and Algorithm 1
# ----------------------------------------------------------------------------
def center_offset(xbar: np.ndarray, x: np.ndarray, L: int) -> int:
    """theta_c = argmin_theta ||R_theta xbar - x||^2 over the grid (Algorithm 1, centring step)."""
    r = rotate(xbar, grid_angle(np.arange(L), L))
    diff = r - x[None]
    return int(np.argmin(np.sum(diff.real ** 2 + diff.imag ** 2, axis=(1, 2))))


def residual_histogram(y, s_true, s_hat, x_true, L):
    """One trial of Algorithm 1: returns (counts [L], c, r [N]) with r_j = (s_j - s_hat_j + c) mod L."""
    xbar = align_mean(y, s_hat, L)
    c = center_offset(xbar, x_true, L)
    r = (np.asarray(s_true) - np.asarray(s_hat) + c) % L
    return np.bincount(r, minlength=L).astype(np.int64), c, r


def vm_ratio(kappa: float) -> float:
    """A(kappa) = I_1(kappa) / I_0(kappa) (scipy exponentially scaled Bessel functions)."""
    return float(special.ive(1, kappa) / special.ive(0, kappa))


def fit_kappa(mean_cos: float) -> float:
    """Maximum-likelihood von Mises concentration with the mean direction fixed at 0: A(kappa) = mean cos."""
    if mean_cos <= 0.0:
        return 0.0
    if mean_cos >= 1.0 - 1e-12:
        return 1e12
    hi = 1.0
    while vm_ratio(hi) < mean_cos:
        hi *= 2.0
    return float(optimize.brentq(lambda k: vm_ratio(k) - mean_cos, 0.0, hi, xtol=1e-13, rtol=1e-14, maxiter=500))


def fit_prior(counts: np.ndarray, L: int, Lw: int, l0: int | None = None, kind: int = 0, step: float = 1.0):
    """rho_bar (Algorithm 1, pooled over trials) restricted to the window and renormalised.

    kind 0: the learned histogram itself; a window position u (grid units, non-integer
    for step < 1) takes the value of the grid bin nearest to it, floor(u + 1/2) mod L.
    kind 1: von Mises fit log rho_bar[l] = kappa cos theta_l - log Z on the window,
    kappa from A(kappa) = sum_l rho_bar[l] cos(2 pi l/L).
    Returns (log_rho_bar [Lw], kappa).
    """
    counts = np.asarray(counts, dtype=np.float64)
    rho_bar = counts / counts.sum()
    offs = window_offsets(L, Lw, l0, step)
    if kind == 0:
        bins = np.mod(np.floor(np.asarray(offs, dtype=np.float64) + 0.5).astype(np.int64), L)
        v = rho_bar[bins]
        v = v / v.sum()
        with np.errstate(divide="ignore"):
            return np.log(v), 0.0
    mc = float(np.sum(rho_bar * np.cos(grid_angle(np.arange(L), L))))
    kappa = fit_kappa(mc)
    t = kappa * np.cos(grid_angle(offs, L))
    return t - _logsumexp(t, axis=0), kappa


# ----------------------------------------------------------------------------
# marginal log-likelihood and its gradient (Fisher identity)
# ----------------------------------------------------------------------------
def vm_log_rho(logits: np.ndarray, kappa: float, L: int, l0: int | None = None, step: float = 1.0) -> np.ndarray:
    """log rho_l = kappa cos theta_l + eta_l - log sum_win exp(kappa cos theta + eta)."""
    Lw = np.asarray(logits).size
    t = kappa * np.cos(grid_angle(window_offsets(L, Lw, l0, step), L)) + np.asarray(logits, dtype=np.float64)
    return t - _logsumexp(t, axis=0)


def loglik(y, x, logits, kappa, L, sigma2, l0=None, shifts=None, step=1.0) -> float:
    y = np.asarray(y, dtype=np.complex128)
    N, Kp1, Q = y.shape
    Lw = np.asarray(logits).size
    offs = window_offsets(L, Lw, l0, step)
    yt = y if shifts is None else align(y, np.asarray(shifts), L)
    _, _, lse = posterior(np.asarray(x, dtype=np.complex128), yt, vm_log_rho(logits, kappa, L, l0, step), L, offs,
                          sigma2)
    return marginal_loglik(lse, Kp1 * Q, sigma2)


def loglik_grad(y, x, logits, kappa, L, sigma2, l0=None, shifts=None, step=1.0):
    """(loglik, dx, dlogits, dkappa).  dx = dl/dRe x + i dl/dIm x = (2/sigma^2)(num - N x),
    dl/deta_l = W[l] - N rho_l, dl/dkappa = sum_l (W[l] - N rho_l) cos theta_l."""
    y = np.asarray(y, dtype=np.complex128)
    x = np.asarray(x, dtype=np.complex128)
    N, Kp1, Q = y.shape
    Lw = np.asarray(logits).size
    offs = window_offsets(L, Lw, l0, step)
    yt = y if shifts is None else align(y, np.asarray(shifts), L)
    lr = vm_log_rho(logits, kappa, L, l0, step)
    w, _, lse = posterior(x, yt, lr, L, offs, sigma2)
    W = w.sum(axis=0)
    back = np.exp(1j * np.outer(grid_angle(offs, L), kbar(Kp1 - 1)))
    num = np.einsum("jk,jkq->kq", w @ back, yt)
    dx = (2.0 / sigma2) * (num - N * x)
    rho = np.exp(lr)
    dl = W - N * rho
    dk = float(np.sum(dl * np.cos(grid_angle(offs, L))))
    return marginal_loglik(lse, Kp1 * Q, sigma2), dx, dl, dk


# ----------------------------------------------------------------------------
# relative error up to rotation, Sec. 2.2
# ----------------------------------------------------------------------------
def relerr(x_hat: np.ndarray, x: np.ndarray, n_grid: int = 4096) -> float:
    """min_theta ||R_theta I_hat - I||_F / ||I||_F on the coefficient vector, k > 0 rows counted twice."""
    x_hat = np.asarray(x_hat, dtype=np.complex128)
    x = np.asarray(x, dtype=np.complex128)
    K = x.shape[0] - 1
    wk = np.where(kbar(K) > 0, 2.0, 1.0)[:, None]

    def f(theta):
        d = rotate(x_hat, theta) - x
        return float(np.sum(wk * (d.real ** 2 + d.imag ** 2)))

    grid = TWO_PI * np.arange(n_grid) / n_grid
    vals = np.array([f(t) for t in grid])
    i = int(np.argmin(vals))
    h = TWO_PI / n_grid
    res = optimize.minimize_scalar(f, bracket=(grid[i] - h, grid[i], grid[i] + h), method="golden",
                                   options={"xtol": 1e-12})
    best = min(float(res.fun), float(vals[i]))
    return math.sqrt(max(best, 0.0)) / math.sqrt(float(np.sum(wk * (x.real ** 2 + x.imag ** 2))))
