"""Pixel images of the steerable model (Sec. 1, Eq. fb_expansion2 with the Fourier-Bessel basis of
App. A): I(r, theta) = sum_{|k| <= K} sum_{q=1..Q} a_{k,q} u^{k,q}(r, theta) on an n x n pixel grid,
with a_{-k,q} = conj(a_{k,q}) so that I is real, plus white pixel noise.

Basis: u^{k,q}(r, theta) = N_{k,q} J_|k|(R_{|k|,q} r / c) e^{i k theta} for r <= c and 0 beyond, R_{k,q} the
q-th positive zero of J_k, N_{k,q} = 1 / (c sqrt(pi) |J_{k+1}(R_{k,q})|), c = (n - 1) / 2 (App. A).
Pixel (row iy, column ix) sits at x = ix - c, y = iy - c, r = |(x, y)|, theta = atan2(y, x).  Rotating
the coefficients by phi (a_k e^{-i k phi}) rotates the image: I(r, theta - phi).

The rendering is the forward model of the data only (it draws the observations the front end
receives); it holds none of the estimation arithmetic.
"""
from __future__ import annotations

import numpy as np
from scipy import special


def render_matrix(n: int, K: int, Q: int) -> np.ndarray:
    """Real matrix [n*n, Q + 2 K Q] mapping (a_0q, Re a_kq, Im a_kq for k >= 1) to pixel values, in the order
    of the stored coefficients [K+1][Q] (k = 0 first; then per k >= 1, per q, the Re then the Im column)."""
    c = (n - 1) / 2.0
    iy, ix = np.mgrid[0:n, 0:n]
    x, y = (ix - c).ravel(), (iy - c).ravel()
    r, th = np.hypot(x, y), np.arctan2(y, x)
    inside = r <= c
    cols = []
    for k in range(K + 1):
        zeros = special.jn_zeros(k, Q)
        for q in range(Q):
            f = np.where(inside, special.jv(k, zeros[q] * r / c), 0.0) / (c * np.sqrt(np.pi) * abs(special.jv(k + 1, zeros[q])))
            if k == 0:
                cols.append(f)
            else:
                cols.append(2.0 * f * np.cos(k * th))   # coefficient of Re a_kq (u^k and u^-k together)
                cols.append(-2.0 * f * np.sin(k * th))  # coefficient of Im a_kq
    return np.stack(cols, axis=1)


def real_params(a: np.ndarray) -> np.ndarray:
    """[..., K+1, Q] complex -> [..., Q + 2 K Q] real in the column order of render_matrix."""
    a = np.asarray(a, dtype=np.complex128)
    head = a[..., 0, :].real
    rest = np.stack([a[..., 1:, :].real, a[..., 1:, :].imag], axis=-1).reshape(a.shape[:-2] + (-1,))
    return np.concatenate([head, rest], axis=-1)


def render(a: np.ndarray, n: int, A: np.ndarray | None = None) -> np.ndarray:
    """Images [..., n, n] of coefficient arrays a [..., K+1, Q]."""
    a = np.asarray(a)
    K, Q = a.shape[-2] - 1, a.shape[-1]
    if A is None:
        A = render_matrix(n, K, Q)
    return (real_params(a) @ A.T).reshape(a.shape[:-2] + (n, n))


def noisy_images(a: np.ndarray, n: int, sigma: float, seed: int, A: np.ndarray | None = None) -> np.ndarray:
    """render(a) plus i.i.d. N(0, sigma^2) on every pixel."""
    img = render(a, n, A)
    return img + sigma * np.random.default_rng(seed).standard_normal(img.shape)
