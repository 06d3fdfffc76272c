"""Seeded 1-D multi-reference alignment instances (Sec. 3.1.1 and App. B) and their
coefficient-space form.

1-D model: x in R^L, observations v_i = roll(x, s_i) + eps_i with shifts s_i uniform on
{0, .., L-1} and eps_i ~ N(0, sigma^2 I) (roll(x, s)[n] = x[n - s mod L]).

Coefficient form (odd L): the DFT of a real signal holds everything in its entries
k = 0 .. (L-1)/2, and a cyclic shift by s multiplies entry k by exp(-2 pi i k s / L), the
rotation of Eq. (fb_rotation) with theta = 2 pi s / L.  Scaling a_0 = V_0 / sqrt(L) and
a_k = sqrt(2 / L) V_k (k >= 1) makes the sum of |a_k|^2 over the stored entries equal the
signal-space squared norm (Parseval), so distances, and with them every likelihood, are
those of the 1-D model.  The noise then has E|eps_k|^2 = 2 sigma^2 on the entries k >= 1
(circular) and is real with variance sigma^2 at k = 0; the 2-D model's
exp(-|d|^2 / sigma2) with sigma2 = 2 sigma^2 is the exact density in both cases (a real
difference d at k = 0 gives exp(-d^2 / (2 sigma^2))).  A second, all-zero radial column
pads the stored entries to an even count; it adds nothing to any distance.

This module draws data and changes basis only; it holds none of the estimation
arithmetic.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class Instance1D:
    L: int
    N: int
    sigma: float
    x: np.ndarray  # float64 [L]
    s: np.ndarray  # int64 [N]
    v: np.ndarray  # float64 [N, L] observations
    eps: np.ndarray  # float64 [N, L] the noise that was added


def make_instance_1d(L: int, N: int, sigma: float, seed: int = 0, x: np.ndarray | None = None,
                     shifts: np.ndarray | None = None) -> Instance1D:
    """x ~ N(0, I_L) unless given; shifts uniform unless given; v_i = roll(x, s_i) + sigma N(0, I)."""
    rng = np.random.default_rng(seed)
    if x is None:
        x = rng.standard_normal(L)
    s = rng.integers(0, L, size=N).astype(np.int64) if shifts is None else np.asarray(shifts, dtype=np.int64)
    eps = sigma * rng.standard_normal((N, L))
    idx = (np.arange(L)[None, :] - s[:, None]) % L
    v = np.asarray(x, dtype=np.float64)[idx] + eps
    return Instance1D(L=L, N=N, sigma=float(sigma), x=np.asarray(x, dtype=np.float64), s=s, v=v, eps=eps)


def coeffs_1d(v: np.ndarray) -> np.ndarray:
    """Scaled DFT coefficients [..., K+1, 2] (K = (L-1)/2, second column zero) of real signals [..., L], odd L."""
    v = np.asarray(v, dtype=np.float64)
    L = v.shape[-1]
    if L % 2 != 1:
        raise ValueError("the coefficient form is written for odd L")
    V = np.fft.fft(v, axis=-1)[..., : (L - 1) // 2 + 1]
    scale = np.full(V.shape[-1], np.sqrt(2.0 / L))
    scale[0] = np.sqrt(1.0 / L)
    a = np.zeros(V.shape + (2,), dtype=np.complex128)
    a[..., 0] = V * scale
    return a


def signal_1d(a: np.ndarray, L: int) -> np.ndarray:
    """The real signal [..., L] whose coefficient form is a [..., K+1, 2] (inverse of coeffs_1d)."""
    a = np.asarray(a, dtype=np.complex128)[..., 0]
    scale = np.full(a.shape[-1], np.sqrt(2.0 / L))
    scale[0] = np.sqrt(1.0 / L)
    V = a / scale
    full = np.zeros(a.shape[:-1] + (L,), dtype=np.complex128)
    full[..., : a.shape[-1]] = V
    full[..., L - a.shape[-1] + 1:] = np.conj(V[..., 1:][..., ::-1])
    return np.real(np.fft.ifft(full, axis=-1))


def sigma2_coeff(sigma: float) -> float:
    """The 2-D model's noise variance per stored complex entry for 1-D noise sigma: 2 sigma^2."""
    return 2.0 * float(sigma) ** 2
