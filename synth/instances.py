"""Synthetic MRA instances in coefficient space.

Recipe (one instance):

* signal ``x[k, q]`` for ``k = 0..K`` (angular index, only k >= 0 is stored
  because a real image satisfies a_{-k,q} = conj(a_{k,q}), Sec. 1) and
  ``q = 0..Q-1`` (radial index).  ``x[k, q] ~ CN(0, exp(-k^2 / decay))``,
  ``x[0, q]`` real, then scaled so that ``||x||_2 = 1`` over the stored entries.
* shifts ``s_i`` uniform on the grid ``{0, .., L-1}`` (rotation 2 pi s_i / L);
  the paper draws its rotations from such a grid too (Sec. 2.2, E. coli test).
* noise: i.i.d. circular complex Gaussian with E|eps|^2 = sigma^2 on every
  stored entry (Eq. MRA_Model_FB).  The SNR is the paper's pixel-space SNR,
  ||I||_F^2 / (n_pix sigma^2) (Sec. 1), for the paper's 129 x 129 images
  (n_pix = 16641, Sec. 2.2 and Sec. 4).  An orthonormal steerable basis keeps
  the per-coefficient noise variance equal to the pixel variance (App. A) and
  ||I||_F^2 equals the two-sided coefficient energy |a_0|^2 + 2 sum_{k>0} |a_k|^2,
  so sigma^2 = (|x_0|^2 + 2 sum_{k>0} |x_k|^2) / (16641 SNR).
* observation ``y_i = x o exp(-2 pi i k s_i / L) + eps_i`` (Eq. MRA_Model_FB).
* ``offgrid=True``: continuous rotations r_i = s_i + f_i grid units with f_i uniform on
  [-1/2, 1/2); ``s_i`` is then the nearest grid point and ``rot`` holds r_i (the
  workload of the denser-resolution window, Sec. 3.3).

The generator uses numpy's PCG64 stream seeded per instance.
"""
from __future__ import annotations

import dataclasses

import numpy as np

# Workload shapes.  Each entry is a coefficient-space stand-in for the paper's
# sPCA-expanded projection images (the ribosome data set is not used).
CONFIGS = {
    # plain Synch-EM: |k| <= 10, Q = 8, N = 500, L = 72, SNR 1/10, window 24, 20 iterations
    1: dict(K=10, Q=8, N=500, L=72, Lw=24, snr=1 / 10, decay=50.0, iters=20, P=100, gamma=100.0),
    # Synch-EM at scale: |k| <= 32, Q = 24, N = 1e5, L = 360, SNR 1/50, window 36, 50 iterations
    2: dict(K=32, Q=24, N=100_000, L=360, Lw=36, snr=1 / 50, decay=400.0, iters=50, P=100, gamma=100.0),
    # differentiable log-likelihood: |k| <= 16, Q = 16, N = 2e4, L = 180, SNR 1/20
    3: dict(K=16, Q=16, N=20_000, L=180, Lw=36, snr=1 / 20, decay=50.0, iters=30, P=100, gamma=100.0),
    # mixed precision at the largest size: |k| <= 48, Q = 32, N = 1e6, L = 720, window 72, SNR 1/100
    5: dict(K=48, Q=32, N=1_000_000, L=720, Lw=72, snr=1 / 100, decay=50.0, iters=50, P=100, gamma=100.0),
}


def config(n: int) -> dict:
    return dict(CONFIGS[n])


NPIX = 129 * 129  # pixels of the paper's projection images


def image_energy(x: np.ndarray) -> float:
    """||I||_F^2 of the real image with stored coefficients x (k < 0 half = conjugate of k > 0)."""
    return float(np.sum(np.abs(x[0]) ** 2) + 2.0 * np.sum(np.abs(x[1:]) ** 2))


def sigma2_for_snr(snr: float, x: np.ndarray) -> float:
    """Noise variance per coefficient for pixel-space SNR = ||I||_F^2 / (n_pix sigma^2)."""
    return image_energy(x) / (NPIX * snr)


def make_signal(K: int, Q: int, decay: float, rng: np.random.Generator) -> np.ndarray:
    k = np.arange(K + 1, dtype=np.float64)[:, None]
    std = np.sqrt(np.exp(-(k ** 2) / decay)) * np.ones((1, Q))
    x = (rng.standard_normal((K + 1, Q)) + 1j * rng.standard_normal((K + 1, Q))) * (std / np.sqrt(2.0))
    x[0, :] = rng.standard_normal(Q) * std[0, :]
    x /= np.linalg.norm(x)
    return x


def random_init(K: int, Q: int, decay: float, seed: int) -> np.ndarray:
    """A random starting point for plain EM: a fresh draw of the signal prior."""
    return make_signal(K, Q, decay, np.random.default_rng(seed))


@dataclasses.dataclass
class Instance:
    K: int
    Q: int
    N: int
    L: int
    sigma2: float
    x: np.ndarray  # complex128 [K+1, Q]
    s: np.ndarray  # int64 [N]
    y: np.ndarray  # complex128 [N, K+1, Q]
    rot: np.ndarray | None = None  # float64 [N] exact rotations in grid units (offgrid instances)


def make_instance(K: int, Q: int, N: int, L: int, snr: float | None = None, decay: float = 50.0,
                  seed: int = 0, sigma2: float | None = None, shifts: np.ndarray | None = None,
                  x: np.ndarray | None = None, offgrid: bool = False) -> Instance:
    """Draw one instance.  ``sigma2`` overrides ``snr``; ``sigma2 = 0`` is noise free."""
    rng = np.random.default_rng(seed)
    if x is None:
        x = make_signal(K, Q, decay, rng)
    if sigma2 is None:
        sigma2 = sigma2_for_snr(snr, x)
    if shifts is None:
        s = rng.integers(0, L, size=N).astype(np.int64)
    else:
        s = np.asarray(shifts, dtype=np.int64)
    rot = None
    if offgrid:
        rot = s + rng.uniform(-0.5, 0.5, size=N)
    k = np.arange(K + 1, dtype=np.float64)
    phase = np.exp(-2j * np.pi * np.outer(s if rot is None else rot, k) / L)  # [N, K+1]
    y = x[None, :, :] * phase[:, :, None]
    if sigma2 > 0:
        noise = rng.standard_normal((N, K + 1, Q)) + 1j * rng.standard_normal((N, K + 1, Q))
        y = y + noise * np.sqrt(sigma2 / 2.0)
    return Instance(K=K, Q=Q, N=N, L=L, sigma2=float(sigma2), x=x, s=s, y=y, rot=rot)


def to_c64(a: np.ndarray) -> np.ndarray:
    """Contiguous complex64 copy (the device storage type of observations)."""
    return np.ascontiguousarray(a, dtype=np.complex64)


def c64_round(a: np.ndarray) -> np.ndarray:
    """The complex128 values that a complex64 copy of ``a`` holds exactly."""
    return to_c64(a).astype(np.complex128)


def _bf16_rne_bits(f: np.ndarray) -> np.ndarray:
    """uint16 bit patterns of float32 values rounded to the nearest bfloat16, ties to even (finite inputs)."""
    u = np.ascontiguousarray(f, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = u + 0x7FFF + ((u >> 16) & 1)
    return (u >> 16).astype(np.uint16)


def bf16_split(y: np.ndarray) -> np.ndarray:
    """The BF16 hi/lo storage of complex64 observations: for each pair of complex values,
    one 16-byte group with bf16 hi = rn(v) of (re0, im0, re1, im1), then bf16 lo = rn(v - hi)
    of the same four values.  Returns a uint16 array of shape [count / 2, 8]."""
    f = to_c64(y).reshape(-1).view(np.float32).reshape(-1, 4)  # [groups, 4]
    hi = _bf16_rne_bits(f)
    hi_f = (hi.astype(np.uint32) << 16).view(np.float32)
    lo = _bf16_rne_bits(f - hi_f)
    return np.ascontiguousarray(np.concatenate([hi, lo], axis=1))


def bf16_merge(groups: np.ndarray, shape) -> np.ndarray:
    """complex128 values hi + lo held by a BF16 hi/lo split (exact in float32)."""
    g = np.asarray(groups, dtype=np.uint16).reshape(-1, 8).astype(np.uint32) << 16
    f = g.view(np.float32)
    v = (f[:, :4] + f[:, 4:]).astype(np.float32).reshape(-1)
    return v.view(np.complex64).astype(np.complex128).reshape(shape)


def config4_instances(seed: int = 4000, n_inst: int = 64, n_max: int | None = None) -> list[dict]:
    """The batched workload: n_inst independent problems with N ~ U[1000, 50000],
    K ~ U{8..40}, Q = 16, L = 360, window Lw ~ U{12..72}, pixel SNR log-uniform on
    [1/100, 1/5], 30 iterations each.  The list is fixed by ``seed``; ``n_max`` caps N
    (smaller test versions of the same list).  Each entry's ``seed`` draws its data."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_inst):
        N = int(rng.integers(1000, 50001))
        K = int(rng.integers(8, 41))
        Lw = int(rng.integers(12, 73))
        snr = float(np.exp(rng.uniform(np.log(1 / 100), np.log(1 / 5))))
        if n_max is not None:
            N = min(N, n_max)
        out.append(dict(N=N, K=K, Q=16, L=360, Lw=Lw, snr=snr, decay=50.0, iters=30, seed=seed + 1 + i))
    return out
