"""Shared helpers of the GPU parity tests (marshalling of numpy inputs to device tensors)."""
import numpy as np
import torch

import synth


def dev_y(y_c128: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(synth.to_c64(y_c128)).cuda()


def dev(a: np.ndarray, dtype=None) -> torch.Tensor:
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().numpy()


def rel_err(a, b) -> float:
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


# Tolerances of the GPU (FP32 arithmetic, FP64 cross-image sums) against the FP64 oracle, per EM step
# from identical inputs: relative 1e-5 in the image coefficients, absolute 1e-5 in the posterior weights.
TOL_X = 1e-5
TOL_W = 1e-5


def loglik_scale(y64, x, sigma2) -> float:
    """Magnitude of the terms that the log-likelihood sums (its value can be a small difference of them):
    beta sum_j ||y_j||^2 + N beta ||x||^2 + N M |log(pi sigma^2)|."""
    N = y64.shape[0]
    M = y64.shape[1] * y64.shape[2]
    beta = 1.0 / sigma2
    return float(beta * np.sum(np.abs(y64) ** 2) + N * beta * np.sum(np.abs(x) ** 2)
                 + N * M * abs(np.log(np.pi * sigma2)))


# FP32 per-image log-sum-exp against the FP64 oracle: relative to the summed terms
TOL_LL = 1e-7
