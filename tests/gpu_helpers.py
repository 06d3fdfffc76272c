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
