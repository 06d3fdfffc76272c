"""Thin ctypes binding of libmra (include/mra.h).

Each function here has the name of the C entry point it calls and only
marshals arguments: torch CUDA tensors become device pointers, the current
torch stream becomes the cudaStream_t.  All computation happens in the CUDA
kernels of libmra; there is no CPU fallback.  If the library is missing the
import of any entry point raises.

Complex arrays are torch complex tensors (complex64 observations, complex128
state), which store interleaved (re, im) pairs exactly as the C ABI expects.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_int, c_int32, c_size_t, c_void_p

import torch

from . import build as _build

MRA_OK = 0
STATUS = {0: "ok", -1: "invalid argument", -2: "host allocation failed", -3: "CUDA runtime error",
          -4: "device wait timed out", -5: "non-finite value", -6: "workspace too small"}


class MraError(RuntimeError):
    def __init__(self, fn: str, status: int):
        super().__init__(f"{fn} failed: {STATUS.get(status, status)} ({status})")
        self.status = status


class mra_dims(ctypes.Structure):
    _fields_ = [("N", c_int32), ("K", c_int32), ("Q", c_int32), ("L", c_int32), ("sigma2", c_double)]


class mra_em_params(ctypes.Structure):
    _fields_ = [("Lw", c_int32), ("l0", c_int32), ("gamma", c_double), ("log_rho_bar", c_void_p),
                ("gamma_a_inv", c_void_p), ("update_rho", c_int32), ("tol", c_double), ("max_iters", c_int32),
                ("check_every", c_int32), ("sweep_ms", c_void_p), ("step", c_double)]


class mra_instance(ctypes.Structure):
    _fields_ = [("dims", mra_dims), ("prm", mra_em_params), ("y", c_void_p), ("y_format", c_int32),
                ("shift", c_void_p), ("x_inout", c_void_p), ("log_rho_inout", c_void_p), ("stats_out", c_void_p)]


_lib = None
_SIGS = {
    "mra_status_string": (ctypes.c_char_p, [c_int]),
    "mra_device_info": (c_int, [POINTER(c_int32), POINTER(c_int32)]),
    "mra_em_workspace_bytes": (c_size_t, [POINTER(mra_dims), c_int32]),
    "mra_em_step": (c_int, [POINTER(mra_dims), POINTER(mra_em_params)] + [c_void_p] * 9 + [c_void_p, c_size_t, c_void_p]),
    "mra_em_step_noalloc": (c_int, [POINTER(mra_dims), POINTER(mra_em_params)] + [c_void_p] * 9 + [c_void_p]),
    "mra_em_run": (c_int, [POINTER(mra_dims), POINTER(mra_em_params)] + [c_void_p] * 4 + [POINTER(c_int32), c_void_p,
                                                                                          c_void_p, c_void_p, c_size_t,
                                                                                          c_void_p]),
    "mra_em_step_hl": (c_int, [POINTER(mra_dims), POINTER(mra_em_params)] + [c_void_p] * 9 + [c_void_p, c_size_t,
                                                                                             c_void_p]),
    "mra_em_run_hl": (c_int, [POINTER(mra_dims), POINTER(mra_em_params)] + [c_void_p] * 4 + [POINTER(c_int32), c_void_p,
                                                                                             c_void_p, c_void_p,
                                                                                             c_size_t, c_void_p]),
    "mra_y_split_bf16": (c_int, [c_void_p, ctypes.c_int64, c_void_p, c_void_p]),
    "mra_em_autotune": (c_int, [POINTER(mra_dims), POINTER(mra_em_params), c_void_p, c_int32, c_void_p, c_void_p,
                                c_void_p, POINTER(c_int32), c_void_p, c_size_t, c_void_p]),
    "mra_em_batched_workspace_bytes": (c_size_t, [POINTER(mra_instance), c_int32]),
    "mra_em_run_batched": (c_int, [POINTER(mra_instance), c_int32, c_int32, POINTER(c_int32), POINTER(ctypes.c_float),
                                   c_void_p, c_size_t, c_void_p]),
    "mra_loglik_grad": (c_int, [POINTER(mra_dims), c_int32, c_int32, c_double, c_void_p, c_void_p, c_void_p, c_void_p,
                                c_double, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "mra_sync_workspace_bytes": (c_size_t, [POINTER(mra_dims), c_int32]),
    "mra_sync_pairwise": (c_int, [POINTER(mra_dims), c_void_p, c_int32, c_void_p, c_void_p]),
    "mra_sync_ppm": (c_int, [c_int32, c_int32, c_void_p, c_int32, c_int32, c_void_p, c_void_p]),
    "mra_sync_match": (c_int, [POINTER(mra_dims), c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "mra_template_match": (c_int, [POINTER(mra_dims), c_void_p, c_void_p, c_void_p, c_void_p]),
    "mra_fb_setup_workspace_bytes": (c_size_t, [c_int32, c_int32, c_int32]),
    "mra_fb_setup": (c_int, [c_int32, c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "mra_fb_operand_bytes": (c_size_t, [c_int32, c_int32, c_int32]),
    "mra_fb_pack": (c_int, [c_int32, c_int32, c_int32, c_void_p, c_void_p, c_void_p]),
    "mra_fb_project": (c_int, [c_int32, c_int32, c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_int32, c_void_p]),
    "mra_spca_workspace_bytes": (c_size_t, [POINTER(mra_dims)]),
    "mra_spca_fit": (c_int, [POINTER(mra_dims), c_void_p, c_void_p, c_void_p, c_void_p, POINTER(c_int32),
                             POINTER(c_int32), c_void_p, c_size_t, c_void_p]),
    "mra_spca_project": (c_int, [POINTER(mra_dims), c_void_p, c_int32, c_int32, c_void_p, c_void_p, c_void_p]),
    "mra_hermitian_eig": (c_int, [c_int32, c_void_p, c_void_p, c_void_p]),
    "mra_sync": (c_int, [POINTER(mra_dims), c_void_p, c_int32, c_int32, c_int32, c_void_p, c_void_p, c_size_t,
                         c_void_p]),
    "mra_align_mean": (c_int, [POINTER(mra_dims), c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "mra_prior_hist": (c_int, [POINTER(mra_dims), c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                               c_size_t, c_void_p]),
    "mra_fit_prior": (c_int, [c_int32, c_int32, c_int32, c_double, c_void_p, c_int32, c_void_p, c_void_p, c_void_p]),
    "mra_relerr": (c_int, [c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_void_p]),
    "mra_ws_status": (c_int, [c_void_p, c_void_p]),
    "mra_em_step_noalloc_status": (c_int, [c_void_p]),
    "mra_selftest_wait_timeout": (c_int, [c_int32, c_void_p, c_void_p]),
    "mra_selftest_grid_barrier": (c_int, [c_int32, c_void_p, c_void_p]),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libmra.so (building it in-tree first if it is missing); raise if that fails."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"libmra.so not built at {path}")
        _build.build_library()
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def exported_symbols() -> list[str]:
    return list(_SIGS)


# ---------------------------------------------------------------- marshalling helpers
def _p(t):
    if t is None:
        return None
    if isinstance(t, int):
        return c_void_p(t)
    if not t.is_cuda:
        raise ValueError("libmra takes device tensors")
    if not t.is_contiguous():
        raise ValueError("libmra takes contiguous tensors")
    return c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return c_void_p(s.cuda_stream)


def _check(fn: str, st: int):
    if st != MRA_OK:
        raise MraError(fn, st)


def dims(N: int, K: int, Q: int, L: int, sigma2: float) -> mra_dims:
    return mra_dims(int(N), int(K), int(Q), int(L), float(sigma2))


def em_params(Lw: int, l0: int | None = None, gamma: float = 0.0, log_rho_bar=None, gamma_a_inv=None,
              update_rho: bool = True, tol: float = 0.0, max_iters: int = 1, check_every: int | None = None,
              sweep_ms=None, step: float = 1.0):
    """sweep_ms: optional host ctypes float array [max_iters] that receives each sweep's device time.
    step: spacing of the window's rotations in grid units (1 = the grid, < 1 the denser window)."""
    if l0 is None:
        l0 = -(Lw // 2)
    p = mra_em_params(int(Lw), int(l0), float(gamma), _p(log_rho_bar), _p(gamma_a_inv), 1 if update_rho else 0,
                      float(tol), int(max_iters), int(check_every if check_every else max_iters),
                      ctypes.cast(sweep_ms, c_void_p) if sweep_ms is not None else None, float(step))
    p._keep = (log_rho_bar, gamma_a_inv, sweep_ms)  # keep buffers alive with the struct
    return p


def mra_em_workspace_bytes(d: mra_dims, Lw: int) -> int:
    return int(load().mra_em_workspace_bytes(ctypes.byref(d), int(Lw)))


def mra_sync_workspace_bytes(d: mra_dims, P: int) -> int:
    return int(load().mra_sync_workspace_bytes(ctypes.byref(d), int(P)))


def workspace(nbytes: int, device=None) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device or "cuda")


def mra_device_info():
    a, b = c_int32(), c_int32()
    _check("mra_device_info", load().mra_device_info(ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


# ---------------------------------------------------------------- entry points
def mra_em_step(d, prm, y, shift, x_in, log_rho_in, x_out, log_rho_out, loglik_out=None, step_out=None, w_out=None,
                ws=None, stream=None):
    _check("mra_em_step", load().mra_em_step(ctypes.byref(d), ctypes.byref(prm), _p(y), _p(shift), _p(x_in),
                                             _p(log_rho_in), _p(x_out), _p(log_rho_out), _p(loglik_out), _p(step_out),
                                             _p(w_out), _p(ws), ws.numel(), _stream(stream)))


def mra_em_step_noalloc(d, prm, y, shift, x_in, log_rho_in, x_out, log_rho_out, loglik_out=None, step_out=None,
                        w_out=None, stream=None):
    """mra_em_step without a workspace argument: the library's fixed 8 MiB device array serves as scratch."""
    _check("mra_em_step_noalloc", load().mra_em_step_noalloc(ctypes.byref(d), ctypes.byref(prm), _p(y), _p(shift),
                                                             _p(x_in), _p(log_rho_in), _p(x_out), _p(log_rho_out),
                                                             _p(loglik_out), _p(step_out), _p(w_out),
                                                             _stream(stream)))


def mra_em_run(d, prm, y, shift, x_inout, log_rho_inout, stats_out=None, x_traj_out=None, ws=None, stream=None) -> int:
    it = c_int32(0)
    _check("mra_em_run", load().mra_em_run(ctypes.byref(d), ctypes.byref(prm), _p(y), _p(shift), _p(x_inout),
                                           _p(log_rho_inout), ctypes.byref(it), _p(stats_out), _p(x_traj_out), _p(ws),
                                           ws.numel(), _stream(stream)))
    return it.value


def mra_y_split_bf16(y, y_hl_out, stream=None):
    """y (complex64, any shape) -> its BF16 hi/lo split in y_hl_out (same byte size, 16-byte groups)."""
    _check("mra_y_split_bf16", load().mra_y_split_bf16(_p(y), int(y.numel()), _p(y_hl_out), _stream(stream)))


def mra_em_step_hl(d, prm, y_hl, shift, x_in, log_rho_in, x_out, log_rho_out, loglik_out=None, step_out=None,
                   w_out=None, ws=None, stream=None):
    _check("mra_em_step_hl", load().mra_em_step_hl(ctypes.byref(d), ctypes.byref(prm), _p(y_hl), _p(shift), _p(x_in),
                                                   _p(log_rho_in), _p(x_out), _p(log_rho_out), _p(loglik_out),
                                                   _p(step_out), _p(w_out), _p(ws), ws.numel(), _stream(stream)))


def mra_em_run_hl(d, prm, y_hl, shift, x_inout, log_rho_inout, stats_out=None, x_traj_out=None, ws=None,
                  stream=None) -> int:
    it = c_int32(0)
    _check("mra_em_run_hl", load().mra_em_run_hl(ctypes.byref(d), ctypes.byref(prm), _p(y_hl), _p(shift),
                                                 _p(x_inout), _p(log_rho_inout), ctypes.byref(it), _p(stats_out),
                                                 _p(x_traj_out), _p(ws), ws.numel(), _stream(stream)))
    return it.value


def mra_em_autotune(d, prm, y, shift, x, log_rho, ws, y_format=0, stream=None):
    """Time every applicable EM sweep on this problem and cache the fastest; returns (kind, images, stages):
    kind 1 warp, 2 batch, 3 chunked (0 none applies); images per batch or chunk; ring stages or CTAs per SM."""
    ch = (c_int32 * 3)()
    _check("mra_em_autotune", load().mra_em_autotune(ctypes.byref(d), ctypes.byref(prm), _p(y), int(y_format),
                                                     _p(shift), _p(x), _p(log_rho), ch, _p(ws), ws.numel(),
                                                     _stream(stream)))
    return tuple(ch)


def instances(items):
    """ctypes array of mra_instance from dicts with keys d, prm, y, x, log_rho and optional shift, stats, y_format.
    The tensors must stay alive while the array is used."""
    arr = (mra_instance * len(items))()
    for a, it in zip(arr, items):
        a.dims = it["d"]
        a.prm = it["prm"]
        a.y = _p(it["y"])
        a.y_format = int(it.get("y_format", 0))
        a.shift = _p(it.get("shift"))
        a.x_inout = _p(it["x"])
        a.log_rho_inout = _p(it["log_rho"])
        a.stats_out = _p(it.get("stats"))
    return arr


def mra_em_batched_workspace_bytes(arr) -> int:
    return int(load().mra_em_batched_workspace_bytes(arr, len(arr)))


def mra_em_run_batched(arr, ws, tune=True, stream=None):
    """All instances in one graph launch; returns (iterations per instance, device ms of the launch)."""
    n = len(arr)
    it = (c_int32 * n)()
    ms = ctypes.c_float(0.0)
    _check("mra_em_run_batched", load().mra_em_run_batched(arr, n, 1 if tune else 0, it, ctypes.byref(ms), _p(ws),
                                                           ws.numel(), _stream(stream)))
    return list(it), ms.value


def mra_loglik_grad(d, Lw, l0, y, shift, x, logits, kappa, loglik_out, dx_out=None, dlogits_out=None, dkappa_out=None,
                    ws=None, stream=None, step=1.0):
    _check("mra_loglik_grad", load().mra_loglik_grad(ctypes.byref(d), int(Lw), int(l0), float(step), _p(y), _p(shift),
                                                     _p(x),
                                                     _p(logits), float(kappa), _p(loglik_out), _p(dx_out),
                                                     _p(dlogits_out), _p(dkappa_out), _p(ws), ws.numel(),
                                                     _stream(stream)))


def mra_sync_pairwise(d, y, P, rel_out, stream=None):
    _check("mra_sync_pairwise", load().mra_sync_pairwise(ctypes.byref(d), _p(y), int(P), _p(rel_out), _stream(stream)))


def mra_sync_ppm(L, P, rel, n_power, n_ppm, phi_out, stream=None):
    _check("mra_sync_ppm", load().mra_sync_ppm(int(L), int(P), _p(rel), int(n_power), int(n_ppm), _p(phi_out),
                                               _stream(stream)))


def mra_sync_match(d, y, P, phi, shift_out, ws, stream=None):
    _check("mra_sync_match", load().mra_sync_match(ctypes.byref(d), _p(y), int(P), _p(phi), _p(shift_out), _p(ws),
                                                   ws.numel(), _stream(stream)))


def mra_fb_setup_workspace_bytes(n, K, Q) -> int:
    return int(load().mra_fb_setup_workspace_bytes(int(n), int(K), int(Q)))


def mra_fb_setup(n, K, Q, P_out, zeros_out, ws, stream=None):
    _check("mra_fb_setup", load().mra_fb_setup(int(n), int(K), int(Q), _p(P_out), _p(zeros_out), _p(ws), ws.numel(),
                                               _stream(stream)))


def mra_fb_operand_bytes(n, K, Q) -> int:
    return int(load().mra_fb_operand_bytes(int(n), int(K), int(Q)))


def mra_fb_pack(n, K, Q, P, op_out, stream=None):
    _check("mra_fb_pack", load().mra_fb_pack(int(n), int(K), int(Q), _p(P), _p(op_out), _stream(stream)))


def mra_fb_project(N, n, K, Q, images, op, y_out, fast=False, stream=None):
    """op: the packed projection operand of mra_fb_pack (see fb_operand)."""
    _check("mra_fb_project", load().mra_fb_project(int(N), int(n), int(K), int(Q), _p(images), _p(op), _p(y_out),
                                                   1 if fast else 0, _stream(stream)))


def fb_operand(n, K, Q, P, stream=None) -> torch.Tensor:
    """The packed projection operand of P (a byte tensor) for mra_fb_project."""
    op = workspace(mra_fb_operand_bytes(n, K, Q), P.device)
    mra_fb_pack(n, K, Q, P, op, stream)
    return op


def mra_spca_workspace_bytes(d) -> int:
    return int(load().mra_spca_workspace_bytes(ctypes.byref(d)))


def mra_spca_fit(d, y, basis_out, ws, stream=None):
    """Returns (K2, Q2, counts [K+1] numpy int32, eigenvalues [K+1, Q] numpy float64)."""
    import numpy as np

    counts = np.zeros(d.K + 1, dtype=np.int32)
    eigs = np.zeros((d.K + 1, d.Q), dtype=np.float64)
    K2, Q2 = c_int32(0), c_int32(0)
    _check("mra_spca_fit", load().mra_spca_fit(ctypes.byref(d), _p(y), _p(basis_out), eigs.ctypes.data,
                                               counts.ctypes.data, ctypes.byref(K2), ctypes.byref(Q2), _p(ws),
                                               ws.numel(), _stream(stream)))
    return K2.value, Q2.value, counts, eigs


def mra_spca_project(d, y, K2, Q2, basis, y_out, stream=None):
    _check("mra_spca_project", load().mra_spca_project(ctypes.byref(d), _p(y), int(K2), int(Q2), _p(basis),
                                                       _p(y_out), _stream(stream)))


def mra_hermitian_eig(A):
    """Host eigen-decomposition of a Hermitian numpy matrix: (w descending, V columns)."""
    import numpy as np

    A = np.asfortranarray(np.asarray(A, dtype=np.complex128))
    n = A.shape[0]
    w = np.zeros(n, dtype=np.float64)
    V = np.zeros((n, n), dtype=np.complex128, order="F")
    _check("mra_hermitian_eig", load().mra_hermitian_eig(n, A.ctypes.data, w.ctypes.data, V.ctypes.data))
    return w, V


def mra_template_match(d, y, ref, shift_out, stream=None):
    _check("mra_template_match", load().mra_template_match(ctypes.byref(d), _p(y), _p(ref), _p(shift_out),
                                                           _stream(stream)))


def mra_sync(d, y, P, n_power, n_ppm, shift_out, ws, stream=None):
    _check("mra_sync", load().mra_sync(ctypes.byref(d), _p(y), int(P), int(n_power), int(n_ppm), _p(shift_out),
                                       _p(ws), ws.numel(), _stream(stream)))


def mra_align_mean(d, y, shift, x_out, ws, stream=None):
    _check("mra_align_mean", load().mra_align_mean(ctypes.byref(d), _p(y), _p(shift), _p(x_out), _p(ws), ws.numel(),
                                                   _stream(stream)))


def mra_prior_hist(d, y, shift_true, shift_est, x_true, hist_inout, center_out=None, ws=None, stream=None):
    _check("mra_prior_hist", load().mra_prior_hist(ctypes.byref(d), _p(y), _p(shift_true), _p(shift_est), _p(x_true),
                                                   _p(hist_inout), _p(center_out), _p(ws), ws.numel(),
                                                   _stream(stream)))


def mra_fit_prior(L, Lw, l0, counts, kind, log_prior_out, kappa_out=None, stream=None, step=1.0):
    _check("mra_fit_prior", load().mra_fit_prior(int(L), int(Lw), int(l0), float(step), _p(counts), int(kind),
                                                 _p(log_prior_out), _p(kappa_out), _stream(stream)))


def mra_relerr(K, Q, x_hat, x, err_out, stream=None):
    _check("mra_relerr", load().mra_relerr(int(K), int(Q), _p(x_hat), _p(x), _p(err_out), _stream(stream)))


def mra_ws_status(ws, stream=None) -> int:
    return int(load().mra_ws_status(_p(ws), _stream(stream)))


def mra_em_step_noalloc_status(stream=None) -> int:
    return int(load().mra_em_step_noalloc_status(_stream(stream)))


def mra_selftest_wait_timeout(limit_us, status_out, stream=None):
    """Run the bounded-wait self-test; status_out (device int32[1]) receives MRA_ETIMEOUT (-4) or MRA_OK."""
    _check("mra_selftest_wait_timeout", load().mra_selftest_wait_timeout(int(limit_us), _p(status_out),
                                                                         _stream(stream)))


def mra_selftest_grid_barrier(limit_us, scratch, stream=None):
    """Run the grid-barrier self-test; scratch (device int32[4]) receives the status in scratch[2]."""
    _check("mra_selftest_grid_barrier", load().mra_selftest_grid_barrier(int(limit_us), _p(scratch),
                                                                         _stream(stream)))
