"""GPU parity of the denser-resolution window (Sec. 3.3): Lw rotations 2 pi step (l0 + i) / L
with step < 1, off the grid.  Every sweep (warp per image, CTA batch, chunked two-read, and the
tile sweep for rows of Q not a multiple of 8) against the FP64 oracle on the same inputs, the
window prior (Algorithm 1 histogram and von Mises fit) and the log-likelihood gradient on such a
window, plus properties at sizes the oracle does not reach."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import synth
from gpu_helpers import TOL_LL, TOL_W, TOL_X, dev, dev_y, host, loglik_scale, rel_err

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]


def _step(mra, inst, y64, x, log_rho, Lw, l0, step, shifts=None, gamma=0.0, log_rho_bar=None):
    d = mra.dims(inst.N, inst.K, inst.Q, inst.L, inst.sigma2)
    lrb = dev(log_rho_bar) if log_rho_bar is not None else None
    prm = mra.em_params(Lw, l0=l0, gamma=gamma, log_rho_bar=lrb, step=step)
    xi, lri = dev(x.astype(np.complex128)), dev(np.asarray(log_rho, dtype=np.float64))
    xo, lro = torch.empty_like(xi), torch.empty_like(lri)
    ll = torch.empty(1, dtype=torch.float64, device="cuda")
    stp = torch.empty(1, dtype=torch.float64, device="cuda")
    w = torch.empty((inst.N, Lw), dtype=torch.float32, device="cuda")
    ws = mra.workspace(mra.mra_em_workspace_bytes(d, Lw))
    sh = dev(shifts.astype(np.int32)) if shifts is not None else None
    mra.mra_em_step(d, prm, dev_y(y64), sh, xi, lri, xo, lro, ll, stp, w, ws)
    torch.cuda.synchronize()
    assert mra.mra_ws_status(ws) == 0
    return host(xo), host(lro), float(ll.item()), float(stp.item()), host(w)


def _compare(mra, inst, x, log_rho, Lw, l0, step, shifts=None, **kw):
    y64 = synth.c64_round(inst.y)
    xg, lrg, llg, stg, wg = _step(mra, inst, y64, x, log_rho, Lw, l0, step, shifts=shifts, **kw)
    st = O.em_step(y64, x, log_rho, inst.L, inst.sigma2, Lw=Lw, l0=l0, shifts=shifts, step=step, **kw)
    assert rel_err(xg, st.x) <= TOL_X, rel_err(xg, st.x)
    assert np.max(np.abs(wg - st.w)) <= TOL_W, np.max(np.abs(wg - st.w))
    np.testing.assert_allclose(np.exp(lrg), np.exp(st.log_rho), atol=1e-5, rtol=0)
    assert abs(llg - st.loglik) <= TOL_LL * loglik_scale(y64, x, inst.sigma2), (llg, st.loglik)
    assert abs(stg - st.step) <= 1e-5 * math.sqrt(st.step) + 1e-10, (stg, st.step)
    return xg, st


@pytest.fixture(params=["cta", "warp", "chunk", "cta-tdg", "tc"])
def sweep(request, monkeypatch):
    """cta-tdg: the batch sweep with its distance-unit table read from global memory."""
    monkeypatch.setenv("MRA_SWEEP", request.param.split("-")[0])
    if request.param.endswith("-tdg"):
        monkeypatch.setenv("MRA_SWEEP_TDG", "1")
    return request.param


# (K, Q, N, L, Lw, l0, step): a one-chunk window, a wide one, the paper's example at a reduced L
# (Lw = 2 L + 1, l0 = -L, step = BW / (2 L) with BW = 18), a window off centre, and one of more
# than 512 rotations (the split sweep's transform in two passes of tensor-memory columns)
SHAPES = [
    (12, 16, 1500, 90, 31, -15, 0.35),
    (8, 16, 900, 120, 201, -100, 0.4),
    (10, 8, 700, 60, 121, -60, 0.15),
    (6, 24, 1100, 72, 47, -9, 0.6),
    (10, 16, 600, 360, 601, -300, 0.5),
]


@pytest.mark.parametrize("K,Q,N,L,Lw,l0,step", SHAPES)
def test_dense_em_step_matches_oracle(gpu_lib, sweep, K, Q, N, L, Lw, l0, step):
    inst = synth.make_instance(K, Q, N, L, snr=1 / 5, decay=50.0, seed=8100 + Lw, offgrid=True)
    y64 = synth.c64_round(inst.y)
    x0 = O.align_mean(y64, inst.s, inst.L)
    rng = np.random.default_rng(Lw)
    lr = np.log(rng.random(Lw) + 0.2)
    lr -= np.log(np.exp(lr).sum())
    _compare(gpu_lib, inst, x0, lr, Lw, l0, step, shifts=inst.s)


@pytest.mark.parametrize("kind", ["warp", "cta", "tc"])
def test_dense_paper_example_window_full_workload_shape(gpu_lib, kind, monkeypatch):
    """The paper's example of the denser window at the Synch-EM workload's shape: the range
    [-pi BW/L, pi BW/L] with BW = 36 at spacing pi BW/L^2 (Lw = 2 L + 1 = 721 rotations 0.05 grid units
    apart, |k| <= 32, Q = 24, L = 360).  Its unit tables do not fit in shared memory next to the image
    rings, so the warp sweep and the batch sweep read them from global memory; the split sweep runs
    its transform in two passes of tensor-memory columns and keeps the first distances of its table
    in shared memory."""
    monkeypatch.setenv("MRA_SWEEP", kind)
    K, Q, L = 32, 24, 360
    inst = synth.make_instance(K, Q, 300, L, snr=1 / 50, decay=400.0, seed=8150, offgrid=True)
    x0 = O.align_mean(synth.c64_round(inst.y), inst.s, inst.L)
    Lw = 2 * L + 1
    _compare(gpu_lib, inst, x0, np.log(np.full(Lw, 1 / Lw)), Lw, -L, 36 / (2 * L), shifts=inst.s)


def test_dense_em_step_tile_sweep_odd_rows(gpu_lib):
    """Rows of Q = 6 (not a multiple of 8) take the tile sweep and its window twiddle table."""
    inst = synth.make_instance(5, 6, 800, 40, snr=1 / 3, decay=20.0, seed=8200, offgrid=True)
    x0 = O.align_mean(synth.c64_round(inst.y), inst.s, inst.L)
    Lw = 25
    _compare(gpu_lib, inst, x0, np.log(np.full(Lw, 1 / Lw)), Lw, -12, 0.5, shifts=inst.s)


def test_dense_em_step_prior_gamma_and_empty_bins(gpu_lib, sweep):
    inst = synth.make_instance(12, 16, 1200, 90, snr=1 / 10, decay=50.0, seed=8300, offgrid=True)
    Lw, l0, step = 41, -20, 0.25
    t = 3.0 * np.cos(2 * np.pi * step * (l0 + np.arange(Lw)) / inst.L)
    lrb = t - np.log(np.exp(t).sum())
    lrb[:3] = -np.inf  # empty bins
    x0 = O.align_mean(synth.c64_round(inst.y), inst.s, inst.L)
    _compare(gpu_lib, inst, x0, lrb.copy(), Lw, l0, step, shifts=inst.s, gamma=50.0, log_rho_bar=lrb)


def test_dense_em_run_trajectory(gpu_lib, sweep):
    mra = gpu_lib
    inst = synth.make_instance(12, 16, 2000, 90, snr=1 / 5, decay=50.0, seed=8400, offgrid=True)
    y64 = synth.c64_round(inst.y)
    Lw, l0, step, T = 37, -18, 1 / 3, 4
    x0 = O.align_mean(y64, inst.s, inst.L)
    lr0 = np.log(np.full(Lw, 1 / Lw))
    d = mra.dims(inst.N, inst.K, inst.Q, inst.L, inst.sigma2)
    prm = mra.em_params(Lw, l0=l0, max_iters=T, step=step)
    ws = mra.workspace(mra.mra_em_workspace_bytes(d, Lw))
    x, lr = dev(x0), dev(lr0)
    traj = torch.empty((T, inst.K + 1, inst.Q), dtype=torch.complex128, device="cuda")
    assert mra.mra_em_run(d, prm, dev_y(y64), dev(inst.s.astype(np.int32)), x, lr, None, traj, ws) == T
    xs, lrs = x0, lr0
    for t in range(T):
        st = O.em_step(y64, xs, lrs, inst.L, inst.sigma2, Lw=Lw, l0=l0, shifts=inst.s, step=step)
        assert rel_err(host(traj[t]), st.x) <= TOL_X * (t + 1), (t, rel_err(host(traj[t]), st.x))
        xs, lrs = st.x, st.log_rho
    np.testing.assert_allclose(np.exp(host(lr)), np.exp(lrs), atol=1e-5 * T, rtol=0)


@pytest.mark.parametrize("Lw,l0,step", [(201, -100, 0.4), (61, -30, 1.0)])
def test_wide_window_warp_sweep_hands_out_images(gpu_lib, monkeypatch, Lw, l0, step):
    """More images (7,000) than two per warp of the persistent grid (152 CTAs x 16 warps), so that the warp
    sweep on a window wider than one unit chunk hands the rest out one at a time from its counter; three
    EM iterations in one run (the counter must be clear again at every sweep) against the oracle."""
    monkeypatch.setenv("MRA_SWEEP", "warp")
    mra = gpu_lib
    inst = synth.make_instance(8, 16, 7000, 120, snr=1 / 5, decay=50.0, seed=8450 + Lw, offgrid=step != 1.0)
    y64 = synth.c64_round(inst.y)
    T = 3
    x0 = O.align_mean(y64, inst.s, inst.L)
    lr0 = np.log(np.full(Lw, 1 / Lw))
    d = mra.dims(inst.N, inst.K, inst.Q, inst.L, inst.sigma2)
    prm = mra.em_params(Lw, l0=l0, max_iters=T, step=step)
    ws = mra.workspace(mra.mra_em_workspace_bytes(d, Lw))
    x, lr = dev(x0), dev(lr0)
    traj = torch.empty((T, inst.K + 1, inst.Q), dtype=torch.complex128, device="cuda")
    assert mra.mra_em_run(d, prm, dev_y(y64), dev(inst.s.astype(np.int32)), x, lr, None, traj, ws) == T
    assert mra.mra_ws_status(ws) == 0
    xs, lrs = x0, lr0
    for t in range(T):
        st = O.em_step(y64, xs, lrs, inst.L, inst.sigma2, Lw=Lw, l0=l0, shifts=inst.s, step=step)
        assert rel_err(host(traj[t]), st.x) <= TOL_X * (t + 1), (t, rel_err(host(traj[t]), st.x))
        xs, lrs = st.x, st.log_rho
    np.testing.assert_allclose(np.exp(host(lr)), np.exp(lrs), atol=1e-5 * T, rtol=0)


def test_dense_window_on_grid_points_equals_grid_window(gpu_lib, sweep):
    """Property at the full size of the Synch-EM workload's shape (|k| <= 32, Q = 24, L = 360, window 36,
    N = 20,000): a step-1/4 window whose prior is zero off the grid points gives the grid window's result."""
    mra = gpu_lib
    c = synth.config(2)
    inst = synth.make_instance(c["K"], c["Q"], 20_000, c["L"], c["snr"], c["decay"], seed=8500)
    y = dev_y(inst.y)
    sh = dev(inst.s.astype(np.int32))
    d = mra.dims(inst.N, inst.K, inst.Q, inst.L, inst.sigma2)
    x0 = dev(O.align_mean(synth.c64_round(inst.y[:2000]), inst.s[:2000], inst.L))
    Lw, m = 37, 4
    l0 = -(Lw // 2)
    lr = np.log(np.full(Lw, 1 / Lw))
    Lwd = m * (Lw - 1) + 1
    lrd = np.full(Lwd, -np.inf)
    lrd[::m] = lr

    def run(Lw_, l0_, lr_, step):
        prm = mra.em_params(Lw_, l0=l0_, step=step)
        xo = torch.empty_like(x0)
        lro = torch.empty(Lw_, dtype=torch.float64, device="cuda")
        ll = torch.empty(1, dtype=torch.float64, device="cuda")
        ws = mra.workspace(mra.mra_em_workspace_bytes(d, Lw_))
        mra.mra_em_step(d, prm, y, sh, x0, dev(lr_), xo, lro, ll, None, None, ws)
        torch.cuda.synchronize()
        return host(xo), host(lro), float(ll.item())

    xg, lrg, llg = run(Lw, l0, lr, 1.0)
    xd, lrdo, lld = run(Lwd, m * l0, lrd, 1.0 / m)
    assert rel_err(xd, xg) <= 2 * TOL_X, rel_err(xd, xg)
    np.testing.assert_allclose(np.exp(lrdo[::m]), np.exp(lrg), atol=1e-6, rtol=0)
    assert np.all(np.exp(lrdo[np.arange(Lwd) % m != 0]) == 0.0)
    assert abs(lld - llg) <= 1e-6 * abs(llg)


def test_dense_noise_free_off_grid_rotations_recovered(gpu_lib, sweep):
    """Images rotated by off-grid angles of the window, nearly noise free: the weights are one-hot at each
    image's angle and the M-step returns the signal, at N = 30,000."""
    mra = gpu_lib
    K, Q, L, N = 16, 16, 180, 30_000
    Lw, l0, step = 61, -30, 0.2
    rng = np.random.default_rng(5)
    x = synth.make_signal(K, Q, 50.0, rng)
    idx = rng.integers(0, Lw, N)
    rot = step * (l0 + idx)
    y = x[None] * np.exp(-2j * np.pi * np.outer(rot, np.arange(K + 1)) / L)[:, :, None]
    # neighbouring angles of the window 60 sigma^2 apart in squared distance
    dth = 2 * np.pi * step / L
    sigma2 = float(np.sum(np.abs(x) ** 2 * np.abs(1 - np.exp(-1j * np.arange(K + 1) * dth))[:, None] ** 2)) / 60
    d = mra.dims(N, K, Q, L, sigma2)
    prm = mra.em_params(Lw, l0=l0, step=step)
    xi = dev(x)
    xo = torch.empty_like(xi)
    lro = torch.empty(Lw, dtype=torch.float64, device="cuda")
    w = torch.empty((N, Lw), dtype=torch.float32, device="cuda")
    ws = mra.workspace(mra.mra_em_workspace_bytes(d, Lw))
    mra.mra_em_step(d, prm, dev_y(y), None, xi, dev(np.log(np.full(Lw, 1 / Lw))), xo, lro, None, None, w, ws)
    torch.cuda.synchronize()
    wh = host(w)
    assert np.array_equal(np.argmax(wh, axis=1), idx)
    assert np.min(wh[np.arange(N), idx]) > 1 - 1e-5
    assert rel_err(host(xo), x) <= 1e-5
    np.testing.assert_allclose(np.exp(host(lro)), np.bincount(idx, minlength=Lw) / N, atol=1e-6)


@pytest.mark.parametrize("kind", [0, 1])
def test_dense_fit_prior_matches_oracle(gpu_lib, kind):
    mra = gpu_lib
    L = 360
    rng = np.random.default_rng(77)
    th = rng.vonmises(0.0, 30.0, 200_000)
    counts = np.bincount(np.floor(np.mod(th, 2 * np.pi) * L / (2 * np.pi) + 0.5).astype(int) % L, minlength=L)
    for Lw, l0, step in [(721, -360, 0.05), (97, -48, 0.5), (64, -11, 0.3)]:
        lp = torch.empty(Lw, dtype=torch.float64, device="cuda")
        kap = torch.empty(1, dtype=torch.float64, device="cuda")
        mra.mra_fit_prior(L, Lw, l0, dev(counts.astype(np.int32)), kind, lp, kap, step=step)
        want, k_o = O.fit_prior(counts, L, Lw, l0=l0, kind=kind, step=step)
        got = host(lp)
        assert np.array_equal(np.isfinite(got), np.isfinite(want))
        f = np.isfinite(want)
        np.testing.assert_allclose(got[f], want[f], rtol=0, atol=1e-9)
        assert abs(float(kap.item()) - k_o) <= 1e-9 * max(1.0, k_o)


def test_dense_loglik_grad_matches_oracle(gpu_lib):
    mra = gpu_lib
    inst = synth.make_instance(16, 16, 3000, 180, snr=1 / 10, decay=50.0, seed=8600, offgrid=True)
    y64 = synth.c64_round(inst.y)
    Lw, l0, step = 73, -36, 0.5
    d = mra.dims(inst.N, inst.K, inst.Q, inst.L, inst.sigma2)
    x = O.align_mean(y64, inst.s, inst.L)
    eta = 0.2 * np.random.default_rng(3).standard_normal(Lw)
    kappa = 2.0
    ws = mra.workspace(mra.mra_em_workspace_bytes(d, Lw))
    ll = torch.empty(1, dtype=torch.float64, device="cuda")
    dx = torch.empty((inst.K + 1, inst.Q), dtype=torch.complex128, device="cuda")
    de = torch.empty(Lw, dtype=torch.float64, device="cuda")
    dk = torch.empty(1, dtype=torch.float64, device="cuda")
    mra.mra_loglik_grad(d, Lw, l0, dev_y(y64), dev(inst.s.astype(np.int32)), dev(x), dev(eta), kappa, ll, dx, de, dk,
                        ws, step=step)
    torch.cuda.synchronize()
    llo, dxo, deo, dko = O.loglik_grad(y64, x, eta, kappa, inst.L, inst.sigma2, l0=l0, shifts=inst.s, step=step)
    assert abs(float(ll.item()) - llo) <= TOL_LL * loglik_scale(y64, x, inst.sigma2)
    # dx = (2/sigma^2)(num - N x): against the scale of num
    scale = 2.0 / inst.sigma2 * inst.N * np.linalg.norm(x)
    assert np.linalg.norm(host(dx) - dxo) <= TOL_X * scale
    np.testing.assert_allclose(host(de), deo, rtol=0, atol=TOL_W * inst.N)
    assert abs(float(dk.item()) - dko) <= TOL_W * inst.N * Lw


def test_dense_window_argument_checks(gpu_lib):
    mra = gpu_lib
    d = mra.dims(100, 3, 8, 40, 0.1)
    y = torch.zeros((100, 4, 8), dtype=torch.complex64, device="cuda")
    x = torch.zeros((4, 8), dtype=torch.complex128, device="cuda")
    for Lw, l0, step in [(81, -40, 0.5), (10, 0, 1.5), (10, 0, -0.5), (5, 0, float("nan"))]:
        lr = torch.zeros(Lw, dtype=torch.float64, device="cuda")
        ws = mra.workspace(mra.mra_em_workspace_bytes(d, Lw))
        with pytest.raises(RuntimeError):
            mra.mra_em_step(d, mra.em_params(Lw, l0=l0, step=step), y, None, x, lr, x.clone(), lr.clone(), None,
                            None, None, ws)
    # (Lw - 1) step < L: 79 steps of 0.5 span 39.5 < 40 grid units
    lr = torch.zeros(80, dtype=torch.float64, device="cuda")
    ws = mra.workspace(mra.mra_em_workspace_bytes(d, 80))
    mra.mra_em_step(d, mra.em_params(80, l0=-40, step=0.5), y, None, x, lr, x.clone(), lr.clone(), None, None, None,
                    ws)
    torch.cuda.synchronize()


def test_dense_autotune_and_batched(gpu_lib):
    """The autotuner keys its choice by the step too, and a batched run mixes grid and dense instances."""
    mra = gpu_lib
    T = 3
    items, probs = [], []
    for i, (Lw, l0, step) in enumerate([(36, -18, 1.0), (36, -18, 0.5), (91, -45, 0.2)]):
        inst = synth.make_instance(12, 16, 1500, 120, snr=1 / 5, decay=50.0, seed=8700 + i, offgrid=True)
        y64 = synth.c64_round(inst.y)
        x0 = O.align_mean(y64, inst.s, inst.L)
        lr = np.log(np.full(Lw, 1 / Lw))
        d = mra.dims(inst.N, inst.K, inst.Q, inst.L, inst.sigma2)
        prm = mra.em_params(Lw, l0=l0, max_iters=T, step=step)
        items.append(dict(d=d, prm=prm, y=dev_y(y64), shift=dev(inst.s.astype(np.int32)), x=dev(x0), log_rho=dev(lr)))
        probs.append((inst, y64, x0, lr, Lw, l0, step))
    arr = mra.instances(items)
    ws = mra.workspace(mra.mra_em_batched_workspace_bytes(arr))
    iters, _ = mra.mra_em_run_batched(arr, ws, tune=True)
    assert iters == [T] * 3
    for (inst, y64, x0, lr, Lw, l0, step), it in zip(probs, items):
        xs, lrs = x0, lr
        for t in range(T):
            st = O.em_step(y64, xs, lrs, inst.L, inst.sigma2, Lw=Lw, l0=l0, shifts=inst.s, step=step)
            xs, lrs = st.x, st.log_rho
        assert rel_err(host(it["x"]), xs) <= TOL_X * T, (step, rel_err(host(it["x"]), xs))
