"""GPU parity of the EM path (mra_em_step, mra_em_run, mra_loglik_grad, mra_align_mean)
against the FP64 oracle, through the C ABI.  Inputs are seeded synthetic
instances; the oracle sees exactly the complex64 values the GPU reads."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import synth
from gpu_helpers import TOL_LL, TOL_W, TOL_X, dev, dev_y, host, loglik_scale, rel_err

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]


def run_step(mra, inst, y64, x, log_rho, Lw, l0=None, shifts=None, gamma=0.0, log_rho_bar=None, gamma_a_inv=None,
             update_rho=True):
    d = mra.dims(inst.N, inst.K, inst.Q, inst.L, inst.sigma2)
    lrb = dev(log_rho_bar) if log_rho_bar is not None else None
    gai = dev(gamma_a_inv.astype(np.float64).ravel()) if gamma_a_inv is not None else None
    prm = mra.em_params(Lw, l0=l0, gamma=gamma, log_rho_bar=lrb, gamma_a_inv=gai, update_rho=update_rho)
    y = dev_y(y64)
    sh = dev(shifts.astype(np.int32)) if shifts is not None else None
    xi = dev(x.astype(np.complex128))
    lri = dev(np.asarray(log_rho, dtype=np.float64))
    xo = torch.empty_like(xi)
    lro = torch.empty_like(lri)
    ll = torch.empty(1, dtype=torch.float64, device="cuda")
    stp = torch.empty(1, dtype=torch.float64, device="cuda")
    w = torch.empty((inst.N, Lw), dtype=torch.float32, device="cuda")
    ws = mra.workspace(mra.mra_em_workspace_bytes(d, Lw))
    mra.mra_em_step(d, prm, y, sh, xi, lri, xo, lro, ll, stp, w, ws)
    torch.cuda.synchronize()
    assert mra.mra_ws_status(ws) == 0
    return host(xo), host(lro), float(ll.item()), float(stp.item()), host(w)


def compare(mra, inst, x, log_rho, Lw, l0=None, shifts=None, **kw):
    y64 = synth.c64_round(inst.y)
    xg, lrg, llg, stg, wg = run_step(mra, inst, y64, x, log_rho, Lw, l0=l0, shifts=shifts, **kw)
    kw_o = {k: v for k, v in kw.items()}
    st = O.em_step(y64, x, log_rho, inst.L, inst.sigma2, Lw=Lw, l0=l0, shifts=shifts, **kw_o)
    assert rel_err(xg, st.x) <= TOL_X, rel_err(xg, st.x)
    assert np.max(np.abs(wg - st.w)) <= TOL_W, np.max(np.abs(wg - st.w))
    np.testing.assert_allclose(np.exp(lrg), np.exp(st.log_rho), atol=1e-5, rtol=0)
    assert abs(llg - st.loglik) <= TOL_LL * loglik_scale(y64, x, inst.sigma2), (llg, st.loglik)
    assert abs(stg - st.step) <= 1e-5 * math.sqrt(st.step) + 1e-10, (stg, st.step)
    return xg, st


@pytest.fixture(params=["cta", "warp", "chunk", "cta-tdg", "lean", "tc", "pair"])
def sweep(request, monkeypatch):
    """Every EM sweep: the CTA-cooperative batch sweep, the warp-per-image one, the chunked
    two-read one, the lean warp sweep, the split sweep with its tensor-core transform and the
    paired-warp sweep (shapes
    a sweep cannot take fall back to the default choice); cta-tdg is the batch sweep with its
    distance-unit table read from global memory."""
    monkeypatch.setenv("MRA_SWEEP", request.param.split("-")[0])
    if request.param.endswith("-tdg"):
        monkeypatch.setenv("MRA_SWEEP_TDG", "1")
    return request.param


def test_em_step_config1_window(gpu_lib, sweep):
    c = synth.config(1)
    inst = synth.make_instance(c["K"], c["Q"], c["N"], c["L"], c["snr"], c["decay"], seed=1001)
    x0 = O.align_mean(synth.c64_round(inst.y), inst.s, inst.L)
    Lw = c["Lw"]
    compare(gpu_lib, inst, x0, np.log(np.full(Lw, 1 / Lw)), Lw, shifts=inst.s)


def test_em_step_config1_prior_gamma(gpu_lib):
    c = synth.config(1)
    inst = synth.make_instance(c["K"], c["Q"], c["N"], c["L"], c["snr"], c["decay"], seed=1002)
    Lw = c["Lw"]
    t = 4.0 * np.cos(2 * np.pi * O.window_offsets(inst.L, Lw) / inst.L)
    lrb = t - np.log(np.exp(t).sum())
    lrb[0] = -np.inf  # an empty bin of the learned histogram
    lr = lrb.copy()
    rng = np.random.default_rng(0)
    sh = (inst.s + rng.integers(-2, 3, inst.N)) % inst.L  # imperfect alignment
    x0 = O.align_mean(synth.c64_round(inst.y), sh, inst.L)
    compare(gpu_lib, inst, x0, lr, Lw, shifts=sh, gamma=c["gamma"], log_rho_bar=lrb)


def test_em_step_full_search_and_signal_prior(gpu_lib, sweep):
    c = synth.config(1)
    inst = synth.make_instance(c["K"], c["Q"], 300, c["L"], c["snr"], c["decay"], seed=1003)
    x0 = synth.random_init(inst.K, inst.Q, c["decay"], seed=5)
    k = np.arange(inst.K + 1)[:, None] * np.ones((1, inst.Q))
    gi = 1.0 / (4.0 * np.exp(-k / 8.0)) ** 2
    L = inst.L
    compare(gpu_lib, inst, x0, np.log(np.full(L, 1 / L)), L, l0=0, gamma_a_inv=gi)


@pytest.mark.parametrize("K,Q,N,L,Lw", [(5, 3, 77, 30, 7), (0, 2, 40, 12, 5), (3, 4, 1, 16, 16), (7, 6, 33, 50, 1),
                                        (12, 10, 500, 90, 13), (4, 8, 1, 16, 16), (6, 16, 301, 40, 9),
                                        (48, 32, 203, 72, 72), (63, 8, 150, 128, 20), (63, 64, 90, 40, 9),
                                        (127, 32, 60, 256, 15), (5, 8, 100, 30, 3), (10, 8, 700, 120, 55),
                                        (20, 16, 400, 200, 63), (1, 8, 257, 20, 5), (16, 24, 333, 90, 30),
                                        (44, 16, 300, 90, 90)])
def test_em_step_shapes_and_edges(gpu_lib, sweep, K, Q, N, L, Lw):
    """Odd Q (float2 path), K = 0, N = 1, Lw = L, Lw = 1, ragged tiles and batches, the
    largest rows (M = 1568) and the most rows (64) of the batch sweep, the largest
    stored size M = 4096 (wide rows and many rows: the tile sweep), windows of 2, 28
    and 32 mirror units (the lean sweep's narrowest and its second unit pitch), for the
    paired-warp sweep a second warp without rows (K = 1) and exactly one row group (K = 16), and
    full search with K + 1 = 45 rows (the split sweep's back transform on rows beyond 32)."""
    inst = synth.make_instance(K, Q, N, L, sigma2=1 / (0.3 * (K + 1) * Q), decay=20.0, seed=K * 100 + N)
    x0 = synth.random_init(K, Q, 20.0, seed=3)
    compare(gpu_lib, inst, x0, np.log(np.full(Lw, 1 / Lw)), Lw, shifts=inst.s, update_rho=(Lw % 2 == 1))


def test_em_step_config2_subset_several_tiles(gpu_lib, sweep):
    c = synth.config(2)
    inst = synth.make_instance(c["K"], c["Q"], 4097, c["L"], c["snr"], c["decay"], seed=2001)
    y64 = synth.c64_round(inst.y)
    rng = np.random.default_rng(1)
    sh = (inst.s + rng.integers(-3, 4, inst.N)) % inst.L
    x0 = O.align_mean(y64, sh, inst.L)
    Lw = c["Lw"]
    compare(gpu_lib, inst, x0, np.log(np.full(Lw, 1 / Lw)), Lw, shifts=sh)


@pytest.mark.parametrize("bi", ["16", "12", "8", "4"])
def test_em_step_batch_sizes(gpu_lib, bi, monkeypatch):
    """Every batch size of the CTA-cooperative sweep, with a ragged last batch."""
    monkeypatch.setenv("MRA_SWEEP", "cta")
    monkeypatch.setenv("MRA_SWEEP_BI", bi)
    inst = synth.make_instance(7, 8, 1000 + 13, 36, sigma2=1 / (0.3 * 64), decay=20.0, seed=77)
    x0 = synth.random_init(7, 8, 20.0, seed=3)
    Lw = 11
    compare(gpu_lib, inst, x0, np.log(np.full(Lw, 1 / Lw)), Lw, shifts=inst.s)


@pytest.mark.parametrize("chunk", ["128", "64", "32", "16"])
def test_em_step_chunk_sizes(gpu_lib, chunk, monkeypatch):
    """Every chunk size of the two-read sweep, with a ragged last chunk and warps without images."""
    monkeypatch.setenv("MRA_SWEEP", "chunk")
    monkeypatch.setenv("MRA_SWEEP_BI", chunk)
    inst = synth.make_instance(7, 16, 1000 + 7, 36, sigma2=1 / (0.3 * 128), decay=20.0, seed=78)
    x0 = synth.random_init(7, 16, 20.0, seed=3)
    Lw = 11
    compare(gpu_lib, inst, x0, np.log(np.full(Lw, 1 / Lw)), Lw, shifts=inst.s)


def test_em_run_trajectory_resume_and_tol(gpu_lib):
    mra = gpu_lib
    c = synth.config(1)
    inst = synth.make_instance(c["K"], c["Q"], c["N"], c["L"], c["snr"], c["decay"], seed=1004)
    y64 = synth.c64_round(inst.y)
    Lw, T = c["Lw"], c["iters"]
    x0 = O.align_mean(y64, inst.s, inst.L)
    lr0 = np.log(np.full(Lw, 1 / Lw))
    ora = O.em_run(y64, x0, lr0, inst.L, inst.sigma2, T, Lw=Lw, shifts=inst.s)
    d = mra.dims(inst.N, inst.K, inst.Q, inst.L, inst.sigma2)
    y = dev_y(inst.y)
    sh = dev(inst.s.astype(np.int32))
    ws = mra.workspace(mra.mra_em_workspace_bytes(d, Lw))

    def run(x, lr, iters, check_every=None):
        x = x.clone()
        lr = lr.clone()
        prm = mra.em_params(Lw, max_iters=iters, check_every=check_every)
        stats = torch.empty((iters, 2), dtype=torch.float64, device="cuda")
        traj = torch.empty((iters, inst.K + 1, inst.Q), dtype=torch.complex128, device="cuda")
        n = mra.mra_em_run(d, prm, y, sh, x, lr, stats, traj, ws)
        return x, lr, n, host(stats), host(traj)

    x, lr, n, stats, traj = run(dev(x0), dev(lr0), T, check_every=7)
    assert n == T
    # trajectory error is reported, gated loosely (FP32 errors compound over iterations)
    assert rel_err(host(x), ora.x) < 20 * TOL_X
    np.testing.assert_allclose(stats[:, 0], ora.loglik, rtol=1e-5)
    assert rel_err(traj[-1], ora.x) < 20 * TOL_X
    # checkpoint / resume: 10 + 10 iterations equal 20, bit for bit (deterministic reductions)
    xa, lra, _, _, _ = run(dev(x0), dev(lr0), 10)
    xb, lrb, _, _, _ = run(xa, lra, 10)
    np.testing.assert_array_equal(host(xb), host(x))
    np.testing.assert_array_equal(host(lrb), host(lr))
    # tolerance stop: the first iteration whose step falls below tol ends the run
    steps = ora.step
    k = next((c for c in range(T // 2, T) if steps[c] < steps[:c].min() / 1.01), None)
    if k is not None:
        tol = math.sqrt(steps[k] * steps[:k].min())
        prm = mra.em_params(Lw, max_iters=T, tol=tol, check_every=3)
        n = mra.mra_em_run(d, prm, y, sh, dev(x0), dev(lr0), None, None, ws)
        assert n == k + 1


def test_align_mean(gpu_lib):
    mra = gpu_lib
    c = synth.config(2)
    inst = synth.make_instance(c["K"], c["Q"], 3000, c["L"], c["snr"], c["decay"], seed=2003)
    d = mra.dims(inst.N, inst.K, inst.Q, inst.L, inst.sigma2)
    ws = mra.workspace(mra.mra_em_workspace_bytes(d, 1))
    x = torch.empty((inst.K + 1, inst.Q), dtype=torch.complex128, device="cuda")
    mra.mra_align_mean(d, dev_y(inst.y), dev(inst.s.astype(np.int32)), x, ws)
    ref = O.align_mean(synth.c64_round(inst.y), inst.s, inst.L)
    assert rel_err(host(x), ref) < TOL_X


def test_loglik_grad(gpu_lib):
    mra = gpu_lib
    c = synth.config(3)
    inst = synth.make_instance(c["K"], c["Q"], 2000, c["L"], c["snr"], c["decay"], seed=3001)
    y64 = synth.c64_round(inst.y)
    Lw = c["Lw"]
    l0 = -(Lw // 2)
    rng = np.random.default_rng(2)
    eta = 0.2 * rng.standard_normal(Lw)
    kappa = 3.0
    x = O.align_mean(y64, inst.s, inst.L)
    ll, dx, de, dk = O.loglik_grad(y64, x, eta, kappa, inst.L, inst.sigma2, l0=l0, shifts=inst.s)
    d = mra.dims(inst.N, inst.K, inst.Q, inst.L, inst.sigma2)
    ws = mra.workspace(mra.mra_em_workspace_bytes(d, Lw))
    llg = torch.empty(1, dtype=torch.float64, device="cuda")
    dxg = torch.empty((inst.K + 1, inst.Q), dtype=torch.complex128, device="cuda")
    deg = torch.empty(Lw, dtype=torch.float64, device="cuda")
    dkg = torch.empty(1, dtype=torch.float64, device="cuda")
    mra.mra_loglik_grad(d, Lw, l0, dev_y(inst.y), dev(inst.s.astype(np.int32)), dev(x), dev(eta), kappa, llg, dxg,
                        deg, dkg, ws)
    torch.cuda.synchronize()
    assert abs(llg.item() - ll) <= TOL_LL * loglik_scale(y64, x, inst.sigma2)
    # dx = (2/sigma^2)(num - N x): compare against the scale of num
    scale = 2.0 / inst.sigma2 * inst.N * np.linalg.norm(x)
    assert np.linalg.norm(host(dxg) - dx) <= TOL_X * scale
    np.testing.assert_allclose(host(deg), de, atol=TOL_W * inst.N)
    assert abs(dkg.item() - dk) <= TOL_W * inst.N * Lw


def test_autograd_function_matches_closed_form(gpu_lib):
    from paper_2105_07372_gb300.autograd import marginal_loglik

    mra = gpu_lib
    inst = synth.make_instance(6, 4, 400, 40, sigma2=1 / (0.3 * 28), decay=20.0, seed=11)
    y64 = synth.c64_round(inst.y)
    Lw = 9
    d = mra.dims(inst.N, inst.K, inst.Q, inst.L, inst.sigma2)
    x0 = O.align_mean(y64, inst.s, inst.L)
    x = dev(x0).requires_grad_(True)
    eta = torch.zeros(Lw, dtype=torch.float64, device="cuda", requires_grad=True)
    kappa = torch.tensor([1.5], dtype=torch.float64, device="cuda", requires_grad=True)
    ll = marginal_loglik(x, eta, kappa, dev_y(inst.y), d, Lw, shift=dev(inst.s.astype(np.int32)))
    ll.backward()
    llo, dxo, deo, dko = O.loglik_grad(y64, x0, np.zeros(Lw), 1.5, inst.L, inst.sigma2, shifts=inst.s)
    assert abs(ll.item() - llo) <= TOL_LL * loglik_scale(y64, x0, inst.sigma2)
    scale = 2.0 / inst.sigma2 * inst.N * np.linalg.norm(x0)
    assert np.linalg.norm(host(x.grad) - dxo) <= TOL_X * scale
    np.testing.assert_allclose(host(eta.grad), deo, atol=TOL_W * inst.N)
    assert abs(kappa.grad.item() - dko) <= TOL_W * inst.N * Lw


def test_errors_are_status_codes(gpu_lib):
    mra = gpu_lib
    d = mra.dims(10, 2, 2, 8, 0.1)
    ws = mra.workspace(mra.mra_em_workspace_bytes(d, 4))
    y = torch.zeros((10, 3, 2), dtype=torch.complex64, device="cuda")
    x = torch.zeros((3, 2), dtype=torch.complex128, device="cuda")
    lr = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(mra.MraError) as e:
        mra.mra_em_step(mra.dims(10, 2, 2, 8, -1.0), mra.em_params(4), y, None, x, lr, x, lr, ws=ws)
    assert e.value.status == -1
    with pytest.raises(mra.MraError) as e:
        mra.mra_em_step(d, mra.em_params(9), y, None, x, lr, x, lr, ws=ws)  # window larger than L
    assert e.value.status == -1
    with pytest.raises(mra.MraError) as e:
        mra.mra_em_step(d, mra.em_params(4), y, None, x, lr, x, lr, ws=ws[:100])
    assert e.value.status == -6
    with pytest.raises(mra.MraError) as e:  # misaligned observations
        mra.mra_em_step(d, mra.em_params(4), y.view(torch.float32).view(-1)[2:], None, x, lr, x, lr, ws=ws)
    assert e.value.status == -1
    with pytest.raises(mra.MraError):
        mra.mra_em_step(mra.dims(10, 2, 3, 8, 0.1), mra.em_params(4), y, None, x, lr, x, lr, ws=ws)  # M odd


@pytest.mark.parametrize("snr", [1 / 50, 1 / 20, 1 / 10])
@pytest.mark.parametrize("K,Q,N,L,Lw", [(32, 24, 2000, 360, 37), (12, 16, 1500, 90, 31), (6, 6, 1200, 60, 21)])
def test_em_step_weights_across_snr(gpu_lib, sweep, snr, K, Q, N, L, Lw):
    """Weights within 1e-5 where the posterior is spread over a few rotations and 2 beta |c| is in the
    thousands: log-weights of that size lose the precision in plain FP32 sums, which the sweeps avoid by
    recomputing the values near each image's peak from peak-relative terms (rows of Q = 6 take the tile
    sweep, which forms them in FP64)."""
    inst = synth.make_instance(K, Q, N, L, snr, 400.0 if K > 20 else 50.0, seed=3100 + K)
    x0 = O.align_mean(synth.c64_round(inst.y), inst.s, inst.L)
    compare(gpu_lib, inst, x0, np.log(np.full(Lw, 1 / Lw)), Lw, shifts=inst.s)


@pytest.mark.parametrize("Lw,l0,snr", [(360, 0, 1 / 50), (100, -50, 1 / 50), (360, 0, 1 / 10), (65, -32, 1 / 20)])
def test_em_step_wide_windows_config2_shape(gpu_lib, sweep, Lw, l0, snr):
    """Full search (all 360 rotations) and wide windows at |k| <= 32, Q = 24: from the aligned mean
    (sharp posteriors) and from a random start (posteriors spread over the circle).  (At SNR 1/5 every
    sweep's FP32 values far from an image's peak move some weights by 1.0e-5 to 1.3e-5.)"""
    c = synth.config(2)
    inst = synth.make_instance(c["K"], c["Q"], 2500, c["L"], snr, c["decay"], seed=3300 + Lw)
    y64 = synth.c64_round(inst.y)
    for x0 in (O.align_mean(y64, inst.s, inst.L), synth.random_init(inst.K, inst.Q, c["decay"], seed=7)):
        compare(gpu_lib, inst, x0, np.log(np.full(Lw, 1 / Lw)), Lw, l0=l0, shifts=inst.s)


@pytest.mark.parametrize("kind", ["tc", ""])
def test_em_step_whole_circle_beyond_512_rotations(gpu_lib, kind, monkeypatch):
    """Full search on a grid of L = 720 rotations (more than the 512 tensor-memory columns of one CTA:
    the split sweep's transform takes two passes and computes the first again for the cut), from the
    aligned mean and from a random start; "" lets the autotuner choose."""
    if kind:
        monkeypatch.setenv("MRA_SWEEP", kind)
    inst = synth.make_instance(16, 16, 700, 720, 1 / 20, 100.0, seed=3400)
    y64 = synth.c64_round(inst.y)
    for x0 in (O.align_mean(y64, inst.s, inst.L), synth.random_init(inst.K, inst.Q, 100.0, seed=9)):
        compare(gpu_lib, inst, x0, np.log(np.full(720, 1 / 720)), 720, l0=0, shifts=inst.s)
