"""The BF16 hi/lo storage of y: the split kernel against a numpy round-to-nearest-even
split (bit for bit), and the EM step / run on split y against the FP64 oracle fed
the values hi + lo that the kernels read (same tolerances as the complex64 path).
The error against the oracle on the unsplit y is printed for each case."""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from gpu_helpers import TOL_W, TOL_X, dev, host, rel_err

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]


def _dev_hl(y):
    g = synth.bf16_split(y)  # uint16 [groups, 8]
    return torch.from_numpy(g.view(np.int16)).cuda()


def test_split_kernel_is_bit_exact(gpu_lib):
    mra = gpu_lib
    rng = np.random.default_rng(11)
    y = (rng.standard_normal(4096) + 1j * rng.standard_normal(4096)) * 10.0 ** rng.uniform(-30, 30, 4096)
    y[:8] = [0, -0.0, 1 + 1j, -1 - 1j, 1.00390625 + 1.01171875j, 3.4e38, -1e-38, 2.0 ** -126]  # ties and extremes
    yd = torch.from_numpy(synth.to_c64(y)).cuda()
    out = torch.empty(y.size * 4, dtype=torch.int16, device="cuda")
    mra.mra_y_split_bf16(yd, out)
    torch.cuda.synchronize()
    want = synth.bf16_split(y).view(np.int16).reshape(-1)
    np.testing.assert_array_equal(host(out), want)


@pytest.fixture(params=["cta", "chunk", "cta-tdg"])
def sweep(request, monkeypatch):
    """Both sweeps that read the split format: the CTA batch sweep and the chunked two-read sweep
    (cta-tdg: the batch sweep with its distance-unit table read from global memory)."""
    monkeypatch.setenv("MRA_SWEEP", request.param.split("-")[0])
    if request.param.endswith("-tdg"):
        monkeypatch.setenv("MRA_SWEEP_TDG", "1")
    return request.param


@pytest.mark.parametrize("N,L,window", [(2000, 720, True), (600, 180, False)])
def test_em_step_hl_config5_shapes(gpu_lib, sweep, N, L, window):
    """|k| <= 48, Q = 32: the window of 72 around aligned images at L = 720, or the whole grid
    of L = 180 (the oracle's literal distances over 720 rotations would need tens of GB)."""
    mra = gpu_lib
    c = synth.config(5)
    inst = synth.make_instance(c["K"], c["Q"], N, L, c["snr"], c["decay"], seed=5000 + N)
    y_hl = synth.bf16_merge(synth.bf16_split(inst.y), inst.y.shape)
    if window:
        Lw, l0, sh = c["Lw"], None, inst.s
        x0 = O.align_mean(y_hl, sh, inst.L)
    else:
        Lw, l0, sh = inst.L, 0, None
        x0 = synth.random_init(inst.K, inst.Q, c["decay"], seed=9)
    lr = np.log(np.full(Lw, 1.0 / Lw))
    d = mra.dims(inst.N, inst.K, inst.Q, inst.L, inst.sigma2)
    prm = mra.em_params(Lw, l0=l0)
    ws = mra.workspace(mra.mra_em_workspace_bytes(d, Lw))
    xi, lri = dev(x0), dev(lr)
    xo, lro = torch.empty_like(xi), torch.empty_like(lri)
    w = torch.empty((N, Lw), dtype=torch.float32, device="cuda")
    ll = torch.empty(1, dtype=torch.float64, device="cuda")
    shd = dev(sh.astype(np.int32)) if sh is not None else None
    mra.mra_em_step_hl(d, prm, _dev_hl(inst.y), shd, xi, lri, xo, lro, ll, None, w, ws)
    torch.cuda.synchronize()
    assert mra.mra_ws_status(ws) == 0
    ref = O.em_step(y_hl, x0, lr, inst.L, inst.sigma2, Lw=Lw, l0=l0, shifts=sh)
    ex, ew = rel_err(host(xo), ref.x), np.max(np.abs(host(w) - ref.w))
    assert ex <= TOL_X, ex
    assert ew <= TOL_W, ew
    full = O.em_step(synth.c64_round(inst.y), x0, lr, inst.L, inst.sigma2, Lw=Lw, l0=l0, shifts=sh)
    print(f"\nbf16 hi/lo, N={N}, Lw={Lw}: vs oracle on hi+lo x {ex:.2e} w {ew:.2e}; vs oracle on complex64 y "
          f"x {rel_err(host(xo), full.x):.2e} w {np.max(np.abs(host(w) - full.w)):.2e}")


def test_em_step_hl_dense_window_table_in_global_memory(gpu_lib):
    """The split format on the paper's dense window at |k| <= 32, Q = 24, L = 360 (721 rotations 0.05 grid
    units apart, off-grid rotations): the batch sweep's distance-unit table does not fit in shared memory
    next to its ring, so it reads the table from global memory."""
    mra = gpu_lib
    K, Q, L, N = 32, 24, 360, 300
    inst = synth.make_instance(K, Q, N, L, snr=1 / 50, decay=400.0, seed=5400, offgrid=True)
    y_hl = synth.bf16_merge(synth.bf16_split(inst.y), inst.y.shape)
    Lw, l0, step = 2 * L + 1, -L, 36 / (2 * L)
    x0 = O.align_mean(y_hl, inst.s, L)
    lr = np.log(np.full(Lw, 1.0 / Lw))
    d = mra.dims(N, K, Q, L, inst.sigma2)
    ws = mra.workspace(mra.mra_em_workspace_bytes(d, Lw))
    xi, lri = dev(x0), dev(lr)
    xo, lro = torch.empty_like(xi), torch.empty_like(lri)
    w = torch.empty((N, Lw), dtype=torch.float32, device="cuda")
    ll = torch.empty(1, dtype=torch.float64, device="cuda")
    mra.mra_em_step_hl(d, mra.em_params(Lw, l0=l0, step=step), _dev_hl(inst.y), dev(inst.s.astype(np.int32)),
                       xi, lri, xo, lro, ll, None, w, ws)
    torch.cuda.synchronize()
    assert mra.mra_ws_status(ws) == 0
    ref = O.em_step(y_hl, x0, lr, L, inst.sigma2, Lw=Lw, l0=l0, shifts=inst.s, step=step)
    assert rel_err(host(xo), ref.x) <= TOL_X, rel_err(host(xo), ref.x)
    assert np.max(np.abs(host(w) - ref.w)) <= TOL_W, np.max(np.abs(host(w) - ref.w))


def test_em_run_hl_first_10k_images_of_config5(gpu_lib, sweep):
    """The first 10,000 images of the largest workload: two EM iterations on the window."""
    mra = gpu_lib
    c = synth.config(5)
    inst = synth.make_instance(c["K"], c["Q"], 10_000, c["L"], c["snr"], c["decay"], seed=5001)
    y_hl = synth.bf16_merge(synth.bf16_split(inst.y), inst.y.shape)
    Lw = c["Lw"]
    x0 = O.align_mean(y_hl, inst.s, inst.L)
    lr = np.log(np.full(Lw, 1.0 / Lw))
    T = 2
    d = mra.dims(inst.N, inst.K, inst.Q, inst.L, inst.sigma2)
    prm = mra.em_params(Lw, max_iters=T)
    ws = mra.workspace(mra.mra_em_workspace_bytes(d, Lw))
    x, lrd = dev(x0), dev(lr)
    traj = torch.empty((T, inst.K + 1, inst.Q), dtype=torch.complex128, device="cuda")
    n = mra.mra_em_run_hl(d, prm, _dev_hl(inst.y), dev(inst.s.astype(np.int32)), x, lrd, None, traj, ws)
    assert n == T
    xs, lro = x0, lr
    for t in range(T):
        st = O.em_step(y_hl, xs, lro, inst.L, inst.sigma2, Lw=Lw, shifts=inst.s)
        e = rel_err(host(traj[t]), st.x)
        assert e <= TOL_X * (t + 1), (t, e)
        xs, lro = st.x, st.log_rho
    print(f"\nbf16 hi/lo, first 10k images, {T} iterations: x error {rel_err(host(x), xs):.2e}; "
          f"x vs truth {O.relerr(host(x), inst.x):.3e}")


def test_hl_error_against_unsplit_y_first_10k_config5(gpu_lib):
    """The error of the storage format itself, on the first 10,000 images of the largest workload
    (|k| <= 48, Q = 32, L = 720, window 72): EM on the BF16 hi/lo split against the FP64 oracle on the
    complex64 observations (not on hi + lo), two iterations from the aligned mean.  The split keeps
    each real value to within 2^-16 of itself, so every result moves by that order: the bounds below
    are the per-value error times the data's own scale (the mean image norm over ||x|| for x, the
    mean squared image norm times 2 beta per image for the log-likelihood), with a factor of 4."""
    mra = gpu_lib
    c = synth.config(5)
    inst = synth.make_instance(c["K"], c["Q"], 10_000, c["L"], c["snr"], c["decay"], seed=5001)
    y64 = synth.c64_round(inst.y)
    Lw = c["Lw"]
    x0 = O.align_mean(y64, inst.s, inst.L)
    lr = np.log(np.full(Lw, 1.0 / Lw))
    T = 2
    d = mra.dims(inst.N, inst.K, inst.Q, inst.L, inst.sigma2)
    prm = mra.em_params(Lw, max_iters=T)
    ws = mra.workspace(mra.mra_em_workspace_bytes(d, Lw))
    x, lrd = dev(x0), dev(lr)
    traj = torch.empty((T, inst.K + 1, inst.Q), dtype=torch.complex128, device="cuda")
    stats = torch.empty((T, 2), dtype=torch.float64, device="cuda")
    assert mra.mra_em_run_hl(d, prm, _dev_hl(inst.y), dev(inst.s.astype(np.int32)), x, lrd, stats, traj, ws) == T
    eps = 2.0 ** -16
    ynorm = np.linalg.norm(y64.reshape(inst.N, -1), axis=1)
    xs, lro = x0, lr
    for t in range(T):
        st = O.em_step(y64, xs, lro, inst.L, inst.sigma2, Lw=Lw, shifts=inst.s)
        ex = rel_err(host(traj[t]), st.x)
        el = abs(float(host(stats)[t, 0]) - st.loglik)
        bx = 4 * eps * ynorm.mean() / np.linalg.norm(st.x)
        bl = 4 * eps * (2 / inst.sigma2) * float((ynorm ** 2).sum())
        print(f"\nbf16 hi/lo vs FP64 oracle on complex64 y, iteration {t + 1}: x rel err {ex:.2e} (bound {bx:.1e}); "
              f"loglik abs err {el:.3e} of |loglik| {abs(st.loglik):.4e} (rel {el / abs(st.loglik):.2e}, bound {bl:.1e})")
        assert ex <= bx, (t, ex, bx)
        assert el <= bl, (t, el, bl)
        xs, lro = st.x, st.log_rho
