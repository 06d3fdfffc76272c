"""Parity at the full benchmark size (|k| <= 32, Q = 24, N = 100,000, L = 360, window 36)
in the launch configuration that bench.py times.  Posterior weights are checked on
sampled images (each image's weights depend only on that image and the state);
the M-step output and the log-likelihood against the full oracle sweep; the
matching step on sampled queries."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import synth
from gpu_helpers import TOL_LL, TOL_W, TOL_X, dev, dev_y, host, loglik_scale, rel_err

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]


@pytest.fixture(scope="module")
def cfg2():
    c = synth.config(2)
    inst = synth.make_instance(c["K"], c["Q"], c["N"], c["L"], c["snr"], c["decay"], seed=2000)
    return c, inst, synth.c64_round(inst.y)


def test_em_step_full_size(gpu_lib, cfg2):
    mra = gpu_lib
    c, inst, y64 = cfg2
    rng = np.random.default_rng(7)
    sh = (inst.s + rng.integers(-4, 5, inst.N)) % inst.L
    x0 = O.align_mean(y64, sh, inst.L)
    Lw = c["Lw"]
    t = 2.0 * np.cos(2 * np.pi * O.window_offsets(inst.L, Lw) / inst.L)
    lrb = t - np.log(np.exp(t).sum())
    d = mra.dims(inst.N, inst.K, inst.Q, inst.L, inst.sigma2)
    prm = mra.em_params(Lw, gamma=c["gamma"], log_rho_bar=dev(lrb))
    xo = torch.empty((inst.K + 1, inst.Q), dtype=torch.complex128, device="cuda")
    lro = torch.empty(Lw, dtype=torch.float64, device="cuda")
    ll = torch.empty(1, dtype=torch.float64, device="cuda")
    stp = torch.empty(1, dtype=torch.float64, device="cuda")
    w = torch.empty((inst.N, Lw), dtype=torch.float32, device="cuda")
    ws = mra.workspace(mra.mra_em_workspace_bytes(d, Lw))
    mra.mra_em_step(d, prm, dev_y(inst.y), dev(sh.astype(np.int32)), dev(x0), dev(lrb), xo, lro, ll, stp, w, ws)
    torch.cuda.synchronize()
    assert mra.mra_ws_status(ws) == 0
    wg = host(w)
    # sampled images, one by one
    idx = np.sort(rng.choice(inst.N, 400, replace=False))
    idx = np.concatenate([idx, [0, inst.N - 1]])
    wo, _, _ = O.posterior(x0, O.align(y64[idx], sh[idx], inst.L), lrb, inst.L, O.window_offsets(inst.L, Lw),
                           inst.sigma2)
    assert np.max(np.abs(wg[idx] - wo)) <= TOL_W
    assert np.allclose(wg.sum(axis=1), 1.0, atol=1e-5)
    # global outputs against the full oracle step
    st = O.em_step(y64, x0, lrb, inst.L, inst.sigma2, Lw=Lw, gamma=c["gamma"], log_rho_bar=lrb, shifts=sh)
    assert rel_err(host(xo), st.x) <= TOL_X
    np.testing.assert_allclose(np.exp(host(lro)), np.exp(st.log_rho), atol=1e-5, rtol=0)
    assert abs(ll.item() - st.loglik) <= TOL_LL * loglik_scale(y64, x0, inst.sigma2)
    assert abs(stp.item() - st.step) <= 1e-5 * math.sqrt(st.step) + 1e-10


def test_match_full_size_sampled(gpu_lib, cfg2):
    mra = gpu_lib
    c, inst, y64 = cfg2
    P = c["P"]
    rng = np.random.default_rng(8)
    phi = rng.integers(0, inst.L, P).astype(np.int32)
    d = mra.dims(inst.N, inst.K, inst.Q, inst.L, inst.sigma2)
    ws = mra.workspace(mra.mra_sync_workspace_bytes(d, P))
    out = torch.empty(inst.N, dtype=torch.int32, device="cuda")
    mra.mra_sync_match(d, dev_y(inst.y), P, dev(phi), out, ws)
    g = host(out)
    idx = np.concatenate([np.arange(P), rng.choice(np.arange(P, inst.N), 2000, replace=False), [inst.N - 1]])
    mism = 0
    for i in idx:
        dd = np.sum(np.abs(y64[i][None] - y64[:P]) ** 2, axis=(1, 2))
        if i < P:
            dd[i] = np.inf
        order = np.argsort(dd)
        if g[i] != phi[order[0]]:
            scale = np.sum(np.abs(y64[i]) ** 2) + np.max(np.sum(np.abs(y64[:P]) ** 2, axis=(1, 2)))
            assert dd[order[1]] - dd[order[0]] <= 2e-5 * scale and g[i] == phi[order[1]], i
            mism += 1
    assert mism <= 10


def test_pairwise_full_size_sampled(gpu_lib, cfg2):
    mra = gpu_lib
    c, inst, y64 = cfg2
    P = c["P"]
    d = mra.dims(inst.N, inst.K, inst.Q, inst.L, inst.sigma2)
    rel = torch.empty((P, P), dtype=torch.int32, device="cuda")
    mra.mra_sync_pairwise(d, dev_y(inst.y), P, rel)
    g = host(rel)
    rng = np.random.default_rng(9)
    for _ in range(150):
        i, j = sorted(rng.choice(P, 2, replace=False))
        r = O.relative_rotation(y64[i], y64[j], inst.L)
        if g[i, j] != r:
            rvj = O.rotate(y64[j], -O.grid_angle(np.arange(inst.L), inst.L))
            dd = np.sum(np.abs(y64[i][None] - rvj) ** 2, axis=(1, 2))
            scale = np.sum(np.abs(y64[i]) ** 2) + np.sum(np.abs(y64[j]) ** 2)
            assert dd[g[i, j]] - dd[r] <= 2e-5 * scale
