"""GPU parity of Synchronize and Match, the rotation prior and the relative error,
through the C ABI.  Integer outputs must match the oracle exactly except where
the oracle itself certifies a near-tie (its margin below the FP32 resolution
of the GPU's arithmetic), in which case either choice is accepted."""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from gpu_helpers import dev, dev_y, host

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

TIE = 2e-5  # relative margin below which an FP32 decision may differ from the FP64 one


def pair_dists(vi, vj, L):
    rvj = O.rotate(vj, -O.grid_angle(np.arange(L), L))
    diff = vi[None] - rvj
    return np.sum(diff.real ** 2 + diff.imag ** 2, axis=(1, 2))


def test_pairwise_relative_rotations(gpu_lib):
    mra = gpu_lib
    c = synth.config(1)
    inst = synth.make_instance(c["K"], c["Q"], 60, c["L"], c["snr"], c["decay"], seed=1101)
    y64 = synth.c64_round(inst.y)
    P = 40
    d = mra.dims(inst.N, inst.K, inst.Q, inst.L, inst.sigma2)
    rel = torch.empty((P, P), dtype=torch.int32, device="cuda")
    mra.mra_sync_pairwise(d, dev_y(inst.y), P, rel)
    g = host(rel)
    ref = O.pairwise_relative(y64[:P], inst.L)
    bad = 0
    for i in range(P):
        assert g[i, i] == 0
        for j in range(i + 1, P):
            assert g[j, i] == (inst.L - g[i, j]) % inst.L
            if g[i, j] != ref[i, j]:
                dd = pair_dists(y64[i], y64[j], inst.L)
                scale = np.sum(np.abs(y64[i]) ** 2) + np.sum(np.abs(y64[j]) ** 2)
                assert dd[g[i, j]] - dd[ref[i, j]] <= TIE * scale, (i, j)
                bad += 1
    assert bad <= 3


def test_ppm_from_oracle_relative_rotations(gpu_lib):
    mra = gpu_lib
    c = synth.config(2)
    inst = synth.make_instance(c["K"], c["Q"], 100, c["L"], c["snr"], c["decay"], seed=2101)
    y64 = synth.c64_round(inst.y)
    P = 100
    rel = O.pairwise_relative(y64[:P], inst.L)
    ang = O.ppm_angles(rel, inst.L)
    ref = O.ppm(rel, inst.L)
    phi = torch.empty(P, dtype=torch.int32, device="cuda")
    mra.mra_sync_ppm(inst.L, P, dev(rel.astype(np.int32)), 50, 100, phi)
    g = host(phi)
    frac = ang * inst.L / (2 * np.pi) + 0.5
    near_half = np.abs(frac - np.round(frac)) < 1e-3  # angle within 1e-3 grid steps of a rounding boundary
    for i in range(P):
        if g[i] != ref[i]:
            assert near_half[i] and ((g[i] - ref[i]) % inst.L in (1, inst.L - 1)), i


def test_match_given_oracle_phi(gpu_lib):
    mra = gpu_lib
    c = synth.config(1)
    inst = synth.make_instance(c["K"], c["Q"], 700, c["L"], c["snr"], c["decay"], seed=1102)
    y64 = synth.c64_round(inst.y)
    P = 100
    rng = np.random.default_rng(3)
    phi = rng.integers(0, inst.L, P).astype(np.int32)
    d = mra.dims(inst.N, inst.K, inst.Q, inst.L, inst.sigma2)
    ws = mra.workspace(mra.mra_sync_workspace_bytes(d, P))
    out = torch.empty(inst.N, dtype=torch.int32, device="cuda")
    mra.mra_sync_match(d, dev_y(inst.y), P, dev(phi), out, ws)
    g = host(out)
    ref = O.match(y64, P, phi)
    for i in np.nonzero(g != ref)[0]:
        dd = np.sum(np.abs(y64[i][None] - y64[:P]) ** 2, axis=(1, 2))
        if i < P:
            dd[i] = np.inf
        order = np.argsort(dd)
        scale = np.sum(np.abs(y64[i]) ** 2) + np.max(np.sum(np.abs(y64[:P]) ** 2, axis=(1, 2)))
        assert dd[order[1]] - dd[order[0]] <= TIE * scale, i
        assert g[i] in (phi[order[0]], phi[order[1]])


def test_sync_full_config1_and_noise_free(gpu_lib):
    mra = gpu_lib
    # noise free: the whole chain recovers s_i - s_0 exactly
    L, P, N = 8, 24, 300
    rng = np.random.default_rng(0)
    base = np.concatenate([np.arange(L), np.arange(L)])
    sp = np.concatenate([base, rng.integers(0, L, P - base.size)])
    s = np.concatenate([rng.permutation(sp), rng.integers(0, L, N - P)])
    inst = synth.make_instance(4, 4, N, L, sigma2=1e-12, decay=8.0, seed=2, shifts=s)
    d = mra.dims(N, 4, 4, L, 1e-12)
    ws = mra.workspace(mra.mra_sync_workspace_bytes(d, P))
    out = torch.empty(N, dtype=torch.int32, device="cuda")
    mra.mra_sync(d, dev_y(inst.y), P, 50, 100, out, ws)
    np.testing.assert_array_equal(host(out), (s - s[0]) % L)


def run_stages(mra, inst, P):
    """The chain mra_sync and its three stages on the same input; the chain must equal the
    composition of the stages exactly (same kernels, same order)."""
    d = mra.dims(inst.N, inst.K, inst.Q, inst.L, inst.sigma2)
    y = dev_y(inst.y)
    ws = mra.workspace(mra.mra_sync_workspace_bytes(d, P))
    rel = torch.empty((P, P), dtype=torch.int32, device="cuda")
    phi = torch.empty(P, dtype=torch.int32, device="cuda")
    sm = torch.empty(inst.N, dtype=torch.int32, device="cuda")
    chain = torch.empty(inst.N, dtype=torch.int32, device="cuda")
    mra.mra_sync_pairwise(d, y, P, rel)
    mra.mra_sync_ppm(inst.L, P, rel, 50, 100, phi)
    mra.mra_sync_match(d, y, P, phi, sm, ws)
    mra.mra_sync(d, y, P, 50, 100, chain, ws)
    np.testing.assert_array_equal(host(chain), host(sm))
    return host(rel), host(phi), host(chain)


@pytest.mark.parametrize("cfg,N,P,seed", [(1, None, None, 1103), (1, None, 40, 1105), (2, 5000, 100, 2103)])
def test_sync_chain_certified(gpu_lib, cfg, N, P, seed):
    """Every image where mra_sync differs from the oracle's Synchronize and Match traces to a
    certified near-tie of the pairwise, PPM-rounding or match stage; at the benchmark's shape
    (|k| <= 32, Q = 24, L = 360, P = 100) on 5,000 images as well as at |k| <= 10."""
    from sync_certify import certify_chain

    c = synth.config(cfg)
    N = N or c["N"]
    P = P or c["P"]
    inst = synth.make_instance(c["K"], c["Q"], N, c["L"], c["snr"], c["decay"], seed=seed)
    y64 = synth.c64_round(inst.y)
    g_rel, g_phi, g_chain = run_stages(gpu_lib, inst, P)
    rep = certify_chain(y64, P, inst.L, g_rel, g_phi, g_chain)
    assert not rep["uncertified"], (rep["uncertified"][:10], rep["causes"])
    print(f"cfg {cfg} N {N} P {P}: {rep['mismatch']} images differ, all certified: {dict(rep['causes'])}, "
          f"{rep['rel_ties']} pairwise near-ties")


def test_prior_hist_and_fit(gpu_lib):
    mra = gpu_lib
    c = synth.config(1)
    inst = synth.make_instance(c["K"], c["Q"], c["N"], c["L"], c["snr"], c["decay"], seed=1104)
    y64 = synth.c64_round(inst.y)
    rng = np.random.default_rng(4)
    s_hat = (inst.s + rng.integers(-3, 4, inst.N) + 11) % inst.L  # a global offset plus errors
    counts, cref, _ = O.residual_histogram(y64, inst.s, s_hat, inst.x, inst.L)
    d = mra.dims(inst.N, inst.K, inst.Q, inst.L, inst.sigma2)
    ws = mra.workspace(mra.mra_em_workspace_bytes(d, 1))
    hist = torch.zeros(inst.L, dtype=torch.int32, device="cuda")
    center = torch.zeros(1, dtype=torch.int32, device="cuda")
    mra.mra_prior_hist(d, dev_y(inst.y), dev(inst.s.astype(np.int32)), dev(s_hat.astype(np.int32)),
                       dev(inst.x), hist, center, ws)
    assert int(center.item()) == cref
    np.testing.assert_array_equal(host(hist), counts)
    for kind in (0, 1):
        for Lw in (c["Lw"], 7, inst.L):
            lp_ref, k_ref = O.fit_prior(counts, inst.L, Lw, kind=kind)
            lp = torch.empty(Lw, dtype=torch.float64, device="cuda")
            kap = torch.empty(1, dtype=torch.float64, device="cuda")
            mra.mra_fit_prior(inst.L, Lw, -(Lw // 2), hist, kind, lp, kap)
            g = host(lp)
            fin = np.isfinite(lp_ref)
            np.testing.assert_array_equal(np.isfinite(g), fin)
            np.testing.assert_allclose(g[fin], lp_ref[fin], atol=1e-10)
            assert abs(kap.item() - k_ref) <= 1e-8 * max(1.0, k_ref)


@pytest.mark.parametrize("kappa", [0.5, 8.0, 45.0, 60.0, 400.0])
def test_von_mises_concentration(gpu_lib, kappa):
    """The CUDA Bessel-ratio solve against the oracle's scipy one, on both sides of the series switch."""
    mra = gpu_lib
    rng = np.random.default_rng(int(kappa * 10))
    L = 720
    th = rng.vonmises(0.0, kappa, 200_000)
    r = np.floor(np.mod(th, 2 * np.pi) * L / (2 * np.pi) + 0.5).astype(int) % L
    counts = np.bincount(r, minlength=L).astype(np.int32)
    lp_ref, k_ref = O.fit_prior(counts, L, 72, kind=1)
    lp = torch.empty(72, dtype=torch.float64, device="cuda")
    kap = torch.empty(1, dtype=torch.float64, device="cuda")
    mra.mra_fit_prior(L, 72, -36, dev(counts), 1, lp, kap)
    assert abs(kap.item() - k_ref) <= 1e-8 * k_ref
    np.testing.assert_allclose(host(lp), lp_ref, atol=1e-8)


def test_relerr(gpu_lib):
    mra = gpu_lib
    x = synth.make_signal(10, 8, 50.0, np.random.default_rng(1))
    rng = np.random.default_rng(2)
    for trial in range(4):
        xh = O.rotate(x, rng.uniform(0, 2 * np.pi)) + 0.05 * (rng.standard_normal(x.shape) + 1j * rng.standard_normal(x.shape))
        out = torch.empty(1, dtype=torch.float64, device="cuda")
        mra.mra_relerr(10, 8, dev(xh), dev(x), out)
        assert abs(out.item() - O.relerr(xh, x)) <= 1e-9
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    mra.mra_relerr(10, 8, dev(O.rotate(x, 0.123)), dev(x), out)
    assert out.item() < 1e-7
