"""Synthetic reproductions of the paper's parameter studies (Sec. 4: prior weighting,
window width, signal prior) on one device, through the library's calls only.

    gamma_study      iterations to the stopping tolerance and relative error of Synch-EM
                     for prior weights gamma (Sec. 4, "Prior weighting")
    bw_study         relative error of Synch-EM for window widths BW (Sec. 4,
                     "Performance with different BW"), with a signal prior
    signal_prior_study
                     relative error and iterations of Synch-EM and full-search EM for the
                     decay parameter of Gamma_a = diag((4 e^{-k/beta})^2) (Sec. 4,
                     "Performance with signal prior"), and without a signal prior
    pearson_study    1-D MRA (Sec. 3.1.1): fraction of Pearson coefficients between the shifted
                     signal's entries and the noise's entries with p < 0.05, before
                     synchronization, after angular synchronization (PPM over all images) and
                     after Synchronize and Match
    degraded_study   1-D MRA: relative error of EM, template matching + EM and PPM
                     synchronization + EM against SNR (Sec. 3.1.1, degraded performance)
    dense_study      relative error of Synch-EM on images with continuous (off-grid) rotations
                     for the grid window and the denser-resolution window (Sec. 3.3): the
                     same number of rotations over a narrower range, or the same range at a
                     finer spacing

Each trial draws a fresh instance (observation model of Eq. MRA_Model_FB), runs
Synchronize and Match, learns the window prior from one trial of Algorithm 1 on the
same instance (its rotations are known, as in the paper's Monte-Carlo learning) and
runs EM to tol = 1e-5 or T iterations.  The paper's BW = 2 h corresponds to the window
Lw = BW + 1 (offsets -h .. h).  Results are means over trials.

    python -m paper_2105_07372_gb300.experiments gamma|bw|prior|dense|pearson|degraded [--n N] [--trials R]
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np
import torch

from . import mra, pipeline


def _instance(K, Q, N, L, snr, decay, seed, dev, offgrid=False):
    import synth  # the seeded generator of the observation model (data only)

    inst = synth.make_instance(K, Q, N, L, snr, decay, seed=seed, offgrid=offgrid)
    y = torch.from_numpy(synth.to_c64(inst.y)).to(dev)
    return inst, y, torch.from_numpy(inst.s.astype(np.int32)).to(dev), torch.from_numpy(inst.x).to(dev)


def gamma_inv(K, Q, beta, dev):
    """Diagonal of Gamma_a^{-1} for Gamma_a = diag((4 e^{-k/beta})^2) over the stored [K+1][Q] entries."""
    k = np.arange(K + 1, dtype=np.float64)[:, None] * np.ones((1, Q))
    return torch.from_numpy((1.0 / (4.0 * np.exp(-k / beta)) ** 2).ravel()).to(dev)


def synch_em_trial(y, s_true, x_true, d, *, Lw, gamma, P=100, tol=1e-5, T=1000, gamma_a_inv=None, ws=None,
                   step=1.0, shift=None):
    """Synchronize and Match, one trial of Algorithm 1, Synch-EM to tol: (iterations, relative error).
    step < 1: the denser window of Lw rotations step grid units apart; shift: reuse a synchronization."""
    if ws is None:
        ws = pipeline.workspaces(d, Lw, P, y.device)
    if shift is None:
        shift = pipeline.synchronize(y, d, P, ws)
    log_prior, _, _ = pipeline.learn_prior(y, d, s_true, shift, x_true, Lw, -(Lw // 2), 0, ws, step=step)
    x = torch.empty((d.K + 1, d.Q), dtype=torch.complex128, device=y.device)
    mra.mra_align_mean(d, y, shift, x, ws.em)
    log_rho = log_prior.clone()
    prm = mra.em_params(Lw, gamma=gamma, log_rho_bar=log_prior, gamma_a_inv=gamma_a_inv, tol=tol, max_iters=T,
                        check_every=25, step=step)
    n = mra.mra_em_run(d, prm, y, shift, x, log_rho, None, None, ws.em)
    return n, pipeline.relerr(x, x_true, d)


def full_em_trial(y, x_true, d, x0, *, tol=1e-5, T=1000, gamma_a_inv=None, ws=None):
    """Full-search EM from x0 to tol: (iterations, relative error)."""
    if ws is None:
        ws = mra.workspace(mra.mra_em_workspace_bytes(d, d.L), y.device)
    x = x0.clone()
    log_rho = torch.full((d.L,), -math.log(d.L), dtype=torch.float64, device=y.device)
    prm = mra.em_params(d.L, l0=0, gamma=0.0, gamma_a_inv=gamma_a_inv, tol=tol, max_iters=T, check_every=25)
    n = mra.mra_em_run(d, prm, y, None, x, log_rho, None, None, ws)
    return n, pipeline.relerr(x, x_true, d)


def gamma_study(snrs=(1 / 20, 1 / 50, 1 / 100), gammas=(0.0, 1.0, 10.0, 100.0), *, K=32, Q=24, N=5000, L=360,
                BW=36, trials=3, decay=400.0, seed=6000, dev="cuda"):
    out = []
    Lw = BW + 1
    for si, snr in enumerate(snrs):
        rows = {g: [] for g in gammas}
        for t in range(trials):
            inst, y, s, x = _instance(K, Q, N, L, snr, decay, seed + 100 * si + t, dev)
            d = mra.dims(N, K, Q, L, inst.sigma2)
            ws = pipeline.workspaces(d, Lw, 100, dev)
            for g in gammas:
                rows[g].append(synch_em_trial(y, s, x, d, Lw=Lw, gamma=g, ws=ws))
        for g in gammas:
            it, err = np.mean([r[0] for r in rows[g]]), np.mean([r[1] for r in rows[g]])
            out.append({"snr": snr, "gamma": g, "iters": float(it), "relerr": float(err)})
    return out


def bw_study(snrs=(1 / 20, 1 / 50), bws=(8, 16, 24, 32, 48, 64), *, K=32, Q=24, N=10000, L=360, trials=2,
             decay=400.0, beta=8.0, gamma=100.0, seed=6500, dev="cuda"):
    out = []
    gi = gamma_inv(K, Q, beta, dev)
    for si, snr in enumerate(snrs):
        errs = {b: [] for b in bws}
        for t in range(trials):
            inst, y, s, x = _instance(K, Q, N, L, snr, decay, seed + 100 * si + t, dev)
            d = mra.dims(N, K, Q, L, inst.sigma2)
            for b in bws:
                errs[b].append(synch_em_trial(y, s, x, d, Lw=b + 1, gamma=gamma, gamma_a_inv=gi)[1])
        for b in bws:
            out.append({"snr": snr, "BW": b, "relerr": float(np.mean(errs[b]))})
    return out


def signal_prior_study(snrs=(1 / 20, 1 / 50), betas=(None, 4.0, 8.0, 16.0), *, K=32, Q=24, N=5000, L=360, BW=36,
                       trials=2, decay=400.0, gamma=100.0, seed=7000, dev="cuda"):
    import synth

    out = []
    for si, snr in enumerate(snrs):
        acc = {b: {"sem": [], "em": []} for b in betas}
        for t in range(trials):
            inst, y, s, x = _instance(K, Q, N, L, snr, decay, seed + 100 * si + t, dev)
            d = mra.dims(N, K, Q, L, inst.sigma2)
            x0 = torch.from_numpy(synth.random_init(K, Q, decay, seed=seed + 7 * t + si)).to(dev)
            for b in betas:
                gi = gamma_inv(K, Q, b, dev) if b is not None else None
                acc[b]["sem"].append(synch_em_trial(y, s, x, d, Lw=BW + 1, gamma=gamma, gamma_a_inv=gi))
                acc[b]["em"].append(full_em_trial(y, x, d, x0, gamma_a_inv=gi))
        for b in betas:
            for kind in ("sem", "em"):
                r = acc[b][kind]
                out.append({"snr": snr, "beta": b, "method": "Synch-EM" if kind == "sem" else "EM",
                            "iters": float(np.mean([v[0] for v in r])), "relerr": float(np.mean([v[1] for v in r]))})
    return out


def dense_study(snrs=(1 / 5, 1 / 20, 1 / 50), *, K=32, Q=24, N=10000, L=360, trials=2, decay=400.0,
                windows=((37, 1.0), (37, 0.25), (145, 0.25)), gamma=100.0, seed=8000, dev="cuda"):
    """Images rotated by continuous angles (off the grid).  For each window (Lw, step): relative error and
    iterations of Synch-EM from one shared synchronization per trial; (37, 1) is the grid window BW = 36,
    (37, 1/4) the same number of rotations over a quarter of the range, (145, 1/4) the same range at a
    quarter of the spacing."""
    out = []
    for si, snr in enumerate(snrs):
        acc = {w: [] for w in windows}
        for t in range(trials):
            inst, y, s, x = _instance(K, Q, N, L, snr, decay, seed + 100 * si + t, dev, offgrid=True)
            d = mra.dims(N, K, Q, L, inst.sigma2)
            ws = pipeline.workspaces(d, max(w[0] for w in windows), 100, dev)
            shift = pipeline.synchronize(y, d, 100, ws)
            for (Lw, step) in windows:
                acc[(Lw, step)].append(synch_em_trial(y, s, x, d, Lw=Lw, gamma=gamma, ws=ws, step=step, shift=shift))
        for (Lw, step) in windows:
            r = acc[(Lw, step)]
            out.append({"snr": snr, "Lw": Lw, "step": step, "range_grid_units": (Lw - 1) * step,
                        "iters": float(np.mean([v[0] for v in r])), "relerr": float(np.mean([v[1] for v in r]))})
    return out


# ---------------------------------------------------------------- 1-D MRA through the coefficient form
def _dims_1d(inst, mra):
    return mra.dims(inst.N, (inst.L - 1) // 2, 2, inst.L, 2.0 * inst.sigma ** 2)


def _coeff_dev(v, dev):
    import synth

    return torch.from_numpy(synth.to_c64(synth.coeffs_1d(v))).to(dev)


def _pearson_fraction(a, b, alpha=0.05):
    """Fraction of the L x L Pearson coefficients r(a[:, i], b[:, j]) whose two-sided p-value (Student t with N - 2
    degrees of freedom, t = r sqrt((N - 2) / (1 - r^2))) is below alpha."""
    from scipy import stats

    n = a.shape[0]
    az = (a - a.mean(0)) / np.sqrt(((a - a.mean(0)) ** 2).sum(0))
    bz = (b - b.mean(0)) / np.sqrt(((b - b.mean(0)) ** 2).sum(0))
    r = np.clip(az.T @ bz, -0.999999, 0.999999)
    t = r * np.sqrt((n - 2) / (1 - r ** 2))
    p = 2 * stats.t.sf(np.abs(t), n - 2)
    return float(np.mean(p < alpha))


def _aligned_pair(inst, shat):
    """(shifted signal after alignment, noise after alignment): roll(x, s - s_hat) and roll(eps, -s_hat)."""
    L = inst.L
    idx = (np.arange(L)[None, :] - (inst.s - shat)[:, None]) % L
    a = inst.x[idx]
    b = np.stack([np.roll(e, -int(sh)) for e, sh in zip(inst.eps, shat)])
    return a, b


def pearson_study(*, L=21, sigma=2.0, N=1000, trials=20, P=100, seed=9500, dev="cuda"):
    """Sec. 3.1.1: 1-D MRA with x ~ N(0, I_21), sigma = 2, N = 1000.  Returns the mean fractions of p < 0.05."""
    import synth

    out = {"before": [], "ppm": [], "synch_and_match": []}
    for t in range(trials):
        inst = synth.make_instance_1d(L, N, sigma, seed=seed + t)
        d = _dims_1d(inst, mra)
        y = _coeff_dev(inst.v, dev)
        idx = (np.arange(L)[None, :] - inst.s[:, None]) % L
        out["before"].append(_pearson_fraction(inst.x[idx], inst.eps))
        # angular synchronization over all images: pairwise rotations and the projected power method
        rel = torch.empty((N, N), dtype=torch.int32, device=dev)
        mra.mra_sync_pairwise(d, y, N, rel)
        phi = torch.empty(N, dtype=torch.int32, device=dev)
        mra.mra_sync_ppm(L, N, rel, 50, 100, phi)
        out["ppm"].append(_pearson_fraction(*_aligned_pair(inst, phi.cpu().numpy().astype(np.int64))))
        ws = mra.workspace(mra.mra_sync_workspace_bytes(d, P), dev)
        sh = torch.empty(N, dtype=torch.int32, device=dev)
        mra.mra_sync(d, y, P, 50, 100, sh, ws)
        out["synch_and_match"].append(_pearson_fraction(*_aligned_pair(inst, sh.cpu().numpy().astype(np.int64))))
    return {k: float(np.mean(v)) for k, v in out.items()}


def _relerr_1d(xhat, x):
    """min over cyclic shifts ||roll(xhat, s) - x|| / ||x|| (1-D relative error up to a shift)."""
    return float(min(np.linalg.norm(np.roll(xhat, s) - x) for s in range(x.size)) / np.linalg.norm(x))


def degraded_study(snrs=(1 / 8, 1 / 4, 1 / 2, 1, 2, 4), *, L=21, N=500, trials=10, T=1000, tol=1e-6, seed=9600, dev="cuda"):
    """Sec. 3.1.1 (degraded performance): relative error of EM from a random start, of template matching (first
    observation as reference) + EM and of PPM synchronization over all images + EM, each EM over all L shifts with a
    uniform start, against the SNR ||x||^2 / (L sigma^2)."""
    import synth

    rows = []
    for si, snr in enumerate(snrs):
        acc = {"EM": [], "TM+EM": [], "Synch+EM": []}
        for t in range(trials):
            rng = np.random.default_rng(seed + 100 * si + t)
            x = rng.standard_normal(L)
            sigma = float(np.linalg.norm(x) / np.sqrt(L * snr))
            inst = synth.make_instance_1d(L, N, sigma, seed=seed + 100 * si + t, x=x)
            d = _dims_1d(inst, mra)
            y = _coeff_dev(inst.v, dev)
            ws = mra.workspace(mra.mra_em_workspace_bytes(d, L), dev)

            def em_from(x0, shift):
                xc = x0.clone()
                lr = torch.full((L,), -np.log(L), dtype=torch.float64, device=dev)
                prm = mra.em_params(L, l0=0, max_iters=T, tol=tol, check_every=50)
                mra.mra_em_run(d, prm, y, shift, xc, lr, None, None, ws)
                return _relerr_1d(synth.signal_1d(xc.cpu().numpy(), L), x)

            x0 = torch.from_numpy(synth.coeffs_1d(rng.standard_normal(L))).to(dev)
            acc["EM"].append(em_from(x0, None))
            tm = pipeline.template_match(y, d, y[0])
            xa = torch.empty_like(x0)
            mra.mra_align_mean(d, y, tm, xa, ws)
            acc["TM+EM"].append(em_from(xa, tm))
            rel = torch.empty((N, N), dtype=torch.int32, device=dev)
            mra.mra_sync_pairwise(d, y, N, rel)
            phi = torch.empty(N, dtype=torch.int32, device=dev)
            mra.mra_sync_ppm(L, N, rel, 50, 100, phi)
            mra.mra_align_mean(d, y, phi, xa, ws)
            acc["Synch+EM"].append(em_from(xa, phi))
        for k, v in acc.items():
            rows.append({"snr": snr, "method": k, "relerr": float(np.mean(v))})
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("study", choices=("gamma", "bw", "prior", "dense", "pearson", "degraded"))
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--trials", type=int, default=None)
    a = ap.parse_args()
    kw = {}
    if a.n:
        kw["N"] = a.n
    if a.trials:
        kw["trials"] = a.trials
    mra.load()
    fn = {"gamma": gamma_study, "bw": bw_study, "prior": signal_prior_study, "dense": dense_study,
          "pearson": pearson_study, "degraded": degraded_study}[a.study]
    res = fn(**kw)
    for row in (res if isinstance(res, list) else [res]):
        print(json.dumps(row), flush=True)


if __name__ == "__main__":
    main()
