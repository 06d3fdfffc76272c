"""The parameter studies of Sec. 4 (prior weight gamma, window width BW, signal prior)
run end to end through the library on small synthetic instances.  Their outcomes are
statistical (the paper reports trends over trials), so the test checks that every
study runs and returns sane values, plus two properties that hold by construction:
the signal prior with a flat covariance limit changes nothing, and a window of 8
offsets cannot beat one that holds the same offsets and more by a wide margin."""
import math

import pytest
import torch

pytestmark = pytest.mark.gpu


def test_studies_run_and_are_sane(gpu_lib):
    from paper_2105_07372_gb300 import experiments as E

    g = E.gamma_study(snrs=(1 / 50,), gammas=(0.0, 100.0), N=1500, trials=1)
    assert len(g) == 2 and all(1 <= r["iters"] <= 1000 and 0 < r["relerr"] < 1 for r in g)
    b = E.bw_study(snrs=(1 / 50,), bws=(8, 48), N=1500, trials=1)
    err = {r["BW"]: r["relerr"] for r in b}
    assert all(0 < v < 1 for v in err.values())
    assert err[48] <= err[8] + 0.02, err
    p = E.signal_prior_study(snrs=(1 / 50,), betas=(None, 8.0), N=1500, trials=1)
    assert len(p) == 4 and all(0 < r["relerr"] < 1 and r["iters"] >= 1 for r in p)


def test_flat_signal_prior_limit(gpu_lib):
    """Gamma_a^{-1} = 0 is the flat image prior: the run equals the one without gamma_a_inv."""
    import numpy as np

    from paper_2105_07372_gb300 import experiments as E
    from paper_2105_07372_gb300 import mra, pipeline

    inst, y, s, x = E._instance(8, 8, 800, 60, 1 / 20, 50.0, 123, "cuda")
    d = mra.dims(inst.N, inst.K, inst.Q, inst.L, inst.sigma2)
    zero = torch.zeros((inst.K + 1) * inst.Q, dtype=torch.float64, device="cuda")
    n0, e0 = E.synch_em_trial(y, s, x, d, Lw=13, gamma=10.0, T=20)
    n1, e1 = E.synch_em_trial(y, s, x, d, Lw=13, gamma=10.0, T=20, gamma_a_inv=zero)
    assert n0 == n1 and math.isclose(e0, e1, rel_tol=1e-12, abs_tol=1e-15)


def test_dense_study_runs_and_finer_spacing_does_not_hurt(gpu_lib):
    """Off-grid rotations at a high SNR: the window of the same range at a quarter of the spacing holds the grid
    window's rotations among others, so its error cannot be much larger (it is expected to be smaller)."""
    from paper_2105_07372_gb300 import experiments as E

    r = E.dense_study(snrs=(1 / 5,), N=2000, trials=1, windows=((37, 1.0), (145, 0.25)))
    err = {(v["Lw"], v["step"]): v["relerr"] for v in r}
    assert all(0 < e < 1 for e in err.values())
    assert err[(145, 0.25)] <= err[(37, 1.0)] + 0.005, err


def test_pearson_and_degraded_studies_run(gpu_lib):
    """1-D studies (Sec. 3.1.1) on small runs: before synchronization the fraction of Pearson p-values below 0.05
    is the test's nominal level (independent entries); synchronization by PPM over all images raises it; the
    degraded-performance study returns sane errors for its three methods."""
    from paper_2105_07372_gb300 import experiments as E

    r = E.pearson_study(trials=3)
    assert 0.02 <= r["before"] <= 0.09, r
    assert r["ppm"] > r["before"], r
    rows = E.degraded_study(snrs=(2.0,), trials=2, N=300)
    assert {v["method"] for v in rows} == {"EM", "TM+EM", "Synch+EM"}
    assert all(0 <= v["relerr"] < 1.5 for v in rows), rows
