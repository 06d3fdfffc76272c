"""Host-side helpers of the pipeline and the experiments, on the CPU: the window chosen to hold a given mass of
the learned residual histogram (Sec. 3.3), and the pieces of the Pearson diagnostic of Sec. 3.1.1 (p-values,
the aligned signal/noise pair, the 1-D relative error up to a shift) against library routines and identities."""
import numpy as np
import pytest
import torch
from scipy import stats

import synth
from paper_2105_07372_gb300 import experiments, pipeline


def _window_mass(h, L, Lw):
    """Mass of the offsets -Lw//2 .. Lw - 1 - Lw//2 (mod L), by a loop."""
    return sum(h[o % L] for o in range(-(Lw // 2), Lw - (Lw // 2)))


@pytest.mark.parametrize("seed", range(6))
def test_window_for_mass_is_the_smallest_window(seed):
    rng = np.random.default_rng(seed)
    L = int(rng.integers(5, 40))
    h = np.zeros(L)
    centre = rng.integers(-3, 4)
    for o in rng.normal(centre, 2.0, 200).round().astype(int):
        h[o % L] += 1
    mass = float(rng.uniform(0.3, 1.0))
    Lw = pipeline.window_for_mass(torch.from_numpy(h), L, mass)
    assert _window_mass(h, L, Lw) >= mass * h.sum()
    assert Lw == 1 or _window_mass(h, L, Lw - 1) < mass * h.sum()


def test_window_for_mass_edges():
    L = 12
    h = np.zeros(L)
    h[0] = 5
    assert pipeline.window_for_mass(torch.from_numpy(h), L, 1.0) == 1
    h[L - 1] = 5  # offset -1 joins at Lw = 2 (offsets -1, 0)
    assert pipeline.window_for_mass(torch.from_numpy(h), L, 1.0) == 2
    h[:] = 0
    h[3] = 1  # offset +3 needs offsets -3 .. 3
    assert pipeline.window_for_mass(torch.from_numpy(h), L, 1.0) == 7
    assert pipeline.window_for_mass(torch.ones(L, dtype=torch.float64), L, 1.0) == L


def test_pearson_fraction_against_scipy():
    rng = np.random.default_rng(3)
    n, L = 300, 6
    a = rng.standard_normal((n, L))
    b = 0.3 * a[:, ::-1] + rng.standard_normal((n, L))
    want = np.mean([stats.pearsonr(a[:, i], b[:, j])[1] < 0.05 for i in range(L) for j in range(L)])
    assert experiments._pearson_fraction(a, b) == pytest.approx(want, abs=1e-12)


def test_pearson_fraction_of_independent_columns_is_alpha():
    rng = np.random.default_rng(4)
    n, L, reps = 400, 10, 40
    f = np.mean([experiments._pearson_fraction(rng.standard_normal((n, L)), rng.standard_normal((n, L)))
                 for _ in range(reps)])
    assert abs(f - 0.05) < 4 * np.sqrt(0.05 * 0.95 / (L * L * reps))


def test_aligned_pair_sums_to_the_aligned_observation():
    inst = synth.make_instance_1d(21, 50, 1.3, seed=5)
    shat = np.random.default_rng(6).integers(0, 21, 50)
    a, b = experiments._aligned_pair(inst, shat)
    back = np.stack([np.roll(v, -int(s)) for v, s in zip(inst.v, shat)])
    np.testing.assert_allclose(a + b, back, atol=1e-12)
    a0, _ = experiments._aligned_pair(inst, inst.s)  # exact alignment leaves x itself
    np.testing.assert_allclose(a0, np.broadcast_to(inst.x, a0.shape), atol=0)


def test_relerr_1d_up_to_a_shift():
    x = np.random.default_rng(7).standard_normal(15)
    assert experiments._relerr_1d(np.roll(x, 4), x) < 1e-15
    assert experiments._relerr_1d(1.1 * np.roll(x, -2), x) == pytest.approx(0.1, rel=1e-12)
