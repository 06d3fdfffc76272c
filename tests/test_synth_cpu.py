"""The seeded input generator against its stated recipe (CPU): unit-norm signals with a real k = 0 row and the
exp(-k^2 / decay) variance profile, the two-sided image energy against a rendered pixel image, the pixel-space
SNR, circular complex noise of variance sigma^2 on every stored entry, grid and off-grid rotations."""
import numpy as np
import pytest

import synth


def test_signal_is_unit_norm_with_real_k0_row():
    for seed in range(5):
        x = synth.make_signal(12, 7, 30.0, np.random.default_rng(seed))
        assert abs(np.linalg.norm(x) - 1.0) < 1e-14
        assert np.all(x[0].imag == 0.0)


def test_signal_variance_profile():
    """E|x_kq|^2 / E|x_0q|^2 = exp(-k^2 / decay) (k > 0 rows complex, k = 0 real with the same variance),
    up to the common per-draw normalisation."""
    K, Q, decay, n = 8, 32, 20.0, 400
    rng = np.random.default_rng(7)
    p = np.mean([np.mean(np.abs(synth.make_signal(K, Q, decay, rng)) ** 2, axis=1) for _ in range(n)], axis=0)
    want = np.exp(-np.arange(K + 1) ** 2 / decay)
    np.testing.assert_allclose(p / p[0], want, rtol=0.08, atol=2e-3)


@pytest.mark.parametrize("K,Q,n", [(10, 8, 65), (20, 10, 97)])
def test_image_energy_is_the_rendered_pixel_energy(K, Q, n):
    """||I||_F^2 of the rendered real image equals |x_0|^2 + 2 sum_{k>0} |x_k|^2 (orthonormal basis, App. A)."""
    x = synth.make_signal(K, Q, 50.0, np.random.default_rng(K))
    img = synth.render(x, n)
    assert abs(float(np.sum(img ** 2)) - synth.image_energy(x)) <= 1e-3 * synth.image_energy(x)


def test_sigma2_is_the_pixel_space_snr():
    x = synth.make_signal(6, 4, 20.0, np.random.default_rng(3))
    for snr in (1 / 50, 1.0, 4.0):
        s2 = synth.sigma2_for_snr(snr, x)
        assert s2 * synth.NPIX * snr == pytest.approx(synth.image_energy(x), rel=1e-14)
        inst = synth.make_instance(6, 4, 3, 10, snr=snr, x=x, seed=1)
        assert inst.sigma2 == pytest.approx(s2, rel=1e-14)


def test_noise_is_circular_with_variance_sigma2_on_every_entry():
    K, Q, N, L, s2 = 4, 6, 20000, 16, 0.37
    x = synth.make_signal(K, Q, 10.0, np.random.default_rng(4))
    inst = synth.make_instance(K, Q, N, L, sigma2=s2, x=x, seed=5)
    eps = inst.y - x[None] * np.exp(-2j * np.pi * np.outer(inst.s, np.arange(K + 1)) / L)[:, :, None]
    n = N * Q
    for k in range(K + 1):
        e = eps[:, k, :].ravel()
        assert abs(np.mean(np.abs(e) ** 2) / s2 - 1) < 6 * np.sqrt(1 / n)
        assert abs(np.mean(e * e)) / s2 < 6 / np.sqrt(n)  # circular: E eps^2 = 0
        assert abs(np.var(e.real) / (s2 / 2) - 1) < 8 * np.sqrt(2 / n)


def test_rotations_on_and_off_the_grid():
    K, Q, N, L = 5, 3, 500, 24
    x = synth.make_signal(K, Q, 10.0, np.random.default_rng(6))
    g = synth.make_instance(K, Q, N, L, sigma2=0.0, x=x, seed=7)
    assert g.rot is None and g.s.min() >= 0 and g.s.max() < L
    np.testing.assert_allclose(g.y, x[None] * np.exp(-2j * np.pi * np.outer(g.s, np.arange(K + 1)) / L)[:, :, None],
                               atol=1e-15)
    o = synth.make_instance(K, Q, N, L, sigma2=0.0, x=x, seed=7, offgrid=True)
    f = o.rot - o.s
    assert f.min() >= -0.5 and f.max() < 0.5 and np.std(f) > 0.25
    np.testing.assert_allclose(o.y, x[None] * np.exp(-2j * np.pi * np.outer(o.rot, np.arange(K + 1)) / L)[:, :, None],
                               atol=1e-15)
