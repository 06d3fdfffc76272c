"""Pins for the FP64 oracle against things other than itself.

Each test ties one oracle function to brute force, a library routine, a closed
form or an invariant fixed by the paper, so that a dropped term, a wrong sign,
a wrong index or a transposed operand in the oracle fails at least one of them.
"""
import cmath
import itertools
import math

import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def soft(snr, K, Q):
    """A noise variance that keeps the posteriors of small test instances spread over several rotations."""
    return 1.0 / (snr * (K + 1) * Q)


def tiny(seed=0, K=2, Q=2, N=3, L=5, snr=0.5):
    return synth.make_instance(K=K, Q=Q, N=N, L=L, sigma2=soft(snr, K, Q), decay=4.0, seed=seed)


# --------------------------------------------------------------------------- rotations
def test_rotation_group_law_and_sign():
    """R_a R_b = R_{a+b}; rotating by 2 pi is the identity; the model's sign (Eq. fb_rotation)."""
    rng = np.random.default_rng(1)
    a = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
    np.testing.assert_allclose(O.rotate(O.rotate(a, 0.3), 1.1), O.rotate(a, 1.4), atol=1e-14)
    np.testing.assert_allclose(O.rotate(a, 2 * math.pi), a, atol=1e-13)
    # entry (k, q) picks up exp(-i k phi), written out element by element
    phi = 0.7
    for k in range(4):
        for q in range(3):
            assert abs(O.rotate(a, phi)[k, q] - a[k, q] * cmath.exp(-1j * k * phi)) < 1e-14


# --------------------------------------------------------------------------- E-step by brute force
def _dist2_loops(x, v, theta):
    s = 0.0
    for k in range(x.shape[0]):
        for q in range(x.shape[1]):
            d = x[k, q] * cmath.exp(-1j * k * theta) - v[k, q]
            s += d.real * d.real + d.imag * d.imag
    return s


@pytest.mark.parametrize("Lw,l0,step", [(5, -2, 1.0), (3, -1, 1.0), (4, 0, 1.0), (5, -2, 0.37), (4, -3, 0.5)])
def test_posterior_and_loglik_by_joint_enumeration(Lw, l0, step):
    """Enumerate all Lw^N joint rotations: marginals equal w_jl, log-sum equals the log-likelihood.
    step < 1: the denser window's angles 2 pi step (l0 + i) / L, off the grid."""
    inst = tiny(seed=3)
    L, N, sigma2 = inst.L, inst.N, inst.sigma2
    x = synth.make_signal(inst.K, inst.Q, 4.0, np.random.default_rng(9))
    rng = np.random.default_rng(5)
    rho = rng.random(Lw) + 0.1
    rho /= rho.sum()
    offs = [(l0 + i) * step for i in range(Lw)]
    M = (inst.K + 1) * inst.Q
    logp = {}
    for combo in itertools.product(range(Lw), repeat=N):
        lp = 0.0
        for j, li in enumerate(combo):
            lp += math.log(rho[li]) - _dist2_loops(x, inst.y[j], 2 * math.pi * offs[li] / L) / sigma2
            lp -= M * math.log(math.pi * sigma2)
        logp[combo] = lp
    mx = max(logp.values())
    Z = sum(math.exp(v - mx) for v in logp.values())
    marg = np.zeros((N, Lw))
    for combo, v in logp.items():
        p = math.exp(v - mx) / Z
        for j, li in enumerate(combo):
            marg[j, li] += p
    st = O.em_step(inst.y, x, np.log(rho), L, sigma2, Lw=Lw, l0=l0, step=step)
    np.testing.assert_allclose(st.w, marg, atol=1e-12)
    assert abs(st.loglik - (mx + math.log(Z))) < 1e-9 * abs(st.loglik)


# --------------------------------------------------------------------------- M-step optimality
def _Q(a, w, y, log_rho, offs, L, sigma2, gamma_a_inv):
    """Q(a, rho | a_t, rho_t) of Eq. (expectation_step) + log p(a), written with loops over j, l."""
    val = 0.0
    for j in range(y.shape[0]):
        for i, l in enumerate(offs):
            val += w[j, i] * (log_rho[i] - _dist2_loops(a, y[j], 2 * math.pi * l / L) / sigma2)
    if gamma_a_inv is not None:
        val -= float(np.sum(gamma_a_inv * np.abs(a) ** 2))
    return val


@pytest.mark.parametrize("with_prior,step", [(False, 1.0), (True, 1.0), (False, 0.45)])
def test_mstep_maximises_Q(with_prior, step):
    inst = tiny(seed=11, N=4, L=6)
    L, sigma2 = inst.L, inst.sigma2
    Lw, l0 = 4, -2
    x = synth.make_signal(inst.K, inst.Q, 4.0, np.random.default_rng(2))
    lr = np.log(np.full(Lw, 1.0 / Lw))
    gi = None
    if with_prior:
        k = np.arange(inst.K + 1)[:, None] * np.ones((1, inst.Q))
        gi = 1.0 / (4.0 * np.exp(-k / 8.0)) ** 2
    st = O.em_step(inst.y, x, lr, L, sigma2, Lw=Lw, l0=l0, gamma_a_inv=gi, step=step)
    offs = [(l0 + i) * step for i in range(Lw)]
    q0 = _Q(st.x, st.w, inst.y, lr, offs, L, sigma2, gi)
    rng = np.random.default_rng(4)
    h = 1e-5
    # stationarity by central differences along every real coordinate
    for k in range(inst.K + 1):
        for q in range(inst.Q):
            for unit in (1.0, 1j):
                e = np.zeros_like(st.x)
                e[k, q] = unit * h
                g = (_Q(st.x + e, st.w, inst.y, lr, offs, L, sigma2, gi)
                     - _Q(st.x - e, st.w, inst.y, lr, offs, L, sigma2, gi)) / (2 * h)
                assert abs(g) < 1e-5 * max(1.0, abs(q0))
    for _ in range(5):
        d = 1e-2 * (rng.standard_normal(st.x.shape) + 1j * rng.standard_normal(st.x.shape))
        assert _Q(st.x + d, st.w, inst.y, lr, offs, L, sigma2, gi) < q0


def test_rho_update_maximises_lagrangian():
    """rho_{t+1} maximises sum W log rho + gamma sum rho_bar log rho on the simplex (App. C)."""
    inst = tiny(seed=21, N=6, L=7)
    Lw, l0 = 5, -2
    x = synth.make_signal(inst.K, inst.Q, 4.0, np.random.default_rng(3))
    lrb = np.log(np.array([0.05, 0.2, 0.5, 0.2, 0.05]))
    gamma = 3.0
    st = O.em_step(inst.y, x, np.log(np.full(Lw, 0.2)), inst.L, inst.sigma2, Lw=Lw, l0=l0, gamma=gamma, log_rho_bar=lrb)
    rho = np.exp(st.log_rho)
    assert abs(rho.sum() - 1) < 1e-14
    ratio = (st.W + gamma * np.exp(lrb)) / rho  # the Lagrange multiplier, equal for every l
    np.testing.assert_allclose(ratio, ratio[0], rtol=1e-12)

    def obj(r):
        return float(np.sum(st.W * np.log(r)) + gamma * np.sum(np.exp(lrb) * np.log(r)))

    rng = np.random.default_rng(0)
    for _ in range(50):
        r = rng.dirichlet(np.ones(Lw))
        assert obj(r) <= obj(rho) + 1e-12


# --------------------------------------------------------------------------- EM monotonicity
@pytest.mark.parametrize("gamma,with_prior,Lw", [(0.0, False, 24), (10.0, False, 24), (5.0, True, 12), (0.0, False, 72)])
def test_map_objective_nondecreasing(gamma, with_prior, Lw):
    c = synth.config(1)
    inst = synth.make_instance(K=6, Q=4, N=120, L=c["L"], sigma2=soft(0.2, 6, 4), decay=20.0, seed=7)
    L = inst.L
    gi = None
    if with_prior:
        k = np.arange(inst.K + 1)[:, None] * np.ones((1, inst.Q))
        gi = 1.0 / (4.0 * np.exp(-k / 8.0)) ** 2
    lrb = None
    if gamma > 0:
        t = 3.0 * np.cos(2 * np.pi * O.window_offsets(L, Lw) / L)
        lrb = t - np.log(np.sum(np.exp(t)))
    x = synth.random_init(inst.K, inst.Q, 20.0, seed=99)
    lr = np.log(np.full(Lw, 1.0 / Lw)) if lrb is None else lrb.copy()
    kw = dict(Lw=Lw, gamma=gamma, log_rho_bar=lrb, gamma_a_inv=gi)
    prev = O.map_objective(inst.y, x, lr, L, inst.sigma2, **kw)
    for _ in range(12):
        st = O.em_step(inst.y, x, lr, L, inst.sigma2, **kw)
        x, lr = st.x, st.log_rho
        cur = O.map_objective(inst.y, x, lr, L, inst.sigma2, **kw)
        assert cur >= prev - 1e-9 * abs(prev)
        prev = cur


# --------------------------------------------------------------------------- reduction to full-search EM (FFT form)
def _standard_em_fft(y, x, rho_full, L, sigma2):
    """Plain EM over all L rotations written with numpy.fft: S_jl = Re sum_k c_jk e^{-2 pi i k l/L}."""
    N, Kp1, Q = y.shape
    c = np.einsum("jkq,kq->jk", np.conj(y), x)  # c_jk = sum_q conj(y) x
    cpad = np.zeros((N, L), dtype=np.complex128)
    cpad[:, :Kp1] = c
    S = np.fft.fft(cpad, axis=1).real  # sum_k c_k e^{-2 pi i k l / L}
    nx = np.sum(np.abs(x) ** 2)
    ny = np.sum(np.abs(y) ** 2, axis=(1, 2))
    t = np.log(rho_full)[None, :] - (nx + ny[:, None] - 2 * S) / sigma2
    m = t.max(axis=1, keepdims=True)
    w = np.exp(t - m)
    w /= w.sum(axis=1, keepdims=True)
    Wk = np.fft.ifft(w, axis=1)[:, :Kp1] * L  # sum_l w_jl e^{+2 pi i k l / L}
    xn = np.einsum("jk,jkq->kq", Wk, y) / N
    W = w.sum(axis=0)
    return xn, W / W.sum(), w


def test_full_window_uniform_prior_is_standard_em():
    inst = synth.make_instance(K=5, Q=3, N=40, L=16, sigma2=soft(0.3, 5, 3), decay=10.0, seed=12)
    L = inst.L
    x = synth.random_init(inst.K, inst.Q, 10.0, seed=5)
    rng = np.random.default_rng(8)
    rho_full = rng.random(L) + 0.2
    rho_full /= rho_full.sum()
    l0 = -(L // 2)
    offs = O.window_offsets(L, L, l0)
    st = O.em_step(inst.y, x, np.log(rho_full[np.mod(offs, L)]), L, inst.sigma2, Lw=L, l0=l0, gamma=0.0)
    xn, rn, w = _standard_em_fft(inst.y, x, rho_full, L, inst.sigma2)
    np.testing.assert_allclose(st.x, xn, atol=1e-12)
    np.testing.assert_allclose(np.exp(st.log_rho), rn[np.mod(offs, L)], atol=1e-12)
    np.testing.assert_allclose(st.w, w[:, np.mod(offs, L)], atol=1e-12)


# --------------------------------------------------------------------------- equivariance
@pytest.mark.parametrize("Lw,l0,step", [(5, -1, 1.0), (7, -6, 1.0), (6, -2, 0.4)])
def test_opposite_rotation_sign_is_the_reflected_window(Lw, l0, step):
    """The opposite rotation convention (v = a e^{+ik theta}) is the paper's one with the window reflected,
    l -> -l: EM on the conjugated observations and signal, over the window -(l0 + Lw - 1) .. -l0 with the prior
    read backwards, gives the weights and prior read backwards and the conjugated signal (non-symmetric
    windows, on and off the grid)."""
    inst = tiny(seed=13, N=5, L=9)
    L, sigma2 = inst.L, inst.sigma2
    x = synth.make_signal(inst.K, inst.Q, 4.0, np.random.default_rng(14))
    rho = np.random.default_rng(15).random(Lw) + 0.2
    rho /= rho.sum()
    st = O.em_step(inst.y, x, np.log(rho), L, sigma2, Lw=Lw, l0=l0, step=step)
    sr = O.em_step(np.conj(inst.y), np.conj(x), np.log(rho[::-1]), L, sigma2, Lw=Lw, l0=-(l0 + Lw - 1),
                   step=step)
    np.testing.assert_allclose(sr.w, st.w[:, ::-1], atol=1e-13)
    np.testing.assert_allclose(sr.x, np.conj(st.x), atol=1e-13)
    np.testing.assert_allclose(sr.log_rho, st.log_rho[::-1], atol=1e-12)
    assert abs(sr.loglik - st.loglik) <= 1e-10 * abs(st.loglik)


def test_em_equivariant_under_global_rotation():
    inst = synth.make_instance(K=6, Q=4, N=60, L=24, sigma2=soft(0.3, 6, 4), decay=20.0, seed=31)
    L, g = inst.L, 5
    x0 = O.align_mean(inst.y, inst.s, L)
    lr = np.log(np.full(9, 1 / 9))
    a = O.em_step(inst.y, x0, lr, L, inst.sigma2, Lw=9)
    yr = O.rotate(inst.y, 2 * np.pi * g / L)
    b = O.em_step(yr, O.rotate(x0, 2 * np.pi * g / L), lr, L, inst.sigma2, Lw=9)
    np.testing.assert_allclose(b.w, a.w, atol=1e-12)
    np.testing.assert_allclose(b.x, O.rotate(a.x, 2 * np.pi * g / L), atol=1e-12)
    assert abs(a.loglik - b.loglik) < 1e-9 * abs(a.loglik)


def test_sync_invariant_under_global_rotation():
    inst = synth.make_instance(K=5, Q=4, N=50, L=24, sigma2=soft(2.0, 5, 4), decay=20.0, seed=41)
    s1, _, _ = O.synchronize_and_match(inst.y, 12, inst.L)
    s2, _, _ = O.synchronize_and_match(O.rotate(inst.y, 2 * np.pi * 7 / inst.L), 12, inst.L)
    np.testing.assert_array_equal(s1, s2)


# --------------------------------------------------------------------------- noise-free recovery
def _covering_shifts(L, P, N, rng):
    base = np.concatenate([np.arange(L), np.arange(L)])  # every rotation twice inside S_P
    sp = np.concatenate([base, rng.integers(0, L, P - base.size)])
    return np.concatenate([rng.permutation(sp), rng.integers(0, L, N - P)])


def test_noise_free_synchronize_and_match_exact():
    L, P, N = 8, 24, 60
    rng = np.random.default_rng(0)
    s = _covering_shifts(L, P, N, rng)
    inst = synth.make_instance(K=4, Q=3, N=N, L=L, sigma2=0.0, decay=8.0, seed=2, shifts=s)
    shat, phi, rel = O.synchronize_and_match(inst.y, P, L)
    np.testing.assert_array_equal(shat, (s - s[0]) % L)
    x0 = O.align_mean(inst.y, shat, L)
    np.testing.assert_allclose(x0, O.rotate(inst.x, 2 * np.pi * s[0] / L), atol=1e-12)
    assert O.relerr(x0, inst.x) < 1e-9
    counts, c, r = O.residual_histogram(inst.y, s, shat, inst.x, L)
    assert counts[0] == N and np.all(r == 0)
    lp, _ = O.fit_prior(counts, L, 5)
    assert lp[2] == 0.0 and np.all(np.isneginf(np.delete(lp, 2)))


def test_prior_residual_sign_matches_em_window():
    """A biased shift estimate for some images shows up at the same offset in the residual
    histogram and in the EM posterior (tiny noise): r_j indexes the EM window."""
    L, N = 12, 30
    rng = np.random.default_rng(3)
    s = rng.integers(0, L, N)
    inst = synth.make_instance(K=4, Q=3, N=N, L=L, sigma2=1e-6, decay=8.0, seed=4, shifts=s)
    shat = s.copy()
    shat[:6] = (shat[:6] + 2) % L  # six images estimated 2 grid steps too far
    counts, c, r = O.residual_histogram(inst.y, s, shat, inst.x, L)
    assert c == 0
    Lw = 7
    xbar = O.align_mean(inst.y, shat, L)
    st = O.em_step(inst.y, inst.x, np.log(np.full(Lw, 1 / Lw)), L, inst.sigma2, Lw=Lw, shifts=shat)
    offs = O.window_offsets(L, Lw)
    peak = offs[np.argmax(st.w, axis=1)] % L
    np.testing.assert_array_equal(peak, r)
    assert np.all(r[:6] == L - 2) and np.all(r[6:] == 0)
    del xbar


# --------------------------------------------------------------------------- synchronization pieces
def test_relative_rotation_matches_fft_cross_correlation():
    rng = np.random.default_rng(6)
    for trial in range(5):
        K, Q, L = 5, 3, 30
        vi = rng.standard_normal((K + 1, Q)) + 1j * rng.standard_normal((K + 1, Q))
        vj = rng.standard_normal((K + 1, Q)) + 1j * rng.standard_normal((K + 1, Q))
        C = np.sum(np.conj(vi) * vj, axis=1)  # C_k
        cp = np.zeros(L, dtype=np.complex128)
        cp[:K + 1] = C
        score = L * np.fft.ifft(cp).real  # Re sum_k C_k e^{+2 pi i k l / L}
        assert O.relative_rotation(vi, vj, L) == int(np.argmax(score))


def test_power_iteration_matches_eigh():
    rng = np.random.default_rng(8)
    P, L = 30, 64
    th = rng.integers(0, L, P)
    rel = (th[None, :] - th[:, None]) % L  # exact theta_j - theta_i
    noise = rng.random((P, P)) < 0.2
    rnd = rng.integers(0, L, (P, P))
    rel = np.where(noise, rnd, rel)
    rel = np.triu(rel, 1)
    rel = (rel - rel.T) % L
    H = O.sync_matrix(rel, L)
    z = O.power_iteration(H, 500)
    evals, evecs = np.linalg.eigh(H)
    u = evecs[:, -1]
    assert abs(abs(np.vdot(u, z)) - 1.0) < 1e-10
    # and the leading eigenvector carries the rotations: phases of e^{i theta}
    phi = O.ppm(rel, L, 50, 100)
    d = (phi - th) % L
    dev = (d - d[0] + L // 2) % L - L // 2  # circular deviation from one image's offset
    assert np.max(np.abs(dev)) <= 4
    wrong = (phi + th) % L  # the opposite sign convention would scatter over the circle
    devw = (wrong - wrong[0] + L // 2) % L - L // 2
    assert np.max(np.abs(devw)) > 8


def test_match_excludes_self_and_picks_nearest():
    rng = np.random.default_rng(2)
    y = rng.standard_normal((10, 3, 2)) + 1j * rng.standard_normal((10, 3, 2))
    y[7] = y[2] + 1e-3
    y[1] = y[4] + 1e-3
    phi = np.arange(5) * 10
    s = O.match(y, 5, phi)
    assert s[7] == phi[2] and s[1] == phi[4] and s[4] == phi[1]
    for i in range(10):
        cands = [n for n in range(5) if n != i]
        dd = [np.sum(np.abs(y[i] - y[n]) ** 2) for n in cands]
        assert s[i] == phi[cands[int(np.argmin(dd))]]


# --------------------------------------------------------------------------- von Mises prior fit
def test_von_mises_fit_recovers_kappa():
    rng = np.random.default_rng(12)
    L, kappa = 360, 40.0
    th = rng.vonmises(0.0, kappa, 400_000)
    r = np.floor(np.mod(th, 2 * np.pi) * L / (2 * np.pi) + 0.5).astype(int) % L
    counts = np.bincount(r, minlength=L)
    lp, k_hat = O.fit_prior(counts, L, 72, kind=1)
    assert abs(k_hat - kappa) / kappa < 0.02
    assert abs(np.sum(np.exp(lp)) - 1.0) < 1e-12


def test_vm_ratio_series():
    """A(kappa) against the power series of I_1 and I_0."""
    for k in (0.1, 1.0, 5.0, 20.0):
        i0 = sum((k / 2) ** (2 * m) / math.factorial(m) ** 2 for m in range(80))
        i1 = sum((k / 2) ** (2 * m + 1) / (math.factorial(m) * math.factorial(m + 1)) for m in range(80))
        assert abs(O.vm_ratio(k) - i1 / i0) < 1e-13


# --------------------------------------------------------------------------- gradient
def test_loglik_gradient_central_differences():
    inst = synth.make_instance(K=3, Q=2, N=25, L=20, sigma2=soft(0.5, 3, 2), decay=6.0, seed=17)
    L, Lw = inst.L, 7
    rng = np.random.default_rng(1)
    x = synth.random_init(inst.K, inst.Q, 6.0, seed=3)
    eta = 0.3 * rng.standard_normal(Lw)
    kappa = 2.5
    ll, dx, de, dk = O.loglik_grad(inst.y, x, eta, kappa, L, inst.sigma2)
    h = 1e-6
    for k in range(inst.K + 1):
        for q in range(inst.Q):
            for part, unit in ((0, 1.0), (1, 1j)):
                e = np.zeros_like(x)
                e[k, q] = unit * h
                g = (O.loglik(inst.y, x + e, eta, kappa, L, inst.sigma2)
                     - O.loglik(inst.y, x - e, eta, kappa, L, inst.sigma2)) / (2 * h)
                an = dx[k, q].real if part == 0 else dx[k, q].imag
                assert abs(g - an) <= 1e-6 * max(1.0, abs(an))
    for l in range(Lw):
        e = np.zeros(Lw)
        e[l] = h
        g = (O.loglik(inst.y, x, eta + e, kappa, L, inst.sigma2) - O.loglik(inst.y, x, eta - e, kappa, L, inst.sigma2)) / (2 * h)
        assert abs(g - de[l]) <= 1e-6 * max(1.0, abs(de[l]))
    g = (O.loglik(inst.y, x, eta, kappa + h, L, inst.sigma2) - O.loglik(inst.y, x, eta, kappa - h, L, inst.sigma2)) / (2 * h)
    assert abs(g - dk) <= 1e-6 * max(1.0, abs(dk))
    assert abs(np.sum(de)) < 1e-9  # the logits are defined up to a constant


# --------------------------------------------------------------------------- relative error and step
def test_relerr_continuous_rotation_and_scale():
    x = synth.make_signal(8, 5, 20.0, np.random.default_rng(4))
    assert O.relerr(O.rotate(x, 1.2345), x) < 1e-9
    assert abs(O.relerr(1.1 * O.rotate(x, -0.77), x) - 0.1) < 1e-9
    # k>0 rows count twice: perturbing only row k=1 by d gives sqrt(2|d|^2)/||I||
    y = x.copy()
    y[0, 0] += 0.01  # a real k=0 perturbation cannot be rotated away
    wnorm = math.sqrt(np.sum(np.abs(x[0]) ** 2) + 2 * np.sum(np.abs(x[1:]) ** 2))
    assert O.relerr(y, x) <= 0.01 / wnorm + 1e-12


def test_step_is_zero_for_grid_rotation():
    x = synth.make_signal(5, 3, 20.0, np.random.default_rng(5))
    L = 40
    assert O.step_size(O.rotate(x, 2 * np.pi * 13 / L), x, L) < 1e-26
    assert O.step_size(x + 0.1, x, L) > 0


# --------------------------------------------------------------------------- denser-resolution window (Sec. 3.3)
@pytest.mark.parametrize("m", [2, 3, 4])
def test_dense_window_on_grid_points_equals_grid_window(m):
    """A window of step 1/m whose prior is zero off the grid points is the grid window:
    same weights there (zero elsewhere), same a_{t+1}, likelihood and rho_{t+1}."""
    inst = synth.make_instance(K=4, Q=3, N=40, L=30, sigma2=soft(0.4, 4, 3), decay=6.0, seed=31)
    L, sigma2 = inst.L, inst.sigma2
    Lw, l0 = 7, -3
    rng = np.random.default_rng(8)
    x = synth.make_signal(inst.K, inst.Q, 6.0, np.random.default_rng(6))
    rho = rng.random(Lw) + 0.2
    rho /= rho.sum()
    rb = rng.random(Lw) + 0.1
    rb /= rb.sum()
    g = O.em_step(inst.y, x, np.log(rho), L, sigma2, Lw=Lw, l0=l0, gamma=3.0, log_rho_bar=np.log(rb),
                  shifts=inst.s)
    Lwd = m * (Lw - 1) + 1
    lrd = np.full(Lwd, -np.inf)
    lrd[::m] = np.log(rho)
    lrbd = np.full(Lwd, -np.inf)
    lrbd[::m] = np.log(rb)
    d = O.em_step(inst.y, x, lrd, L, sigma2, Lw=Lwd, l0=m * l0, gamma=3.0, log_rho_bar=lrbd, shifts=inst.s,
                  step=1.0 / m)
    tol = 1e-12
    np.testing.assert_allclose(d.w[:, ::m], g.w, atol=tol)
    off = np.ones(Lwd, dtype=bool)
    off[::m] = False
    assert np.all(d.w[:, off] == 0.0)
    assert np.max(np.abs(d.x - g.x)) <= tol * np.max(np.abs(g.x))
    assert abs(d.loglik - g.loglik) <= tol * abs(g.loglik)
    np.testing.assert_allclose(np.exp(d.log_rho[::m]), np.exp(g.log_rho), atol=tol)
    assert abs(d.step - g.step) <= tol * max(1.0, g.step)


def test_dense_window_noise_free_recovers_off_grid_rotations():
    """Images rotated by off-grid angles of the window and nearly noise free: each posterior is one-hot at its
    angle and the M-step returns the signal (the rotation is undone exactly at non-grid angles)."""
    K, Q, L, N = 6, 4, 36, 30
    Lw, l0, step = 21, -10, 0.3
    rng = np.random.default_rng(13)
    x = synth.make_signal(K, Q, 8.0, np.random.default_rng(14))
    idx = rng.integers(0, Lw, N)
    ang = 2 * math.pi * step * (l0 + idx) / L
    y = np.stack([x * np.exp(-1j * np.arange(K + 1) * a)[:, None] for a in ang])
    sigma2 = 1e-5 * float(np.sum(np.abs(x) ** 2))
    st = O.em_step(y, x, np.log(np.full(Lw, 1.0 / Lw)), L, sigma2, Lw=Lw, l0=l0, step=step)
    np.testing.assert_allclose(st.w, np.eye(Lw)[idx], atol=1e-12)
    assert np.max(np.abs(st.x - x)) < 1e-12 * np.max(np.abs(x))
    np.testing.assert_allclose(st.W, np.bincount(idx, minlength=Lw), atol=1e-10)


@pytest.mark.parametrize("kappa,l0", [(0.7, 0), (3.0, -80), (9.0, 17)])
def test_dense_von_mises_normaliser_is_bessel(kappa, l0):
    """n equally spaced angles around the whole circle (Lw step = L): sum exp(kappa cos theta) = n I0(kappa) up to
    aliasing terms 2 n I_n(kappa), below 1e-100 here; the window prior is kappa cos theta - log(n I0(kappa))."""
    from scipy import special

    L, step = 40, 0.25
    n = int(L / step)
    lr = O.vm_log_rho(np.zeros(n), kappa, L, l0=l0, step=step)
    th = 2 * math.pi * step * (l0 + np.arange(n)) / L
    np.testing.assert_allclose(lr, kappa * np.cos(th) - math.log(n * special.i0(kappa)), atol=1e-12)


def test_dense_histogram_prior_takes_nearest_grid_bin():
    """Counts 3 : 1 in bins 0 and 1 of L = 12; window positions -2 .. 2 grid units at step 1/4.
    floor(u + 1/2) puts [-1/2, 1/2) in bin 0 and [1/2, 3/2) in bin 1: four positions each, the
    others empty, so the window prior is 3/16 on the first four and 1/16 on the next four."""
    counts = np.zeros(12, dtype=np.int64)
    counts[0], counts[1] = 3, 1
    lp, _ = O.fit_prior(counts, 12, 17, l0=-8, kind=0, step=0.25)
    want = np.zeros(17)
    want[6:10] = 3 / 16   # u = -0.5, -0.25, 0, 0.25
    want[10:14] = 1 / 16  # u = 0.5, 0.75, 1, 1.25
    np.testing.assert_allclose(np.exp(lp), want, atol=1e-15)
    # step 1 reads the grid bins themselves
    lp1, _ = O.fit_prior(counts, 12, 5, l0=-2, kind=0)
    np.testing.assert_allclose(np.exp(lp1), [0, 0, 0.75, 0.25, 0], atol=1e-15)


def test_dense_loglik_gradient_central_differences():
    inst = synth.make_instance(K=3, Q=2, N=20, L=24, sigma2=soft(0.5, 3, 2), decay=6.0, seed=19)
    L, Lw, l0, step = inst.L, 9, -4, 0.6
    rng = np.random.default_rng(2)
    x = synth.random_init(inst.K, inst.Q, 6.0, seed=5)
    eta = 0.3 * rng.standard_normal(Lw)
    kappa = 1.5
    kw = dict(l0=l0, step=step)
    ll, dx, de, dk = O.loglik_grad(inst.y, x, eta, kappa, L, inst.sigma2, **kw)
    h = 1e-6
    for k in range(inst.K + 1):
        for q in range(inst.Q):
            for part, unit in ((0, 1.0), (1, 1j)):
                e = np.zeros_like(x)
                e[k, q] = unit * h
                g = (O.loglik(inst.y, x + e, eta, kappa, L, inst.sigma2, **kw)
                     - O.loglik(inst.y, x - e, eta, kappa, L, inst.sigma2, **kw)) / (2 * h)
                an = dx[k, q].real if part == 0 else dx[k, q].imag
                assert abs(g - an) <= 1e-6 * max(1.0, abs(an))
    g = (O.loglik(inst.y, x, eta, kappa + h, L, inst.sigma2, **kw)
         - O.loglik(inst.y, x, eta, kappa - h, L, inst.sigma2, **kw)) / (2 * h)
    assert abs(g - dk) <= 1e-6 * max(1.0, abs(dk))


# --------------------------------------------------------------------------- template matching, 1-D MRA, App. B
def test_template_match_noise_free_and_sign():
    """Images that are the reference rotated by s_j come back with s_j (the sign of the relative rotation)."""
    K, Q, L = 6, 3, 40
    ref = synth.make_signal(K, Q, 20.0, np.random.default_rng(21))
    s = np.random.default_rng(22).integers(0, L, 25)
    y = np.stack([O.rotate(ref, 2 * np.pi * sj / L) for sj in s])
    np.testing.assert_array_equal(O.template_match(y, ref, L), s)


def test_1d_coefficient_form_preserves_distances_and_shifts():
    """Parseval in the coefficient form of synth.mra1d: ||roll(x, s) - v||^2 in signal space equals the stored-entry
    distance after rotating the coefficients by 2 pi s / L, for every s."""
    rng = np.random.default_rng(5)
    L = 21
    x, v = rng.standard_normal(L), rng.standard_normal(L)
    ax, av = synth.coeffs_1d(x), synth.coeffs_1d(v)
    for s in range(L):
        d_sig = float(np.sum((np.roll(x, s) - v) ** 2))
        diff = O.rotate(ax, 2 * np.pi * s / L) - av
        assert abs(d_sig - float(np.sum(np.abs(diff) ** 2))) < 1e-10 * max(1.0, d_sig)
    np.testing.assert_allclose(synth.signal_1d(ax, L), x, atol=1e-13)


def test_template_match_1d_against_signal_space_brute_force():
    """Template matching in the coefficient form equals argmin_l ||ref - roll(v_j, -l)||^2 in signal space."""
    inst = synth.make_instance_1d(21, 200, 1.5, seed=9)
    ref = inst.v[0]
    want = np.array([int(np.argmin([np.sum((ref - np.roll(vj, -l)) ** 2) for l in range(21)])) for vj in inst.v])
    got = O.template_match(synth.coeffs_1d(inst.v), synth.coeffs_1d(ref), 21)
    np.testing.assert_array_equal(got, want)


def test_1d_em_step_in_coefficient_form_equals_signal_space_em():
    """One EM step of the 1-D model written in signal space (posterior over all L cyclic shifts with
    exp(-||v_j - roll(x, l)||^2 / (2 sigma^2)), x_new = mean_j sum_l w_jl roll(v_j, -l), rho_new = mean_j w_j)
    against the oracle's EM step on the coefficient form with sigma2 = 2 sigma^2 (whole grid, l0 = 0)."""
    L, N, sigma = 15, 60, 0.9
    inst = synth.make_instance_1d(L, N, sigma, seed=41)
    x0 = np.random.default_rng(42).standard_normal(L)
    rho = np.random.default_rng(43).random(L) + 0.3
    rho /= rho.sum()
    # signal space, written out
    logw = np.empty((N, L))
    for j in range(N):
        for l in range(L):
            logw[j, l] = np.log(rho[l]) - np.sum((inst.v[j] - np.roll(x0, l)) ** 2) / (2 * sigma ** 2)
    w = np.exp(logw - logw.max(axis=1, keepdims=True))
    w /= w.sum(axis=1, keepdims=True)
    x_new = np.zeros(L)
    for j in range(N):
        for l in range(L):
            x_new += w[j, l] * np.roll(inst.v[j], -l)
    x_new /= N
    rho_new = w.mean(axis=0)
    # coefficient form through the oracle
    st = O.em_step(synth.coeffs_1d(inst.v), synth.coeffs_1d(x0), np.log(rho), L, synth.sigma2_coeff(sigma),
                   Lw=L, l0=0)
    np.testing.assert_allclose(st.w, w, atol=1e-12)
    np.testing.assert_allclose(synth.signal_1d(st.x, L), x_new, atol=1e-12)
    np.testing.assert_allclose(np.exp(st.log_rho), rho_new, atol=1e-12)


def test_tm_shift_pmf_two_point_closed_form():
    """L = 2: p[0] = P(A_0 > A_1) = Phi((R[0] - R[1]) / (sqrt 2 sigma_c)) for the independent model."""
    from scipy import stats

    x = np.array([1.3, -0.4])
    sigma = 0.8
    R0, R1 = float(x @ x), 2 * x[0] * x[1]
    sc = sigma * np.linalg.norm(x)
    p = O.tm_shift_pmf(x, sigma)
    assert abs(p[0] - stats.norm.cdf((R0 - R1) / (np.sqrt(2) * sc))) < 1e-9
    assert abs(p.sum() - 1.0) < 1e-9


def test_tm_shift_pmf_against_monte_carlo_of_its_model():
    """The pmf integral against argmax frequencies of independent N(R_xx[l], sigma_c^2) draws (the model App. B
    integrates), and its symmetry p[m] = p[L - m]."""
    rng = np.random.default_rng(31)
    L, sigma = 21, 3.0
    x = rng.standard_normal(L)
    p = O.tm_shift_pmf(x, sigma)
    R = np.array([np.dot(x, np.roll(x, -l)) for l in range(L)])
    sc = sigma * np.linalg.norm(x)
    n = 400_000
    A = R[None, :] + sc * rng.standard_normal((n, L))
    freq = np.bincount(np.argmax(A, axis=1), minlength=L) / n
    assert np.all(np.abs(freq - p) <= 5 * np.sqrt(p * (1 - p) / n) + 1e-6), np.abs(freq - p).max()
    np.testing.assert_allclose(p[1:], p[1:][::-1], atol=1e-9)
    assert abs(p.sum() - 1.0) < 1e-9


# --------------------------------------------------------------------------- Fourier-Bessel front end (App. A)
@pytest.mark.parametrize("k,q", [(0, 1), (0, 7), (3, 2), (12, 5), (30, 20)])
def test_fb_normalisation_closed_form(k, q):
    """N_{k,q} makes the continuous basis function unit-norm on the disk: 2 pi int_0^c N^2 J_k(R r/c)^2 r dr = 1
    (equivalently c^2 J_{k+1}(R)^2 / 2 = int_0^c J_k(R r/c)^2 r dr, the Lommel integral at a zero)."""
    from scipy import integrate, special

    c = 64.0
    R = special.jn_zeros(k, q)[-1]
    Nkq = 1.0 / (c * math.sqrt(math.pi) * abs(special.jv(k + 1, R)))
    val = 2 * math.pi * integrate.quad(lambda r: (Nkq * special.jv(k, R * r / c)) ** 2 * r, 0, c, limit=400)[0]
    assert abs(val - 1.0) < 1e-9


def test_fb_project_recovers_rendered_coefficients():
    """Images rendered by the data generator (its own evaluation of the basis) come back through the oracle's least
    squares: the two implementations of App. A's basis agree."""
    K, Q, n = 6, 5, 41
    a = np.stack([synth.make_signal(K, Q, 10.0, np.random.default_rng(s)) for s in range(3)])
    img = synth.render(a, n)
    np.testing.assert_allclose(O.fb_project(img, K, Q), a, atol=1e-11)


def test_fb_rotation_by_quarter_turn():
    """Steerability on the pixel grid: the image rotated by pi/2, I'(x, y) = I(y, -x), i.e. I'[iy][ix] =
    I[n-1-ix][iy], has the coefficients a_k e^{-i k pi/2} (Eq. fb_rotation)."""
    K, Q, n = 8, 4, 33
    a = synth.make_signal(K, Q, 20.0, np.random.default_rng(3))
    img = synth.render(a[None], n)[0]
    iy, ix = np.mgrid[0:n, 0:n]
    rot = img[n - 1 - ix, iy]
    want = a * np.exp(-1j * np.arange(K + 1) * np.pi / 2)[:, None]
    np.testing.assert_allclose(O.fb_project(rot[None], K, Q)[0], want, atol=1e-11)


def test_fb_pixel_noise_is_nearly_white_in_coefficients():
    """White pixel noise of variance s^2 gives coefficients of variance ~ s^2 per stored complex entry (the discrete
    basis is nearly orthonormal; App. A): within 3% on average and 10% per entry over 4000 draws."""
    K, Q, n, s = 4, 4, 41, 1.0
    noise = np.random.default_rng(8).standard_normal((4000, n, n)) * s
    v = np.mean(np.abs(O.fb_project(noise, K, Q)) ** 2, axis=0)
    assert abs(v.mean() - s ** 2) < 0.03
    assert np.all(np.abs(v - s ** 2) < 0.1)


# --------------------------------------------------------------------------- steerable PCA (App. A)
def _lowrank(N, K, Q, r, var, sigma2, seed):
    """a_ik = sum_{j<r} z_ikj u_kj + noise with known orthonormal u_k [Q, r] and E|z|^2 = var[j]."""
    rng = np.random.default_rng(seed)
    U = []
    a = np.zeros((N, K + 1, Q), dtype=np.complex128)
    for k in range(K + 1):
        M = rng.standard_normal((Q, r)) + 1j * rng.standard_normal((Q, r))
        Uk, _ = np.linalg.qr(M)
        U.append(Uk)
        z = (rng.standard_normal((N, r)) + 1j * rng.standard_normal((N, r))) * np.sqrt(np.asarray(var) / 2)
        a[:, k, :] = z @ Uk.T
    a += (rng.standard_normal(a.shape) + 1j * rng.standard_normal(a.shape)) * math.sqrt(sigma2 / 2)
    return a, U


def test_spca_recovers_known_low_rank_subspaces():
    """Rank 2 per k with variances 5 and 2 over unit noise: two components kept at every k, their span is the true
    one (principal angles below 0.05), eigenvalues var + sigma^2 within 5%, U^H U = I, max entries real positive."""
    N, K, Q = 20000, 4, 10
    a, U = _lowrank(N, K, Q, 2, [5.0, 2.0], 1.0, seed=41)
    f = O.spca_fit(a, 1.0)
    np.testing.assert_array_equal(f.counts, 2)
    assert (f.K2, f.Q2) == (K, 2)
    for k in range(K + 1):
        B = f.bases[k]
        s = np.linalg.svd(B.conj().T @ U[k], compute_uv=False)
        assert np.all(s > np.cos(0.05))
        np.testing.assert_allclose(f.eigs[k][:2], [6.0, 3.0], rtol=0.05)
        np.testing.assert_allclose(B.conj().T @ B, np.eye(2), atol=1e-12)
        for j in range(2):
            i = int(np.argmax(np.abs(B[:, j])))
            assert abs(B[i, j].imag) < 1e-12 and B[i, j].real > 0


def test_spca_is_steerable_and_scalar_case():
    """Rotating every image (a_ik e^{-i k theta_i}) leaves each C_k unchanged, so b rotates the same way; with Q = 1
    the basis is [1] and b = a wherever mean |a_k|^2 exceeds sigma^2 (1 + 1/sqrt N)^2."""
    N, K, Q = 3000, 5, 6
    a, _ = _lowrank(N, K, Q, 1, [4.0], 0.5, seed=42)
    th = np.random.default_rng(43).uniform(0, 2 * np.pi, N)
    ph = np.exp(-1j * np.outer(th, np.arange(K + 1)))[:, :, None]
    f, fr = O.spca_fit(a, 0.5), O.spca_fit(a * ph, 0.5)
    b, br = O.spca_project(a, f), O.spca_project(a * ph, fr)
    np.testing.assert_allclose(br, b * ph[:, : f.K2 + 1], atol=1e-10)
    a1 = a[:, :, :1]
    f1 = O.spca_fit(a1, 0.5)
    keep = np.mean(np.abs(a1[:, :, 0]) ** 2, axis=0) > 0.5 * (1 + 1 / math.sqrt(N)) ** 2
    np.testing.assert_array_equal(f1.counts, keep.astype(int))
    b1 = O.spca_project(a1, f1)
    np.testing.assert_allclose(b1[:, :, 0], a1[:, : f1.K2 + 1, 0] * keep[None, : f1.K2 + 1], atol=1e-13)
