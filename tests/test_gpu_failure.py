"""Device-side failure detection without a GPU fault: a bounded mbarrier wait on a
barrier nothing arrives on gives up after its limit and reports MRA_ETIMEOUT, and
the context stays usable (an EM step afterwards still matches the oracle)."""
import time

import numpy as np
import pytest
import torch

import oracle as O
import synth
from gpu_helpers import TOL_X, dev, dev_y, host, rel_err

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives(gpu_lib):
    mra = gpu_lib
    st = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    t0 = time.perf_counter()
    mra.mra_selftest_wait_timeout(20_000, st)  # 20 ms
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    assert st.item() == -4  # MRA_ETIMEOUT
    assert 0.015 <= dt < 5.0, dt
    # the context is intact: an ordinary step runs and matches the oracle
    inst = synth.make_instance(4, 8, 200, 24, sigma2=1 / (0.3 * 40), decay=20.0, seed=91)
    y64 = synth.c64_round(inst.y)
    Lw = 7
    d = mra.dims(inst.N, inst.K, inst.Q, inst.L, inst.sigma2)
    x0 = O.align_mean(y64, inst.s, inst.L)
    lr = np.log(np.full(Lw, 1.0 / Lw))
    xo = torch.empty((inst.K + 1, inst.Q), dtype=torch.complex128, device="cuda")
    lro = torch.empty(Lw, dtype=torch.float64, device="cuda")
    ws = mra.workspace(mra.mra_em_workspace_bytes(d, Lw))
    mra.mra_em_step(d, mra.em_params(Lw), dev_y(y64), dev(inst.s.astype(np.int32)), dev(x0), dev(lr), xo, lro,
                    ws=ws)
    torch.cuda.synchronize()
    assert mra.mra_ws_status(ws) == 0
    ref = O.em_step(y64, x0, lr, inst.L, inst.sigma2, Lw=Lw, shifts=inst.s)
    assert rel_err(host(xo), ref.x) <= TOL_X


def test_selftest_rejects_bad_limits(gpu_lib):
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(gpu_lib.MraError):
        gpu_lib.mra_selftest_wait_timeout(0, st)


def test_grid_barrier_times_out_and_batched_run_still_works(gpu_lib):
    """The persistent batched kernel's grid barrier: one CTA never arrives, every waiting CTA gives up
    after the limit and reports MRA_ETIMEOUT; a persistent batched run afterwards matches the oracle."""
    mra = gpu_lib
    scratch = torch.full((4,), 7, dtype=torch.int32, device="cuda")
    t0 = time.perf_counter()
    mra.mra_selftest_grid_barrier(20_000, scratch)  # 20 ms
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    assert int(scratch[2].item()) == -4  # MRA_ETIMEOUT
    assert 0.015 <= dt < 5.0, dt
    T = 2
    inst = synth.make_instance(12, 16, 700, 60, sigma2=1 / (0.3 * 13 * 16), decay=20.0, seed=93)
    y64 = synth.c64_round(inst.y)
    Lw = 11
    d = mra.dims(inst.N, inst.K, inst.Q, inst.L, inst.sigma2)
    x0 = O.align_mean(y64, inst.s, inst.L)
    lr = np.log(np.full(Lw, 1.0 / Lw))
    it = dict(d=d, prm=mra.em_params(Lw, max_iters=T), y=dev_y(y64), shift=dev(inst.s.astype(np.int32)),
              x=dev(x0), log_rho=dev(lr))
    arr = mra.instances([it])
    ws = mra.workspace(mra.mra_em_batched_workspace_bytes(arr))
    iters, _ = mra.mra_em_run_batched(arr, ws, tune=False)
    assert iters == [T]
    xs, lrs = x0, lr
    for _ in range(T):
        st = O.em_step(y64, xs, lrs, inst.L, inst.sigma2, Lw=Lw, shifts=inst.s)
        xs, lrs = st.x, st.log_rho
    assert rel_err(host(it["x"]), xs) <= TOL_X * T


def test_grid_barrier_selftest_rejects_bad_limits(gpu_lib):
    scratch = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(gpu_lib.MraError):
        gpu_lib.mra_selftest_grid_barrier(0, scratch)
