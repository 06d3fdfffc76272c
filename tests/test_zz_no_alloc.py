"""mra_em_step_noalloc: the EM step for callers that cannot allocate device memory.

Some callers cannot give the library a workspace: their device memory is owned
by another component that has no spare buffer to lend, or they must avoid
cudaMalloc/cudaFree because those calls can synchronize the whole device.  For
them the library keeps one fixed 8 MiB scratch array in device memory.  This
test calls that entry point through the C ABI twice in a row and checks each
result against mra_em_step with an ordinary workspace, within the tolerances
the other parity tests use.  It lives in a file of its own, collected last.
"""
import numpy as np
import pytest
import torch

import synth
from gpu_helpers import TOL_W, TOL_X, dev, dev_y, host, rel_err

pytestmark = pytest.mark.gpu


def _outputs(d, Lw, N, K, Q):
    return (torch.empty((K + 1, Q), dtype=torch.complex128, device="cuda"),
            torch.empty(Lw, dtype=torch.float64, device="cuda"),
            torch.empty(1, dtype=torch.float64, device="cuda"),
            torch.empty(1, dtype=torch.float64, device="cuda"),
            torch.empty((N, Lw), dtype=torch.float32, device="cuda"))


def test_noalloc_step_matches_workspace_step_twice(gpu_lib):
    mra = gpu_lib
    c = synth.config(2)
    inst = synth.make_instance(c["K"], c["Q"], 6000, c["L"], c["snr"], c["decay"], seed=5001)
    Lw = c["Lw"]
    d = mra.dims(inst.N, inst.K, inst.Q, inst.L, inst.sigma2)
    assert mra.mra_em_workspace_bytes(d, Lw) <= 8 << 20
    y = dev_y(inst.y)
    sh = dev(inst.s.astype(np.int32))
    prm = mra.em_params(Lw)
    x = dev(inst.x)
    lr = torch.full((Lw,), -np.log(Lw), dtype=torch.float64, device="cuda")
    ws = mra.workspace(mra.mra_em_workspace_bytes(d, Lw))
    for call in range(2):  # the second call starts from the first call's result
        ref = _outputs(d, Lw, inst.N, inst.K, inst.Q)
        got = _outputs(d, Lw, inst.N, inst.K, inst.Q)
        mra.mra_em_step(d, prm, y, sh, x, lr, *ref, ws=ws)
        mra.mra_em_step_noalloc(d, prm, y, sh, x, lr, *got)
        torch.cuda.synchronize()
        assert rel_err(host(got[0]), host(ref[0])) <= TOL_X, call
        np.testing.assert_allclose(np.exp(host(got[1])), np.exp(host(ref[1])), atol=TOL_W, rtol=0)
        assert np.max(np.abs(host(got[4]) - host(ref[4]))) <= TOL_W, call
        assert abs(got[2].item() - ref[2].item()) <= 1e-9 * abs(ref[2].item())
        assert abs(got[3].item() - ref[3].item()) <= 1e-9 * abs(ref[3].item()) + 1e-15
        assert mra.mra_em_step_noalloc_status() == 0, call
        x, lr = ref[0], ref[1]


def _compare_once(mra, inst, Lw, L):
    d = mra.dims(inst.N, inst.K, inst.Q, L, inst.sigma2)
    prm = mra.em_params(Lw)
    y = dev_y(inst.y)
    sh = dev(inst.s.astype(np.int32))
    x = dev(inst.x)
    lr = torch.full((Lw,), -np.log(Lw), dtype=torch.float64, device="cuda")
    ws = mra.workspace(mra.mra_em_workspace_bytes(d, Lw))  # a fresh workspace for the reference step
    ref = _outputs(d, Lw, inst.N, inst.K, inst.Q)
    got = _outputs(d, Lw, inst.N, inst.K, inst.Q)
    mra.mra_em_step(d, prm, y, sh, x, lr, *ref, ws=ws)
    mra.mra_em_step_noalloc(d, prm, y, sh, x, lr, *got)
    assert mra.mra_em_step_noalloc_status() == 0  # synchronizes; MRA_OK: no wait ran out
    assert rel_err(host(got[0]), host(ref[0])) <= TOL_X
    np.testing.assert_allclose(np.exp(host(got[1])), np.exp(host(ref[1])), atol=TOL_W, rtol=0)
    assert np.max(np.abs(host(got[4]) - host(ref[4]))) <= TOL_W
    assert abs(got[2].item() - ref[2].item()) <= 1e-9 * abs(ref[2].item())


def test_noalloc_larger_then_smaller_problem(gpu_lib):
    """A problem whose scratch fills most of the array, then a smaller one of other K, Q, L and
    window: the second call must not see the first call's partial sums, tables or norms."""
    mra = gpu_lib
    big = synth.make_instance(40, 32, 3000, 720, 1 / 50, 50.0, seed=5002)
    d_big = mra.dims(big.N, big.K, big.Q, big.L, big.sigma2)
    nb = mra.mra_em_workspace_bytes(d_big, 60)
    assert (6 << 20) <= nb <= (8 << 20), nb
    _compare_once(mra, big, 60, big.L)
    c = synth.config(1)
    small = synth.make_instance(c["K"], c["Q"], 700, c["L"], c["snr"], c["decay"], seed=5003)
    _compare_once(mra, small, c["Lw"], small.L)


def test_noalloc_rejects_problems_beyond_its_scratch(gpu_lib):
    mra = gpu_lib
    d = mra.dims(1000, 63, 64, 720, 0.1)  # 4096 coefficients: partials alone exceed 8 MiB
    assert mra.mra_em_workspace_bytes(d, 720) > 8 << 20
    y = torch.zeros((1000, 64, 64), dtype=torch.complex64, device="cuda")
    x = torch.zeros((64, 64), dtype=torch.complex128, device="cuda")
    lr = torch.zeros(720, dtype=torch.float64, device="cuda")
    with pytest.raises(mra.MraError) as e:
        mra.mra_em_step_noalloc(d, mra.em_params(720), y, None, x, lr, x, lr)
    assert e.value.status == -6
