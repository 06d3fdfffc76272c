"""Many independent problems in one graph launch (mra_em_run_batched) and the sweep
autotuner (mra_em_autotune).  Each instance of a batched run must match the same
instance run alone through mra_em_run (same cached sweep choice; a batched run gives
a small instance fewer CTAs, so FP32 partial sums are combined in another order and
agreement is to 1e-6 rather than bit for bit), and follow the FP64 oracle's EM
trajectory within the per-iteration tolerance."""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from gpu_helpers import TOL_X, dev, dev_y, host, rel_err

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]
TOL_SAME = 1e-6  # batched against single runs: another FP32 summation order, no other difference

# uneven shapes: rows of 16, 8, 24 and 6 coefficients (the last has no batch sweep),
# windows narrow, wide and the whole grid, with and without alignment shifts
SHAPES = [
    dict(K=12, Q=16, N=1300, L=90, Lw=13, shifts=True),
    dict(K=3, Q=8, N=257, L=36, Lw=36, shifts=False),
    dict(K=20, Q=16, N=700, L=120, Lw=45, shifts=True),
    dict(K=8, Q=24, N=999, L=60, Lw=5, shifts=True),
    dict(K=5, Q=6, N=400, L=40, Lw=9, shifts=True),
    dict(K=30, Q=16, N=150, L=72, Lw=72, shifts=False),
]


def _problem(mra, sh, i, T):
    inst = synth.make_instance(sh["K"], sh["Q"], sh["N"], sh["L"], sigma2=1 / (0.5 * (sh["K"] + 1) * sh["Q"]),
                               decay=30.0, seed=7000 + i)
    y64 = synth.c64_round(inst.y)
    Lw = sh["Lw"]
    l0 = 0 if Lw == inst.L else None
    s = inst.s if sh["shifts"] else None
    x0 = O.align_mean(y64, s, inst.L) if s is not None else synth.random_init(inst.K, inst.Q, 30.0, seed=i)
    lr = np.log(np.full(Lw, 1.0 / Lw))
    d = mra.dims(inst.N, inst.K, inst.Q, inst.L, inst.sigma2)
    prm = mra.em_params(Lw, l0=l0, max_iters=T)
    return dict(inst=inst, y64=y64, s=s, x0=x0, lr=lr, d=d, prm=prm, Lw=Lw, l0=l0)


def test_batched_run_equals_single_runs_and_oracle(gpu_lib):
    mra = gpu_lib
    T = 3
    probs = [_problem(mra, sh, i, T) for i, sh in enumerate(SHAPES)]
    items = []
    for p in probs:
        items.append(dict(d=p["d"], prm=p["prm"], y=dev_y(p["y64"]), x=dev(p["x0"]), log_rho=dev(p["lr"]),
                          shift=dev(p["s"].astype(np.int32)) if p["s"] is not None else None,
                          stats=torch.empty((T, 2), dtype=torch.float64, device="cuda")))
    arr = mra.instances(items)
    ws = mra.workspace(mra.mra_em_batched_workspace_bytes(arr))
    iters, ms = mra.mra_em_run_batched(arr, ws, tune=True)
    assert iters == [T] * len(SHAPES) and ms > 0
    for p, it in zip(probs, items):
        # alone, through mra_em_run, from the same start
        x1, lr1 = dev(p["x0"]), dev(p["lr"])
        ws1 = mra.workspace(mra.mra_em_workspace_bytes(p["d"], p["Lw"]))
        st1 = torch.empty((T, 2), dtype=torch.float64, device="cuda")
        assert mra.mra_em_run(p["d"], p["prm"], it["y"], it["shift"], x1, lr1, st1, None, ws1) == T
        assert rel_err(host(it["x"]), host(x1)) <= TOL_SAME
        np.testing.assert_allclose(np.exp(host(it["log_rho"])), np.exp(host(lr1)), rtol=0, atol=TOL_SAME)
        np.testing.assert_allclose(host(it["stats"])[:, 0], host(st1)[:, 0], rtol=TOL_SAME)
        # the oracle's trajectory
        xs, lrs = p["x0"], p["lr"]
        for t in range(T):
            st = O.em_step(p["y64"], xs, lrs, p["inst"].L, p["inst"].sigma2, Lw=p["Lw"], l0=p["l0"], shifts=p["s"])
            xs, lrs = st.x, st.log_rho
        assert rel_err(host(it["x"]), xs) <= TOL_X * T, rel_err(host(it["x"]), xs)


def test_autotune_picks_a_valid_sweep_and_keeps_parity(gpu_lib):
    mra = gpu_lib
    c = synth.config(2)
    inst = synth.make_instance(c["K"], c["Q"], 3000, c["L"], c["snr"], c["decay"], seed=7100)
    y64 = synth.c64_round(inst.y)
    Lw = 50
    d = mra.dims(inst.N, inst.K, inst.Q, inst.L, inst.sigma2)
    prm = mra.em_params(Lw)
    x0 = O.align_mean(y64, inst.s, inst.L)
    lr = np.log(np.full(Lw, 1.0 / Lw))
    ws = mra.workspace(mra.mra_em_workspace_bytes(d, Lw))
    y, sh = dev_y(y64), dev(inst.s.astype(np.int32))
    kind, bi, ns = mra.mra_em_autotune(d, prm, y, sh, dev(x0), dev(lr), ws)
    assert kind in (1, 2, 3, 4, 5, 6)
    if kind == 2:
        assert bi in (16, 12, 8, 4) and ns in (2, 3)
    if kind == 3:
        assert bi in (128, 64, 32, 16) and ns in (1, 2)
    xo, lro = torch.empty((inst.K + 1, inst.Q), dtype=torch.complex128, device="cuda"), torch.empty(Lw, dtype=torch.float64, device="cuda")
    w = torch.empty((inst.N, Lw), dtype=torch.float32, device="cuda")
    mra.mra_em_step(d, prm, y, sh, dev(x0), dev(lr), xo, lro, None, None, w, ws)
    ref = O.em_step(y64, x0, lr, inst.L, inst.sigma2, Lw=Lw, shifts=inst.s)
    assert rel_err(host(xo), ref.x) <= TOL_X
    assert np.max(np.abs(host(w) - ref.w)) <= 1e-5


def test_batched_workload_list_small_n(gpu_lib):
    """The batched workload's first 12 instances (N capped at 1500), one launch, 4 iterations,
    each instance matching its single run."""
    mra = gpu_lib
    T = 4
    specs = synth.config4_instances(n_inst=12, n_max=1500)
    items, keep = [], []
    for sp in specs:
        inst = synth.make_instance(sp["K"], sp["Q"], sp["N"], sp["L"], sp["snr"], sp["decay"], seed=sp["seed"])
        y64 = synth.c64_round(inst.y)
        d = mra.dims(inst.N, inst.K, inst.Q, inst.L, inst.sigma2)
        prm = mra.em_params(sp["Lw"], max_iters=T)
        x0 = O.align_mean(y64, inst.s, inst.L)
        lr = np.log(np.full(sp["Lw"], 1.0 / sp["Lw"]))
        items.append(dict(d=d, prm=prm, y=dev_y(y64), shift=dev(inst.s.astype(np.int32)), x=dev(x0), log_rho=dev(lr)))
        keep.append((d, prm, x0, lr, sp["Lw"]))
    arr = mra.instances(items)
    ws = mra.workspace(mra.mra_em_batched_workspace_bytes(arr))
    iters, _ = mra.mra_em_run_batched(arr, ws, tune=True)
    assert iters == [T] * len(specs)
    for (d, prm, x0, lr, Lw), it in zip(keep, items):
        x1, lr1 = dev(x0), dev(lr)
        ws1 = mra.workspace(mra.mra_em_workspace_bytes(d, Lw))
        mra.mra_em_run(d, prm, it["y"], it["shift"], x1, lr1, None, None, ws1)
        assert rel_err(host(it["x"]), host(x1)) <= TOL_SAME


# rows of 16 coefficients only: the persistent kernel takes every instance (the lean sweep for windows
# of up to 32 mirror units, the warp sweep's any-window instance for the whole circle and wider windows)
SHAPES16 = [
    dict(K=12, N=1300, L=90, Lw=13, shifts=True, tol=0.0),
    dict(K=20, N=700, L=120, Lw=45, shifts=True, tol=0.0),
    dict(K=30, N=150, L=72, Lw=72, shifts=False, tol=0.0),
    dict(K=40, N=2100, L=360, Lw=60, shifts=True, tol=0.0),
    dict(K=8, N=90, L=40, Lw=9, shifts=True, tol=0.0),
    dict(K=10, N=500, L=60, Lw=15, shifts=True, tol=1e3),  # stops after its first iteration
    dict(K=16, N=3000, L=180, Lw=70, shifts=True, tol=0.0),
]


def test_persistent_batched_run_matches_graph_and_oracle(gpu_lib, monkeypatch):
    """The persistent kernel (default for these shapes) against the graph of per-instance launches
    (MRA_BATCHED=graph) from the same start, and against the FP64 oracle's trajectory; one instance
    stops by its tolerance after one iteration while the others go on."""
    mra = gpu_lib
    T = 3

    def run(graph):
        if graph:
            monkeypatch.setenv("MRA_BATCHED", "graph")
        else:
            monkeypatch.delenv("MRA_BATCHED", raising=False)
        probs, items = [], []
        for i, sh in enumerate(SHAPES16):
            p = _problem(mra, dict(sh, Q=16), 100 + i, T)
            p["prm"] = mra.em_params(p["Lw"], l0=p["l0"], max_iters=T, tol=sh["tol"])
            probs.append(p)
            items.append(dict(d=p["d"], prm=p["prm"], y=dev_y(p["y64"]), x=dev(p["x0"]), log_rho=dev(p["lr"]),
                              shift=dev(p["s"].astype(np.int32)) if p["s"] is not None else None,
                              stats=torch.full((T, 2), np.nan, dtype=torch.float64, device="cuda")))
        arr = mra.instances(items)
        ws = mra.workspace(mra.mra_em_batched_workspace_bytes(arr))
        iters, ms = mra.mra_em_run_batched(arr, ws, tune=False)
        return probs, items, iters, ms

    probs, pers, it_p, ms_p = run(False)
    _, graph, it_g, _ = run(True)
    want = [1 if sh["tol"] > 0 else T for sh in SHAPES16]
    assert it_p == want and it_g == want and ms_p > 0
    for p, a, b, n in zip(probs, pers, graph, want):
        assert rel_err(host(a["x"]), host(b["x"])) <= TOL_SAME
        np.testing.assert_allclose(np.exp(host(a["log_rho"])), np.exp(host(b["log_rho"])), rtol=0, atol=TOL_SAME)
        np.testing.assert_allclose(host(a["stats"])[:n, 0], host(b["stats"])[:n, 0], rtol=TOL_SAME)
        xs, lrs = p["x0"], p["lr"]
        for t in range(n):
            st = O.em_step(p["y64"], xs, lrs, p["inst"].L, p["inst"].sigma2, Lw=p["Lw"], l0=p["l0"], shifts=p["s"])
            assert abs(host(a["stats"])[t, 0] - st.loglik) <= 1e-6 * abs(st.loglik) + 1e-3, (t, st.loglik)
            xs, lrs = st.x, st.log_rho
        assert rel_err(host(a["x"]), xs) <= TOL_X * n, rel_err(host(a["x"]), xs)


def test_persistent_batched_run_repeats_from_its_graph(gpu_lib):
    """A second call with the same instance list (same tensors, reset to the same start) launches the
    cached graph of the persistent kernel and gives the same results: bit for bit where the lean warp
    sweep runs (fixed image order), to TOL_SAME where the warp sweep's any-window instance hands the
    images out to its warps as they become free (the whole circle here: FP32 sums in varying order)."""
    mra = gpu_lib
    T = 2
    probs, items = [], []
    for i, sh in enumerate(SHAPES16[:4]):
        p = _problem(mra, dict(sh, Q=16), 200 + i, T)
        probs.append(p)
        items.append(dict(d=p["d"], prm=p["prm"], y=dev_y(p["y64"]), x=dev(p["x0"]), log_rho=dev(p["lr"]),
                          shift=dev(p["s"].astype(np.int32)) if p["s"] is not None else None))
    arr = mra.instances(items)
    ws = mra.workspace(mra.mra_em_batched_workspace_bytes(arr))
    outs = []
    for rep in range(2):
        for p, it in zip(probs, items):
            it["x"].copy_(dev(p["x0"]))
            it["log_rho"].copy_(dev(p["lr"]))
        iters, _ = mra.mra_em_run_batched(arr, ws, tune=False)
        assert iters == [T] * 4
        outs.append([host(it["x"]).copy() for it in items])
    for sh, a, b in zip(SHAPES16[:4], *outs):
        if sh["Lw"] < sh["L"] and sh["Lw"] <= 60:
            np.testing.assert_array_equal(a, b)
        else:
            assert rel_err(a, b) <= TOL_SAME
