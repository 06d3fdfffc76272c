"""bench.py's reference arm (the FP64 oracle on the host cores) on the CPU: one JSON line carrying the
benchmark contract's keys, the oracle baseline and a zero-copy end-to-end entry; under torchrun with two
ranks only rank 0 does the work and prints.  Also the sweep-choice report under an environment override."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

KEYS = ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
        "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e")


def _json_lines(cmd, timeout=600):
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=timeout)
    assert r.returncode == 0, r.stderr[-3000:]
    return [json.loads(s) for s in r.stdout.splitlines() if s.startswith("{")]


def _bench():
    # imported inside the tests: importing bench sets the BLAS thread-count defaults of the process
    import bench

    return bench


def _check_line(d, n_gpus, steps, warmup):
    bench = _bench()
    for k in KEYS:
        assert k in d, k
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert (d["n_gpus"], d["steps"], d["warmup"]) == (n_gpus, steps, warmup)
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["higher_is_better"] is True and d["dtype"] == "f64" and d["vs_baseline"] is None
    assert d["config"]["workload"].startswith("Synch-EM")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["sample"]
    assert cb["cores"] == cb["host"]["nproc"] >= 1 and cb["host"]["cpu_model"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_prints_one_contract_line():
    lines = _json_lines([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1"])
    assert len(lines) == 1
    _check_line(lines[0], 1, 2, 1)


def test_reference_arm_dense_workload_names_its_window():
    lines = _json_lines([sys.executable, "bench.py", "--impl", "reference", "--config", "dense", "--steps", "1",
                         "--warmup", "0"])
    assert len(lines) == 1
    _check_line(lines[0], 1, 1, 0)
    c = lines[0]["config"]
    assert c["Lw"] == 2 * c["L"] + 1 and c["l0"] == -c["L"] and 0 < c["step"] < 1


def test_reference_arm_under_torchrun_two_ranks():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    lines = _json_lines([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                         "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
                         "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"])
    assert len(lines) == 1
    _check_line(lines[0], 2, 1, 0)


def test_sweep_choice_follows_the_environment(monkeypatch):
    bench = _bench()
    tuned = (1, 0, 0)
    monkeypatch.delenv("MRA_SWEEP", raising=False)
    assert bench._effective_choice(tuned) == tuned
    monkeypatch.setenv("MRA_SWEEP", "chunk")
    monkeypatch.setenv("MRA_SWEEP_BI", "64")
    monkeypatch.setenv("MRA_SWEEP_NS", "2")
    assert bench._effective_choice(tuned) == [3, 64, 2]
    monkeypatch.setenv("MRA_SWEEP", "cta")
    monkeypatch.delenv("MRA_SWEEP_BI")
    monkeypatch.delenv("MRA_SWEEP_NS")
    assert bench._effective_choice(tuned) == [2, 0, 0]


def test_oracle_on_several_cores_equals_the_oracle_on_all_images():
    """The worker-process split of the CPU baseline adds the slices' M-step sums (Eq. coefficients_update):
    its EM step equals the oracle's em_step over all images at once."""
    import numpy as np

    import oracle as O
    import synth

    bench = _bench()
    inst = synth.make_instance(6, 4, 301, 36, 1 / 10, 50.0, seed=91)
    Lw = 9
    x0 = O.align_mean(inst.y, inst.s, inst.L)
    lr0 = np.log(np.full(Lw, 1.0 / Lw))
    ref = O.em_step(inst.y, x0, lr0, inst.L, inst.sigma2, Lw=Lw, shifts=inst.s)
    pool = bench.OracleCores(3)
    try:
        pool.load(inst.y, inst.s, inst.L, inst.sigma2, Lw)
        x1, lr1, ll = pool.em_step(x0, lr0)
    finally:
        pool.close()
    np.testing.assert_allclose(x1, ref.x, rtol=0, atol=1e-13)
    np.testing.assert_allclose(lr1, ref.log_rho, rtol=0, atol=1e-12)
    assert abs(ll - ref.loglik) <= 1e-10 * abs(ref.loglik)


def test_cpu_baseline_reports_all_cores_and_one_core():
    import synth

    bench = _bench()
    c = dict(synth.config(1))
    inst = synth.make_instance(c["K"], c["Q"], 400, c["L"], c["snr"], c["decay"], seed=92)
    cb = bench.cpu_baseline(inst, c, repeats=2)
    assert cb["kind"] == "oracle" and cb["value"] > 0 and cb["one_core"]["value"] > 0
    assert cb["cores"] == cb["host"]["nproc"] and cb["one_core"]["cores"] == 1
