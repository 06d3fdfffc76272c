#!/usr/bin/env python
"""Benchmark: Synch-EM on one GB300 at |k| <= 32, Q = 24, N = 100,000, L = 360, window 36, 50 EM iterations.

One step = the whole hot path over one resident instance:
  Synchronize and Match (P = 100) -> one trial of Algorithm 1 on the instance
  (residual histogram + window prior) -> align and average -> 50 EM iterations
  (one graph-captured mra_em_run).
Metric: image-rotation evaluations per second, N * Lw * iterations / step time.
Also reported: the sweep kernel's HBM roofline fraction, an end-to-end number
through the public API with host buffers, the FP64 CPU oracle on a bounded
sample, clocks during the timed region, and time to converge against
full-search EM at equal error on the same GPU.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--no-ttc]
"""
import os

# Every oracle process runs its BLAS on one thread: the CPU legs use the host's cores through
# worker processes (one per core), whose number is the core count they report.
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse  # noqa: E402
import ctypes  # noqa: E402
import hashlib  # noqa: E402
import json  # noqa: E402
import math  # noqa: E402
import subprocess  # noqa: E402
import sys  # noqa: E402
import tempfile  # noqa: E402
import time  # noqa: E402

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

CFG = 2
METRIC = "EM image-rotation evals/s"
UNIT = "evals/s"


def dense_config():
    """The denser-resolution window of Sec. 3.3 on the Synch-EM workload: the range [-pi BW/L, pi BW/L]
    (BW = 36) sampled at spacing pi BW/L^2, i.e. Lw = 2 L + 1 rotations 0.05 grid units apart, on images
    whose rotations are continuous (off the grid)."""
    c = synth.config(CFG)
    c.update(Lw=2 * c["L"] + 1, l0=-c["L"], step=36 / (2 * c["L"]), offgrid=True)
    return c


def workload_config(c):
    dense = c.get("step", 1.0) != 1.0
    name = "Synch-EM dense window" if dense else "Synch-EM"
    w = (f"Lw={c['Lw']} step={c['step']:g} (range {(c['Lw'] - 1) * c['step']:g} grid units, off-grid rotations)"
         if dense else f"Lw={c['Lw']}")
    out = {"workload": f"{name} |k|<={c['K']} Q={c['Q']} N={c['N']} L={c['L']} {w} "
                       f"SNR=1/{round(1 / c['snr'])} T={c['iters']} P={c['P']} gamma={c['gamma']}",
           "K": c["K"], "Q": c["Q"], "N": c["N"], "L": c["L"], "Lw": c["Lw"], "iters": c["iters"], "P": c["P"],
           "snr": c["snr"], "l2": "inputs larger than L2 (y is 633.6 MB per sweep)"}
    if dense:
        out.update(step=c["step"], l0=c["l0"])
    return out


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def fp32_alu_peak_tflops():
    """FP32 CUDA-core peak of a GB300 from its unit counts and clock: 152 SMs x 128 FP32 lanes x 2 flop (FMA)
    x 2.07 GHz maximum SM clock."""
    return 152 * 128 * 2 * 2.07e9 / 1e12


def traffic_kernel():
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            return json.load(f)["kernel"].split("<")[0]
    except Exception:
        return None


def traffic_for():
    """DRAM bytes per sweep launch from the committed ncu summary, if the kernel source is unchanged since."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
        sha = hashlib.sha256(b"".join(open(os.path.join(ROOT, s), "rb").read() for s in t["sources"])).hexdigest()
        if t.get("source_sha256") == sha:
            return float(t["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


class Clocks:
    def __init__(self, out):
        self.out = out
        self.p = None

    def __enter__(self):
        try:
            self.f = open(self.out, "w")
            self.p = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200", "-i", str(self._gpu())],
                stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.p = None
        return self

    @staticmethod
    def _gpu():
        v = os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0]
        return v if v.isdigit() else "0"

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            self.p.wait()
            self.f.close()

    def summary(self):
        try:
            rows = [r.split(",") for r in open(self.out).read().strip().splitlines()]
            sm = [float(r[1]) for r in rows]
            mx = float(rows[0][2])
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip().lower() == "active"})
            return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": reasons, "samples": len(rows)}
        except Exception as e:  # no nvidia-smi
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "error": str(e)[:80]}


# ------------------------------------------------------------------ replicas across ranks (no data-path collective)
def replica_seed(rank: int) -> int:
    """Each rank draws its own independent instance (replicas, weak scaling)."""
    return 1000 * CFG + rank


def max_over_ranks(values, world: int, device):
    """Elementwise maximum of per-rank timings (one all-reduce of a few floats; no-op at world 1)."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def whole_job_value(world: int, units_per_rank: float, ms: float) -> float:
    """Units all ranks processed per second, against the slowest rank's time."""
    return world * units_per_rank / (ms / 1e3)


# ------------------------------------------------------------------ CPU oracle (baseline and reference arm)
def host_info():
    """Host core count (the cores this process may run on) and CPU model."""
    try:
        ncores = len(os.sched_getaffinity(0))
    except AttributeError:
        ncores = os.cpu_count() or 1
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                model = line.split(":", 1)[1].strip()
                if line.startswith("Model name"):
                    break
    except Exception:
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return {"nproc": ncores, "cpu_count": os.cpu_count(), "cpu_model": model or "unknown",
            "machine": os.uname().machine}


def _oracle_worker(conn):
    """One worker process: holds a slice of the images and runs the oracle's EM step on it."""
    import oracle as O

    y64, s, L, sigma2, Lw, l0, step = conn.recv()
    conn.send("ready")
    while True:
        msg = conn.recv()
        if msg is None:
            return
        x, lr = msg
        st = O.em_step(y64, x, lr, L, sigma2, Lw=Lw, shifts=s, l0=l0, step=step)
        conn.send((y64.shape[0] * st.x, st.W, st.loglik))


class OracleCores:
    """The FP64 oracle's EM step (Algorithm Synch-EM, flat image prior, gamma = 0) on several host cores:
    the images are split into equal slices, worker process i runs the oracle's em_step on slice i, and
    the parent adds the slices' M-step sums as Eq. coefficients_update does (num = sum_i N_i a_i,
    a_{t+1} = num / N, W_t = sum_i W_i, rho_{t+1} = W_t / N) and the log-likelihoods.  One worker
    calls the oracle on all images at once."""

    def __init__(self, workers: int):
        import multiprocessing as mp

        self.workers = max(1, int(workers))
        self.procs, self.conns = [], []
        if self.workers > 1:
            ctx = mp.get_context("spawn")  # safe whether or not this process already uses the GPU
            for _ in range(self.workers):
                a, b = ctx.Pipe()
                p = ctx.Process(target=_oracle_worker, args=(b,), daemon=True)
                p.start()
                self.procs.append(p)
                self.conns.append(a)

    def load(self, y64, s, L, sigma2, Lw, l0=None, step=1.0):
        self.N, self.L, self.sigma2, self.Lw, self.l0, self.stp = y64.shape[0], L, sigma2, Lw, l0, step
        if self.workers == 1:
            self.y64, self.s = y64, s
            return
        bounds = np.linspace(0, self.N, self.workers + 1).astype(int)
        for i, cn in enumerate(self.conns):
            a, b = bounds[i], bounds[i + 1]
            cn.send((y64[a:b], s[a:b], L, sigma2, Lw, l0, step))
        for cn in self.conns:
            assert cn.recv() == "ready"

    def em_step(self, x, lr):
        """Returns (a_{t+1}, log rho_{t+1}, loglik)."""
        import oracle as O

        if self.workers == 1:
            st = O.em_step(self.y64, x, lr, self.L, self.sigma2, Lw=self.Lw, shifts=self.s, l0=self.l0,
                           step=self.stp)
            return st.x, st.log_rho, st.loglik
        for cn in self.conns:
            cn.send((x, lr))
        num, W, ll = 0.0, 0.0, 0.0
        for cn in self.conns:
            n_i, w_i, l_i = cn.recv()
            num, W, ll = num + n_i, W + w_i, ll + l_i
        x_new = num / self.N
        with np.errstate(divide="ignore"):
            lr_new = np.log(W / np.sum(W))
        return x_new, lr_new, ll

    def close(self):
        for cn in self.conns:
            try:
                cn.send(None)
            except (BrokenPipeError, OSError):
                pass
        for p in self.procs:
            p.join(timeout=10)
        self.procs, self.conns = [], []


def oracle_timing(inst, c, workers, per_worker, iters, repeats=5, n_cap=None):
    """Median over `repeats` of `iters` oracle EM iterations on workers x per_worker images of the
    workload (capped at n_cap), from the aligned mean with a uniform window prior."""
    import oracle as O

    n_img = min(workers * per_worker, n_cap or inst.N, inst.N)
    y64 = synth.c64_round(inst.y[:n_img])
    s = inst.s[:n_img]
    Lw = c["Lw"]
    x0 = O.align_mean(y64, s, inst.L)
    lr0 = np.log(np.full(Lw, 1.0 / Lw))
    pool = OracleCores(workers)
    try:
        pool.load(y64, s, inst.L, inst.sigma2, Lw, c.get("l0"), c.get("step", 1.0))
        pool.em_step(x0, lr0)  # warm the workers (imports, first allocation)
        times = []
        for _ in range(repeats):
            x, lr = x0, lr0
            t0 = time.perf_counter()
            for _ in range(iters):
                x, lr, _ = pool.em_step(x, lr)
            times.append(time.perf_counter() - t0)
    finally:
        pool.close()
    dt = float(np.median(times))
    return {"value": n_img * Lw * iters / dt, "cores": pool.workers, "n_img": n_img, "iters": iters,
            "seconds_median": dt, "seconds_all": [round(t, 3) for t in times]}


def cpu_baseline(inst, c, repeats=5):
    """The oracle on all host cores (worker processes) and on one core; median of `repeats` each."""
    info = host_info()
    wide = c["Lw"] > 64
    per_worker, iters = ((max(60, 1500 * 37 // c["Lw"]), 1) if wide else (1500, 2))
    allc = oracle_timing(inst, c, info["nproc"], per_worker, iters, repeats)
    one = oracle_timing(inst, c, 1, per_worker * 2, iters, repeats)
    unit_note = "image-rotation evals/s of oracle em_step (FP64 numpy, one BLAS thread per process)"
    return {"value": allc["value"], "unit": UNIT, "cores": allc["cores"], "kind": "oracle",
            "sample": f"{unit_note}: {allc['n_img']} of the {inst.N} images split over {allc['cores']} worker "
                      f"processes, {allc['iters']} iteration(s) per repeat, median of {repeats} "
                      f"({allc['seconds_median']:.2f} s)",
            "one_core": {"value": one["value"], "cores": 1,
                         "sample": f"{one['n_img']} images, {one['iters']} iteration(s), median of {repeats} "
                                   f"({one['seconds_median']:.2f} s)"},
            "host": info}


def run_reference(args, c):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O

    info = host_info()
    workers = info["nproc"]
    per_worker = 600 if c["Lw"] <= 64 else max(30, 600 * 37 // c["Lw"])
    n_img = workers * per_worker
    inst = synth.make_instance(c["K"], c["Q"], n_img, c["L"], c["snr"], c["decay"], seed=1000 * CFG,
                               offgrid=c.get("offgrid", False))
    y64 = synth.c64_round(inst.y)
    Lw = c["Lw"]
    x0 = O.align_mean(y64, inst.s, inst.L)
    lr0 = np.log(np.full(Lw, 1.0 / Lw))
    pool = OracleCores(workers)
    try:
        pool.load(y64, inst.s, inst.L, inst.sigma2, Lw, c.get("l0"), c.get("step", 1.0))
        x, lr = x0, lr0
        for _ in range(args.warmup):
            x, lr, _ = pool.em_step(x, lr)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            x, lr, _ = pool.em_step(x, lr)
        wall = time.perf_counter() - t0
    finally:
        pool.close()
    value = args.steps * n_img * Lw / wall
    sample = (f"oracle em_step (FP64 numpy, one BLAS thread per process) on {n_img} images of the workload "
              f"split over {workers} worker processes, 1 EM iteration per step")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(c),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle", "sample": sample,
                             "host": info},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu")
    ap.add_argument("--no-ttc", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--config", default=str(CFG), choices=("1", "2", "4", "5", "dense", "tm", "fb"),
                    help="2: Synch-EM at N=1e5 (default); 1: the small Synch-EM workload (N=500, |k|<=10, Q=8, "
                         "L=72, window 24, SNR 1/10, 20 iterations); 4: 64 uneven instances in one graph launch; "
                         "5: N=1e6 with y in the BF16 hi/lo split; dense: the workload of 2 with the "
                         "denser-resolution window (2L+1 rotations over BW = 36) on off-grid rotations; tm: "
                         "template matching of the images of 2 against the first one; fb: the Fourier-Bessel "
                         "front end on 10,000 images of 129 x 129 pixels")
    args = ap.parse_args()
    c = dense_config() if args.config == "dense" else synth.config(1 if args.config == "1" else CFG)
    if args.impl == "reference":
        return run_reference(args, c)
    if args.config == "4":
        return bench_batched(args)
    if args.config == "5":
        return bench_bf16(args)
    if args.config == "tm":
        return bench_template_match(args)
    if args.config == "fb":
        return bench_fb(args)

    import torch
    import torch.distributed as dist

    from paper_2105_07372_gb300 import mra, pipeline

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    mra.load()

    # ---- inputs resident in HBM (each rank its own independent instance: replicas)
    inst = synth.make_instance(c["K"], c["Q"], c["N"], c["L"], c["snr"], c["decay"], seed=replica_seed(rank),
                               offgrid=c.get("offgrid", False))
    y_host = torch.from_numpy(synth.to_c64(inst.y)).pin_memory()
    y = y_host.to(dev)
    s_true = torch.from_numpy(inst.s.astype(np.int32)).to(dev)
    x_true = torch.from_numpy(inst.x).to(dev)
    N, K, Q, L, Lw, T, P = c["N"], c["K"], c["Q"], c["L"], c["Lw"], c["iters"], c["P"]
    d = mra.dims(N, K, Q, L, inst.sigma2)
    ws = pipeline.workspaces(d, Lw, P, dev)
    l0 = c.get("l0", -(Lw // 2))
    wstep = c.get("step", 1.0)
    shift = torch.empty(N, dtype=torch.int32, device=dev)
    hist = torch.zeros(L, dtype=torch.int32, device=dev)
    log_prior = torch.empty(Lw, dtype=torch.float64, device=dev)
    kappa = torch.empty(1, dtype=torch.float64, device=dev)
    x = torch.empty((K + 1, Q), dtype=torch.complex128, device=dev)
    log_rho = torch.empty(Lw, dtype=torch.float64, device=dev)
    stats = torch.empty((T, 2), dtype=torch.float64, device=dev)
    sweep_ms = (ctypes.c_float * T)()
    sweep_times = []

    def step(timed_sweeps, yb=None, sb=None, xb=None):
        yb = y if yb is None else yb
        sb = s_true if sb is None else sb
        xb = x_true if xb is None else xb
        mra.mra_sync(d, yb, P, 50, 100, shift, ws.sync)
        hist.zero_()
        mra.mra_prior_hist(d, yb, sb, shift, xb, hist, None, ws.em)
        mra.mra_fit_prior(L, Lw, l0, hist, 0, log_prior, kappa, step=wstep)
        mra.mra_align_mean(d, yb, shift, x, ws.em)
        log_rho.copy_(log_prior)
        prm = mra.em_params(Lw, l0=l0, gamma=c["gamma"], log_rho_bar=log_prior, max_iters=T,
                            sweep_ms=sweep_ms if timed_sweeps else None, step=wstep)
        n = mra.mra_em_run(d, prm, yb, shift, x, log_rho, stats, None, ws.em)
        if timed_sweeps:
            sweep_times.extend(list(sweep_ms)[:n])
        return n

    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        step(False)
    # the autotuner picks the EM sweep for this shape from one timed sweep of each candidate,
    # at the state a step starts from (outside the timed region, like the warm-up)
    mra.mra_sync(d, y, P, 50, 100, shift, ws.sync)
    mra.mra_align_mean(d, y, shift, x, ws.em)
    log_rho.copy_(log_prior)
    tuned = _effective_choice(mra.mra_em_autotune(
        d, mra.em_params(Lw, l0=l0, gamma=c["gamma"], log_rho_bar=log_prior, step=wstep), y, shift, x, log_rho, ws.em))
    torch.cuda.synchronize()
    # kernels of ours per step: sync 4, prior hist 5, fit 1, align 4, em_run 2 + T x (the sweep's kernels:
    # three for the split sweep, else one; and the finalize) + 1
    launches_per_step = 4 + 5 + 1 + 4 + 2 + ((3 if tuned[0] == 5 else 1) + 1) * T + 1

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    clk = _clocks(rank)
    with clk:
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step(True)
        e1.record(stream)
        barrier()
    ms = max_over_ranks([e0.elapsed_time(e1) / args.steps], world, dev)[0]
    evals_per_step = N * Lw * T
    value = whole_job_value(world, evals_per_step, ms)

    # ---- roofline of the dominant kernel (the EM sweep): algorithmic bytes = one read of y; algorithmic
    # FP32 flops per image = 8 M (correlation) + 4 Lw (K+1) (window transform) + 4 Lw (K+1) (back
    # transform) + 8 M (accumulation).  The bound is whichever takes longer at its peak: HBM for the
    # 36-rotation window, FP32 ALU for the 721-rotation dense window.
    bytes_per_sweep = N * (K + 1) * Q * 8
    flops_per_sweep = N * (16 * (K + 1) * Q + 8 * Lw * (K + 1))
    avg_sweep_s = float(np.mean(sweep_times)) / 1e3
    peak, peak_kind = peaks()
    alu_peak = fp32_alu_peak_tflops()
    traffic = traffic_for()
    kernel = {1: "k_sweep_v2", 2: "k_sweep_v3", 3: "k_sweep_v4", 4: "k_sweep_v5",
              5: "k_tc_corr+k_tc_trans+k_tc_accum", 6: "k_sweep_v6"}.get(tuned[0], "k_em_sweep")
    hbm_side = {"achieved": bytes_per_sweep / avg_sweep_s / 1e9, "peak": peak, "unit": "GB/s"}
    alu_side = {"achieved": flops_per_sweep / avg_sweep_s / 1e12, "peak": alu_peak, "unit": "TFLOP/s"}
    hbm_bound = bytes_per_sweep / (peak * 1e9) >= flops_per_sweep / (alu_peak * 1e12)
    dom = hbm_side if hbm_bound else alu_side
    roofline = {"bound": "hbm" if hbm_bound else "alu", "achieved": dom["achieved"], "peak": dom["peak"],
                "unit": dom["unit"], "frac": dom["achieved"] / dom["peak"],
                "traffic": traffic if kernel == traffic_kernel() and wstep == 1.0 else None,
                "peak_source": f"{peak_kind} hbm_gbs" if hbm_bound else
                               "derived FP32 CUDA-core peak: 152 SMs x 128 FMA/clk x 2 flop x 2.07 GHz",
                "other": ({"bound": "alu", **alu_side, "frac": alu_side["achieved"] / alu_peak} if hbm_bound else
                          {"bound": "hbm", **hbm_side, "frac": hbm_side["achieved"] / peak}),
                "kernel": kernel, "sweep_choice": {"kind": tuned[0], "batch": tuned[1], "stages_or_ctas": tuned[2]},
                "algorithmic_bytes_per_launch": bytes_per_sweep, "algorithmic_flops_per_launch": flops_per_sweep,
                "avg_launch_ms": avg_sweep_s * 1e3, "launches_timed": len(sweep_times)}
    em_ms = float(np.sum(sweep_times)) / args.steps

    # ---- end to end through the public API with host buffers (H2D of the step's inputs, D2H of its result)
    x_host = torch.empty((K + 1, Q), dtype=torch.complex128).pin_memory()
    lr_host = torch.empty(Lw, dtype=torch.float64).pin_memory()
    s_true_h = s_true.cpu().pin_memory()
    x_true_h = x_true.cpu().pin_memory()
    h2d = y_host.numel() * 8 + s_true_h.numel() * 4 + x_true_h.numel() * 16
    d2h = x_host.numel() * 16 + lr_host.numel() * 8

    # Every step's inputs are copied from pinned host memory inside the timed region, double-buffered:
    # the copies for step i + 1 run on a second stream while step i computes on the other buffers (all
    # host-to-device copies go through that stream, so that none queues behind another on the main one).
    ybufs, sbufs, xbufs = (y, torch.empty_like(y)), (s_true, torch.empty_like(s_true)), (x_true, torch.empty_like(x_true))
    cstream = torch.cuda.Stream()
    ready = (torch.cuda.Event(), torch.cuda.Event())
    done = (torch.cuda.Event(), torch.cuda.Event())

    def put(b):  # H2D of a step's inputs into buffers b once the step that last read them has finished
        with torch.cuda.stream(cstream):
            cstream.wait_event(done[b])
            sbufs[b].copy_(s_true_h, non_blocking=True)
            xbufs[b].copy_(x_true_h, non_blocking=True)
            ybufs[b].copy_(y_host, non_blocking=True)
            ready[b].record(cstream)

    def e2e_run(nsteps):
        for b in (0, 1):
            done[b].record(stream)
        put(0)
        for i in range(nsteps):
            b = i % 2
            stream.wait_event(ready[b])
            if i + 1 < nsteps:
                put(1 - b)
            step(False, ybufs[b], sbufs[b], xbufs[b])
            done[b].record(stream)
            x_host.copy_(x, non_blocking=True)
            lr_host.copy_(log_rho, non_blocking=True)

    e2e_run(2)
    barrier()
    e0.record(stream)
    e2e_run(args.steps)
    e1.record(stream)
    barrier()
    e2e_ms = max_over_ranks([e0.elapsed_time(e1) / args.steps], world, dev)[0]
    e2e = {"value": whole_job_value(world, evals_per_step, e2e_ms), "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
           "pipelining": "each step's inputs (y, and the true shifts and signal of the prior trial) copied from "
                         "pinned host memory on a second stream into the other of two device buffer sets while the "
                         "previous step computes; the first step's copy is not overlapped"}

    relerr_final = pipeline.relerr(x, x_true, d)

    # ---- time to converge against full-search EM at equal error (same GPU, same instance)
    ttc = None
    if not args.no_ttc and rank == 0 and wstep == 1.0:
        ttc = time_to_converge(mra, pipeline, c, inst, d, y, s_true, x_true, ws, dev)

    # ---- CPU oracle baseline (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(inst, c)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": dict(workload_config(c), parallelism="replicas" if world > 1 else "single"),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches_per_step * args.steps, "clocks": clk.summary(),
                "em_only": {"ms_per_step": em_ms, "evals_per_s": evals_per_step / (em_ms / 1e3)},
                "relerr_final": relerr_final, "ttc": ttc}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def time_to_converge(mra, pipeline, c, inst, d, y, s_true, x_true, ws, dev):
    """Full-search EM (random start, all L rotations, uniform rho) against Synch-EM on the same
    GPU and instance: seconds and iterations to the stopping tolerance, and the time Synch-EM
    needs to reach the full-search error (within 1%), for the configured window and for the
    window chosen from the learned distribution (99.9% of its mass)."""
    import torch

    N, K, Q, L, Lw, P = c["N"], c["K"], c["Q"], c["L"], c["Lw"], c["P"]
    tol, tmax = 1e-5, 1000
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        torch.cuda.synchronize()
        ev0.record()
        r = fn()
        ev1.record()
        torch.cuda.synchronize()
        return r, ev0.elapsed_time(ev1) / 1e3

    x0 = torch.from_numpy(synth.random_init(K, Q, c["decay"], seed=77)).to(dev)
    ws_full = mra.workspace(mra.mra_em_workspace_bytes(d, L), dev)
    full_ws = pipeline.Workspaces(em=ws_full, sync=ws.sync)
    pipeline.full_search_em(y, d, x0, iters=3, ws=full_ws)  # warm
    full, t_full = timed(lambda: pipeline.full_search_em(y, d, x0, iters=tmax, ws=full_ws, tol=tol, check_every=25))
    e_full = pipeline.relerr(full.x, x_true, d)
    target = e_full * 1.01
    out = {"full_search_s": t_full, "full_search_iters": full.iters, "full_search_relerr": e_full, "tol": tol,
           "equal_error_target": target}

    shift = pipeline.synchronize(y, d, P, ws)
    _, _, hist = pipeline.learn_prior(y, d, s_true, shift, x_true, Lw, -(Lw // 2), 0, ws)
    lw_auto = pipeline.window_for_mass(hist, L, 0.999)
    for tag, lw in (("window", Lw), ("window_auto", lw_auto)):
        wse = pipeline.Workspaces(em=mra.workspace(mra.mra_em_workspace_bytes(d, lw), dev), sync=ws.sync)

        def run(max_iters, traj=None, lw=lw, wse=wse):
            sh = pipeline.synchronize(y, d, P, wse)
            lp, _, _ = pipeline.learn_prior(y, d, s_true, sh, x_true, lw, -(lw // 2), 0, wse)
            return pipeline.synch_em(y, d, P=P, Lw=lw, iters=max_iters, gamma=c["gamma"], log_rho_bar=lp, ws=wse,
                                     shift=sh, tol=tol, check_every=25, stats=False, x_traj=traj)

        traj = torch.empty((tmax, K + 1, Q), dtype=torch.complex128, device=dev)
        r = run(tmax, traj)
        errs = [pipeline.relerr(traj[i].contiguous(), x_true, d) for i in range(r.iters)]
        hit = next((i + 1 for i, e in enumerate(errs) if e <= target), None)
        res = {"Lw": lw, "iters_to_tol": r.iters, "relerr_at_tol": errs[-1] if errs else None}
        _, t_tol = timed(lambda: run(tmax))
        res["seconds_to_tol"] = t_tol
        if hit is not None:
            _, t_hit = timed(lambda: run(hit))
            res.update({"iters_to_equal_error": hit, "seconds_to_equal_error": t_hit, "speedup": t_full / t_hit})
        else:
            res.update({"iters_to_equal_error": None, "seconds_to_equal_error": None, "speedup": None})
        out[tag] = res
    return out


def _timed_steps(step, args, clk):
    import torch

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    with clk:
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            step()
        e1.record()
        torch.cuda.synchronize()
    return e0.elapsed_time(e1) / args.steps


def _effective_choice(tuned):
    """The sweep the timed steps use: MRA_SWEEP (with MRA_SWEEP_BI / _NS) overrides the autotuner's choice."""
    kind = {"warp": 1, "cta": 2, "chunk": 3, "lean": 4, "tc": 5, "pair": 6}.get(os.environ.get("MRA_SWEEP", ""))
    if kind is None:
        return tuned
    return [kind, int(os.environ.get("MRA_SWEEP_BI", 0) or 0), int(os.environ.get("MRA_SWEEP_NS", 0) or 0)]


def _clocks(rank=0):
    """The clock samples go to $MRA_CLOCKS_DIR (kept for inspection) or to the temporary directory."""
    d = os.environ.get("MRA_CLOCKS_DIR") or tempfile.gettempdir()
    return Clocks(os.path.join(d, f"mra_clocks_rank{rank}.csv"))


def bench_batched(args):
    """64 independent instances of uneven N, K and window, 30 EM iterations each, in one graph launch
    per step (mra_em_run_batched, sweeps chosen by the autotuner).  Inputs resident in HBM; each
    instance starts from the average of its synchronized images."""
    import torch

    from paper_2105_07372_gb300 import mra, pipeline

    mra.load()
    dev = torch.device("cuda", 0)
    specs = synth.config4_instances()
    items, starts = [], []
    evals = 0
    ybytes = 0
    for sp in specs:
        inst = synth.make_instance(sp["K"], sp["Q"], sp["N"], sp["L"], sp["snr"], sp["decay"], seed=sp["seed"])
        yh = torch.from_numpy(synth.to_c64(inst.y))
        y = yh.to(dev)
        d = mra.dims(inst.N, inst.K, inst.Q, inst.L, inst.sigma2)
        ws = pipeline.workspaces(d, sp["Lw"], 100, dev)
        shift = pipeline.synchronize(y, d, 100, ws)
        x = torch.empty((inst.K + 1, inst.Q), dtype=torch.complex128, device=dev)
        mra.mra_align_mean(d, y, shift, x, ws.em)
        lr = torch.full((sp["Lw"],), -math.log(sp["Lw"]), dtype=torch.float64, device=dev)
        prm = mra.em_params(sp["Lw"], max_iters=sp["iters"])
        items.append(dict(d=d, prm=prm, y=y, shift=shift, x=x.clone(), log_rho=lr.clone()))
        starts.append((x, lr))
        evals += inst.N * sp["Lw"] * sp["iters"]
        ybytes += inst.N * (inst.K + 1) * inst.Q * 8 * sp["iters"]
        del ws
    arr = mra.instances(items)
    ws = mra.workspace(mra.mra_em_batched_workspace_bytes(arr), dev)
    t_tune = time.perf_counter()
    mra.mra_em_run_batched(arr, ws, tune=True)  # the autotuner runs here, once per shape
    t_tune = time.perf_counter() - t_tune
    exec_ms = []

    def step():
        for it, (x0, lr0) in zip(items, starts):
            it["x"].copy_(x0)
            it["log_rho"].copy_(lr0)
        _, ms = mra.mra_em_run_batched(arr, ws, tune=False)
        exec_ms.append(ms)

    clk = _clocks()
    ms = _timed_steps(step, args, clk)
    launch_ms = float(np.mean(exec_ms[args.warmup:]))
    peak, peak_kind = peaks()
    achieved = ybytes / (launch_ms / 1e3) / 1e9
    line = {"metric": METRIC, "value": evals / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{len(specs)} independent MRA instances, N~U[1000,50000] (sum "
                                   f"{sum(s['N'] for s in specs)}), K~U{{8..40}}, Q=16, L=360, Lw~U{{12..72}}, "
                                   "SNR log-U[1/100,1/5], 30 EM iterations each, one graph launch "
                                   + ("(per-instance launches)" if os.environ.get("MRA_BATCHED") == "graph"
                                      else "(one persistent kernel for all iterations)"),
                       "parallelism": "single", "l2": "inputs larger than L2"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "peak_source": f"{peak_kind} hbm_gbs", "kernel": ("whole batched graph" if os.environ.get("MRA_BATCHED") == "graph"
                                                  else "k_em_batched (persistent, in the batched graph)"),
                         "algorithmic_bytes_per_launch": ybytes, "avg_launch_ms": launch_ms},
            "autotune_s": t_tune, "graph_launch_ms": launch_ms, "clocks": clk.summary(),
            "gpu_launches": (sum(4 + 2 * sp["iters"] + 1 for sp in specs) if os.environ.get("MRA_BATCHED") == "graph"
                             else sum(4 + 1 for sp in specs) + 1) * args.steps}
    print(json.dumps(line), flush=True)


def bench_bf16(args):
    """N = 1e6 images at |k| <= 48, Q = 32, L = 720, window 72, y stored as the BF16 hi/lo split,
    50 EM iterations (mra_em_run_hl) from the average of the aligned images."""
    import torch

    from paper_2105_07372_gb300 import mra

    mra.load()
    dev = torch.device("cuda", 0)
    c = synth.config(5)
    N, K, Q, L, Lw, T = c["N"], c["K"], c["Q"], c["L"], c["Lw"], c["iters"]
    x_true = synth.make_signal(K, Q, c["decay"], np.random.default_rng(5000))
    sigma2 = synth.sigma2_for_snr(c["snr"], x_true)
    M = (K + 1) * Q
    y_hl = torch.empty((N, M, 2), dtype=torch.float32, device=dev)  # 8 bytes per complex value
    shift = torch.empty(N, dtype=torch.int32, device=dev)
    chunk = 50_000
    stage = torch.empty((chunk, K + 1, Q), dtype=torch.complex64, device=dev)
    for i0 in range(0, N, chunk):
        n = min(chunk, N - i0)
        inst = synth.make_instance(K, Q, n, L, seed=5000 + 1 + i0 // chunk, sigma2=sigma2, x=x_true)
        stage[:n].copy_(torch.from_numpy(synth.to_c64(inst.y)))
        mra.mra_y_split_bf16(stage[:n], y_hl[i0:i0 + n])
        shift[i0:i0 + n].copy_(torch.from_numpy(inst.s.astype(np.int32)))
    del stage
    d = mra.dims(N, K, Q, L, sigma2)
    ws = mra.workspace(mra.mra_em_workspace_bytes(d, Lw), dev)
    x0 = torch.from_numpy(x_true * 0.9).to(dev)  # a start near the truth; the sweeps do the same work anywhere
    lr0 = torch.full((Lw,), -math.log(Lw), dtype=torch.float64, device=dev)
    x, lr = x0.clone(), lr0.clone()
    # the autotuner times the sweeps that read the split format (batch and chunked) from the start state
    tuned = _effective_choice(mra.mra_em_autotune(d, mra.em_params(Lw), y_hl, shift, x, lr, ws, y_format=1))
    x, lr = x0.clone(), lr0.clone()
    sweep_ms = (ctypes.c_float * T)()
    sweeps = []

    def step():
        x.copy_(x0)
        lr.copy_(lr0)
        n = mra.mra_em_run_hl(d, mra.em_params(Lw, max_iters=T, sweep_ms=sweep_ms), y_hl, shift, x, lr, None, None,
                              ws)
        sweeps.extend(list(sweep_ms)[:n])

    clk = _clocks()
    ms = _timed_steps(step, args, clk)
    sw = float(np.mean(sweeps[args.warmup * T:])) / 1e3
    ybytes = N * M * 8
    peak, peak_kind = peaks()
    line = {"metric": METRIC, "value": N * Lw * T / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16 hi/lo storage, f32 arithmetic", "data": "synthetic",
            "config": {"workload": f"EM |k|<={K} Q={Q} N={N} L={L} Lw={Lw} SNR=1/100 T={T}, y as BF16 hi/lo",
                       "parallelism": "single", "l2": "inputs larger than L2 (12.5 GB per sweep)"},
            "roofline": {"bound": "hbm", "achieved": ybytes / sw / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": ybytes / sw / 1e9 / peak, "traffic": None, "peak_source": f"{peak_kind} hbm_gbs",
                         "kernel": {2: "k_sweep_v3", 3: "k_sweep_v4"}.get(tuned[0], "?") + " (BF16 hi/lo)",
                         "sweep_choice": {"kind": tuned[0], "batch": tuned[1], "stages_or_ctas": tuned[2]},
                         "algorithmic_bytes_per_launch": ybytes,
                         "avg_launch_ms": sw * 1e3},
            "clocks": clk.summary(), "gpu_launches": (2 + 2 * T + 1) * args.steps}
    print(json.dumps(line), flush=True)


def bench_template_match(args):
    """Template matching (Sec. 2.1.1) of the Synch-EM workload's images (|k| <= 32, Q = 24, N = 1e5, L = 360,
    SNR 1/50) against the first observation: one mra_template_match per step, N L image-rotation evaluations."""
    import torch

    from paper_2105_07372_gb300 import mra

    mra.load()
    dev = torch.device("cuda", 0)
    c = synth.config(CFG)
    N, K, Q, L = c["N"], c["K"], c["Q"], c["L"]
    inst = synth.make_instance(K, Q, N, L, c["snr"], c["decay"], seed=replica_seed(0))
    y = torch.from_numpy(synth.to_c64(inst.y)).to(dev)
    d = mra.dims(N, K, Q, L, inst.sigma2)
    out = torch.empty(N, dtype=torch.int32, device=dev)
    ref = y[0].clone()

    def step():
        mra.mra_template_match(d, y, ref, out)

    clk = _clocks()
    ms = _timed_steps(step, args, clk)
    M = (K + 1) * Q
    ybytes = N * M * 8
    flops = N * (8 * M + 4 * L * (K + 1))  # correlation + the transform over all L shifts, per image
    peak, peak_kind = peaks()
    alu = fp32_alu_peak_tflops()
    hbm_bound = ybytes / (peak * 1e9) >= flops / (alu * 1e12)
    ach_h, ach_a = ybytes / (ms / 1e3) / 1e9, flops / (ms / 1e3) / 1e12
    hit = float((out.cpu().numpy().astype(np.int64) == (inst.s - inst.s[0]) % L).mean())
    line = {"metric": "template-matching image-rotation evals/s", "value": N * L / (ms / 1e3), "unit": UNIT,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"template matching |k|<={K} Q={Q} N={N} L={L} SNR=1/{round(1 / c['snr'])}, "
                                   f"reference = first observation", "parallelism": "single",
                       "l2": "inputs larger than L2 (633.6 MB per launch)"},
            "roofline": {"bound": "hbm" if hbm_bound else "alu", "achieved": ach_h if hbm_bound else ach_a,
                         "peak": peak if hbm_bound else alu, "unit": "GB/s" if hbm_bound else "TFLOP/s",
                         "frac": ach_h / peak if hbm_bound else ach_a / alu, "traffic": None,
                         "peak_source": f"{peak_kind} hbm_gbs" if hbm_bound else
                                        "derived FP32 CUDA-core peak: 152 SMs x 128 FMA/clk x 2 flop x 2.07 GHz",
                         "kernel": "k_template_match", "algorithmic_bytes_per_launch": ybytes,
                         "algorithmic_flops_per_launch": flops, "avg_launch_ms": ms},
            "fraction_true_relative_shift": hit, "clocks": clk.summary(), "gpu_launches": args.steps}
    print(json.dumps(line), flush=True)


def bench_fb(args):
    """The Fourier-Bessel front end (App. A) at the paper's image size: N = 10,000 images of 129 x 129 pixels
    onto |k| <= 32, Q = 24 (the coefficient shape of the Synch-EM workload): one mra_fb_project per step on the
    tensor cores (six BF16 piece products, FP32 accuracy; the three-product fast mode timed beside it); the
    one-time mra_fb_setup and packing are timed separately."""
    import torch

    from paper_2105_07372_gb300 import mra, pipeline

    mra.load()
    dev = torch.device("cuda", 0)
    n, K, Q, N = 129, 32, 24, 10_000
    c = synth.config(CFG)
    A = torch.from_numpy(synth.render_matrix(n, K, Q)).to(dev, torch.float32)  # data generation only
    x = synth.make_signal(K, Q, c["decay"], np.random.default_rng(11))
    s = np.random.default_rng(12).integers(0, c["L"], N)
    a = x[None] * np.exp(-2j * np.pi * np.outer(s, np.arange(K + 1)) / c["L"])[:, :, None]
    sigma = math.sqrt(synth.sigma2_for_snr(c["snr"], x))
    coeff = torch.from_numpy(synth.real_params(a)).to(dev, torch.float32)
    images = (coeff @ A.T).reshape(N, n, n)
    images += sigma * torch.randn(images.shape, generator=torch.Generator(device=dev).manual_seed(13), device=dev)
    del A, coeff
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    P = pipeline.fb_projection(n, K, Q, dev)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    y = torch.empty((N, K + 1, Q), dtype=torch.complex64, device=dev)

    def step(fast=False):
        mra.mra_fb_project(N, n, K, Q, images, P, y, fast)

    clk = _clocks()
    ms = _timed_steps(step, args, clk)
    ms_tf32 = _timed_steps(lambda: step(True), args, _clocks())
    flops = 2.0 * N * n * n * 2 * (K + 1) * Q
    alu = fp32_alu_peak_tflops()
    bf16 = 1943.5
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            bf16 = float(json.load(f)["bf16_tflops"])
    except Exception:
        pass

    # steerable PCA of the projected coefficients: the fit (second moments on the GPU, eigenvectors on the
    # host) once, then the reduced coefficients by CGEMM
    step()
    d = mra.dims(N, K, Q, c["L"], sigma ** 2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    yr, d2, basis, counts = pipeline.spca(y, d)
    torch.cuda.synchronize()
    spca_s = time.perf_counter() - t0
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.steps):
        mra.mra_spca_project(d, y, d2.K, d2.Q, basis, yr)
    ev1.record()
    torch.cuda.synchronize()
    spca_proj_ms = ev0.elapsed_time(ev1) / args.steps
    # white pixel noise of variance sigma^2 stays (nearly) white with the same variance per coefficient (App. A)
    noise_ratio = float(torch.mean(torch.abs(y.cpu().to(torch.complex128) - torch.from_numpy(a)) ** 2) / sigma ** 2)
    line = {"metric": "Fourier-Bessel projected images/s", "value": N / (ms / 1e3), "unit": "images/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"Fourier-Bessel front end: N={N} images {n}x{n} onto |k|<={K} Q={Q} "
                                   f"(SNR 1/{round(1 / c['snr'])})", "parallelism": "single",
                       "l2": f"inputs larger than L2 ({N * n * n * 4 / 1e6:.0f} MB of pixels per launch)"},
            "roofline": {"bound": "tensor", "achieved": 6 * flops / (ms / 1e3) / 1e12, "peak": bf16,
                         "unit": "TFLOP/s", "frac": 6 * flops / (ms / 1e3) / 1e12 / bf16, "traffic": None,
                         "peak_source": "measured bf16_tflops (burst); achieved counts the six BF16 products",
                         "kernel": "k_gemm3<0> (tcgen05, mra_fb_project)", "algorithmic_flops_per_launch": flops,
                         "fp32_equivalent_tflops": flops / (ms / 1e3) / 1e12, "fp32_alu_peak": alu,
                         "avg_launch_ms": ms},
            "fast": {"ms_per_step": ms_tf32, "images_per_s": N / (ms_tf32 / 1e3),
                     "achieved_tflops_bf16": 3 * flops / (ms_tf32 / 1e3) / 1e12, "peak_tflops": bf16,
                     "frac": 3 * flops / (ms_tf32 / 1e3) / 1e12 / bf16},
            "setup_s": setup_s, "coefficient_noise_variance_over_pixel_variance": noise_ratio,
            "spca": {"fit_s": spca_s, "project_ms": spca_proj_ms, "reduced_shape": [d2.K + 1, d2.Q],
                     "kept_per_k": [int(v) for v in counts]},
            "clocks": clk.summary(), "gpu_launches": args.steps}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
