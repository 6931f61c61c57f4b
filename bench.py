"""Benchmark of the Monte Carlo KBC LBM hot path on one GB300 (or N, one ensemble per rank).

Workload (default): M = 64 randomized Taylor-Green samples on 64^3, Re = 800, Ma = 0.025,
shifted FP32 populations, pull streaming; the whole ensemble advances in one launch per
lattice step.  One bench step = one output interval: S = 50 fused stream+collide updates
of every sample, then the ensemble reductions the interval feeds (per-sample kinetic
energy E_m(t), ensemble mean and variance velocity fields, all FP64).

metric: ensemble GLUPS (lattice-node updates per second, summed over ranks), with the
stepper's achieved HBM bandwidth against the measured copy bandwidth.  Inputs (one
ensemble of 2.55 GB of populations) exceed the 129 MB L2, so no flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(name="rtgv_64cube_x64_fp32_pull", N=64, M=64, Re=800.0, Ma=0.025, precision="fp32",
                pattern="pull", updates_per_step=50, seed=1)
KINDS = ["direct", "staged", "prefetch", "prefetch_packed", "async_ring2", "async_ring3", "exact_gamma"]
KERNEL_NAMES = ["k_step_batch", "k_step_staged", "k_step_prefetch", "k_step_prefetch", "k_step_async", "k_step_async",
                "k_step_batch"]
BYTES_PER_LU = {"fp64": 2 * 19 * 8, "fp32": 2 * 19 * 4, "fp16": 2 * 19 * 2}
STEPPER_SOURCES = ["paper_2608_23786_gb300/csrc/stepper.cu", "paper_2608_23786_gb300/csrc/collide.cuh",
                   "paper_2608_23786_gb300/csrc/storage.cuh", "paper_2608_23786_gb300/csrc/lattice.cuh",
                   "paper_2608_23786_gb300/csrc/stepper_impl.cuh", "paper_2608_23786_gb300/csrc/stepper_launch.cuh",
                   "paper_2608_23786_gb300/csrc/stepper_staged.cuh", "paper_2608_23786_gb300/csrc/stepper_async.cuh",
                   "paper_2608_23786_gb300/csrc/stepper_f32_pull.cu"]
# DRAM bytes (read + write) per launch of the stepper on this workload, from one ncu capture of the
# kernel built from sources with this digest and launched with this shape (kind, vec, block); the
# capture ran 16 of the 64 samples (318.8 MB read + 267.5 MB written) and is scaled by 64/16.
# Reported as null when the sources or the launch shape differ.
NCU_TRAFFIC = {"sha256": "45155e47dc0715a2", "launch": (3, 2, 128), "bytes_per_launch": 4 * (318.808576e6 + 267.662848e6)}


def stepper_digest():
    """Digest of the stepper's code: the sources with their line comments, trailing blanks and
    empty lines removed, so that a change of wording in a comment keeps the traffic record (the
    sources hold no string literal with a double slash)."""
    h = hashlib.sha256()
    for p in STEPPER_SOURCES:
        with open(os.path.join(ROOT, p), encoding="utf-8") as f:
            for line in f:
                code = line.split("//", 1)[0].rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region: one `nvidia-smi -lms 100`
    process streams a line every 100 ms; entering waits for its first line (at most 5 s) so that
    the samples cover the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.samples = []
        self._proc = None
        self._t = None
        self._first = threading.Event()

    def _read(self):
        for line in self._proc.stdout:
            parts = [p.strip() for p in line.strip().split(",")]
            if len(parts) == 6:
                self.samples.append(parts)
                self._first.set()

    def __enter__(self):
        try:
            self._proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                           "--format=csv,noheader,nounits", "-lms", "100"],
                                          stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            return self
        self._t = threading.Thread(target=self._read, daemon=True)
        self._t.start()
        self._first.wait(5.0)
        return self

    def __exit__(self, *a):
        if self._proc is not None:
            self._proc.terminate()
            try:
                self._proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self._proc.kill()
            self._t.join(timeout=5)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4) if s[2 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def oracle_sample(wl, budget_s=10.0, max_samples=2):
    """The FP64 oracle as it stands on a bounded sample of the workload: `max_samples` samples,
    as many updates as fit the time budget (whole output intervals are not required), then the
    same reductions.  Returns (GLUPS, description, cores)."""
    import oracle
    from oracle import stats
    import ensemble_inputs as gen
    un = oracle.units(wl["N"], wl["Re"], wl["Ma"])
    X = gen.draw_params(wl["seed"], max_samples)
    f = oracle.init_ensemble(wl["N"], X, un["ulat"], lattice=wl.get("lattice", 19))
    lu, steps = 0, 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        oracle.step(f, un["omega"])
        steps += 1
        lu += max_samples * wl["N"] ** 3
    _, u = oracle.moments(f)
    up = stats.to_physical(u, un["ulat"])
    stats.kinetic_energy(up)
    stats.mean_var(up)
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    desc = (f"{max_samples} of {wl['M']} samples x {steps} updates of {wl['N']}^3 (a step of the workload is "
            f"{wl['updates_per_step']} updates), then E(t) and mean/var; FP64 C oracle, OpenMP over planes")
    return lu / dt / 1e9, desc, cores


# The 128^3 x 32 target shape and the other large configurations, measured after the default timed region
# (each entry times its own stepper launches with CUDA events on the ensemble's stream, for about
# half a second, with its own clock record).  (name, N, M, Re, Ma, precision, pattern)
TARGETS = [("rtgv_128cube_x32_fp32_pull", 128, 32, 1600.0, 0.0125, "fp32", "pull"),
           ("rtgv_128cube_x32_fp32_aa", 128, 32, 1600.0, 0.0125, "fp32", "aa"),
           ("rtgv_128cube_x32_fp16_pull", 128, 32, 1600.0, 0.0125, "fp16", "pull"),
           ("rtgv_128cube_x32_fp16_aa", 128, 32, 1600.0, 0.0125, "fp16", "aa"),
           ("rtgv_512cube_x4_fp16_aa", 512, 4, 6400.0, 0.003125, "fp16", "aa")]
# the D3Q27 library at the target shape (FP16 storage: the configuration furthest from the roofline)
TARGETS_D3Q27 = [("rtgv_128cube_x32_fp16_pull_d3q27", 128, 32, 1600.0, 0.0125, "fp16", "pull"),
                 ("rtgv_128cube_x32_fp16_aa_d3q27", 128, 32, 1600.0, 0.0125, "fp16", "aa")]
LEVELS = [(64, 64, 400.0, 0.025, 1, 1), (128, 32, 1600.0, 0.0125, 4, 2), (256, 8, 3200.0, 0.00625, 16, 3)]
ALU_KINDS = [("fp64_fma", 2.0), ("fp32_fma", 2.0), ("fp32x2_fma", 2.0), ("half2_fma", 2.0), ("fp32_rcp", 1.0)]


def _timed_steps(stream, fn, est_s, target_s=0.5, lo=4, hi=2000):
    """Number of calls of `fn` (one step or macro step) that fill about target_s seconds, from
    a first estimate of one call's time est_s."""
    return int(min(hi, max(lo, round(target_s / max(est_s, 1e-6)))))


def _event_time(stream, fn, n):
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    fn(n)
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / 1e3


def measure_targets(dev, stream, peaks, peak_kind, lattice=19):
    """The 128^3 x 32 target configuration (FP32 and FP16 shifted storage, pull and
    AA), the 512^3 x 4 FP16 AA configuration, and the three-level batch (FP32 pull, FP16 AA),
    each with the library's default launch shape: GLUPS and HBM fraction of the stepper from
    CUDA events over whole steps (every step is one stepper launch; a batch macro step is one
    graph replay of its sub-steps)."""
    import torch
    from paper_2608_23786_gb300 import Ensemble, mclbm
    import ensemble_inputs as gen
    out = {}
    runs = [t + (lattice,) for t in TARGETS] + ([t + (27,) for t in TARGETS_D3Q27] if lattice == 19 else [])
    for name, N, M, Re, Ma, prec, pat, q in runs:
        mclbm.load(lattice=q)
        ens = Ensemble(N, M, Re=Re, Ma=Ma, precision=prec, pattern=pat, seed=2, device=dev, stream=stream,
                       lattice=q).init(gen.draw_params(2, M))
        step = lambda n: ens.step(n)  # noqa: E731
        step(4)
        est = _event_time(stream, step, 4) / 4
        n = _timed_steps(stream, step, est)
        n += n % 2  # whole AA step pairs
        with ClockSampler(dev.index or 0) as clk:
            sec = _event_time(stream, step, n)
        mclbm.mclbm_device_status(ens.ctx)
        lu = M * N**3 * n
        bpl = BYTES_PER_LU[prec] * q // 19
        ach = bpl * lu / sec / 1e9
        launch = launch_desc(mclbm.mclbm_get_launch_parity(ens.ctx, 0),
                             mclbm.mclbm_get_launch_parity(ens.ctx, 1) if pat == "aa" else None)
        out[name] = {"glups": lu / sec / 1e9, "avg_launch_ms": sec / n * 1e3, "steps_timed": n,
                     "bytes_per_lu": bpl, "achieved_gbs": ach, "peak_gbs": peaks["hbm_gbs"], "peak_kind": peak_kind,
                     "frac": ach / peaks["hbm_gbs"], "launch": dict(launch, chosen_by="default"),
                     "clocks": clk.summary()}
        del ens
        torch.cuda.empty_cache()
    for prec, pat in (("fp32", "pull"), ("fp16", "aa")):
        levels = [Ensemble(N, M, Re=Re, Ma=Ma, precision=prec, pattern=pat, seed=seed, device=dev, stream=stream,
                           lattice=lattice).init(gen.draw_params(seed, M)) for N, M, Re, Ma, _, seed in LEVELS]
        subs = [lv[4] for lv in LEVELS]
        b = mclbm.mclbm_batch_create([e.ctx for e in levels], subs)
        macro = lambda n: mclbm.mclbm_batch_step(b, n)  # noqa: E731
        macro(3)
        est = _event_time(stream, macro, 2) / 2
        n = _timed_steps(stream, macro, est, lo=3, hi=200)
        with ClockSampler(dev.index or 0) as clk:
            sec = _event_time(stream, macro, n)
        for e in levels:
            mclbm.mclbm_device_status(e.ctx)
        lu = sum(M * N**3 * sub for (N, M, _, _, sub, _) in LEVELS) * n
        bpl = BYTES_PER_LU[prec] * lattice // 19
        ach = bpl * lu / sec / 1e9
        launch = launch_desc(mclbm.mclbm_batch_get_launch_parity(b, 0),
                             mclbm.mclbm_batch_get_launch_parity(b, 1) if pat == "aa" else None)
        out[f"levels_64x64_128x32_256x8_{prec}_{pat}"] = {
            "glups": lu / sec / 1e9, "ms_per_macro_step": sec / n * 1e3, "macro_steps_timed": n, "substeps": subs,
            "bytes_per_lu": bpl, "achieved_gbs": ach, "peak_gbs": peaks["hbm_gbs"], "peak_kind": peak_kind,
            "frac": ach / peaks["hbm_gbs"], "launch": dict(launch, chosen_by="default"), "graph": True,
            "clocks": clk.summary()}
        mclbm.mclbm_batch_destroy(b)
        del levels
        torch.cuda.empty_cache()
    return out


def measure_alu(dev, stream):
    """Measured arithmetic ceilings of this GPU (fma chains per type, the reciprocal unit):
    results and floating-point operations per second."""
    import torch
    from paper_2608_23786_gb300 import mclbm
    sink = torch.zeros(1, dtype=torch.float64, device=dev)
    out = {}
    for kind, flops_per_result in ALU_KINDS:
        iters = 64
        r, ms = mclbm.mclbm_alu_rate(kind, iters, sink.data_ptr(), stream.cuda_stream)
        iters = int(min(1 << 16, max(64, iters * 50.0 / max(ms, 1e-3))))  # about 50 ms per timed launch
        r, ms = mclbm.mclbm_alu_rate(kind, iters, sink.data_ptr(), stream.cuda_stream)
        out[kind] = {"results_per_s": r, "flops": r * flops_per_result, "ms": ms}
    return out


def run_peaks(args):
    """Measured arithmetic ceilings (FP64, FP32, packed FP32x2 and half2 fma, FP32 reciprocal)
    with the clocks seen while they ran."""
    import torch
    from paper_2608_23786_gb300 import mclbm
    mclbm.load()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    measure_alu(dev, stream)  # warm-up
    with ClockSampler(0) as clk:
        alu = measure_alu(dev, stream)
    print(json.dumps({"metric": "alu_peaks", "unit": "results/s", "alu": alu, "clocks": clk.summary(),
                      "how": "8 blocks x 256 threads per SM, 8 independent chains per thread, CUDA events"}))


def run_stats(args):
    """The ensemble statistics on one ensemble (N = 128, M = 4 unless --N / --M; storage
    --precision, FP32 by default) after 10 steps, each timed once with CUDA events after one
    untimed call: E_m and Z_m, E_m and the mean/variance fields in one pass, the shell spectrum, trace S_2,
    S_p along the axes (p = 2..6), the restriction to 8^3 points, the one-point W1 and the
    vector and component-wise two-point W1 against a second ensemble of the same shape."""
    import torch
    from paper_2608_23786_gb300 import Ensemble, mclbm
    import ensemble_inputs as gen
    mclbm.load()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    N, M, prec = args.N or 128, args.M or 4, args.precision or "fp32"
    A = Ensemble(N, M, Re=1600.0, Ma=1.6 / N, precision=prec, seed=7, device=dev, stream=stream).init(
        gen.draw_params(7, M)).step(10)
    B = Ensemble(N, M, Re=1600.0, Ma=1.6 / N, precision=prec, seed=8, device=dev, stream=stream).init(
        gen.draw_params(8, M)).step(10)
    calls = {"energy_enstrophy": lambda: A.energy(enstrophy=True), "energy_mean_var": lambda: A.energy_mean_var(),
             "spectrum": lambda: A.spectrum(),
             "sf_trace": lambda: A.sf_trace(), "sf_axes_p2_6": lambda: A.sf_axes(6), "restrict_8": lambda: A.restrict(8),
             "w1_1pt": lambda: A.w1(B), "w1_2pt_vector": lambda: A.w1_2pt(B, Q=8, vector=True),
             "w1_2pt_componentwise": lambda: A.w1_2pt(B, Q=8, vector=False)}
    out = {}
    for name, fn in calls.items():
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        out[name] = (time.perf_counter() - t0) * 1e3
    print(json.dumps({"metric": "statistics_ms", "unit": "ms per call (host wall clock around a synchronising call)",
                      "config": {"workload": f"rtgv_{N}cube_x{M}_{prec}_stats", "N": N, "M": M}, "ms": out}))


def run_w1_2pt(args):
    """Two-point W1 (vector W_{1,2}^v and component-wise W_{1,2}) between two RTGV ensembles of
    M samples (100 unless --M, the paper's smaller EOWC ensembles; N = 32 unless --N, 10 steps)
    on the Q^3 restriction grid (Q = 8 unless --Q: 131328 point pairs), each timed once with
    CUDA events on the stream after one untimed call."""
    import torch
    from paper_2608_23786_gb300 import Ensemble, mclbm
    import ensemble_inputs as gen
    mclbm.load()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    N, M, Q = args.N or 32, args.M or 100, args.Q
    A = Ensemble(N, M, Re=1600.0, Ma=1.6 / N, precision="fp32", seed=11, device=dev, stream=stream).init(
        gen.draw_params(11, M)).step(10)
    B = Ensemble(N, M, Re=1600.0, Ma=1.6 / N, precision="fp32", seed=12, device=dev, stream=stream).init(
        gen.draw_params(12, M)).step(10)
    G = Q**3
    out = {}
    for vector, key in ((True, "vector"), (False, "componentwise")):
        A.w1_2pt(B, Q=Q, vector=vector)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        W = A.w1_2pt(B, Q=Q, vector=vector)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        nprob = G * (G + 1) // 2 * (1 if vector else 3)
        out[key] = {"W": W, "ms": ms, "problems": nprob, "us_per_problem": ms * 1e3 / nprob}
    print(json.dumps({"metric": "w1_2pt_ms", "unit": "ms per call (CUDA events)",
                      "config": {"workload": f"w1_2pt_rtgv_{N}cube_x{M}_Q{Q}", "N": N, "M": M, "Q": Q,
                                 "pairs": G * (G + 1) // 2}, "w1_2pt": out}))


def _observables(ens, pmax=6, fields=True):
    """Per-sample statistics of one ensemble (host arrays)."""
    out = {"ke": ens.energy(), "spectrum": ens.spectrum(), "s2": ens.sf_trace(), "sp": ens.sf_axes(pmax)}
    if fields:
        E, mean, var = ens.energy_mean_var()
        out["mean"], out["var"] = mean.cpu().numpy(), var.cpu().numpy()
        out["u"] = [ens.moments(m)[1].cpu().numpy() for m in range(ens.M)]
    return out


def _precision_errors(red, ref):
    """Relative errors of one reduced-precision run's observables against the FP64 run's."""
    def rel(a, b):
        return float(np.max(np.abs(a - b) / np.abs(b)))
    e = {"ke": rel(red["ke"], ref["ke"])}
    S, So = red["spectrum"], ref["spectrum"]
    tot = So.sum(axis=1, keepdims=True)
    for floor in (1e-2, 1e-4, 1e-6):
        big = So >= floor * tot
        e[f"spectrum_bins_ge_{floor:g}_of_total"] = float(np.max(np.abs(S - So)[big] / So[big]))
    e["spectrum_abs_over_total"] = float(np.max(np.abs(S - So) / tot))
    e["s2"] = rel(red["s2"][:, 1:], ref["s2"][:, 1:])
    e["sp"] = rel(red["sp"], ref["sp"])
    if "u" in red:
        e["u_l2"] = float(max(np.linalg.norm(a - b) / np.linalg.norm(b) for a, b in zip(red["u"], ref["u"])))
        e["mean_l2"] = float(np.linalg.norm(red["mean"] - ref["mean"]) / np.linalg.norm(ref["mean"]))
        e["var_l2"] = float(np.linalg.norm(red["var"] - ref["var"]) / np.linalg.norm(ref["var"]))
    return e


def run_precision(args):
    """FP32 and FP16 shifted storage against the plain FP64 GPU stepper (whose parity with the
    oracle the tests establish), per observable, after a fixed horizon:
      - 128^3 x 32 RTGV samples at Re 1600, Ma 0.0125, 500 steps: FP32 and FP16, pull and AA;
        kinetic energy, velocity field (relative L2), E(kappa) (on bins holding >= 1e-2, 1e-4,
        1e-6 of the total, and the largest absolute error over the total), trace S_2, S_p along
        the axes (p = 2..6), mean and variance fields, and the one-point W1 between the reduced-
        precision law and the FP64 law of the same samples as a fraction of the W1 between two
        independent FP64 ensembles (the sampling distance);
      - the three-level batch (64^3 x 64, 128^3 x 32, 256^3 x 8 at Re 400 / 1600 / 3200, 1 : 4 : 16
        sub-steps), FP16 AA and FP32 pull batches against per-level FP64 runs after 10 macro
        steps: per level the same statistics (S_p for p = 2, 3), and the one-point W1 between
        consecutive levels."""
    import torch
    from paper_2608_23786_gb300 import Ensemble, mclbm
    import ensemble_inputs as gen
    mclbm.load()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    res = {"metric": "precision_errors", "unit": "relative error against the FP64 GPU run"}
    # ---- 128^3 x 32
    N, M, Re, Ma, T = 128, args.M or 32, 1600.0, 0.0125, args.T
    XA, XB = gen.draw_params(21, M), gen.draw_params(22, M)

    def run(prec, pat, X, seed):
        return Ensemble(N, M, Re=Re, Ma=Ma, precision=prec, pattern=pat, seed=seed, device=dev,
                        stream=stream).init(X).step(T)

    t0 = time.perf_counter()
    A64 = run("fp64", "pull", XA, 21)
    ref = _observables(A64)
    rA = A64.restrict(8).cpu().numpy()
    del A64
    B64 = run("fp64", "pull", XB, 22)
    rB = B64.restrict(8).cpu().numpy()
    del B64
    torch.cuda.empty_cache()
    from paper_2608_23786_gb300 import mclbm as _m

    def w1_restricted(a, b):
        da, db = torch.as_tensor(a, device=dev), torch.as_tensor(b, device=dev)
        nb = _m.mclbm_w1_work_bytes(a.shape[0], b.shape[0], a.shape[1])
        work = torch.empty(nb, dtype=torch.uint8, device=dev)
        return _m.mclbm_w1_restricted(da.data_ptr(), a.shape[0], db.data_ptr(), b.shape[0], a.shape[1],
                                      work.data_ptr(), nb, stream.cuda_stream)

    w_sampling = w1_restricted(rA, rB)
    table = {}
    for prec, pat in (("fp32", "pull"), ("fp32", "aa"), ("fp16", "pull"), ("fp16", "aa")):
        e = run(prec, pat, XA, 21)
        err = _precision_errors(_observables(e), ref)
        err["w1_to_fp64_law_over_sampling_w1"] = w1_restricted(e.restrict(8).cpu().numpy(), rA) / w_sampling
        table[f"{prec}_{pat}"] = err
        del e
        torch.cuda.empty_cache()
    res["rtgv_128cube_x%d_%dsteps" % (M, T)] = {"errors": table, "sampling_w1": w_sampling,
                                                 "seconds": time.perf_counter() - t0}
    # ---- three-level batch
    t0 = time.perf_counter()
    MACRO = 10
    refs, rrefs = [], []
    for (Nl, Ml, Rel, Mal, sub, seed) in LEVELS:
        e = Ensemble(Nl, Ml, Re=Rel, Ma=Mal, precision="fp64", pattern="pull", seed=seed, device=dev,
                     stream=stream).init(gen.draw_params(seed, Ml)).step(sub * MACRO)
        refs.append(_observables(e, pmax=3, fields=False))
        rrefs.append(e.restrict(8).cpu().numpy())
        del e
        torch.cuda.empty_cache()
    w_ref = [w1_restricted(rrefs[k], rrefs[k + 1]) for k in range(2)]
    batch = {}
    for prec, pat in (("fp32", "pull"), ("fp16", "aa")):
        levels = [Ensemble(Nl, Ml, Re=Rel, Ma=Mal, precision=prec, pattern=pat, seed=seed, device=dev,
                           stream=stream).init(gen.draw_params(seed, Ml)) for Nl, Ml, Rel, Mal, _, seed in LEVELS]
        b = mclbm.mclbm_batch_create([x.ctx for x in levels], [lv[4] for lv in LEVELS])
        mclbm.mclbm_batch_step(b, MACRO)
        mclbm.mclbm_batch_destroy(b)
        per = {}
        for k, x in enumerate(levels):
            per[f"{LEVELS[k][0]}cube_x{LEVELS[k][1]}"] = _precision_errors(_observables(x, pmax=3, fields=False),
                                                                           refs[k])
        rr = [x.restrict(8).cpu().numpy() for x in levels]
        per["w1_consecutive_levels"] = [abs(w1_restricted(rr[k], rr[k + 1]) - w_ref[k]) / w_ref[k] for k in range(2)]
        batch[f"{prec}_{pat}"] = per
        del levels
        torch.cuda.empty_cache()
    res[f"levels_64x64_128x32_256x8_{MACRO}macro"] = {"errors": batch, "w1_consecutive_levels_fp64": w_ref,
                                                     "seconds": time.perf_counter() - t0}
    print(json.dumps(res))


def run_precision_large(args):
    """The error per observable at 512^3 x 4 RTGV samples (Re 6400, Ma 0.003125, 200 steps): FP16 and
    FP32 shifted storage with in-place AA streaming against the plain FP64 GPU stepper (AA) on the
    same samples: kinetic energy, velocity field (relative L2, formed on the GPU), E(kappa), trace
    S_2, S_p along the axes (p = 2..6), mean and variance fields, and the one-point W1 against a
    256^3 x 8 level (Re 3200, Ma 0.00625, 50 steps: the same physical time under diffusive scaling;
    FP64), as the relative change of that distance against the FP64 512^3 law's."""
    import torch
    from paper_2608_23786_gb300 import Ensemble, mclbm
    import ensemble_inputs as gen
    mclbm.load()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    N, M, Re, Ma, T = 512, 4, 6400.0, 0.003125, 200
    X = gen.draw_params(5, M)
    t0 = time.perf_counter()
    lev = Ensemble(256, 8, Re=3200.0, Ma=0.00625, precision="fp64", pattern="aa", seed=6, device=dev,
                   stream=stream).init(gen.draw_params(6, 8)).step(T // 4)
    r256 = lev.restrict(8).cpu().numpy()
    del lev
    torch.cuda.empty_cache()

    def w1_vs_level(e):
        da, db = e.restrict(8), torch.as_tensor(r256, device=dev)
        nb = mclbm.mclbm_w1_work_bytes(M, r256.shape[0], da.shape[1])
        work = torch.empty(nb, dtype=torch.uint8, device=dev)
        return mclbm.mclbm_w1_restricted(da.data_ptr(), M, db.data_ptr(), r256.shape[0], da.shape[1],
                                         work.data_ptr(), nb, stream.cuda_stream)

    def observe(prec):
        e = Ensemble(N, M, Re=Re, Ma=Ma, precision=prec, pattern="aa", seed=5, device=dev,
                     stream=stream).init(X).step(T)
        o = {"ke": e.energy(), "spectrum": e.spectrum(), "s2": e.sf_trace(), "sp": e.sf_axes(6)}
        _, o["mean"], o["var"] = e.energy_mean_var()
        o["u"] = [e.moments(m)[1] for m in range(M)]  # device tensors
        o["w1"] = w1_vs_level(e)
        del e
        torch.cuda.empty_cache()
        return o

    def l2(a, b):
        return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))

    ref = observe("fp64")
    table = {}
    for prec in ("fp16", "fp32"):
        o = observe(prec)
        err = _precision_errors({k: o[k] for k in ("ke", "spectrum", "s2", "sp")},
                                {k: ref[k] for k in ("ke", "spectrum", "s2", "sp")})
        err["u_l2"] = max(l2(a, b) for a, b in zip(o["u"], ref["u"]))
        err["mean_l2"], err["var_l2"] = l2(o["mean"], ref["mean"]), l2(o["var"], ref["var"])
        err["w1_vs_256_level"] = abs(o["w1"] - ref["w1"]) / ref["w1"]
        table[f"{prec}_aa"] = err
        del o
        torch.cuda.empty_cache()
    print(json.dumps({"metric": "precision_errors", "unit": "relative error against the FP64 GPU run",
                      "rtgv_512cube_x4_200steps": {"errors": table, "w1_vs_256_level_fp64": ref["w1"],
                                                   "seconds": time.perf_counter() - t0}}))


def run_reference(args, wl):
    """Reference arm: the FP64 oracle timed on the host cores (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from oracle import stats
    import ensemble_inputs as gen
    un = oracle.units(wl["N"], wl["Re"], wl["Ma"])
    ms, upd = 1, 4  # bounded sample per step: 1 sample x 4 updates of 64^3, then the reductions
    X = gen.draw_params(wl["seed"], ms)
    f = oracle.init_ensemble(wl["N"], X, un["ulat"])

    def one():
        for _ in range(upd):
            oracle.step(f, un["omega"])
        _, u = oracle.moments(f)
        up = stats.to_physical(u, un["ulat"])
        stats.kinetic_energy(up)

    for _ in range(args.warmup):
        one()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one()
    dt = time.perf_counter() - t0
    value = ms * wl["N"] ** 3 * upd * args.steps / dt / 1e9
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = f"{ms} of {wl['M']} samples x {upd} of {wl['updates_per_step']} updates per step, then E(t)"
    print(json.dumps({
        "impl": "reference", "metric": "ensemble_glups", "value": value, "unit": "GLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl["name"], "N": wl["N"], "M": wl["M"], "Re": wl["Re"], "Ma": wl["Ma"],
                   "updates_per_step": wl["updates_per_step"], "l2": "inputs larger than L2"},
        "cpu_baseline": {"value": value, "unit": "GLUPS", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def launch_desc(even, odd=None):
    """The launch shape(s) of a bench line: (kind, vec, block) of pull or AA even steps, and of
    AA odd steps where they differ."""
    d = {"kind": KINDS[even[0]], "vec": even[1], "block": even[2]}
    if odd is not None and tuple(odd[:3]) != tuple(even[:3]):
        d["odd_steps"] = {"kind": KINDS[odd[0]], "vec": odd[1], "block": odd[2]}
    return d


def _cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_report_child(stats_too):
    """The FP64 oracle as it stands, with the OpenMP thread count of this process: cfg1 (32^3 x 1
    deterministic TGV, Re 100, U_lat 0.05, TGV pressure density) timed whole over 200 steps; cfg2
    (64^3 RTGV, Re 800, Ma 0.025) as a per-update rate over the first 10 steps of a few samples;
    with `stats_too`, one snapshot's statistics per sample."""
    import oracle
    from oracle import stats
    import ensemble_inputs as gen
    out = {"threads": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))}
    un = oracle.units(32, 100.0, 0.05 * np.sqrt(3.0))
    f = oracle.init_ensemble(32, None, un["ulat"], density_mode=1, M=1)
    t0 = time.perf_counter()
    oracle.run(f, un["omega"], 200)
    dt = time.perf_counter() - t0
    out["cfg1"] = {"mlups": 32**3 * 200 / dt / 1e6, "seconds": dt, "run": "32^3 x 1, 200 steps, whole"}
    ms = 4 if out["threads"] > 1 else 1
    un = oracle.units(64, 800.0, 0.025)
    f = oracle.init_ensemble(64, gen.draw_params(1, ms), un["ulat"])
    t0 = time.perf_counter()
    oracle.run(f, un["omega"], 10)
    dt = time.perf_counter() - t0
    out["cfg2"] = {"mlups": ms * 64**3 * 10 / dt / 1e6, "seconds": dt,
                   "run": f"{ms} of 64 samples x the first 10 steps of 64^3 (per-update rate)"}
    if stats_too:
        _, u = oracle.moments(f)
        up = stats.to_physical(u, un["ulat"])
        g = oracle.init_ensemble(64, gen.draw_params(2, ms), un["ulat"])
        _, ub = oracle.moments(g)
        ub = stats.to_physical(ub, un["ulat"])
        times = {}
        for name, fn in (("kinetic_energy", lambda: stats.kinetic_energy(up)),
                         ("enstrophy", lambda: stats.enstrophy(up)),
                         ("mean_var", lambda: stats.mean_var(up)),
                         ("energy_spectrum", lambda: stats.energy_spectrum(up)),
                         ("structure_function_trace", lambda: stats.structure_function_trace(up)),
                         ("structure_function_axes_p2_6", lambda: stats.structure_function_axes(up, 6)),
                         ("w1_one_point_8cube", lambda: stats.w1_one_point(stats.restrict(up), stats.restrict(ub)))):
            t0 = time.perf_counter()
            fn()
            times[name] = (time.perf_counter() - t0) / ms * 1e3
        out["stats_ms_per_sample_64cube"] = times
    return out


def run_oracle_report(args):
    """The oracle's timings of the CPU baseline plan on the host (all cores, then one core, each in
    a child process so that OpenMP starts with that thread count), the CPU model, and the GPU's
    cfg1 run (32^3 x 1 x 200 steps: L2-resident, not an HBM figure) beside them."""
    if args.oracle_child:
        print(json.dumps(oracle_report_child(args.oracle_child == "all")))
        return
    nproc = os.cpu_count() or 1
    rep = {"metric": "oracle_report", "cpu_model": _cpu_model(), "nproc": nproc, "oracle": {}}
    for tag, threads in (("all_cores", nproc), ("one_core", 1)):
        env = dict(os.environ, OMP_NUM_THREADS=str(threads))
        res = subprocess.run([sys.executable, os.path.abspath(__file__), "--workload", "oracle_report",
                              "--oracle-child", "all" if tag == "all_cores" else "one"],
                             env=env, capture_output=True, text=True, check=True)
        rep["oracle"][tag] = json.loads(res.stdout.strip().splitlines()[-1])
    import torch
    if torch.cuda.is_available():
        from paper_2608_23786_gb300 import Ensemble, mclbm
        mclbm.load()
        dev = torch.device("cuda", 0)
        stream = torch.cuda.Stream(dev)
        torch.cuda.set_stream(stream)
        gpu = {}
        for prec in ("fp64", "fp32", "fp16"):
            ens = Ensemble(32, 1, Re=100.0, Ma=0.05 * np.sqrt(3.0), precision=prec, init_density=1, device=dev,
                           stream=stream).init_tgv()
            ens.step(200)
            torch.cuda.synchronize()
            ens.init_tgv()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ens.step(200)
            b.record(stream)
            torch.cuda.synchronize()
            sec = a.elapsed_time(b) / 1e3
            gpu[prec] = {"mlups": 32**3 * 200 / sec / 1e6, "ms": sec * 1e3, "memory": "L2-resident"}
        rep["gpu_cfg1"] = gpu
    print(json.dumps(rep))


def run_levels(args, precision):
    """Uneven batch of the diffusive-scaling viscosity sequence in one graph-captured launch per
    sub-step: 64^3 x 64, 128^3 x 32, 256^3 x 8 at Re 400 / 1600 / 3200, Ma 0.025 / 0.0125 / 0.00625,
    1 : 4 : 16 sub-steps per macro step.  One bench step = one macro step.  The statistics the
    levels feed (shell spectra, S_2 / S_3 along axes, W1 between consecutive levels) are timed
    once after the timed region and reported separately."""
    import torch
    from paper_2608_23786_gb300 import Ensemble, mclbm
    import ensemble_inputs as gen
    mclbm.load()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    pattern = "aa" if precision == "fp16" else "pull"
    spec = [(64, 64, 400.0, 0.025, 1, 1), (128, 32, 1600.0, 0.0125, 4, 2), (256, 8, 3200.0, 0.00625, 16, 3)]
    levels = [Ensemble(N, M, Re=Re, Ma=Ma, precision=precision, pattern=pattern, seed=seed, device=dev,
                       stream=stream).init(gen.draw_params(seed, M)) for N, M, Re, Ma, _, seed in spec]
    subs = [sp[4] for sp in spec]
    b = mclbm.mclbm_batch_create([e.ctx for e in levels], subs)
    tuned = mclbm.mclbm_batch_autotune(b, 1)
    for _ in range(max(3, args.warmup)):
        mclbm.mclbm_batch_step(b, 1)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        ev0.record(stream)
        mclbm.mclbm_batch_step(b, args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
    sec = ev0.elapsed_time(ev1) / 1e3
    lu = sum(M * N**3 * sub for (N, M, _, _, sub, _) in spec) * args.steps
    for e in levels:
        mclbm.mclbm_device_status(e.ctx)
    bpl = BYTES_PER_LU[precision]
    peaks, peak_kind = measured_peaks()
    achieved = bpl * lu / sec / 1e9
    # statistics fed by the levels
    t0 = time.perf_counter()
    spectra = [e.spectrum() for e in levels]
    sfa = [e.sf_axes(3) for e in levels]
    w1 = [levels[k].w1(levels[k + 1]) for k in range(2)]
    stats_s = time.perf_counter() - t0
    # two-point W1 between consecutive levels on the 8^3 grid (131328 point pairs; L = 64 and 32)
    w12 = {}
    for vector, key in ((True, "vector"), (False, "componentwise")):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        vals = [levels[k].w1_2pt(levels[k + 1], Q=8, vector=vector) for k in range(2)]
        w12[key] = {"values": vals, "s": time.perf_counter() - t1}
    out = {
        "metric": "ensemble_glups", "value": lu / sec / 1e9, "unit": "GLUPS", "n_gpus": 1, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": sec / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if precision == "fp32" else "f16-storage/f32",
        "data": "synthetic",
        "config": {"workload": f"levels_64x64_128x32_256x8_{precision}_{pattern}", "substeps": subs,
                   "launch": launch_desc(tuned, mclbm.mclbm_batch_get_launch_parity(b, 1) if pattern == "aa" else None),
                   "graph": True,
                   "l2": "inputs larger than L2"},
        "roofline": {"kernel": KERNEL_NAMES[tuned[0]], "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                     "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "peak_kind": peak_kind, "traffic": None},
        "stats_once_s": stats_s, "w1_consecutive_levels": w1, "w1_2pt_consecutive_levels": w12,
        "spectrum_finite": bool(all(np.all(np.isfinite(x)) for x in spectra + sfa)),
        "clocks": clk.summary(),
    }
    mclbm.mclbm_batch_destroy(b)
    print(json.dumps(out))


def run_large(args):
    """512^3 x 4 samples, Re = 6400, Ma = 0.003125, FP16 shifted storage, in-place AA streaming;
    one bench step = 10 updates.  E(k), S_p (p = 2..6) and W1 against a 256^3 x 8 level are timed
    once after the timed region."""
    import torch
    from paper_2608_23786_gb300 import Ensemble, mclbm
    import ensemble_inputs as gen
    mclbm.load()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    S = 10
    ens = Ensemble(512, 4, Re=6400.0, Ma=0.003125, precision="fp16", pattern="aa", seed=5, device=dev,
                   stream=stream).init(gen.draw_params(5, 4))
    tuned = mclbm.mclbm_autotune(ens.ctx, 2)
    for _ in range(max(3, args.warmup)):
        ens.step(S)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        ev0.record(stream)
        ens.step(S * args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
    sec = ev0.elapsed_time(ev1) / 1e3
    mclbm.mclbm_device_status(ens.ctx)
    lu = 4 * 512**3 * S * args.steps
    peaks, peak_kind = measured_peaks()
    achieved = BYTES_PER_LU["fp16"] * lu / sec / 1e9
    ref = Ensemble(256, 8, Re=3200.0, Ma=0.00625, precision="fp16", pattern="aa", seed=6, device=dev,
                   stream=stream).init(gen.draw_params(6, 8)).step(4 * S)
    t0 = time.perf_counter()
    E = ens.spectrum()
    t1 = time.perf_counter()
    Sp = ens.sf_axes(6)
    t2 = time.perf_counter()
    W = ens.w1(ref)
    t3 = time.perf_counter()
    out = {
        "metric": "ensemble_glups", "value": lu / sec / 1e9, "unit": "GLUPS", "n_gpus": 1, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": sec / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f16-storage/f32", "data": "synthetic",
        "config": {"workload": "rtgv_512cube_x4_fp16_aa", "updates_per_step": S, "footprint_gb": 38 * 512**3 * 4 / 1e9,
                   "launch": launch_desc(tuned, mclbm.mclbm_get_launch_parity(ens.ctx, 1)),
                   "l2": "inputs larger than L2"},
        "roofline": {"kernel": KERNEL_NAMES[tuned[0]], "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                     "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "peak_kind": peak_kind, "traffic": None},
        "stats_s": {"spectrum": t1 - t0, "sf_axes_p2_6": t2 - t1, "w1_vs_256": t3 - t2}, "w1": W,
        "stats_finite": bool(np.all(np.isfinite(E)) and np.all(np.isfinite(Sp))),
        "clocks": clk.summary(),
    }
    print(json.dumps(out))


def run_adjoint(args):
    """Adjoint workload alone: dE(T)/dX of 64^3 x M randomized-TGV samples (M = 16 unless --M), T = 500
    FP32 steps (--T), checkpoint every 50; one bench step = one whole gradient (forward with
    checkpoints, segment recomputation, reverse sweep, parameter reduction)."""
    import torch
    from paper_2608_23786_gb300 import Ensemble, mclbm
    import ensemble_inputs as gen
    Q = args.lattice
    mclbm.load(lattice=Q)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    M, T, K = args.M or 16, args.T, 50
    X = gen.draw_params(1, M)
    prec = args.precision or "fp32"
    if prec == "fp64":
        raise SystemExit("the adjoint workload times the FP32 reverse sweep (FP32 or FP16 state)")
    b_state = {"fp32": 4, "fp16": 2}[prec]
    ens = Ensemble(64, M, Re=800.0, Ma=0.025, precision=prec, pattern="pull", device=dev, stream=stream,
                   lattice=Q).init(X)
    need = mclbm.mclbm_grad_required_bytes(ens.ctx, T, K)
    gbuf = torch.empty(need + 256, dtype=torch.uint8, device=dev)
    gptr = (gbuf.data_ptr() + 255) // 256 * 256
    for _ in range(max(3, args.warmup)):
        ens.init(X)
        mclbm.mclbm_grad(ens.ctx, 0, T, K, gptr, need, M)
    torch.cuda.synchronize()
    ph = np.zeros(4)
    with ClockSampler(0) as clk:
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ens.init(X)
            J, G = mclbm.mclbm_grad(ens.ctx, 0, T, K, gptr, need, M)  # synchronises (host results)
            ph += np.array(mclbm.mclbm_grad_timing(ens.ctx))
        sec = time.perf_counter() - t0
    ph /= args.steps
    lu = M * 64**3 * T
    peaks, peak_kind = measured_peaks()
    rev_bytes = Q * (b_state + 4 + 4) * lu  # state read, lambda^{t+1} read, lambda^t written
    achieved = rev_bytes / (ph[2] / 1e3) / 1e9
    out = {
        "metric": "adjoint_glups", "value": lu * args.steps / sec / 1e9, "unit": "GLUPS (whole gradient)",
        "n_gpus": 1, "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": sec / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if prec == "fp32" else "f16-storage/f32", "data": "synthetic",
        "config": {"workload": f"rtgv_64cube_x{M}_{prec}_{T}steps_ckpt{K}_dE", "lattice": f"D3Q{Q}",
                   "l2": "inputs larger than L2"},
        "phases_ms": {"forward": ph[0], "recompute": ph[1], "reverse": ph[2], "reduction": ph[3]},
        "roofline": {"kernel": f"k_adjoint_async<{'float' if prec == 'fp32' else '__half'},2,2>", "bound": "hbm",
                     "achieved": achieved,
                     "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                     "peak_kind": peak_kind, "traffic": None, "algorithmic_bytes_per_lu": Q * (b_state + 8),
                     "reverse_glups": lu / (ph[2] / 1e3) / 1e9},
        "grad_finite": bool(np.all(np.isfinite(G))), "clocks": clk.summary(),
    }
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--precision", default=None, choices=["fp32", "fp16", "fp64"])
    ap.add_argument("--pattern", default=None, choices=["pull", "aa"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end and plain-FP64 legs (profiling)")
    ap.add_argument("--no-targets", action="store_true",
                    help="skip the target-configuration entries (128^3 x 32, 512^3 x 4, three-level batches)")
    ap.add_argument("--N", type=int, default=None, help="override the lattice size (profiling of small cases)")
    ap.add_argument("--M", type=int, default=None, help="override the number of samples (profiling of small cases)")
    ap.add_argument("--launch", default=None, help="kind,vec,block instead of the library default (e.g. 0,2,128)")
    ap.add_argument("--autotune", action="store_true", help="let the library's autotuner pick the launch shape")
    ap.add_argument("--workload", default="ensemble64",
                    choices=["ensemble64", "levels_fp32", "levels_fp16", "large", "adjoint", "oracle_report",
                             "peaks", "stats", "w1_2pt", "precision", "precision_large"],
                    help="ensemble64 (default): 64^3 x 64 FP32; levels_*: 3-level batch; large: 512^3 x 4 FP16 AA; "
                         "adjoint: gradient of E(T), 64^3 x 16, 500 steps; oracle_report: the oracle on cfg1/cfg2 "
                         "(all cores and one core), its statistics per snapshot, and the GPU on cfg1; precision / "
                         "precision_large: FP32 and FP16 storage against the FP64 GPU run per observable (128^3 x 32 "
                         "and the three-level batch / 512^3 x 4)")
    ap.add_argument("--T", type=int, default=500, help="adjoint horizon (steps) of --workload adjoint")
    ap.add_argument("--Q", type=int, default=8, help="restriction grid Q^3 of --workload w1_2pt")
    ap.add_argument("--oracle-child", default=None, choices=["all", "one"], help=argparse.SUPPRESS)
    ap.add_argument("--exact-gamma", action="store_true",
                    help="ensemble workload with the exact entropic gamma (Newton per node) instead of the closed form")
    ap.add_argument("--lattice", type=int, default=19, choices=[19, 27],
                    help="velocity set of the ensemble64 workload: 19 (D3Q19, the paper's) or 27 (D3Q27)")
    args = ap.parse_args()
    if args.workload.startswith("levels"):
        return run_levels(args, args.workload.split("_")[1])
    if args.workload == "large":
        return run_large(args)
    if args.workload == "adjoint":
        return run_adjoint(args)
    if args.workload == "oracle_report":
        return run_oracle_report(args)
    if args.workload == "peaks":
        return run_peaks(args)
    if args.workload == "stats":
        return run_stats(args)
    if args.workload == "w1_2pt":
        return run_w1_2pt(args)
    if args.workload == "precision":
        return run_precision(args)
    if args.workload == "precision_large":
        return run_precision_large(args)
    wl = dict(WORKLOAD)
    if args.N or args.M:
        wl["N"] = args.N or wl["N"]
        wl["M"] = args.M or wl["M"]
    if args.precision:
        wl["precision"] = args.precision
    if args.pattern:
        wl["pattern"] = args.pattern
    if args.N or args.M or args.precision or args.pattern:
        wl["name"] = f"rtgv_{wl['N']}cube_x{wl['M']}_{wl['precision']}_{wl['pattern']}"
    wl["lattice"] = args.lattice
    if args.lattice == 27:
        wl["name"] += "_d3q27"
    if args.exact_gamma:
        wl["name"] += "_exact_gamma"
    if args.impl == "reference":
        return run_reference(args, wl)

    import torch
    import torch.distributed as dist
    from paper_2608_23786_gb300 import Ensemble, mclbm
    import ensemble_inputs as gen

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    mclbm.load()
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    S = wl["updates_per_step"]
    # each rank owns an independent ensemble: samples rank*M .. rank*M + M - 1 of the Philox stream
    X = gen.draw_params(wl["seed"], wl["M"], first_sample=rank * wl["M"])
    ens = Ensemble(wl["N"], wl["M"], Re=wl["Re"], Ma=wl["Ma"], precision=wl["precision"], pattern=wl["pattern"],
                   seed=wl["seed"], device=dev, stream=stream, lattice=wl["lattice"],
                   exact_gamma=args.exact_gamma).init(X)
    # launch shape: the library default, an explicit one, or the autotuner's pick on this ensemble
    # (the autotuner restores the initial state)
    if args.launch:
        kind, vec, block = (int(v) for v in args.launch.split(","))
        mclbm.mclbm_set_launch(ens.ctx, vec, block, kind)
        tuned = (kind, vec, block, None)
    elif args.autotune:
        tuned = mclbm.mclbm_autotune(ens.ctx, 3)
    else:
        tuned = tuple(mclbm.mclbm_get_launch(ens.ctx)) + (None,)
    mean = torch.empty((3,) + (wl["N"],) * 3, dtype=torch.float64, device=dev)
    var = torch.empty_like(mean)
    E = np.zeros(wl["M"])
    kernels_per_step = S + 2  # S stepper launches, one pass for E(t) and the mean/var fields, its energy reduce

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]

    def one_step(i=None):
        if i is not None:
            ev[i][0].record(stream)
        mclbm.mclbm_step(ens.ctx, S)
        if i is not None:
            ev[i][1].record(stream)
        mclbm.mclbm_energy_mean_var(ens.ctx, E, mean.data_ptr(), var.data_ptr())  # synchronises (host E)

    for _ in range(max(3, args.warmup)):
        one_step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        t_start.record(stream)
        for i in range(args.steps):
            one_step(i)
        t_end.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    elapsed = t_start.elapsed_time(t_end) / 1e3
    stepper_s = sum(a.elapsed_time(b) for a, b in ev) / 1e3 / (args.steps * S)  # per launch
    if world > 1:
        t = torch.tensor([elapsed], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed = t.item()
    lu_per_rank = wl["M"] * wl["N"] ** 3 * S * args.steps
    value = lu_per_rank * world / elapsed / 1e9

    # ---- end to end through the public API with host buffers: params H2D from pinned memory,
    # init + S updates + reductions, E and the mean/var fields D2H every step.  The fields of step
    # k travel to the host on a copy stream while step k + 1 computes (two device buffers, each
    # reused only after its copy has finished); E comes back inside the reduction call.
    params_h = torch.from_numpy(X.copy()).pin_memory()
    E_h = torch.empty(wl["M"], dtype=torch.float64).pin_memory()
    mv_h = torch.empty((2, 2, 3) + (wl["N"],) * 3, dtype=torch.float64).pin_memory()
    mv_d = torch.empty((2, 2, 3) + (wl["N"],) * 3, dtype=torch.float64, device=dev)
    copy_stream = torch.cuda.Stream(dev)
    copied = [None, None]  # event: the copy out of buffer b has finished
    e2e_k = [0]

    def e2e_step():
        b = e2e_k[0] & 1
        e2e_k[0] += 1
        if copied[b] is not None:
            copied[b].synchronize()
        mclbm.mclbm_init_ensemble(ens.ctx, params_h.numpy())  # host parameters, H2D inside the call
        mclbm.mclbm_step(ens.ctx, S)
        e = np.zeros(wl["M"])
        mclbm.mclbm_energy_mean_var(ens.ctx, e, mv_d[b, 0].data_ptr(), mv_d[b, 1].data_ptr())  # synchronises
        E_h.copy_(torch.from_numpy(e))
        with torch.cuda.stream(copy_stream):
            mv_h[b].copy_(mv_d[b], non_blocking=True)
            copied[b] = torch.cuda.Event()
            copied[b].record(copy_stream)

    e2e_steps = max(2, args.steps // 4)
    if args.no_e2e:
        e2e_steps = 0
    else:
        e2e_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    copy_stream.synchronize()  # the last step's fields are on the host
    torch.cuda.synchronize()
    e2e_dt = max(time.perf_counter() - t0, 1e-9)
    if world > 1:
        t = torch.tensor([e2e_dt], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_dt = t.item()
    e2e_value = wl["M"] * wl["N"] ** 3 * S * e2e_steps * world / e2e_dt / 1e9

    # ---- plain FP64 single-sample GPU stepper on the same GPU (the method without the ensemble
    # batching or shifted storage), 64^3 x 1
    plain_glups = None
    if not args.no_e2e:
        plain = Ensemble(wl["N"], 1, Re=wl["Re"], Ma=wl["Ma"], precision="fp64", pattern="pull", device=dev,
                         stream=stream, lattice=wl["lattice"]).init(X[:1])
        plain_launch = mclbm.mclbm_autotune(plain.ctx, 5)  # its fastest shape (restores the initial state)
        plain.step(5)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        plain.step(40)
        b.record(stream)
        torch.cuda.synchronize()
        plain_glups = wl["N"] ** 3 * 40 / (a.elapsed_time(b) / 1e3) / 1e9
        del plain

    # ---- adjoint: gradients of E(T) w.r.t. the 24 parameters of 16 samples at 64^3 after 500 FP32
    # steps, checkpoint every 50 (forward, segment recomputation, reverse sweep, reduction)
    adjoint = None
    if not args.no_e2e:
        T4, K4, M4 = 500, 50, 16
        ens4 = Ensemble(64, M4, Re=wl["Re"], Ma=wl["Ma"], precision="fp32", pattern="pull", device=dev,
                        stream=stream, lattice=wl["lattice"]).init(X[:M4])
        need = mclbm.mclbm_grad_required_bytes(ens4.ctx, T4, K4)
        gbuf = torch.empty(need + 256, dtype=torch.uint8, device=dev)
        gptr = (gbuf.data_ptr() + 255) // 256 * 256
        mclbm.mclbm_grad(ens4.ctx, 0, T4, K4, gptr, need, M4)  # warm-up
        ens4.init(X[:M4])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        J4, G4 = mclbm.mclbm_grad(ens4.ctx, 0, T4, K4, gptr, need, M4)
        grad_s = time.perf_counter() - t0
        ph = mclbm.mclbm_grad_timing(ens4.ctx)
        lu4 = M4 * 64**3 * T4
        adj_bytes = 3 * wl["lattice"] * 4 * lu4  # read state + read lambda + write lambda per update
        adjoint = {"workload": "rtgv_64cube_x16_fp32_500steps_ckpt50", "objective": "E(T)",
                   "value": lu4 / grad_s / 1e9, "unit": "GLUPS (whole gradient: forward + recompute + reverse)",
                   "phases_ms": {"forward": ph[0], "recompute": ph[1], "reverse": ph[2], "reduction": ph[3]},
                   "reverse_glups": lu4 / (ph[2] / 1e3) / 1e9,
                   "reverse_achieved_gbs": adj_bytes / (ph[2] / 1e3) / 1e9,
                   "reverse_frac_of_hbm": adj_bytes / (ph[2] / 1e3) / 1e9 / measured_peaks()[0]["hbm_gbs"],
                   "algorithmic_bytes_per_lu_reverse": 3 * wl["lattice"] * 4,
                   "grad_finite": bool(np.all(np.isfinite(G4)))}
        del gbuf, ens4

    peaks, peak_kind = measured_peaks()
    mclbm.mclbm_device_status(ens.ctx)
    main_odd = mclbm.mclbm_get_launch_parity(ens.ctx, 1) if wl["pattern"] == "aa" else None
    targets = alu = plain_ratio = None
    if not args.no_e2e and not args.no_targets:
        del ens
        torch.cuda.empty_cache()
        targets = measure_targets(dev, stream, peaks, peak_kind, lattice=wl["lattice"])
        alu = measure_alu(dev, stream)
        if plain_glups is not None:
            # the plain FP64 stepper's bandwidth against the copy bandwidth (its arithmetic
            # ceiling is the measured FP64 fma rate in alu_measured)
            plain_gbs = plain_glups * BYTES_PER_LU["fp64"] * wl["lattice"] // 19
            plain_ratio = {"achieved_gbs": plain_gbs, "frac_of_hbm": plain_gbs / peaks["hbm_gbs"],
                           "launch": dict(launch_desc(plain_launch), chosen_by="autotuner"),
                           "l2": "80 MB of populations: L2-resident"}
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    bpl = BYTES_PER_LU[wl["precision"]] * wl["lattice"] // 19 * wl["M"] * wl["N"] ** 3
    achieved = bpl / stepper_s / 1e9
    digest = stepper_digest()
    traffic = (NCU_TRAFFIC["bytes_per_launch"]
               if NCU_TRAFFIC["sha256"] == digest and tuple(tuned[:3]) == NCU_TRAFFIC["launch"] and wl["M"] == 64
               and wl["lattice"] == 19
               and wl["N"] == 64 and wl["precision"] == "fp32" and wl["pattern"] == "pull" else None)
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        v, desc, cores = oracle_sample(wl)
        cpu = {"value": v, "unit": "GLUPS", "cores": cores, "kind": "oracle", "sample": desc}
    out = {
        "metric": "ensemble_glups", "value": value, "unit": "GLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if wl["precision"] == "fp32" else
        ("f16-storage/f32" if wl["precision"] == "fp16" else "f64"), "data": "synthetic",
        "config": {"workload": wl["name"], "N": wl["N"], "M_per_gpu": wl["M"], "Re": wl["Re"], "Ma": wl["Ma"],
                   "lattice": f"D3Q{wl['lattice']}", "storage": wl["precision"], "streaming": wl["pattern"],
                   "updates_per_step": S,
                   "reductions_per_step": ["E_m(t)", "mean/var fields"], "l2": f"inputs ({bpl / 1e9:.2f} GB moved per update) "
                         "larger than the 129 MB L2: no flush",
                   "launch": dict(launch_desc(tuned, main_odd),
                                  chosen_by="explicit" if args.launch else ("autotuner" if args.autotune else "default"))},
        "roofline": {"kernel": KERNEL_NAMES[tuned[0]] +
                     f"<{wl['precision']},{wl['pattern']},vec={tuned[1]},block={tuned[2]}>",
                     "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / peaks["hbm_gbs"], "peak_kind": peak_kind,
                     "traffic": traffic, "algorithmic_bytes_per_launch": bpl,
                     "avg_launch_ms": stepper_s * 1e3, "stepper_glups": wl["M"] * wl["N"] ** 3 / stepper_s / 1e9},
        "cpu_baseline": cpu,
        "e2e": None if args.no_e2e else {"value": e2e_value, "unit": "GLUPS",
                                         "h2d_bytes_per_step": int(params_h.numel() * 8),
                                         "d2h_bytes_per_step": int(E_h.numel() * 8 + mv_h[0].numel() * 8)},
        "gpu_launches": kernels_per_step * args.steps,
        "fp64_plain_single_sample": dict({"value": plain_glups, "unit": "GLUPS", "N": wl["N"], "M": 1},
                                         **(plain_ratio or {})),
        "targets": targets,
        "alu_measured": alu,
        "adjoint": adjoint,
        "clocks": clk.summary(),
        "stepper_code_digest": digest,
    }
    print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
