"""Benchmark: batched OMP on partial-DFT measurements, fast vs FFT correlation.

Workload of the headline metric: partial DFT,
complex64 correlation side, 1024 instances sharing one Omega, N = 4096,
M = 1024 random rows, K = 64, complex Gaussian nonzeros, 40 dB AWGN, halt at K
or ||r|| < 1e-6 ||y||.  One step = one cs_omp call on the whole batch: the
initial transform, K identifications with the fast and/or transform
correlation (hybrid switch), K FP64 least-squares updates, all in one
persistent kernel.  Inputs are synthetic and seeded; they stay resident in
HBM for the device-timed value, and go host -> device -> host every step for
the end-to-end value.  L2 is flushed before every timed step: a 256 MB write,
then a read of the same buffer, so that the dirty lines of the write are
written back before the timed region starts instead of inside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  Under torchrun every rank solves its own
batch (weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "OMP solves/s & correlations/s, fast vs FFT/FWHT path, 1 GB300; p50/p99"
WORKLOAD = "partial-DFT complex64 OMP, 1024 instances sharing Omega, N=4096, M=1024, K=64, 40 dB AWGN"
CFG = dict(synth.CONFIG_DFT_C64_BATCH)
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP32 non-tensor peak: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz maximum SM clock
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


# ------------------------------------------------------------------ oracle leg
# Instances of the 1024-instance batch the oracle solves: spread over the
# batch, including instances that land on reused slots of the persistent
# kernel (high indices).
SAMPLE = [0, 1, 151, 303, 304, 455, 607, 608, 609, 700, 811, 900, 1000, 1021, 1022, 1023]


def _oracle_worker(args):
    os.environ["OMP_NUM_THREADS"] = "1"
    kind, N, omega, ys, K, record = args
    from oracle import matrices, omp as oomp
    Phi = matrices.sensing_rows(kind, N, omega)
    out = []
    for y in ys:
        r = oomp.omp(Phi, y.astype(np.complex128 if kind == "dft" else np.float64), K, record_h=record)
        if not record:
            out.append(len(r["support"]))
            continue
        out.append({"support": r["support"], "x": np.asarray(r["x"]), "iters": r["iters"], "gap": r["gap"],
                    "halt": r["halt"], "rn": r["resnorm"][-1] / r["ynorm"] if r["resnorm"] else 0.0,
                    "h": np.stack(r["h"]) if r["h"] else None})
    return out


def _oracle_transform_worker(spec):
    os.environ["OMP_NUM_THREADS"] = "1"
    from oracle import transform as tro
    om, yv = synth.uneven_instance(spec)
    r = tro.omp(spec["kind"], spec["N"], om, yv.astype(np.complex128 if spec["kind"] == "dft" else np.float64),
                spec["K"])
    return {"support": r["support"], "x": np.asarray(r["x"]), "iters": r["iters"], "gap": r["gap"],
            "halt": r["halt"], "rn": r["resnorm"][-1] / r["ynorm"] if r["resnorm"] else 0.0}


def oracle_throughput(inst, idx, cores: int, record: bool = False):
    """Time the FP64 oracle (Algorithm 1.1, dense Phi^H r) on the instances
    `idx` of the batch, spread over `cores` spawned single-threaded
    processes.  Returns (solves/s, wall seconds, per-instance results in the
    order of idx; with `record`, supports, x, ||r||/||y|| and every h)."""
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    idx = list(idx)
    ys = inst["Y"][idx]
    chunks = [list(range(i, len(idx), cores)) for i in range(cores)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_worker, [(inst["kind"], inst["N"], inst["omega"], ys[:0], inst["K"], False)] * cores)  # warm
        t0 = time.perf_counter()
        res = pool.map(_oracle_worker, [(inst["kind"], inst["N"], inst["omega"], ys[c], inst["K"], record)
                                        for c in chunks])
        dt = time.perf_counter() - t0
    out = [None] * len(idx)
    for c, r in zip(chunks, res):
        for i, v in zip(c, r):
            out[i] = v
    return len(idx) / dt, dt, out


def uneven_sample(n_inst: int, count: int = 16, max_work: float = 2e9) -> list[int]:
    """Instances of the uneven batch the transform oracle solves: `count`
    indices spread over the batch among those whose dense least squares
    (M K^3 / 3 flops over a run) stays below max_work, so the oracle leg ends
    in seconds."""
    specs = synth.uneven_batch(n_inst, seed=0)
    ok = [i for i, sp in enumerate(specs) if sp["M"] * sp["K"] ** 3 / 3 <= max_work]
    step = max(1, len(ok) // count)
    return ok[::step][:count]


def oracle_refs(cores: int, n_uneven: int):
    """FP64 oracle results the accuracy report compares with, computed before
    any GPU call: the single WHT FP64 instance, and the sample of the uneven
    batch (transform oracle)."""
    c1 = synth.make_batch(**synth.CONFIG_WHT_FP64_SINGLE)
    ctx = mp.get_context("spawn")
    idx = uneven_sample(n_uneven)
    specs = synth.uneven_batch(n_uneven, seed=0)
    with ctx.Pool(cores) as pool:
        r1 = pool.apply_async(_oracle_worker, [("wht", c1["N"], c1["omega"], c1["Y"], c1["K"], True)])
        ru = pool.map(_oracle_transform_worker, [specs[i] for i in idx])
        r1 = r1.get()[0]
    return {"config1": r1, "uneven": dict(zip(idx, ru))}


def _rel_inf(a, b):
    d = np.max(np.abs(b))
    return float(np.max(np.abs(np.asarray(a) - b)) / (d if d > 0 else 1.0))


def compare_run(ref, supp, iters, x, rn):
    """One instance against its oracle run: support equal up to the first
    near tie (top-two gap <= 1e-3), and where the whole run is comparable the
    iteration count, the l_inf relative x error and the ||r||/||y|| error."""
    near = next((t for t, g in enumerate(ref["gap"]) if g <= 1e-3), len(ref["gap"]))
    got = [int(v) for v in supp[: int(iters)]]
    out = {"support_prefix_equal": got[:near] == list(ref["support"][:near]), "whole_run": near == len(ref["gap"])}
    if out["whole_run"]:
        out["iters_equal"] = int(iters) == int(ref["iters"])
        xr = np.asarray(ref["x"])
        n = min(int(iters), len(xr))
        out["x_err"] = _rel_inf(np.asarray(x)[:n], xr[:n]) if n else 0.0
        out["rn_err"] = abs(float(rn) - float(ref["rn"]))
    return out


def summarize(rows):
    """Worst errors over the compared instances."""
    whole = [r for r in rows if r["whole_run"]]
    return {"instances": len(rows), "support_prefix_equal": sum(r["support_prefix_equal"] for r in rows),
            "whole_runs_compared": len(whole), "iters_equal": sum(r["iters_equal"] for r in whole),
            "x_err_max": max((r["x_err"] for r in whole), default=None),
            "rn_abs_err_max": max((r["rn_err"] for r in whole), default=None)}


# ---------------------------------------------------------------- clock sampler
class ClockSampler:
    FIELDS = "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown," \
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown," \
             "clocks_event_reasons.sw_power_cap"

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 7:
                continue
            try:
                rows.append((float(p[0]), float(p[1]), p[3:7]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------- GPU timing
def correlation_flops(N: int, iters: np.ndarray, t_switch: int, path: str) -> float:
    """FP32 algorithmic flops of the correlations one step performs: one
    transform (5 N log2 N) at t = 1; per later iteration with s atoms either
    the kernel sum (s complex MACs per output = 8 N s flops) or the transform
    path (forward + adjoint transform, 2 x 5 N log2 N)."""
    logn = np.log2(N)
    tr = 5.0 * N * logn
    total = 0.0
    for it in iters.tolist():
        total += tr
        for t in range(2, it + 1):
            s = t - 1
            fast = path == "fast" or (path == "hybrid" and t <= t_switch)
            total += 8.0 * N * s if fast else 2.0 * tr
    return total


def flush_l2(buf):
    import torch
    """Evicts L2: write a buffer twice the L2 size, then read it, leaving L2
    full of clean lines that belong to no input of the timed step."""
    buf.zero_()
    buf.view(torch.float32).sum()  # read back as float32: no widening copy


def _events_ms(fn, steps, warmup, stream, flush=None):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    out = []
    for _ in range(steps):
        if flush is not None:
            flush_l2(flush)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        out.append((e0, e1))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in out]


def secondary(args, dev, plan, inst, stream, flush, refs=None):
    """Measurements beside the headline (not part of the timed step):
    subspace pursuit on the same batch; single-instance latency on the
    partial-WHT FP64 case (N=1024, M=256, K=16, noiseless); fast vs
    transform CoSaMP time per iteration at M=64, N=8192, K=4 (the case the
    paper quotes for CoSaMP, Sec. IV)."""
    import torch
    from paper_1205_4139_gb300 import binding
    from paper_1205_4139_gb300 import costmodel
    out = {}
    B, K = inst["B"], inst["K"]
    y = torch.from_numpy(inst["Y"]).to(dev)
    x = torch.empty(B, K, dtype=torch.complex128, device=dev)
    supp = torch.empty(B, K, dtype=torch.int32, device=dev)
    it = torch.empty(B, dtype=torch.int32, device=dev)
    rn = torch.empty(B, dtype=torch.float64, device=dev)
    ms = _events_ms(lambda: plan.pursuit_into("sp", y, K, x, supp, it, rn, path="fast"), 3, 1, stream, flush)
    out["sp_fast"] = {"solves_per_s": B / (statistics.median(ms) * 1e-3), "ms_per_step_p50": statistics.median(ms),
                      "iters_mean": float(it.float().mean())}

    c1 = dict(synth.CONFIG_WHT_FP64_SINGLE)
    i1 = synth.make_batch(**c1)
    p1 = binding.Plan(c1["N"], i1["omega"], "wht", "fp64")
    y1 = torch.from_numpy(i1["Y"]).to(dev)
    x1 = torch.empty(1, c1["K"], dtype=torch.float64, device=dev)
    s1 = torch.empty(1, c1["K"], dtype=torch.int32, device=dev)
    t1 = torch.empty(1, dtype=torch.int32, device=dev)
    r1 = torch.empty(1, dtype=torch.float64, device=dev)
    lat = {}
    for path in ("fast", "conv", "hybrid"):
        # one solve captured in a CUDA graph, replayed 10^4 times, each
        # replay timed with CUDA events on the replay stream
        gs = torch.cuda.Stream()
        with torch.cuda.stream(gs):
            for _ in range(3):
                p1.omp_into(y1, c1["K"], x1, s1, t1, r1, path=path)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=gs):
            p1.omp_into(y1, c1["K"], x1, s1, t1, r1, path=path)
        torch.cuda.synchronize()
        n_rep = 10000
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_rep)]
        with torch.cuda.stream(gs):
            for e0, e1 in ev:
                e0.record(gs)
                graph.replay()
                e1.record(gs)
        torch.cuda.synchronize()
        v = sorted(1e3 * a.elapsed_time(b) for a, b in ev)
        lat[path] = {"p50_us": statistics.median(v), "p99_us": v[int(0.99 * (len(v) - 1))], "repeats": n_rep}
        assert int(t1.item()) > 0
    out["omp_wht_fp64_single_latency"] = {"config": "partial WHT FP64, N=1024, M=256, K=16, noiseless, 1 instance; "
                                                    "one solve in a CUDA graph, 10^4 replays", **lat}
    if refs and refs.get("config1"):
        r1c = refs["config1"]
        row = compare_run(r1c, s1.cpu().numpy()[0], t1.cpu().numpy()[0], x1.cpu().numpy()[0], r1.cpu().numpy()[0])
        h1, _ = p1.correlate(y1)
        out["omp_wht_fp64_single_latency"]["accuracy"] = {
            **row, "h_err_t1": _rel_inf(h1.cpu().numpy()[0], r1c["h"][0]), "path": "hybrid (last replayed graph)"}

    rng_inst = synth.make_batch("dft", 8192, 64, 4, 256, snr_db=None, prec="fp32", seed=3)
    p3 = binding.Plan(8192, rng_inst["omega"], "dft", "fp32")
    y3 = torch.from_numpy(rng_inst["Y"]).to(dev)
    B3 = y3.shape[0]
    x3 = torch.empty(B3, 4, dtype=torch.complex128, device=dev)
    s3 = torch.empty(B3, 4, dtype=torch.int32, device=dev)
    t3 = torch.empty(B3, dtype=torch.int32, device=dev)
    r3 = torch.empty(B3, dtype=torch.float64, device=dev)
    per_it = {}
    for path in ("fast", "conv"):
        v = _events_ms(lambda: p3.pursuit_into("cosamp", y3, 4, x3, s3, t3, r3, path=path, max_iter=8), 20, 3,
                       stream, flush)
        per_it[path] = statistics.median(v) / max(1.0, float(t3.sum()))
    # the correlation alone, per instance: kernel sums over the K = 4 atoms of
    # an estimate, and one transform (the transform path runs two per
    # iteration: the residual and the correlation)
    h3 = torch.zeros(B3, 8192, dtype=torch.complex64, device=dev)
    sp3 = torch.from_numpy(np.stack([np.sort(np.random.default_rng(b).choice(8192, 4, replace=False))
                                     for b in range(B3)]).astype(np.int32)).to(dev)
    xw3 = torch.ones(B3, 4, dtype=torch.complex64, device=dev)
    corr = {"kernel_sums_s4": statistics.median(_events_ms(lambda: p3.correlate_fast(h3, sp3, xw3, want_h=False),
                                                           20, 3, stream, flush)) / B3,
            "one_transform": statistics.median(_events_ms(lambda: p3.correlate(y3, want_h=False), 20, 3, stream,
                                                          flush)) / B3}
    out["cosamp_M64_N8192_K4"] = {"ms_per_instance_iteration": per_it,
                                  "fast_over_conv": per_it["fast"] / per_it["conv"],
                                  "paper_flop_model": costmodel.cosamp_fast_ratio(8192, 4),
                                  "correlation_ms_per_instance": corr,
                                  "correlation_share_of_iteration": {
                                      "fast": corr["kernel_sums_s4"] / per_it["fast"],
                                      "conv": 2 * corr["one_transform"] / per_it["conv"]}}
    out["wht_fp32_correlate"] = {"N4096": wht_correlate(dev, stream),
                                 "N256": wht_correlate(dev, stream, N=256, M=64, B=1 << 20, tc_default=True)}
    out["large_dft_c64_N4194304_M524288"] = large_single(dev, stream, flush)
    out["serving"] = serving(args.serve_requests)
    out["uneven_batch"] = uneven(args.uneven_instances, refs.get("uneven") if refs else None)
    return out


def wht_correlate(dev, stream, N=4096, M=1024, B=65536, tc_default=False):
    """Batched conventional correlation h = Phi^H r of a partial-WHT FP32 plan
    (cs_correlate), with the radix-16 Hadamard stages as butterflies on the
    CUDA cores (default) and on the tensor cores (CS_PLAN_TENSOR_CORES):
    B residuals of M entries -> B correlations of N entries (inputs and
    outputs about 1.3 GB, beyond L2).  Against HBM: algorithmic bytes per
    correlation = M * 4 (r) + N * 4 (h); the slot map (N * 4) is shared by the
    batch and stays in L2."""
    import torch
    from paper_1205_4139_gb300 import binding
    import ctypes
    rng = np.random.default_rng(9)
    om = synth.draw_omega(N, M, rng)
    r = torch.randn(B, M, dtype=torch.float32, device=dev)
    h = torch.empty(B, N, dtype=torch.float32, device=dev)
    am = torch.empty(B, dtype=torch.int32, device=dev)
    L = binding.load()
    st = ctypes.c_void_p(stream.cuda_stream)
    byts = B * (M * 4 + N * 4)
    hbm = json.load(open(PEAKS_FILE))["hbm_gbs"] if os.path.exists(PEAKS_FILE) else 6800.0
    out = {"workload": f"partial WHT FP32, N={N}, M={M}, {B} residuals, cs_correlate", "bytes": byts}
    names = (("tensor_core_radix16", False), ("tensor_core_radix16_flag", True)) if tc_default else \
        (("cuda_core_butterflies", False), ("tensor_core_radix16", True))
    for name, tc in names:
        plan = binding.Plan(N, om, "wht", "fp32", tensor_cores=tc)

        def call():
            binding._check(L.cs_correlate(plan._h, ctypes.c_void_p(r.data_ptr()), B, ctypes.c_void_p(h.data_ptr()),
                                          ctypes.c_void_p(am.data_ptr()), st))
        ms = statistics.median(_events_ms(call, 10, 3, stream))
        out[name] = {"ms": ms, "correlations_per_s": B / ms * 1e3, "gbs": byts / ms / 1e6,
                     "frac_of_hbm": byts / ms / 1e6 / hbm, "device_error": plan.device_error()}
    return out


def _uneven_gen(spec):
    return synth.uneven_instance(spec)


def uneven(n_inst: int, refs=None):
    """The uneven batch: n_inst instances (4096 by default), N = 2^12 .. 2^16,
    M = N/4 or N/8, K = 8 .. 256, half partial WHT FP32 and half partial DFT
    complex64, each with its own Omega, +-1 or Gaussian nonzeros, noiseless;
    all instances in one cs_omp_batched call (one persistent launch per
    element type and residence: shared-memory N <= 8192, global-memory
    N > 8192).  Plans are built before the timed region; plans, measurements
    and workspaces (several GB) exceed L2."""
    import torch
    from paper_1205_4139_gb300 import binding
    specs = synth.uneven_batch(n_inst, seed=0)
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(16, os.cpu_count() or 1)) as pool:
        data = pool.map(_uneven_gen, specs)
    t0 = time.perf_counter()
    plans = [binding.Plan(sp["N"], om, sp["kind"], "fp32") for sp, (om, yv) in zip(specs, data)]
    torch.cuda.synchronize()
    plan_s = time.perf_counter() - t0
    ys = [torch.from_numpy(yv).cuda() for om, yv in data]
    bt = binding.Batch(plans, ys, [sp["K"] for sp in specs])
    bt.run()
    torch.cuda.synchronize()

    def timed3():
        times = []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            bt.run()
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        return statistics.median(times)
    ms_default = timed3()
    # the project's autotuner: launch shapes per element type and residence,
    # measured on this batch, then the call timed with them
    t0 = time.perf_counter()
    shapes = binding.batch_tune(bt)
    tune_s = time.perf_counter() - t0
    ms = timed3()
    iters = int(bt.iters.sum().item())
    acc = None
    if refs:
        it_n, rn_n = bt.iters.cpu().numpy(), bt.resnorm.cpu().numpy()
        rows = [compare_run(r, bt.supp[i].cpu().numpy(), it_n[i], bt.x[i].cpu().numpy(), rn_n[i])
                for i, r in refs.items()]
        acc = {"sample": f"{len(refs)} instances spread over the batch whose oracle run is short "
                         "(M K^3/3 <= 2e9), transform oracle", **summarize(rows)}
    return {"workload": f"{n_inst} instances, N=2^12..2^16, M=N/4 or N/8, K=8..256, WHT fp32 / DFT c64, "
                        "per-instance Omega, noiseless", "call": "cs_omp_batched", "instances": n_inst,
            "plan_build_s": plan_s, "ms": ms, "solves_per_s": n_inst / ms * 1e3,
            "ms_default_shapes": ms_default, "tuned_shapes": shapes, "tune_s": tune_s,
            "correlations_per_s": iters / ms * 1e3, "iterations": iters,
            "device_error": plans[0].device_error(), "accuracy": acc}


def huge_instance(N=1 << 22, M=1 << 19, K=4096, prefix=32):
    """The one large instance, once: one partial-DFT complex64 instance,
    N = 2^22, M = 2^19, K = 4096, 30 dB, OMP with the FP64 least squares on
    the GPU: hybrid at the switch point tuned on a K = 256 run (the
    headline), then kernel sums throughout and transforms throughout.

    Against the FP64 oracle (Algorithm 1.1 with Phi applied by FFTs; the
    dense oracle cannot hold Phi at this size): OMP's first iterations do not
    depend on K, so the oracle runs the first `prefix` iterations and the GPU
    run is compared on them (support bit-exact up to the first near tie, x of
    a K = prefix run, and the kernel-sum correlation h_s = h_0 - sum x c at
    several s against the oracle's Phi^H r_s).  The whole K = 4096 result is
    checked by properties that hold at any size: K distinct columns, a
    residual orthogonal to them, and the reported residual norm."""
    import torch
    from oracle import transform as tro
    from paper_1205_4139_gb300 import binding
    dev = torch.device("cuda", 0)
    inst = synth.make_batch("dft", N, M, K, 1, snr_db=30, prec="fp32", seed=5)
    plan = binding.Plan(N, inst["omega"], "dft", "fp32")
    y = torch.from_numpy(inst["Y"]).to(dev)
    t_best, _ = plan.tune(y, 256)
    x = torch.empty(1, K, dtype=torch.complex128, device=dev)
    sp = torch.empty(1, K, dtype=torch.int32, device=dev)
    it = torch.empty(1, dtype=torch.int32, device=dev)
    rn = torch.empty(1, dtype=torch.float64, device=dev)

    def timed(path, ts):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        plan.omp_into(y, K, x, sp, it, rn, path=path, t_switch=ts)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    times = {"conv": timed("conv", -1), "fast": timed("fast", -1), "hybrid": timed("hybrid", t_best)}
    ms = times["hybrid"]
    n_it = int(it.item())
    s_ = sp.cpu().numpy()[0][:n_it]
    xv = x.cpu().numpy()[0][:n_it]
    yv = inst["Y"][0].astype(np.complex128)
    r = yv - tro.synthesize("dft", N, inst["omega"], s_, xv)
    h = tro.correlate("dft", N, inst["omega"], r)
    out = {"workload": "partial DFT complex64, N=2^22, M=2^19, K=4096, 30 dB, OMP, FP64 least squares",
           "t_switch": t_best, "ms": ms, "ms_by_path": times, "iters": n_it,
           "distinct_columns": int(len(set(s_.tolist()))),
           "resnorm_reported": float(rn.item()), "resnorm_recomputed": float(np.linalg.norm(r) / np.linalg.norm(yv)),
           "max_abs_h_on_support_over_norm_y": float(np.max(np.abs(h[s_])) / np.linalg.norm(yv)),
           "device_error": plan.device_error()}
    # the first `prefix` iterations against the FP64 oracle
    t0 = time.perf_counter()
    ref = tro.omp("dft", N, inst["omega"], yv, prefix, record_x=True)
    oracle_s = time.perf_counter() - t0
    near = next((t for t, g in enumerate(ref["gap"]) if g <= 1e-3), len(ref["gap"]))
    xp, spp, _, _ = plan.omp(y, prefix, path="hybrid", t_switch=t_best)
    spp = spp.cpu().numpy()[0]
    acc = {"prefix": prefix, "oracle_s": oracle_s, "near_tie_at": near,
           "support_prefix_equal_in_K4096_run": s_[:near].tolist() == ref["support"][:near],
           "support_prefix_equal_in_prefix_run": spp[:near].tolist() == ref["support"][:near]}
    if near >= 1:  # x after the comparable iterations: a K = near run against the oracle's x_near
        xq, _, _, _ = plan.omp(y, near, path="hybrid", t_switch=t_best)
        xr = np.asarray(ref["xs"][near - 1])
        acc["x_err_at_near_tie"] = float(np.max(np.abs(xq.cpu().numpy()[0] - xr)) / np.max(np.abs(xr)))
    h0, _ = plan.correlate(y)
    herr = {}
    for s in sorted({1, 2, 4, 8, 16, 24, prefix - 1}):
        if s > near or s >= prefix:
            continue
        xs, ss, _, _ = plan.omp(y, s, path="fast")
        hs, _ = plan.correlate_fast(h0, ss, xs.to(torch.complex64).contiguous())
        r_s = yv - tro.synthesize("dft", N, inst["omega"], ref["support"][:s], ref["xs"][s - 1])
        want = tro.correlate("dft", N, inst["omega"], r_s)
        herr[str(s)] = float(np.max(np.abs(hs.cpu().numpy()[0] - want)) / np.max(np.abs(want)))
    want0 = tro.correlate("dft", N, inst["omega"], yv)
    herr["0"] = float(np.max(np.abs(h0.cpu().numpy()[0] - want0)) / np.max(np.abs(want0)))
    acc["h_err_by_atoms"] = herr
    out["accuracy_vs_oracle"] = acc
    return out


def _serving_gen(req):
    return synth.serving_instance(req)


def serving(n_req: int, rate: float = 2000.0, workers: int = 16, budget_gb: float = 64.0):
    """The serving workload: Poisson arrivals at 2000 requests/s, N = 2^14 ..
    2^20, M = N/8, K = 32 .. 1024, partial WHT or DFT by a coin, FP32, OMP
    (hybrid switch) or CoSaMP by a coin (CoSaMP's K capped at M/3, the most
    its least squares allow), each request with its own Omega, replayed in
    real time into the request runtime (cs_server_*) with `workers` streams
    and a device-memory budget; latency = completion - arrival.  The same
    requests are then replayed at half the throughput measured at the
    offered rate (a sustainable rate) for the unsaturated latency.  An
    untimed replay of the first requests at once comes first: the first
    solves of each plan size in a process pay one-off costs (growing the
    stream-ordered memory pool, first launches of each kernel) that a
    running server has paid."""
    from paper_1205_4139_gb300 import binding
    reqs = synth.serving_requests(n_req, rate=rate, seed=0)
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(16, os.cpu_count() or 1)) as pool:
        data = pool.map(_serving_gen, reqs)
    q = lambda v, f: v[min(len(v) - 1, int(f * (len(v) - 1) + 0.5))]

    def replay(scale, n=None):
        n = len(reqs) if n is None else n
        srv = binding.Server(workers=workers, budget_bytes=int(budget_gb * (1 << 30)))
        for kind in ("wht", "dft"):  # warm-up: one small job per kind
            w = synth.serving_requests(1, seed=99, log_n_lo=14, log_n_hi=14, k_lo=32, k_hi=32)[0]
            w["kind"] = kind
            om, yv = synth.serving_instance(w)
            srv.submit(kind, "fp32", w["N"], om, yv, w["K"])
        srv.wait_all()
        t0 = time.perf_counter()
        for r, (om, yv) in zip(reqs[:n], data[:n]):
            dt = r["arrival_s"] * scale - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            srv.submit(r["kind"], "fp32", r["N"], om, yv, r["K"], algo=r["algo"])
        res = srv.wait_all()
        srv.close()
        lat = sorted((r["t_done_us"] - r["t_submit_us"]) * 1e-3 for r in res)
        wait = sorted((r["t_admit_us"] - r["t_submit_us"]) * 1e-3 for r in res)
        span = (max(r["t_done_us"] for r in res) - min(r["t_submit_us"] for r in res)) * 1e-6
        offered = len(res) / (reqs[n - 1]["arrival_s"] * scale) if scale > 0 else None
        return {"offered_per_s": offered, "requests": len(res),
                "failed": sum(1 for r in res if r["status"] != 0 or r["device_error"] != 0),
                "solves_per_s": len(res) / span, "latency_ms_p50": q(lat, 0.5), "latency_ms_p99": q(lat, 0.99),
                "queue_wait_ms_p50": q(wait, 0.5), "makespan_s": span}

    replay(0.0, min(len(reqs), 160))  # warm-up: the first requests at once, untimed
    sat = replay(1.0)
    sus = replay(rate / max(1e-9, 0.5 * sat["solves_per_s"]))
    return {"workload": f"{n_req} requests, Poisson, N=2^14..2^20, M=N/8, K=32..1024, WHT/DFT fp32, "
                        "OMP or CoSaMP (CoSaMP K capped at M/3)",
            "workers": workers, "budget_gb": budget_gb, "at_offered_rate": sat, "at_half_saturation": sus}


def large_single(dev, stream, flush, N=1 << 22, M=1 << 19, K=256):
    """One large partial-DFT complex64 instance (30 dB, N = 2^22, M = 2^19,
    K = 256): the transform h_0 = Phi^H y against the HBM roofline, the
    kernel-sum correlation at several support sizes s against L2 traffic,
    and OMP by each path (transforms four-step through global memory)."""
    import torch
    from paper_1205_4139_gb300 import binding
    inst = synth.make_batch("dft", N, M, K, 1, snr_db=30, prec="fp32", seed=5)
    t0 = time.perf_counter()
    plan = binding.Plan(N, inst["omega"], "dft", "fp32")
    plan_ms = (time.perf_counter() - t0) * 1e3
    y = torch.from_numpy(inst["Y"]).to(dev)
    hbm = json.load(open(PEAKS_FILE))["hbm_gbs"] if os.path.exists(PEAKS_FILE) else 6800.0
    out = {"plan_ms": plan_ms, "hbm_peak_gbs": hbm}
    h = torch.empty(1, N, dtype=torch.complex64, device=dev)
    am = torch.empty(1, dtype=torch.int32, device=dev)
    ms = statistics.median(_events_ms(lambda: plan.correlate(y), 20, 3, stream, flush))
    # two passes, each reads and writes N complex64; pass 1 also reads the
    # slot map (4 B per position) and y
    byts = 2 * 2 * 8 * N + 4 * N + 8 * M
    out["transform_h0"] = {"ms": ms, "bytes": byts, "gbs": byts / ms / 1e6, "frac_of_hbm": byts / ms / 1e6 / hbm}
    rng = np.random.default_rng(1)
    fast = {}
    for s_ in (8, 32, 128):
        sp = torch.from_numpy(rng.choice(N, s_, replace=False).astype(np.int32)[None]).to(dev)
        xs = torch.from_numpy((rng.standard_normal(s_) + 1j * rng.standard_normal(s_)).astype(np.complex64)[None]).to(dev)
        ms = statistics.median(_events_ms(lambda: plan.correlate_fast(h, sp, xs, want_h=False), 20, 3, stream, flush))
        l2 = (s_ + 1) * 8 * N
        fast[str(s_)] = {"ms": ms, "l2_gbs": l2 / ms / 1e6, "gcmac_per_s": s_ * N / ms / 1e6}
    out["kernel_sums"] = fast
    x = torch.empty(1, K, dtype=torch.complex128, device=dev)
    sp = torch.empty(1, K, dtype=torch.int32, device=dev)
    it = torch.empty(1, dtype=torch.int32, device=dev)
    rn = torch.empty(1, dtype=torch.float64, device=dev)
    omp = {}
    for path in ("fast", "conv"):
        omp[path] = statistics.median(_events_ms(lambda: plan.omp_into(y, K, x, sp, it, rn, path=path), 3, 1, stream))
    t_best, curve = plan.tune(y, K)
    omp["hybrid_tuned"] = statistics.median(_events_ms(lambda: plan.omp_into(y, K, x, sp, it, rn, path="hybrid"), 3, 1,
                                                       stream))
    out["omp_ms"] = omp
    out["t_switch"] = t_best
    out["t_switch_curve_ms"] = {str(k): round(v, 3) for k, v in curve.items()}
    out["iters"] = int(it.item())
    return out


def accuracy_batch(plan, inst, y_dev, outs, refs, t_switch: int):
    """Errors of the timed step against the FP64 oracle on the SAMPLE
    instances: supports, iteration counts, x and ||r||/||y|| of the hybrid
    step's outputs; h at t = 1 (cs_correlate) and the kernel-sum correlation
    with s = 1 .. K-1 columns (cs_correlate_fast on the GPU's own first s
    columns and coefficients, which cs_omp with K = s returns), each as
    l_inf / ||h||_inf against the oracle's h with s columns."""
    import torch
    x, supp, iters, rn = (t.cpu().numpy() for t in outs)
    rows = [compare_run(refs[i], supp[b], iters[b], x[b], rn[b]) for i, b in enumerate(SAMPLE)]
    K = inst["K"]
    ys = y_dev[torch.tensor(SAMPLE, device=y_dev.device)].contiguous()
    h0, _ = plan.correlate(ys)
    h0n = h0.cpu().numpy()
    h_t1 = max(_rel_inf(h0n[i], refs[i]["h"][0]) for i in range(len(SAMPLE)))
    per_s = {}
    for s_ in range(1, K):
        xs, sp, _, _ = plan.omp(ys, s_, path="fast")
        h, _ = plan.correlate_fast(h0, sp, xs.to(h0.dtype).contiguous())
        hn, spn = h.cpu().numpy(), sp.cpu().numpy()
        errs = [_rel_inf(hn[i], refs[i]["h"][s_]) for i in range(len(SAMPLE))
                if len(refs[i]["h"]) > s_ and spn[i].tolist() == list(refs[i]["support"][:s_])]
        if errs:
            per_s[s_] = max(errs)
    s_sw = min(t_switch, K) - 1
    return {"sample": f"{len(SAMPLE)} of the 1024 instances (indices {SAMPLE[0]}..{SAMPLE[-1]}, slots reused "
                      "past 607)", **summarize(rows),
            "h_err_t1": h_t1, "h_err_at_switch": per_s.get(s_sw), "switch_atoms": s_sw,
            "h_err_kernel_sum_max": max(per_s.values()) if per_s else None,
            "h_err_kernel_sum_worst_s": max(per_s, key=per_s.get) if per_s else None,
            "h_err_definition": "l_inf(h_gpu - h_oracle) / l_inf(h_oracle), same columns and the GPU's coefficients"}


def run_gpu(args, rank: int, world: int, refs=None):
    import torch
    from paper_1205_4139_gb300 import binding, replicas

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    cfg = dict(CFG)
    B, N, M, K = cfg["B"], cfg["N"], cfg["M"], cfg["K"]
    cfg["seed"] = replicas.shard_seed(rank, B)  # rank r solves global instances r*B .. r*B+B-1
    inst = synth.make_batch(**{**cfg, "omega_seed": 0})

    t0 = time.perf_counter()
    plan = binding.Plan(N, inst["omega"], "dft", "fp32")
    plan_ms = (time.perf_counter() - t0) * 1e3
    stream = torch.cuda.current_stream()
    y = torch.from_numpy(inst["Y"]).to(dev)
    x = torch.empty(B, K, dtype=torch.complex128, device=dev)
    supp = torch.empty(B, K, dtype=torch.int32, device=dev)
    iters = torch.empty(B, dtype=torch.int32, device=dev)
    rn = torch.empty(B, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device=dev)

    def step(path, ts):
        plan.omp_into(y, K, x, supp, iters, rn, rel_tol=1e-6, path=path, t_switch=ts)

    def timed(path, ts, steps, warmup):
        for _ in range(warmup):
            step(path, ts)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for e0, e1 in ev:
            flush_l2(flush)
            e0.record(stream)
            step(path, ts)
            e1.record(stream)
        torch.cuda.synchronize()
        return [e0.elapsed_time(e1) for e0, e1 in ev]

    # switch point: the flop-model default of Table I, and the one the
    # library's tuner (cs_plan_tune) measures on this batch, checked below
    # under the benchmark's own protocol
    default_ts = plan.info()["t_switch_default"]
    with ClockSampler(dev.index if dev.index is not None else 0) as clk:
        best_ts, tune = plan.tune(y, K, rel_tol=1e-6)
        fast_ms = timed("fast", -1, max(10, args.steps // 4), args.warmup)
        conv_ms = timed("conv", -1, max(10, args.steps // 4), args.warmup)
        # the tuner times back to back; under this benchmark's protocol (L2
        # flushed before every step) the hybrid at its point is checked
        # against the hybrid at K (kernel sums throughout, the fast path
        # timed just above) and the faster one is the headline switch point
        tuned_ts = best_ts
        probe_ms = timed("hybrid", tuned_ts, max(10, args.steps // 4), args.warmup)
        if statistics.median(fast_ms) < statistics.median(probe_ms):
            best_ts = K
        ts_check = {"tuned": tuned_ts, "hybrid_at_tuned_ms_p50": statistics.median(probe_ms),
                    "hybrid_at_K_ms_p50": statistics.median(fast_ms), "used": best_ts}
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        hyb_ms = timed("hybrid", best_ts, args.steps, args.warmup)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
    it_np = iters.cpu().numpy()
    total_ms = float(sum(hyb_ms))

    # end to end through the same C ABI with host buffers
    y_host = torch.from_numpy(inst["Y"]).pin_memory()
    outs_host = [torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in (x, supp, iters, rn)]
    y_dev = torch.empty_like(y)

    def e2e_step():
        y_dev.copy_(y_host, non_blocking=True)
        plan.omp_into(y_dev, K, x, supp, iters, rn, rel_tol=1e-6, path="hybrid", t_switch=best_ts)
        for h, d in zip(outs_host, (x, supp, iters, rn)):
            h.copy_(d, non_blocking=True)

    for _ in range(args.warmup):
        e2e_step()
    torch.cuda.synchronize()
    e2e_ev = []
    for _ in range(max(10, args.steps // 4)):
        flush_l2(flush)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        e2e_step()
        e1.record(stream)
        e2e_ev.append((e0, e1))
    torch.cuda.synchronize()
    e2e_ms = [a.elapsed_time(b) for a, b in e2e_ev]
    h2d = y.numel() * y.element_size()
    d2h = sum(t.numel() * t.element_size() for t in (x, supp, iters, rn))

    acc = None
    if rank == 0 and refs is not None and refs.get("config2") is not None:
        step("hybrid", best_ts)
        acc = accuracy_batch(plan, inst, y, (x, supp, iters, rn), refs["config2"], best_ts)
    extra = secondary(args, dev, plan, inst, stream, flush, refs) if (rank == 0 and not args.no_extra) else {}

    # max over ranks
    total_ms, e2e_mean, fast_med, conv_med = replicas.max_over_ranks(
        [total_ms, sum(e2e_ms) / len(e2e_ms), statistics.median(fast_ms), statistics.median(conv_ms)], dev)

    # FP32 FMA-pipe peak measured in this run (cs_fma_probe), beside the
    # figure derived from unit counts and the maximum clock
    probe = []
    for _ in range(6):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fl = binding.fma_probe(1 << 14, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        probe.append(fl / (e0.elapsed_time(e1) * 1e-3) / 1e12)
    fp32_measured = max(probe[1:])

    flops = correlation_flops(N, it_np, best_ts, "hybrid")
    per_launch_ms = total_ms / args.steps
    achieved = flops / (per_launch_ms * 1e-3) / 1e12
    solves = B * world * args.steps / (total_ms * 1e-3)
    corr = float(it_np.sum()) * world * args.steps / (total_ms * 1e-3)
    hs = sorted(hyb_ms)
    return {
        "value": solves, "ms_per_step": total_ms / args.steps,
        "p50_ms": statistics.median(hs), "p99_ms": hs[min(len(hs) - 1, int(0.99 * len(hs)))],
        "correlations_per_s": corr, "plan_ms": plan_ms, "t_switch": best_ts, "t_switch_default": default_ts,
        "t_switch_sweep_ms": {str(k): round(v, 4) for k, v in tune.items()}, "t_switch_check": ts_check,
        "fast": {"solves_per_s": B * world / (fast_med * 1e-3), "ms_per_step_p50": fast_med,
                 "frac_of_fp32_peak": correlation_flops(N, it_np, best_ts, "fast") / (fast_med * 1e-3) / 1e12
                 / fp32_measured},
        "conv": {"solves_per_s": B * world / (conv_med * 1e-3), "ms_per_step_p50": conv_med,
                 "frac_of_fp32_peak": correlation_flops(N, it_np, best_ts, "conv") / (conv_med * 1e-3) / 1e12
                 / fp32_measured},
        "e2e": {"value": B * world / (e2e_mean * 1e-3), "unit": "solves/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_measured, "unit": "TFLOP/s",
                     "frac": achieved / fp32_measured, "traffic": None,
                     "peak_source": "FP32 FMA pipe measured in this run (cs_fma_probe, best of 5)",
                     "peak_derived": FP32_PEAK_TFLOPS, "frac_of_derived": achieved / FP32_PEAK_TFLOPS},
        "clocks": clk.summary(),
        "gpu_launches": args.steps,
        "iters_mean": float(it_np.mean()),
        "accuracy": acc,
        "extra": extra,
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--serve-requests", type=int, default=2000, help="requests in the serving measurement")
    ap.add_argument("--uneven-instances", type=int, default=4096, help="instances of the uneven-batch measurement")
    ap.add_argument("--huge", action="store_true",
                    help="run only the one partial-DFT instance N=2^22, M=2^19, K=4096, 30 dB")
    ap.add_argument("--no-extra", action="store_true", help="skip the secondary measurements")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    cores = len(os.sched_getaffinity(0))

    if args.huge:
        print(json.dumps(huge_instance()))
        return

    if args.impl == "reference":
        # The reference arm is the FP64 oracle, timed on the host cores,
        # rank 0 only; each step is a bounded sample of the same workload.
        if rank != 0:
            return
        inst = synth.make_batch(**{**CFG, "B": cores})
        budget_s, t_start = 150.0, time.perf_counter()
        for _ in range(min(args.warmup, 3)):
            oracle_throughput(inst, range(cores), cores)
        vals = []
        while len(vals) < args.steps and (not vals or time.perf_counter() - t_start < budget_s):
            vals.append(oracle_throughput(inst, range(cores), cores)[0])
        v = statistics.median(vals)
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": args.gpus,
                "steps": len(vals), "steps_requested": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * cores / v,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic (seeded)",
                "config": {"workload": WORKLOAD, "kind": "dft", "N": 4096, "M": 1024, "K": 64, "batch": 1024,
                           "snr_db": 40},
                "cpu_baseline": {"value": v, "unit": "solves/s", "cores": cores, "kind": "oracle",
                                 "sample": f"{cores} instances per step, one per core; at most "
                                           f"{int(budget_s)} s of steps"},
                "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    # CPU baseline first (spawned pool, before any GPU call), rank 0 at N=1 only
    cpu, refs = None, None
    if rank == 0 and world == 1:
        inst0 = synth.make_batch(**CFG)
        v, dt, res = oracle_throughput(inst0, SAMPLE, cores, record=True)
        cpu = {"value": v, "unit": "solves/s", "cores": cores, "kind": "oracle",
               "sample": f"{len(SAMPLE)} of the 1024 instances (indices {SAMPLE[0]}..{SAMPLE[-1]}), FP64 dense "
                         f"Algorithm 1.1, {dt:.1f} s wall"}
        refs = {"config2": res}
        if not args.no_extra:
            refs.update(oracle_refs(cores, args.uneven_instances))

    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    r = run_gpu(args, rank, world, refs)
    if rank == 0:
        line = {"metric": METRIC, "value": r["value"], "unit": "solves/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "c64 correlation / f64 least squares",
                "data": "synthetic (seeded)",
                "config": {"workload": WORKLOAD, "kind": "dft", "N": 4096, "M": 1024, "K": 64,
                           "batch_per_gpu": 1024, "snr_db": 40, "path": "hybrid", "t_switch": r["t_switch"],
                           "l2": "flushed (256 MB write, then read) before every timed step"},
                "p50_ms": r["p50_ms"], "p99_ms": r["p99_ms"], "correlations_per_s": r["correlations_per_s"],
                "fast": r["fast"], "conv": r["conv"], "plan_ms": r["plan_ms"],
                "t_switch_default": r["t_switch_default"], "t_switch_sweep_ms": r["t_switch_sweep_ms"],
                "t_switch_check": r["t_switch_check"], "e2e": r["e2e"], "roofline": r["roofline"], "cpu_baseline": cpu, "accuracy": r["accuracy"],
                "clocks": r["clocks"],
                "gpu_launches": r["gpu_launches"], "secondary": r["extra"]}
        print(json.dumps(line))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
