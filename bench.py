#!/usr/bin/env python
"""Benchmark of the Gaussian-sum nonlocal-potential apply on GB300.

Workload: 3D Coulomb potential on [-12,12]^3, 256^3 grid, FP64, seeded mixture
of 8 anisotropic Gaussians (centres U[-3,3]^3, widths U[0.5,1.5], amplitudes
U[0.5,2], seed 20150104).  A step is one apply u = U * rho (Algorithm 1,
"Actual computation": the five FFT passes with the multiplier; the
precomputation is excluded, as in the paper).  Metric: grid points per second
(Mpts/s), whole job.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

N > 1 (torchrun): replicas, one independent apply per rank, no collective in
the data path ("scaling": "weak"); the time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "3D Coulomb 256^3 FP64 Mpts/s at <=1e-12 rel err; HBM roofline fraction"
UNIT = "Mpts/s"
L_BOX = 12.0
FP64_PEAK_TFLOPS = 1.25     # 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz (nominal)
FP32_PEAK_TFLOPS = 80.5     # 152 SMs x 128 FP32 FMA/clk x 2 flop x 2.07 GHz (nominal)
PASS_NAMES_3D = ["xf", "yf", "conv", "yi", "xi"]


def args_parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gsm", "reference"], default="gsm")
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32x2", "fp32"])
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-n", type=int, default=128, help="grid of the reference arm's bounded sample")
    ap.add_argument("--suite", action="store_true",
                    help="measure every config (one JSON line each) instead of the headline line")
    ap.add_argument("--configs", default="1,2,3,4,5", help="with --suite: which configs to run (comma list)")
    ap.add_argument("--passes", default=None, metavar="KERNEL:PRECISION:N",
                    help="time the passes of one tuned plan (e.g. poisson2d:fp64:4096) instead of the headline line")
    return ap.parse_args()


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.rows = []
        if self.proc is None:
            return False
        time.sleep(0.3)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        for row in csv.reader(io.StringIO(out)):
            if len(row) >= 9:
                self.rows.append([c.strip() for c in row])
        return False

    def summary(self):
        rows = getattr(self, "rows", [])
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        loaded = [s for s in sm if s > 0.5 * max(sm)] if sm else []
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# ------------------------------------------------------------------ models
def conv_pass_model(n: int, cbytes: int):
    """Algorithmic work of the z pass (forward FFT, multiply, inverse FFT of
    length M = 2n on (n+1) M pencils): radix-2 flop count 5 M log2 M per
    complex FFT, 2 flops per real-by-complex product; bytes: n complex in and
    out per pencil plus the octant multiplier once."""
    M = 2 * n
    lines = (n + 1) * M
    flops = lines * (2 * 5 * M * np.log2(M) + 2 * M)
    mbytes = 8 if cbytes == 16 else 4
    bytes_ = 2 * cbytes * n * lines + mbytes * (n + 1) ** 3
    return float(flops), float(bytes_)


def apply_model(n: int, cbytes: int):
    """Whole apply: radix-2 flops 70 n^3 log2(2n) (pruning ignored); bytes of the
    minimal padded-FFT pass count (three HBM round trips of the pruned half
    spectrum plus rho, u and the multiplier): for FP64 16 n^3 + 128 (n+1) n^2 +
    8 (n+1)^3."""
    flops = 70.0 * n ** 3 * np.log2(2 * n)
    rb = cbytes // 2
    bytes_ = 2 * rb * n ** 3 + 8 * cbytes * (n + 1) * n * n + rb * (n + 1) ** 3
    return float(flops), float(bytes_)


def kernel_source_hash():
    """Hash of the source that fixes the conv kernel's memory traffic: the FFT
    engine and arithmetic headers and the conv section of the pass file."""
    csrc = os.path.join(ROOT, "paper_1501_04438_gb300", "csrc")
    h = hashlib.sha256()
    for name in ("gsm_fft.cuh", "gsm_arith.cuh"):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(f.read())
    src = open(os.path.join(csrc, "gsm_passes.cu")).read()
    a = src.index("// ------------------------------------------------------------------ pass conv")
    b = src.index("// ------------------------------------------------------------------ pass yi")
    h.update(src[a:b].encode())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str, precision: str):
    """DRAM bytes per launch from the committed ncu summary, only if the kernel
    sources are unchanged since the capture."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
        e = t["kernels"][f"{kernel}:{precision}"]
        if e.get("source_hash", t.get("source_hash")) == kernel_source_hash():
            return e["dram_bytes_per_launch_full_size"]
    except Exception:
        pass
    return None


# ------------------------------------------------------------------ timing
def time_passes(torch, plan, rho, u, steps, flush, stream):
    """K steps; each step is the apply's passes launched one by one with CUDA
    events between them on the launching stream; L2 is flushed between steps
    (outside the events).  Returns per-step and per-pass milliseconds."""
    npass = plan.info()["npasses"]
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(npass + 1)] for _ in range(steps)]
    with torch.cuda.stream(stream):
        for k in range(steps):
            flush.zero_()
            evs[k][0].record(stream)
            for p in range(npass):
                plan.apply_pass(p, rho if p == 0 else None, u if p == npass - 1 else None, stream=stream)
                evs[k][p + 1].record(stream)
    torch.cuda.synchronize()
    step_ms = [evs[k][0].elapsed_time(evs[k][npass]) for k in range(steps)]
    pass_ms = [[evs[k][p].elapsed_time(evs[k][p + 1]) for k in range(steps)] for p in range(npass)]
    return step_ms, pass_ms


def relmax(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


# ------------------------------------------------------------------ multi-rank host logic
def max_over_ranks(x: float, device) -> float:
    """Maximum of a per-rank float over all ranks of the default process group
    (the value itself when there is no group): every rank gets the same result."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(points_per_rank: int, world: int, total_ms_max: float, steps: int):
    """(ms per step, whole-job Mpts/s): every rank applies its own replica, so the
    job processes world * points_per_rank points per step in the slowest rank's time."""
    ms_per_step = total_ms_max / steps
    return ms_per_step, world * points_per_rank / (ms_per_step / 1e3) / 1e6


# ------------------------------------------------------------------ reference arm
def run_reference(a, rank, world):
    """The CPU oracle, as it stands, on the host cores: each step is one apply
    (plan excluded) on a bounded sample of the workload, the same mixture on a
    coarser grid (a.ref_n^3)."""
    if rank != 0:
        return
    import oracle
    from paper_1501_04438_gb300 import workloads as wl
    n = a.ref_n
    rho = wl.coulomb3d_mixture(n, L_BOX)
    prep = oracle.Prepared("coulomb3d", n, L_BOX)
    for _ in range(a.warmup):
        prep.run(rho)
    t0 = time.perf_counter()
    for _ in range(a.steps):
        prep.run(rho)
    dt = (time.perf_counter() - t0) / a.steps
    value = n ** 3 / dt / 1e6
    cores = oracle.max_threads()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"coulomb3d mixture8 L=12 sample {n}^3 (of 256^3)", "kernel": "coulomb3d",
                       "grid": n, "L": L_BOX, "precision": "fp64"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{n}^3 instance of the same seeded mixture, apply only (plan excluded)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ main arm
def main():
    a = args_parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        run_reference(a, rank, world)
        return

    import torch
    import torch.distributed as dist

    import paper_1501_04438_gb300 as gsm
    from paper_1501_04438_gb300 import workloads as wl

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    n = a.n
    prec = a.precision
    dt_io = torch.float32 if prec == "fp32" else torch.float64
    cbytes = 8 if prec == "fp32" else 16

    rho_h = wl.coulomb3d_mixture(n, L_BOX)
    rho = torch.tensor(rho_h, dtype=dt_io, device=dev)
    u = torch.empty_like(rho)
    stream = torch.cuda.Stream(device=dev)
    plan = gsm.Plan("coulomb3d", L_BOX, n, precision=prec, stream=stream)
    tune_report = plan.autotune(stream=stream)   # part of the plan: launch shapes by measurement
    info = plan.info()
    npass = info["npasses"]
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)   # > L2 (129 MiB)

    # warm-up
    time_passes(torch, plan, rho, u, max(1, a.warmup), flush, stream)

    # timed region
    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    barrier()
    with ClockSampler(local) as clk:
        t_wall0 = time.perf_counter()
        step_ms, pass_ms = time_passes(torch, plan, rho, u, a.steps, flush, stream)
        barrier()
        t_wall = time.perf_counter() - t_wall0
    clocks = clk.summary()
    total_ms = max_over_ranks(float(sum(step_ms)), dev)
    ms_per_step, value = job_throughput(n ** 3, world, total_ms, a.steps)

    # dominant kernel and its roofline
    avg_pass = [float(np.mean(x)) for x in pass_ms]
    dom = int(np.argmax(avg_pass))
    dom_name = PASS_NAMES_3D[dom]
    peaks = load_peaks()
    # the driver's measured copy bandwidth; without that file the recipe's fallback figure
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    hbm_src = "of measured" if "hbm_gbs" in peaks else "of fallback"
    f_conv, b_conv = conv_pass_model(n, cbytes)
    f_app, b_app = apply_model(n, cbytes)
    if dom_name == "conv":
        alg_flops, alg_bytes = f_conv, b_conv
    else:
        alg_flops, alg_bytes = None, None
    dom_s = avg_pass[dom] / 1e3
    if prec == "fp32":
        roof = {"bound": "hbm", "achieved": (alg_bytes or b_app) / dom_s / 1e9, "peak": hbm_peak,
                "unit": "GB/s"}
    else:
        peak = FP64_PEAK_TFLOPS if prec == "fp64" else FP32_PEAK_TFLOPS
        roof = {"bound": "alu", "achieved": (alg_flops or f_app) / dom_s / 1e12, "peak": peak,
                "unit": "TFLOP/s"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = profiled_traffic(dom_name, prec)
    roof["kernel"] = f"k_{dom_name} (pass {dom} of {npass})"
    roof["peak_source"] = ("FP64 pipe: 152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz (recipe nominal 1.25 TFLOP/s); "
                           "measured DFMA probe 1.20 TFLOP/s at 2.0 GHz" if prec == "fp64" else
                           ("FP32 pipe nominal (double-float arithmetic)" if prec == "fp32x2" else
                            ("measured HBM copy, MEASURED_PEAKS.json" if "hbm_gbs" in peaks else
                             "fallback HBM figure 6.8 TB/s (no MEASURED_PEAKS.json)")))
    # the five passes as built move 12 (instead of 8) half-spectrum slabs
    b_5 = b_app + 4 * cbytes * (n + 1) * n * n
    hbm_whole = {"bytes_model": b_app, "achieved_gbs": b_app / (ms_per_step / 1e3) / 1e9, "peak_gbs": hbm_peak,
                 "frac": b_app / (ms_per_step / 1e3) / 1e9 / hbm_peak, "peak_source": hbm_src,
                 "bytes_model_5pass": float(b_5), "frac_5pass": b_5 / (ms_per_step / 1e3) / 1e9 / hbm_peak}

    result = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
              "warmup": a.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
              "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32", "fp32x2": "f32x2"}[prec],
              "data": "synthetic",
              "config": {"workload": f"coulomb3d {n}^3 L=12 mixture8 seed 20150104", "kernel": "coulomb3d",
                         "grid": n, "L": L_BOX, "precision": prec, "S": info["S"], "nterms": info["nterms"],
                         "parallelism": f"replicas x{world}" if world > 1 else "single",
                         "l2": "flushed between steps (512 MiB write, outside the events)"},
              "roofline": roof, "hbm_whole_apply": hbm_whole,
              "passes_ms": {PASS_NAMES_3D[p]: avg_pass[p] for p in range(npass)},
              "gpu_launches": a.steps * npass, "clocks": clocks, "wall_s_timed": t_wall,
              "launch_shapes": {PASS_NAMES_3D[p]: {"lines_per_cta": info["launch_nl"][p],
                                                   "threads_per_line": info["launch_threads"][p],
                                                   "elems_per_thread": info["launch_emax"][p]}
                                for p in range(npass)}}
    if os.environ.get("GSM_BENCH_TUNE_REPORT"):
        with open(os.environ["GSM_BENCH_TUNE_REPORT"], "w") as f:
            f.write(tune_report)

    if rank == 0:
        # e2e: host buffers through the C interface, copies inside the timed region
        npd = np.float32 if prec == "fp32" else np.float64
        pin_in = torch.empty(rho.shape, dtype=dt_io, pin_memory=True).numpy()
        pin_out = torch.empty(rho.shape, dtype=dt_io, pin_memory=True).numpy()
        pin_in[...] = rho_h.astype(npd)
        for _ in range(2):
            plan.apply_host(pin_in, pin_out, stream=stream)
        k_e2e = max(3, min(a.steps, 10))
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            plan.apply_host(pin_in, pin_out, stream=stream)
        t_e2e = (time.perf_counter() - t0) / k_e2e
        nbytes = int(pin_in.nbytes)
        result["e2e"] = {"value": n ** 3 / t_e2e / 1e6, "unit": UNIT, "h2d_bytes_per_step": nbytes,
                         "d2h_bytes_per_step": nbytes, "ms_per_step": t_e2e * 1e3,
                         "call": "gsm_apply_host (pinned host arrays)"}
        u_gpu = u.double().cpu().numpy()

        # oracle at full size: CPU baseline and full-size parity
        u_oracle = None
        if not a.no_cpu_baseline and world == 1:
            import oracle
            t0 = time.perf_counter()
            prep = oracle.Prepared("coulomb3d", n, L_BOX)
            t_prep = time.perf_counter() - t0
            t0 = time.perf_counter()
            u_oracle = prep.run(rho_h)
            t_run = time.perf_counter() - t0
            result["cpu_baseline"] = {"value": n ** 3 / t_run / 1e6, "unit": UNIT, "cores": oracle.max_threads(),
                                      "kind": "oracle",
                                      "sample": f"one apply of the full {n}^3 workload (plan excluded, "
                                                f"{t_prep:.1f} s)",
                                      "seconds": t_run}
            result["parity"] = {"rel_err_vs_oracle": relmax(u_gpu, u_oracle), "tolerance": 1e-12,
                                "oracle": "taylor_mode 0 (literal Algorithm 1)"}

        # reduced / split precision forms of the same apply
        if not a.no_variants and prec == "fp64":
            variants = {}
            for vp in ("fp32x2", "fp32"):
                vdt = torch.float32 if vp == "fp32" else torch.float64
                vp_plan = gsm.Plan("coulomb3d", L_BOX, n, precision=vp, stream=stream)
                vp_plan.autotune(stream=stream)
                vr = rho.to(vdt)
                vu = torch.empty_like(vr)
                time_passes(torch, vp_plan, vr, vu, 2, flush, stream)
                sm_, pm_ = time_passes(torch, vp_plan, vr, vu, max(3, a.steps), flush, stream)
                ms = float(np.mean(sm_))
                uv = vu.double().cpu().numpy()
                ref = u_oracle if u_oracle is not None else u_gpu
                vcb = 8 if vp == "fp32" else 16
                _, vb = apply_model(n, vcb)
                vb5 = vb + 4 * vcb * (n + 1) * n * n
                variants[vp] = {"value": n ** 3 / (ms / 1e3) / 1e6, "unit": UNIT, "ms_per_step": ms,
                                "hbm_frac": vb / (ms / 1e3) / 1e9 / hbm_peak,
                                "hbm_frac_5pass": vb5 / (ms / 1e3) / 1e9 / hbm_peak,
                                "rel_err": relmax(uv, ref),
                                "rel_err_vs": "oracle" if u_oracle is not None else "gpu fp64",
                                "passes_ms": {PASS_NAMES_3D[p]: float(np.mean(pm_[p])) for p in range(npass)}}
                vp_plan.destroy()
            result["variants"] = variants
            result["tc_dft32_stage"] = tc_stage_measure(torch, gsm, n, stream, flush)
        print(json.dumps(result), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


# ------------------------------------------------------------------ tensor-core DFT stage
def tc_stage_measure(torch, gsm, n, stream, flush):
    """The length-32 DFT stage of the conv pass's forward transforms (a
    padded line of 2n = 512 as 16 x 32: (n + 1) 2n lines, 16 vectors of 32
    each) three ways: on the tensor cores with FP64-class digit planes
    (gsm_dft32_tc), and through the FFT engine in FP64 and in FP32x2
    (gsm_fft_lines).  Errors against the FP64 engine's result."""
    nvec = (n + 1) * 2 * n * (2 * n // 32)
    torch.manual_seed(7)
    x = torch.complex(torch.randn(nvec, 32, dtype=torch.float64, device=stream.device),
                      torch.randn(nvec, 32, dtype=torch.float64, device=stream.device))
    out = {"vectors": nvec, "bytes_in_out": 2 * x.numel() * 16}

    def timed(fn, reps=5):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        with torch.cuda.stream(stream):
            y = fn()
            for e0, e1 in evs:
                flush.zero_()
                e0.record(stream)
                y = fn()
                e1.record(stream)
        torch.cuda.synchronize()
        return y, float(np.median([a.elapsed_time(b) for a, b in evs]))

    ref, ms64 = timed(lambda: gsm.fft_lines(x, -1, "fp64", stream=stream))
    res = {"fft_engine_fp64": {"ms": ms64}}
    y2, ms2 = timed(lambda: gsm.fft_lines(x, -1, "fp32x2", stream=stream))
    scale = float(ref.abs().max())
    res["fft_engine_fp32x2"] = {"ms": ms2, "rel_err_vs_fp64": float((y2 - ref).abs().max()) / scale}
    try:
        yt, mst = timed(lambda: gsm.dft32_tc(x, -1, stream=stream))
        res["tensor_core_digit_planes"] = {"ms": mst, "rel_err_vs_fp64": float((yt - ref).abs().max()) / scale,
                                           "mma_tflops": nvec / 128 * 84 * 2 * 128 * 64 * 16 / (mst / 1e3) / 1e12}
    except Exception as exc:                 # reported, not hidden
        res["tensor_core_digit_planes"] = {"error": str(exc)}
    out.update(res)
    del x, ref, y2
    torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------------ config suite
def _time_apply(torch, fn, steps, flush, stream):
    """Mean ms of fn() over `steps` runs, CUDA events on `stream`, L2 flushed
    between runs outside the events."""
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with torch.cuda.stream(stream):
        fn()
        for e0, e1 in ev:
            flush.zero_()
            e0.record(stream)
            fn()
            e1.record(stream)
    torch.cuda.synchronize()
    return float(np.mean([a.elapsed_time(b) for a, b in ev]))


def _cpu_leg(run, points: int, sample: str):
    """A config's CPU-baseline leg: the oracle, as it stands, on the host cores.
    `run` does one oracle evaluation (its set-up already done); it is timed, and
    its output also serves as the line's parity reference."""
    import oracle
    t0 = time.perf_counter()
    out = run()
    dt = time.perf_counter() - t0
    return out, {"value": points / dt / 1e6, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
                 "sample": sample, "seconds": dt}


def run_suite_sharded(a, rank: int, world: int, local: int):
    """Config 4 over `world` GPUs: the 48 independent applies split by the LPT
    rule (partition_batch), each rank applying its share with the grouped
    launch; no collective on the data path.  Time = max over ranks."""
    import torch
    import torch.distributed as dist

    import paper_1501_04438_gb300 as gsm
    from paper_1501_04438_gb300 import workloads as wl

    torch.cuda.set_device(local)
    dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    specs = wl.batch_specs()
    mine = gsm.partition_batch([n for n, _ in specs], world)[rank]
    for prec in ("fp64", "fp32"):
        dt = torch.float32 if prec == "fp32" else torch.float64
        plans = [gsm.Plan("coulomb3d", 10.0, specs[i][0], precision=prec, stream=stream) for i in mine]
        rhos = [torch.tensor(wl.mixture((specs[i][0],) * 3, 10.0, specs[i][1]), dtype=dt, device=dev) for i in mine]
        outs = [torch.empty_like(r) for r in rhos]
        dist.barrier()
        ms = _time_apply(torch, lambda: gsm.apply_batched(plans, rhos, outs, stream=stream), max(3, a.steps),
                         flush, stream)
        ms = max_over_ranks(ms, dev)
        npts = sum(n ** 3 for n, _ in specs)
        if rank == 0:
            print(json.dumps({"config": "4 batch48 sharded", "precision": prec, "n_gpus": world,
                              "partition": "LPT on prod(2n) log2 prod(2n)", "ms": ms,
                              "Mpts_s": npts / ms / 1e3, "scaling": "strong"}), flush=True)
        for p in plans:
            p.destroy()
    dist.barrier()
    dist.destroy_process_group()


def run_suite(a):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1:
        return run_suite_sharded(a, int(os.environ.get("RANK", "0")), world, int(os.environ.get("LOCAL_RANK", "0")))
    import torch

    import oracle
    import paper_1501_04438_gb300 as gsm
    from paper_1501_04438_gb300 import workloads as wl

    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    steps = max(3, a.steps)

    def emit(d):
        d["gpu"] = torch.cuda.get_device_name(0)
        print(json.dumps(d), flush=True)

    def precisions_line(cfg, kernel, rho_h, L, n_tuple, u_ref):
        out = {"config": cfg, "kernel": kernel, "grid": list(n_tuple), "L": L, "forms": {}}
        for prec in ("fp64", "fp32x2", "fp32"):
            dt = torch.float32 if prec == "fp32" else torch.float64
            plan = gsm.Plan(kernel, L, n_tuple, precision=prec, stream=stream)
            plan.autotune(stream=stream)
            r = torch.tensor(rho_h, dtype=dt, device=dev)
            u = torch.empty_like(r)
            ms = _time_apply(torch, lambda: plan.apply(r, u, stream=stream), steps, flush, stream)
            uh = u.double().cpu().numpy()
            npts = int(np.prod(n_tuple))
            out["forms"][prec] = {"ms": ms, "Mpts_s": npts / (ms / 1e3) / 1e6,
                                  "rel_err_vs_oracle": relmax(uh, u_ref), "S": plan.info()["S"]}
            plan.destroy()
        return out

    want = {c.strip() for c in a.configs.split(",")}

    if "1" in want:
        # config 1: 3D Coulomb 32^3 on [-8,8]^3, exp(-|x|^2) (the closed-form checks are in the tests)
        rho = wl.coulomb3d_gaussian(32, 8.0, 1.0)
        prep = oracle.Prepared("coulomb3d", 32, 8.0)
        uo, cpu = _cpu_leg(lambda: prep.run(rho), 32 ** 3, "the whole 32^3 config, apply only")
        line = precisions_line("1", "coulomb3d", rho, 8.0, (32, 32, 32), uo)
        line["cpu_baseline"] = cpu
        emit(line)

    if "2" in want:
        # config 2: 3D Coulomb on [-12,12]^3, anisotropic and 8-Gaussian mixture, 128^3 and 256^3
        for n in (128, 256):
            for name, rho in (("2a anisotropic", wl.coulomb3d_anisotropic(n, 12.0, 4.0)),
                              ("2b mixture8", wl.coulomb3d_mixture(n, 12.0))):
                prep = oracle.Prepared("coulomb3d", n, 12.0)
                uo, cpu = _cpu_leg(lambda: prep.run(rho), n ** 3, f"the whole {n}^3 config, apply only")
                line = precisions_line(name, "coulomb3d", rho, 12.0, (n, n, n), uo)
                line["cpu_baseline"] = cpu
                emit(line)

    if "3" in want:
        # config 3: 2D Poisson and Coulomb on [-16,16]^2, 1024^2 and 4096^2, 6 isotropic Gaussians
        params = wl.mixture2d_params()
        for n in (1024, 4096):
            rho = wl.mixture((n, n), 16.0, params)
            for kernel in ("poisson2d", "coulomb2d"):
                prep = oracle.Prepared(kernel, n, 16.0)
                uo, cpu = _cpu_leg(lambda: prep.run(rho), n * n, f"the whole {n}^2 config, apply only")
                line = precisions_line("3", kernel, rho, 16.0, (n, n), uo)
                line["cpu_baseline"] = cpu
                emit(line)

    if "4" in want:
        # config 4: 48 densities, n in {48,64,96,128,160}, [-10,10]^3, 4 Gaussians each
        specs = wl.batch_specs()
        for prec in ("fp64", "fp32"):
            dt = torch.float32 if prec == "fp32" else torch.float64
            t0 = time.perf_counter()
            plans = [gsm.Plan("coulomb3d", 10.0, n, precision=prec, stream=stream) for n, _ in specs]
            plan_s = time.perf_counter() - t0
            for p in plans:
                p.autotune(stream=stream)
            rhos = [torch.tensor(wl.mixture((n, n, n), 10.0, prm), dtype=dt, device=dev) for n, prm in specs]
            outs = [torch.empty_like(r) for r in rhos]
            npts = sum(n ** 3 for n, _ in specs)
            ms_loop = _time_apply(torch, lambda: [p.apply(r, o, stream=stream) for p, r, o in zip(plans, rhos, outs)],
                                  steps, flush, stream)
            loop_out = [o.clone() for o in outs]
            ms_grouped = _time_apply(torch, lambda: gsm.apply_batched(plans, rhos, outs, stream=stream), steps, flush,
                                     stream)
            same = all(torch.equal(x, y) for x, y in zip(outs, loop_out))
            batch = gsm.Batch(plans, rhos, outs, stream=stream)
            ms_graph = _time_apply(torch, lambda: batch.launch(stream=stream), steps, flush, stream)
            batch.wait(stream=stream)          # raises if a bounded wait of the last launch ran out
            same_graph = all(torch.equal(x, y) for x, y in zip(outs, loop_out))
            # CPU-baseline leg on three of the instances, also the parity sample
            errs, cpu_s, cpu_pts = [], 0.0, 0
            for i in (0, len(specs) // 2, len(specs) - 1):
                n, prm = specs[i]
                prep = oracle.Prepared("coulomb3d", n, 10.0, taylor_mode=1)
                rho_i = wl.mixture((n, n, n), 10.0, prm)
                uo, cpu_i = _cpu_leg(lambda: prep.run(rho_i), n ** 3, "")
                cpu_s += cpu_i["seconds"]
                cpu_pts += n ** 3
                errs.append(relmax(outs[i].double().cpu().numpy(), uo))
            cpu = dict(cpu_i, value=cpu_pts / cpu_s / 1e6, seconds=cpu_s,
                       sample="instances 0, 24 and 47 of the 48, apply only")
            emit({"config": "4 batch48", "precision": prec, "instances": len(specs),
                  "sizes": [n for n, _ in specs], "points": npts,
                  "loop": {"ms": ms_loop, "Mpts_s": npts / ms_loop / 1e3},
                  "queue": {"ms": ms_grouped, "Mpts_s": npts / ms_grouped / 1e3, "bitwise_equal_loop": same,
                            "call": "gsm_apply_batched: one launch with a device work queue, status read back"},
                  "graph": {"ms": ms_graph, "Mpts_s": npts / ms_graph / 1e3, "bitwise_equal_loop": same_graph,
                            "call": "gsm_batch_launch: the queue launch recorded in a CUDA graph"},
                  "rel_err_vs_oracle_sampled": errs, "cpu_baseline": cpu, "plans_s": plan_s})
            batch.destroy()
            for p in plans:
                p.destroy()
            del rhos, outs, loop_out

    if "5" not in want:
        return
    # config 5: 192^3 on [-12,12]^3, Hartree energy and gradient, Coulomb and dipolar (n = m = e_z)
    from paper_1501_04438_gb300.autograd import hartree_energy
    n, L = 192, 12.0
    psi_h = wl.psi3d(n, L)
    for kernel in ("coulomb3d", "dipolar3d"):
        plan = gsm.Plan(kernel, L, n, stream=stream)
        plan.autotune(stream=stream)
        psi = torch.tensor(psi_h, device=dev)

        def fwd_bwd():
            p = psi.detach().requires_grad_(True)
            E = hartree_energy(p, plan)
            E.backward()
            return E, p.grad

        with torch.cuda.stream(stream):
            E, g = fwd_bwd()
        torch.cuda.synchronize()
        ms = _time_apply(torch, fwd_bwd, steps, flush, stream)
        (E_o, g_o, _), cpu = _cpu_leg(lambda: oracle.hartree(kernel, psi_h, L, taylor_mode=1),
                                      n ** 3, f"energy and gradient of the whole {n}^3 config, plan included")
        gh = g.cpu().numpy()
        # central differences of the GPU energy, h = 1e-6, real and imaginary parts
        rng = np.random.default_rng(5)
        fd_err = 0.0
        idxs = [tuple(int(v) for v in rng.integers(n // 4, 3 * n // 4, 3)) for _ in range(16)]
        for idx in idxs:
            for unit in (1.0, 1j):
                vals = []
                for sgn in (1, -1):
                    with torch.cuda.stream(stream):
                        p2 = psi.clone()
                        p2[idx] += sgn * 1e-6 * unit
                        e2, _, _ = plan.hartree(p2, stream=stream)
                        e2 = e2.cpu()     # copied on the stream that computed it
                    vals.append(float(e2))
                fd = (vals[0] - vals[1]) / 2e-6
                an = gh[idx].real if unit == 1.0 else gh[idx].imag
                fd_err = max(fd_err, abs(fd - an))
        emit({"config": "5 hartree", "kernel": kernel, "grid": [n] * 3, "L": L,
              "ms_energy_and_gradient": ms, "Mpts_s": n ** 3 / ms / 1e3,
              "energy": float(E.detach()), "rel_err_energy_vs_oracle": abs(float(E.detach()) - E_o) / abs(E_o),
              "rel_err_grad_vs_oracle": float(np.max(np.abs(gh - g_o)) / np.max(np.abs(g_o))),
              "fd_max_abs_err_over_max_grad": fd_err / float(np.max(np.abs(g_o))), "fd_points": 2 * len(idxs),
              "cpu_baseline": cpu})
        plan.destroy()


def run_passes(a):
    """One JSON line: the per-pass milliseconds (median of K steps, L2 flushed
    between steps) of a tuned plan on seeded white noise, for profiling one
    kernel set outside the headline workload."""
    import torch
    import paper_1501_04438_gb300 as gsm
    kernel, prec, n = a.passes.split(":")
    n = int(n)
    d = 3 if kernel.endswith("3d") else 2
    L = L_BOX if d == 3 else 16.0
    dev = torch.device("cuda:0")
    stream = torch.cuda.Stream(dev)
    rho_h = np.random.default_rng(1).standard_normal((n,) * d)
    dt = torch.float32 if prec == "fp32" else torch.float64
    rho = torch.tensor(rho_h, dtype=dt, device=dev)
    u = torch.empty_like(rho)
    plan = gsm.Plan(kernel, L, n, precision=prec, stream=stream)
    plan.autotune(stream=stream)
    flush = torch.empty(512 * 2 ** 20 // 4, dtype=torch.float32, device=dev)
    time_passes(torch, plan, rho, u, max(1, a.warmup), flush, stream)
    _, pass_ms = time_passes(torch, plan, rho, u, a.steps, flush, stream)
    info = plan.info()
    print(json.dumps({"passes": f"{kernel} {prec} {n}^{d}", "steps": a.steps,
                      "passes_ms": [float(np.median(x)) for x in pass_ms],
                      "total_ms": float(sum(np.median(x) for x in pass_ms)),
                      "radix_fwd": info["radix_fwd"], "radix_inv": info["radix_inv"]}))
    plan.destroy()


if __name__ == "__main__":
    if "--suite" in sys.argv:
        run_suite(args_parse())
    elif "--passes" in sys.argv:
        run_passes(args_parse())
    else:
        main()
