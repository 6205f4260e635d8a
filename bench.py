#!/usr/bin/env python3
"""Benchmark of the WR3L deblurring hot path on B300 (one JSON line on rank 0).

Workload: a 1024x1024 float32 synthetic grey image blurred by a 30-degree line
PSF of length 31 (raised-cosine taps, 17x27 support, 71 non-zero taps) with
Gaussian noise sigma=2 and 1% salt-and-pepper; one step is the whole pipeline:
Wiener initialisation + 20 robust regularised Richardson-Lucy iterations
(spatial blur/correlation with constant continuation, TV regulariser).

Metric: Mpixel*iterations/s of RRRL over the whole step (the Wiener image
passes included in the step time; the per-size set-up -- transform tables,
PSF spectrum, tap groups -- is done once by a plan outside the step, as the
paper excludes it).  Inputs stay resident in HBM; L2 is flushed before every
timed step by writing a 256 MiB buffer (L2 is 126 MB).

  python bench.py [--gpus N --steps K --warmup W] [--impl ours|reference]

With N > 1 (launched by torch.distributed.run) every rank deblurs its own
image (independent replicas, weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6400.0
SM_COUNT, FP32_LANES_PER_SM, SM_MAX_MHZ = 148, 128, 2032.0
METRIC = "RRRL Mpixel*iter/s"
UNIT = "Mpx*iter/s"


def forms_arg(text):
    """--forms: "auto" or [fft<T>/|nofft/]<dense|groups>/<all|rule|none>."""
    if text == "auto":
        return text
    parts = text.split("/")
    ok = (len(parts) in (2, 3) and parts[-2] in ("dense", "groups") and parts[-1] in ("all", "rule", "none")
          and (len(parts) == 2 or parts[0] == "nofft" or (parts[0].startswith("fft") and parts[0][3:].isdigit())))
    if not ok:
        raise argparse.ArgumentTypeError(f"bad --forms value {text!r}")
    return text


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["batch512", "learn512", "stream1024"],
                    default="batch512",
                    help="batch512 (default: the largest workload, 512 uneven images), line1024, box256, "
                         "gauss2048, learn512, stream1024 (line1024 frames with overlapped host<->device "
                         "transfers)")
    ap.add_argument("--no-sub", action="store_true",
                    help="batch512 at N=1: skip the line1024, gauss2048 and learn512 sub-measurements")
    ap.add_argument("--schedule", choices=["auto", "fused", "split", "flow", "cluster"], default="auto",
                    help="kernel schedule of the spatial RRRL iterations")
    ap.add_argument("--images", type=int, default=512,
                    help="batch512 only: deblur an evenly spaced subset of this many of the 512 images "
                         "(a smaller case of the same kernels, for profiling)")
    ap.add_argument("--forms", default="auto", type=forms_arg,
                    help="batch512 only: tile forms timed (auto: chosen by db_batch_autotune before capture) "
                         "or fixed as [fft<T>/|nofft/]<2D sums>/<one-axis register windows>, e.g. fft169/dense/all "
                         "(FFT tiles for 2D PSFs with kh*kw >= T; no prefix: the default threshold; nofft/: none) "
                         "(for profiling: the autotuner's own runs are then not launched)")
    ap.add_argument("--rf", choices=["log1p", "lut"], default="log1p",
                    help="evaluation of r_f: log1p (default) or the lookup table of Sec. 4.1")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def peaks():
    try:
        with open(PEAKS_PATH) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle sampling while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        load = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(load) if load else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# DRAM bytes per RRRL iteration on the line1024 workload under the default
# (flow) schedule: one ncu capture of the persistent launch (20 iterations,
# dram__bytes_read.sum + dram__bytes_write.sum, caches flushed before the
# capture), divided by the iteration count.
LINE1024_FLOW_ITER_DRAM_BYTES = (8.488448e6 + 1.435136e6) / 20


# DRAM bytes per pixel and iteration of k_rrl_batch on batch512
# (dram__bytes_read.sum + dram__bytes_write.sum of one full-size launch, 55.93 GB,
# over its 1.735e9 pixel-iterations, forms fft81/dense/all as the autotuner chose
# them).  Set to None when the kernel changes, until it is captured again.
BATCH_DRAM_BYTES_PER_PX_ITER = 32.23


def pinned_copy(array):
    """A page-locked float32 host tensor holding `array`, written by one
    single-threaded copy: rows written by many host threads can stay dirty in
    the caches of several cores, and the device's reads of them ran five
    times slower on B300 hosts."""
    a = np.ascontiguousarray(np.asarray(array, dtype=np.float32))
    t = torch.empty(a.shape, dtype=torch.float32).pin_memory()
    ctypes.memmove(t.data_ptr(), a.ctypes.data, a.nbytes)
    return t


def step_stats(ms_list):
    """Median, minimum and standard deviation of the per-step times (ms)."""
    v = list(ms_list)
    return {"median": statistics.median(v), "min": min(v), "sd": statistics.pstdev(v) if len(v) > 1 else 0.0}


# Algorithmic bytes per pixel and iteration: what the method itself must read
# and write once per iteration, halo re-reads and intermediates excluded.
#   spatial iteration: read u, read f, write u'                        12 B
#   periodic (FFT) iteration, four passes over complex spectra:
#     columns fwd x S inv 12, rows C2R + ratio + packed C2C 16,
#     columns fwd x conj S inv on the packed pair 20, rows inverse +
#     regulariser + update + next forward 20                            68 B
#   reverse mode (adjoint of one iteration): forward recompute 12 +
#     reverse reads u, f, the adjoint and writes the adjoint 16         28 B
ALGO_BYTES = {"spatial": 12.0, "fourier": 68.0, "adjoint": 28.0}


def fp32_peak_tflops(world=1):
    """Nominal FP32 FMA rate: 148 SMs x 128 lanes x 2 flop x 2032 MHz."""
    return world * SM_COUNT * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12


def flops_per_px_iter(h, kind="general"):
    """Algorithmic FP32 flops per pixel and iteration: three tap sums (b, then
    the two correlations) at 2 flops per non-zero tap, plus about 60 for the
    pointwise work (weight, ratio, regulariser, update).  A box PSF is summed
    by sliding windows: about 4 flops per sum whatever its length."""
    if kind.startswith("box"):
        return 3 * 4 + 60
    return 6 * int((np.asarray(h) != 0).sum()) + 60


def hbm_roofline(bytes_per_pxi, pxi, ms, kernel, traffic=None, flops=None, world=1, **extra):
    """Roofline entry against the measured HBM copy bandwidth: achieved =
    algorithmic bytes of the launch / its device time; the FP32 figure of the
    same time is given beside it (`alu`)."""
    hbm_peak, src = peaks()
    ach = bytes_per_pxi * pxi / (ms / 1e3) / 1e9
    d = {"bound": "hbm", "achieved": ach, "peak": hbm_peak * world, "unit": "GB/s",
         "frac": ach / (hbm_peak * world), "traffic": traffic, "kernel": kernel, "kernel_ms": ms,
         "algorithmic_bytes_per_px_iter": bytes_per_pxi, "units_per_launch_px_iter": pxi,
         "peak_src": f"{src} (HBM copy bandwidth, of measured)" if src == "measured" else f"{src} (6.4 TB/s, of fallback)"}
    if flops is not None:
        a = flops / (ms / 1e3) / 1e12
        d["alu"] = {"achieved": a, "peak": fp32_peak_tflops(world), "unit": "TFLOP/s",
                    "frac": a / fp32_peak_tflops(world),
                    "peak_src": "FP32 FMA: 148 SMs x 128 lanes x 2 flop x 2032 MHz (nominal)"}
    d.update(extra)
    return d


def _spatial_model(case, ms_iter, schedule="auto"):
    """One spatial RRRL iteration (12 algorithmic B/px) with its FP32 figure."""
    H, W = case.f.shape
    line1024 = (H, W, int((case.h != 0).sum())) == (1024, 1024, 71)
    traffic = LINE1024_FLOW_ITER_DRAM_BYTES if line1024 and schedule in ("auto", "flow") else None
    return hbm_roofline(ALGO_BYTES["spatial"], H * W, ms_iter,
                        "one RRRL iteration (1/iters of k_rrl_flow; k_rrl_q + k_rrl_update; or k_rrl_spatial)",
                        traffic=traffic, flops=flops_per_px_iter(case.h, case.psf_kind) * H * W)


# DRAM bytes of one periodic iteration on the gauss2048 workload: one ncu
# capture of its four launches (dram__bytes_read.sum + dram__bytes_write.sum,
# caches flushed between passes).  Set to None when the kernels change, until
# they are captured again.
GAUSS2048_ITER_DRAM_BYTES = (67.135488 + 1.007360 + 50.380032 + 4.249856 + 67.135232 + 1.110784
                             + 50.377984 + 11.309056) * 1e6


def _fourier_model(case, ms_iter, schedule="auto"):
    """One periodic RRRL iteration: 68 algorithmic B/px (four passes)."""
    H, W = case.f.shape
    traffic = GAUSS2048_ITER_DRAM_BYTES if case.name == "gauss2048" and (H, W) == (2048, 2048) else None
    return hbm_roofline(ALGO_BYTES["fourier"], H * W, ms_iter,
                        "one Fourier RRRL iteration (k_fourier_cols8 x2, k_fourier_mid8, k_fourier_rows8; "
                        "k_fourier_cols / k_fourier_rows for sides below 64)", traffic=traffic)


def _make(name):
    from paper_1212_2245_b300 import synth
    return {"line1024": synth.case_line1024, "box256": synth.case_box256,
            "gauss2048": synth.case_gauss2048, "gauss3072": synth.case_gauss3072}[name]()


WORKLOADS = {
    "line1024": ("line1024: 1024x1024 f32, 30deg line PSF L=31 (17x27, 71 taps), sigma=2 + 1% salt/pepper, "
                 "Wiener K=0.01 + 20 RRRL (TV, alpha=0.003), spatial blur/correlation", _spatial_model),
    "box256": ("box256: 256x256 f32, horizontal box L=15, sigma=2, row Wiener K=0.006 + 10 RRRL, spatial",
               _spatial_model),
    "gauss2048": ("gauss2048: 2048x2048 f32, 31x31 mixture of 3 Gaussians, sigma=1, Wiener K=0.006 + 30 RRRL "
                  "with Fourier-domain (periodic) blur/correlation", _fourier_model),
    "gauss3072": ("gauss3072: 3072x3072 f32, 25x25 mixture of 3 Gaussians, sigma=2, Wiener K=0.006 + 10 RRRL "
                  "with constant continuation (spatial: 64x64 FFT tiles)", _spatial_model),
}


BATCH512_DESC = ("batch512: 512 f32 images, sides U{128..1024}, half 1D motion (box/raised cosine, L 5-41), "
                 "half 2D Gaussian mixtures 7x7..25x25, sigma=2, Wiener K=0.006 + 10 RRRL; one planned batch "
                 "replayed from a CUDA graph")


def make_case(name="line1024"):
    return _make(name)


def cpu_baseline_oracle(case, budget_s=10.0, max_iters=None):
    """The FP64 oracle as it stands, on the host cores: the Wiener step, then
    RRRL iterations on the full image until about `budget_s` seconds have
    passed (at most the workload's iteration count, at least one)."""
    import oracle
    max_iters = case.iters if max_iters is None else max_iters
    t0 = time.perf_counter()
    u0, u = oracle.wr3l(case.f, case.h, case.params, 1)
    f0 = oracle.condition_input(case.f, case.params.pos_floor)
    n_iters = 1
    while n_iters < max_iters and time.perf_counter() - t0 < budget_s:
        u = oracle.rrrl_step(u, f0, case.h, case.params)
        n_iters += 1
    dt = time.perf_counter() - t0
    H, W = case.f.shape
    return {"value": H * W * n_iters / dt / 1e6, "unit": UNIT, "cores": torch.get_num_threads(),
            "kind": "oracle",
            "sample": f"FP64 oracle (torch CPU ops), Wiener + {n_iters} RRRL iterations on the full "
                      f"{H}x{W} image, {dt:.1f} s"}


def run_reference(args, ws_, rank):
    """Reference arm: the FP64 CPU oracle as it stands, on a bounded sample of
    the same workload per step."""
    if rank != 0:
        return
    import oracle
    if args.workload == "batch512":
        from paper_1212_2245_b300 import synth
        order = batch_sample_order(512)
        n_steps = args.warmup + args.steps
        cases = [synth.batch_case(order[s % len(order)]) for s in range(n_steps)]
        desc = BATCH512_DESC
        sample = ("one FP64 oracle RRRL iteration on one whole image of the batch per step, images taken "
                  "alternately from its 1D-PSF and 2D-PSF halves")
    else:
        case = make_case(args.workload if args.workload in WORKLOADS else "line1024")
        rows = min(128, case.f.shape[0])
        strip = type(case)(case.name, case.g[:rows], case.f[:rows], case.h, case.iters, case.params, case.psf_kind)
        cases = [strip] * (args.warmup + args.steps)
        desc = WORKLOADS[args.workload if args.workload in WORKLOADS else "line1024"][0]
        sample = f"one FP64 oracle RRRL iteration on a {rows}x{case.f.shape[1]} strip of the workload per step"
    pxi, total = 0, 0.0
    times = []
    for s_, c in enumerate(cases):
        f0 = oracle.condition_input(c.f.astype(np.float64), c.params.pos_floor)
        u = oracle.positivity_floor(torch.as_tensor(c.f, dtype=torch.float64), c.params.pos_floor)  # warm start
        t0 = time.perf_counter()
        oracle.rrrl_step(u, f0, c.h, c.params)
        dt = time.perf_counter() - t0
        if s_ >= args.warmup:
            times.append(dt)
            pxi += c.f.size
            total += dt
    val = pxi / total / 1e6
    ms = 1e3 * statistics.mean(times)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "sample": sample},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, world, rank, local, workload=None):
    import paper_1212_2245_b300 as db
    from paper_1212_2245_b300 import _lib

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lib = _lib.load()
    workload = workload or args.workload
    case = make_case(workload)
    desc, model = WORKLOADS[workload]
    H, W = case.f.shape
    iters, p = case.iters, case.params
    f = torch.as_tensor(case.f).to(dev)
    h = torch.as_tensor(case.h).to(dev).contiguous()
    u = torch.empty_like(f)
    u_w = torch.empty_like(f)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(device=dev)

    with torch.cuda.stream(stream):
        # set-up once per image size and PSF (transform tables, PSF spectrum,
        # tap groups): the paper's precomputation, outside the timed step
        plan = db.Plan(H, W, h, p, iters, kind=case.psf_kind)
        plan_w = db.Plan(H, W, h, p, 0, kind=case.psf_kind)  # Wiener only, to split the step time
        stream.synchronize()
        # the plan's schedule and tile form by measurement (db_plan_autotune),
        # unless a schedule was fixed on the command line
        tuned = None
        if args.schedule == "auto":
            sched, form = plan.autotune(f, reps=2)
            tuned = {"schedule": sched, "form": form}
        # warm-up: at least W steps and at least one second of work (clocks
        # ramp up from idle; the first launches also load the modules)
        t0, n = time.perf_counter(), 0
        while n < max(args.warmup, 3) or time.perf_counter() - t0 < 1.0:
            plan.run(f, u, check=False)
            n += 1
            if n % 8 == 0:
                stream.synchronize()
        plan.run(f, u)  # raises on any device flag
        n0 = lib.db_launch_count()
        g_step, g_w = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
        with torch.cuda.graph(g_step, stream=stream):
            plan.run(f, u, check=False)
        n1 = lib.db_launch_count()
        with torch.cuda.graph(g_w, stream=stream):
            plan_w.run(f, u_w, check=False)
        launches_per_step = n1 - n0
        iter_launches = launches_per_step  # the step's graph holds the Wiener passes and the iterations
        for _ in range(2):
            g_step.replay()
            g_w.replay()
        stream.synchronize()
        plan.ws.raise_on_flags("graph replay")

    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
    if world > 1:
        torch.distributed.barrier()
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        t_wall = time.perf_counter()
        with torch.cuda.stream(stream):
            for k in range(K):
                flush.fill_(float(k))
                ev[k][0].record(stream)
                g_step.replay()
                ev[k][1].record(stream)
                flush.fill_(float(k))
                ev[k][2].record(stream)
                g_w.replay()
                ev[k][3].record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
        if world > 1:
            torch.distributed.barrier()
    step_ms = [e[0].elapsed_time(e[1]) for e in ev]
    wiener_ms = [e[2].elapsed_time(e[3]) for e in ev]
    ms = statistics.mean(step_ms)
    ms_iter = max(ms - statistics.mean(wiener_ms), 1e-6)
    if world > 1:
        t = torch.tensor([ms, ms_iter], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms, ms_iter = float(t[0]), float(t[1])

    # status after the timed region
    torch.cuda.synchronize()
    plan.ws.raise_on_flags("timed region")

    # end-to-end through the C ABI with host buffers (db_plan_run_host: copy
    # in, pipeline, copy out; page-locked buffers from db_host_alloc)
    f_host, u_host = db.HostBuffer((H, W)), db.HostBuffer((H, W))
    f_host.copy_from(case.f)
    e2e_ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(K)]
    with torch.cuda.stream(stream):
        plan.run_host(f_host, u_host)  # device buffers of the host path, outside the timed region
        for k in range(K):
            flush.fill_(float(k))
            e2e_ev[k][0].record(stream)
            plan.run_host(f_host, u_host, check=False, sync=False)
            e2e_ev[k][1].record(stream)
    torch.cuda.synchronize()
    plan.ws.raise_on_flags("end-to-end region")
    if not torch.equal(u_host.tensor, u.cpu()):
        raise RuntimeError("host-buffer result differs from the device-buffer result")
    e2e_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in e2e_ev)
    if world > 1:
        t = torch.tensor([e2e_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_ms = float(t[0])

    if rank != 0:
        return
    px_iter = H * W * iters
    value = world * px_iter / (ms / 1e3) / 1e6
    roof = model(case, ms_iter / iters, args.schedule)
    kh, kw = case.h.shape
    fft_form = (tuned or {}).get("form") == "fft" if tuned else (
        args.schedule != "fused" and case.psf_kind == "general" and 2 <= kh <= 48 and 2 <= kw <= 48 and kh * kw >= 225)
    if fft_form and "alu" in roof:  # the FFT tiles do far fewer flops than the direct sums
        roof["alu"] = {"note": "not reported: the FFT tiles form the 2D tap sums with far fewer flops than the "
                               "direct sums"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": ms, "ms_stats": step_stats(step_ms), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": desc, "H": H, "W": W, "iters": iters, "psf": list(case.h.shape),
                   "psf_nnz": int((case.h != 0).sum()), "l2": "flushed before every step (256 MiB write)",
                   "parallelism": f"replicas x{world}"},
        "rrrl_only_mpx_iter_s": world * px_iter / (ms_iter / 1e3) / 1e6,
        "wiener_ms": statistics.mean(wiener_ms),
        "autotuned": tuned,
        "roofline": roof,
        "e2e": {"value": world * px_iter / (e2e_ms / 1e3) / 1e6, "unit": UNIT,
                "h2d_bytes_per_step": H * W * 4, "d2h_bytes_per_step": H * W * 4, "ms_per_step": e2e_ms},
        "gpu_launches": launches_per_step * K,
        "launches_per_step": launches_per_step, "iteration_launches": iter_launches,
        "wall_s_timed": t_wall,
        "clocks": clk.summary(),
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_oracle(case)
    return line


def run_batch(args, world, rank, local):
    """512 uneven images (sides U{128..1024}), own PSF each, Wiener + 10 RRRL,
    as one planned batch replayed from a CUDA graph."""
    import paper_1212_2245_b300 as db
    from paper_1212_2245_b300 import _lib, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lib = _lib.load()
    from paper_1212_2245_b300 import shard
    t0 = time.perf_counter()
    n_img = max(1, min(512, args.images))
    all_cases = [synth.batch_case(i) for i in np.linspace(0, 511, n_img).round().astype(int).tolist()]
    gen_s = time.perf_counter() - t0
    iters = all_cases[0].iters
    px_total = sum(c.f.size for c in all_cases)
    # N ranks: each deblurs its longest-processing-time share of the images
    # (independent problems, no exchange); the whole batch's pixels count
    mine = shard.rank_images(shard.image_costs([c.f.shape for c in all_cases], iters), world, rank)
    cases = [all_cases[i] for i in mine]
    fs = [torch.as_tensor(c.f).to(dev) for c in cases]
    hs = [torch.as_tensor(c.h).to(dev).contiguous() for c in cases]
    ps = [c.params for c in cases]
    kinds = [c.psf_kind for c in cases]
    px = sum(c.f.size for c in cases)
    flops_iter = sum(c.f.size * flops_per_px_iter(c.h, c.psf_kind) for c in cases)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    fixed = None
    if args.forms != "auto":
        parts = args.forms.split("/")
        d, w = parts[-2:]
        fft = -1 if len(parts) == 2 else 0 if parts[0] == "nofft" else int(parts[0][3:])
        fixed = {"fft": fft, "dense": d == "dense", "windows": w}
        set_batch_forms(fixed)
    with torch.cuda.stream(stream):
        t0 = time.perf_counter()
        full = db.Batch(fs, hs, ps, iters, kinds=kinds)
        wien = db.Batch(fs, hs, ps, 0, kinds=kinds, outs=[torch.empty_like(f) for f in fs])
        stream.synchronize()
        plan_s = time.perf_counter() - t0
        # tile forms by measurement (dense sums, one-axis form), before capture
        t0 = time.perf_counter()
        tuned = full.autotune(reps=2) if fixed is None else fixed
        tune_s = time.perf_counter() - t0
        fft_used = tuned.get("fft", -1) != 0  # some 2D PSFs run as FFT tiles
        full.run()
        wien.run()
        n0 = lib.db_launch_count()
        g_full, g_w = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
        with torch.cuda.graph(g_full, stream=stream):
            full.run(check=False)
        n1 = lib.db_launch_count()
        with torch.cuda.graph(g_w, stream=stream):
            wien.run(check=False)
        for _ in range(max(args.warmup, 3)):
            g_full.replay()
            g_w.replay()
        stream.synchronize()
    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
    full.ws.reset_status()
    if world > 1:
        torch.distributed.barrier()
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            for k in range(K):
                flush.fill_(float(k))
                ev[k][0].record(stream)
                g_full.replay()
                ev[k][1].record(stream)
                flush.fill_(float(k))
                ev[k][2].record(stream)
                g_w.replay()
                ev[k][3].record(stream)
        torch.cuda.synchronize()
    full.ws.raise_on_flags("timed region")
    ms = statistics.mean(e[0].elapsed_time(e[1]) for e in ev)
    ms_w = statistics.mean(e[2].elapsed_time(e[3]) for e in ev)
    ms_rrl = ms - ms_w
    # end to end through the C ABI (db_batch_stream_run_host): page-locked
    # host images in, results out, every step; 6 sub-batches (pixel shares
    # 1, 4, 16, 16, 4, 1) whose copies overlap the other sub-batches' runs.
    # Each step starts after the previous one has fully finished (the call's
    # stream waits for its downloads).
    f_host = [pinned_copy(c.f) for c in cases]
    u_host = [torch.empty(c.f.shape, dtype=torch.float32).pin_memory() for c in cases]
    # the sub-batch plans take the tuned forms through the process-wide settings
    set_batch_forms(tuned)
    with torch.cuda.stream(stream):
        bs = db.BatchStream([c.f.shape for c in cases], hs, ps, iters, kinds=kinds, parts=6, device=dev)
        bs.run(f_host, u_host)
    set_batch_forms(None)
    for a, b_ in zip(u_host, full.us):
        if not torch.equal(a, b_.cpu()):
            raise RuntimeError("streamed batch differs from the single batch")
    e2e = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(K)]
    bs.ws.reset_status()
    with torch.cuda.stream(stream):
        for k in range(K):
            flush.fill_(float(k))
            e2e[k][0].record(stream)
            bs.run(f_host, u_host, sync=False)
            e2e[k][1].record(stream)
    torch.cuda.synchronize()
    bs.ws.raise_on_flags("streamed batch")
    e2e_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in e2e)
    e2e_parts = bs.parts
    bs.close()
    if world > 1:
        t = torch.tensor([ms, ms_w, e2e_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms, ms_w, e2e_ms = (float(x) for x in t)
        ms_rrl = ms - ms_w
        ft = torch.tensor([flops_iter], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(ft)
        flops_iter = float(ft[0])
    if rank != 0:
        return
    px = px_total
    pxi = px * iters
    line = {
        "metric": METRIC, "value": pxi / (ms / 1e3) / 1e6, "unit": UNIT, "n_gpus": world,
        "steps": K, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "strong" if world > 1 else "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": BATCH512_DESC, "images": len(all_cases), "pixels": px, "iters": iters,
                   "l2": "inputs 0.7 GB > L2; L2 flushed before every step (256 MiB write)",
                   "parallelism": f"images sharded by LPT over {world} ranks" if world > 1 else "1 GPU"},
        "rrrl_only_mpx_iter_s": pxi / (ms_rrl / 1e3) / 1e6, "wiener_ms": ms_w, "rrrl_ms": ms_rrl,
        "roofline": hbm_roofline(ALGO_BYTES["spatial"], pxi, ms_rrl,
                                 "k_rrl_batch (persistent: all RRRL iterations of all images in one launch)",
                                 traffic=(BATCH_DRAM_BYTES_PER_PX_ITER * pxi
                                          if BATCH_DRAM_BYTES_PER_PX_ITER and len(all_cases) == 512 else None),
                                 flops=None if fft_used else flops_iter * iters, world=world,
                                 **({"alu": {"note": "not reported: the FFT tiles form the 2D tap sums with "
                                                     "far fewer flops than the direct sums"}}
                                    if fft_used else {})),
        "e2e": {"value": pxi / (e2e_ms / 1e3) / 1e6, "unit": UNIT,
                "h2d_bytes_per_step": 4 * px, "d2h_bytes_per_step": 4 * px, "ms_per_step": e2e_ms,
                "path": f"db_batch_stream_run_host (C ABI): {e2e_parts} sub-batches, page-locked host images, "
                        "copies overlapped with the other sub-batches' runs"},
        "gpu_launches": (n1 - n0) * K, "launches_per_step": n1 - n0,
        "plan_s": plan_s, "autotune_s": tune_s if fixed is None else None,
        "autotuned" if fixed is None else "forms": tuned, "generate_s": gen_s, "clocks": clk.summary(),
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_batch(all_cases)
    return line


def set_batch_forms(forms):
    """Process-wide settings under which a batch plan takes the given tile
    forms ({"fft": threshold on kh * kw (0: none, -1: the default), "dense":
    bool, "windows": "all" | "rule" | "none"}; None: the defaults)."""
    import paper_1212_2245_b300 as db
    if forms is None:
        db.set_fft_tiles(0)
        db.set_dense_min(0)
        db.set_one_axis_min(0)
        return
    t = forms.get("fft", -1)
    db.set_fft_tiles(0 if t == -1 else (t or 2305))
    db.set_dense_min(50 if forms["dense"] else 101)
    db.set_one_axis_min({"rule": 0, "all": 1, "none": 256}[forms["windows"]])


def batch_sample_order(n):
    """Images of the batch interleaved from its two halves (1D PSFs, 2D
    Gaussian mixtures): 0, n/2, 1, n/2+1, ..."""
    half = n // 2
    out = []
    for i in range(half):
        out += [i, half + i]
    return out + list(range(2 * half, n))


def cpu_baseline_batch(all_cases, budget_s=10.0):
    """The FP64 oracle as it stands on the host cores: the whole pipeline
    (Wiener + every RRRL iteration) on images of the batch in the interleaved
    order, until about `budget_s` seconds have passed (at least two images)."""
    import oracle
    t0 = time.perf_counter()
    pxi, done = 0, []
    for i in batch_sample_order(len(all_cases)):
        c = all_cases[i]
        oracle.wr3l(c.f, c.h, c.params, c.iters)
        pxi += c.f.size * c.iters
        done.append(i)
        if len(done) >= 2 and time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": pxi / dt / 1e6, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
            "sample": f"FP64 oracle (torch CPU ops), Wiener + {all_cases[0].iters} RRRL on {len(done)} of the "
                      f"batch's images (1D and 2D PSFs alternating: {done}), {dt:.1f} s"}


def run_learn(args, world, rank, local):
    """64 x 512^2 images, 21 learnable row taps, alpha and K: forward (Wiener +
    15 RRRL, checkpoints every 5) + MSE loss gradient + backward (gradients for
    f, taps, alpha, K), one CUDA graph per step; the forward alone beside it."""
    import paper_1212_2245_b300 as db
    from paper_1212_2245_b300 import _lib, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lib = _lib.load()
    from paper_1212_2245_b300 import shard
    case = synth.case_learn512(64)
    N_all, H, W = case.f.shape
    iters, every, p = case.iters, 5, case.params
    # N ranks: each runs forward and backward on its share of the images;
    # the parameter gradients are combined by one all-reduce per step
    mine = shard.rank_images(shard.image_costs([(H, W)] * N_all, iters), world, rank)
    N = len(mine)
    f = torch.as_tensor(case.f[mine]).to(dev)
    g = torch.as_tensor(case.g[mine]).to(dev)
    taps = torch.as_tensor(case.h).to(dev).contiguous()
    u = torch.empty_like(f)
    nck = (iters - 1) // every + 1
    ck = torch.empty(N, nck, H, W, device=dev)
    bws = db.Workspace(lib.db_backward_workspace_bytes(H, W, N, ctypes.byref(_lib.DbPsf(1, taps.shape[1], 0, taps.data_ptr())), every))
    gt = torch.zeros(taps.numel(), dtype=torch.float64, device=dev)
    ga = torch.zeros(1, dtype=torch.float64, device=dev)
    gk = torch.zeros(1, dtype=torch.float64, device=dev)
    gf = torch.empty_like(f)
    gu = torch.empty_like(f)
    stream = torch.cuda.Stream(device=dev)

    wsn = db.Workspace(db.workspace_bytes_n(H, W, N, 1, taps.shape[1], p))

    def forward():  # all images of the rank in one db_deblur_n call
        db.deblur_n(f, taps, p, iters, out=u, ckpt=ck, ckpt_every=every, ws=wsn, check=False)

    def backward_part():  # loss gradient and reverse pass (needs the targets g)
        torch.sub(u, g, out=gu)
        gu.mul_(2.0 / u.numel())
        gt.zero_(); ga.zero_(); gk.zero_()
        db.rrl_backward(f, ck, gu, taps, p, iters, every, gt, ga, gk, grad_f=gf, ws=bws, check=False)

    def step():
        forward()
        backward_part()

    with torch.cuda.stream(stream):
        wsn.reset_status(); bws.reset_status()
        step()
        stream.synchronize()
        wsn.raise_on_flags("forward"); bws.raise_on_flags("backward")
        n0 = lib.db_launch_count()
        g_step, g_fwd = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
        with torch.cuda.graph(g_step, stream=stream):
            step()
        n1 = lib.db_launch_count()
        with torch.cuda.graph(g_fwd, stream=stream):
            forward()
        g_bwd = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g_bwd, stream=stream):
            backward_part()
        for _ in range(max(args.warmup, 3)):
            g_step.replay()
            g_fwd.replay()
        stream.synchronize()
    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
    if world > 1:
        torch.distributed.barrier()
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            for k in range(K):
                ev[k][0].record(stream)
                g_step.replay()
                if world > 1:
                    shard.combine_param_grads([gt, ga, gk], N, N_all)
                ev[k][1].record(stream)
                ev[k][2].record(stream)
                g_fwd.replay()
                ev[k][3].record(stream)
        torch.cuda.synchronize()
    ms = statistics.mean(e[0].elapsed_time(e[1]) for e in ev)
    ms_f = statistics.mean(e[2].elapsed_time(e[3]) for e in ev)
    wsn.raise_on_flags("timed forward"); bws.raise_on_flags("timed backward")
    # end to end: the step's images and targets in from page-locked host
    # memory, the step (forward, loss gradient, backward), the loss and the
    # parameter gradients back to the host.  The targets are needed only by
    # the loss: their copy runs on a second stream while the forward runs.
    f_host, g_host = pinned_copy(case.f[mine]), pinned_copy(case.g[mine])
    out_host = torch.empty(taps.numel() + 3, dtype=torch.float64).pin_memory()
    out_dev = torch.empty(taps.numel() + 3, dtype=torch.float64, device=dev)
    e2e = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(K + 1)]
    side = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        for k in range(K + 1):  # the first pass is untimed (loads the loss kernels)
            e2e[k][0].record(stream)
            f.copy_(f_host, non_blocking=True)
            side.wait_event(e2e[k][0])  # the previous step no longer reads g
            with torch.cuda.stream(side):
                g.copy_(g_host, non_blocking=True)
                g_in = torch.cuda.Event()
                g_in.record(side)
            g_fwd.replay()
            stream.wait_event(g_in)
            g_bwd.replay()
            if world > 1:
                shard.combine_param_grads([gt, ga, gk], N, N_all)
            out_dev[0] = ((u - g) ** 2).mean()
            out_dev[1:1 + taps.numel()].copy_(gt)
            out_dev[1 + taps.numel()] = ga[0]
            out_dev[2 + taps.numel()] = gk[0]
            out_host.copy_(out_dev, non_blocking=True)
            e2e[k][1].record(stream)
            if k == 0:
                stream.synchronize()
    torch.cuda.synchronize()
    e2e_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in e2e[1:])
    if world > 1:
        t = torch.tensor([ms, ms_f, e2e_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms, ms_f, e2e_ms = float(t[0]), float(t[1]), float(t[2])
    if rank != 0:
        return
    pxi = N_all * H * W * iters
    line = {
        "metric": METRIC + " (forward + backward)", "value": pxi / (ms / 1e3) / 1e6, "unit": UNIT,
        "n_gpus": world, "steps": K, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "strong" if world > 1 else "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "learn512: 64 x 512x512 f32, 21 learnable row taps + alpha + K, row Wiener "
                               "+ 15 RRRL (checkpoints every 5), MSE loss, full backward; one CUDA graph per step",
                   "images": N_all, "H": H, "W": W, "iters": iters, "ckpt_every": every,
                   "parallelism": f"images sharded over {world} ranks, gradient all-reduce" if world > 1 else "1 GPU",
                   "l2": "working set 0.6 GB > L2"},
        "forward_only_mpx_iter_s": pxi / (ms_f / 1e3) / 1e6, "forward_ms": ms_f,
        "backward_over_forward": (ms - ms_f) / ms_f,
        "roofline": hbm_roofline(ALGO_BYTES["adjoint"], pxi, ms,
                                 "whole fwd+bwd step (reverse mode: 28 algorithmic B/px*iter)", world=world),
        "e2e": {"value": pxi / (e2e_ms / 1e3) / 1e6, "unit": UNIT,
                "h2d_bytes_per_step": 2 * N_all * H * W * 4, "d2h_bytes_per_step": (taps.numel() + 3) * 8,
                "ms_per_step": e2e_ms},
        "gpu_launches": (n1 - n0) * K, "launches_per_step": n1 - n0, "clocks": clk.summary(),
    }
    return line


def run_stream(args, world, rank, local):
    """Frames of the line1024 workload streamed from pinned host memory:
    upload, Wiener + 20 RRRL (one captured plan per slot) and download of
    consecutive frames overlap on three streams.  Every step deblurs 16
    frames end to end (transfers inside the timed region)."""
    import paper_1212_2245_b300 as db
    from paper_1212_2245_b300 import _lib, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lib = _lib.load()
    case = synth.case_line1024()
    H, W = case.f.shape
    iters, p = case.iters, case.params
    n_frames = 16
    rng = np.random.default_rng(1024)
    frames = []
    for k in range(n_frames):  # 16 distinct frames: the case image, shifted
        frames.append(pinned_copy(np.roll(case.f, (17 * k, 29 * k), axis=(0, 1))))
    outs = [torch.empty(H, W, dtype=torch.float32).pin_memory() for _ in range(n_frames)]
    fs = db.FrameStream(H, W, torch.as_tensor(case.h).to(dev).contiguous(), p, iters, depth=2)
    for _ in range(max(args.warmup, 3)):
        fs.run(frames, outs)
    # kernels per frame, counted on one direct (uncaptured) run of the plan;
    # the streamed frames replay the captured copies of the same launches
    with torch.cuda.stream(fs.compute):
        n0 = lib.db_launch_count()
        fs.plan.run(fs.f[0], fs.u[0])
        launches = (lib.db_launch_count() - n0) * n_frames
    fs.compute.synchronize()
    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(K)]
    if world > 1:
        torch.distributed.barrier()
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for k in range(K):
            ev[k][0].record(fs.h2d)
            fs.run(frames, outs)
            ev[k][1].record(fs.d2h)
        torch.cuda.synchronize()
    ms = statistics.mean(e[0].elapsed_time(e[1]) for e in ev)
    # the same frames without transfers: graph replays back to back
    ev2 = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    with torch.cuda.stream(fs.compute):
        ev2[0].record(fs.compute)
        for k in range(n_frames):
            fs.graphs[k % 2].replay()
        ev2[1].record(fs.compute)
    torch.cuda.synchronize()
    ms_compute = ev2[0].elapsed_time(ev2[1])
    if world > 1:
        t = torch.tensor([ms, ms_compute], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms, ms_compute = float(t[0]), float(t[1])
    fs.close()
    if rank != 0:
        return
    pxi = n_frames * H * W * iters
    line = {
        "metric": METRIC, "value": world * pxi / (ms / 1e3) / 1e6, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "stream1024: 16 frames of the line1024 workload per step, pinned host frames "
                               "uploaded, deblurred (Wiener + 20 RRRL) and downloaded with the transfers "
                               "overlapped (3 streams, 2 device slots)",
                   "frames": n_frames, "H": H, "W": W, "iters": iters,
                   "l2": "16 distinct frames streamed through 2 slots",
                   "parallelism": f"replicas x{world}"},
        "frames_per_s": world * n_frames / (ms / 1e3),
        "compute_only_ms": ms_compute, "transfer_overhead": ms / ms_compute - 1.0,
        # the frames' iterations as in line1024 (per-iteration time from the
        # compute-only replays, Wiener included: a lower bound of the kernel's rate)
        "roofline": _spatial_model(case, ms_compute / n_frames / iters, "auto"),
        "e2e": {"value": world * pxi / (ms / 1e3) / 1e6, "unit": UNIT,
                "h2d_bytes_per_step": 4 * n_frames * H * W, "d2h_bytes_per_step": 4 * n_frames * H * W,
                "ms_per_step": ms},
        "gpu_launches": launches * K, "launches_per_step": launches, "clocks": clk.summary(),
    }
    return line


def main():
    args = parse()
    world, rank, local = dist_env()
    if world > 1:
        backend = "nccl" if args.impl == "ours" else "gloo"
        if args.impl == "ours":
            torch.cuda.set_device(local)
        torch.distributed.init_process_group(backend)
    try:
        if args.impl == "ours" and args.schedule != "auto":
            import paper_1212_2245_b300 as db
            db.set_schedule(args.schedule)
        if args.impl == "ours" and args.rf != "log1p":
            import paper_1212_2245_b300 as db
            db.set_rf_eval(args.rf)
        if args.impl == "reference":
            run_reference(args, world, rank)
            return
        runner = {"batch512": run_batch, "learn512": run_learn, "stream1024": run_stream}.get(args.workload, run_ours)
        line = runner(args, world, rank, local)
        if args.workload == "batch512" and world == 1 and not args.no_sub and args.images == 512:
            # the other workloads at their own sizes, each with its roofline
            sub_args = argparse.Namespace(**{**vars(args), "steps": min(args.steps, 10), "no_cpu_baseline": True})
            line["workloads"] = {}
            for name, fn in (("line1024", run_ours), ("gauss2048", run_ours), ("learn512", run_learn)):
                r = fn(sub_args, world, rank, local, name) if fn is run_ours else fn(sub_args, world, rank, local)
                if r is not None:
                    line["workloads"][name] = {k: r[k] for k in ("value", "unit", "ms_per_step", "roofline", "e2e",
                                                                 "config", "clocks") if k in r}
        if line is not None:
            print(json.dumps(line), flush=True)
    finally:
        if world > 1:
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
