#!/usr/bin/env python3
"""Throughput benchmark of the hierarchical-grid FFT correlator on GB300.

One step = one pass of the whole hot path over one batch of synthetic input:
omni_correlate over C channels x T samples (scatter, forward 2n-D FFT, |F|^2
time integration) followed by omni_visibilities (inverse 2n-D FFT, 1/L,
lag gather) with the accumulator reset.  The headline path is the mixed
precision one (split-FP16 tensor-core DFT-GEMMs); the plain FP32 FFT path is
timed beside it ("fp32_path").  Metric: antenna-samples per second
(N x T x C per step).  The default workload is the 2-level 16x16 / 8x8
hierarchy (N = 16384, 64 channels x 1024 samples of int8 voltages, 2.1 GB per
step, larger than L2, so no flush is needed between steps).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU runs (torchrun, one rank per GPU) are independent replicas: the
channels of different ranks never interact, so there is no collective on the
data path and the result scales weakly.
"""
from __future__ import annotations

import argparse
import hashlib

import numpy as np
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "antenna-samples/s"
UNIT = "antenna*samples/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="hier2")
    ap.add_argument("--precision", default="mixed", choices=["fp32", "mixed", "mixed_bf16"],
                    help="headline path; the other one is timed beside it")
    ap.add_argument("--no-compare", action="store_true", help="skip the FP32 comparison run")
    ap.add_argument("--channels", type=int, default=None,
                    help="run a smaller case of the workload (profiling)")
    ap.add_argument("--samples", type=int, default=None,
                    help="run a smaller case of the workload (profiling)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-direct", action="store_true", help="skip the direct N^2 context run")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-beams", action="store_true", help="skip the beam-space variant")
    ap.add_argument("--no-tiles", action="store_true", help="skip the tile-hybrid variant")
    ap.add_argument("--no-fengine", action="store_true", help="skip the F-engine leg")
    ap.add_argument("--no-others", action="store_true",
                    help="skip the other workloads (1-level 16x16, 3-level, 1024x1024, batch of 48)")
    return ap.parse_args()


def line_config(w, precision, world):
    """The `config` of the JSON line: identical for this arm and the reference arm."""
    return dict(workload_config(w, precision),
                parallelism=f"{world} ranks x {w.channels} channels" if world > 1 else "single GPU")


def workload_config(w, precision):
    return {
        "workload": f"{w.name}: {w.description}",
        "levels": [[lv.n1, lv.n2] for lv in w.levels],
        "antennas": w.n_antennas,
        "channels": w.channels,
        "samples": w.samples,
        "input": w.dtype,
        "precision": precision,
        "l2": "inputs larger than L2 (%.2f GB of voltages per step); no flush"
              % (w.n_antennas * w.channels * w.samples * (2 if w.dtype == "ci8" else 8) / 1e9),
    }


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.out, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.out.close()

    def summary(self):
        if self.proc is None or not self.path:
            return None
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                p = [v.strip() for v in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    smax = float(p[2])
                except ValueError:
                    continue
                for n, v in zip(names, p[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ roofline

# kernel sources behind each pass kind (plus the shared headers)
_PASS_SOURCES = [("lagsum-tcgen05", ("omni_xspec5.cu",)), ("xspec-tcgen05", ("omni_xspec5.cu",)),
                 ("xspec", ("omni_tiles.cu",)), ("tcgen05", ("omni_tc5.cu",)), ("tc", ("omni_tc.cu",)),
                 ("smem3x", ("omni_fft_smem3.cu",)),
                 ("level", ("omni_fft_level.cuh", "omni_fft_level_a.cu", "omni_fft_level_b.cu")),
                 ("smem", ("omni_fft_smem.cuh", "omni_fft_smem_a.cu", "omni_fft_smem_b.cu",
                           "omni_fft_smem_c.cu")),
                 ("reg", ("omni_fft_reg.cuh", "omni_fft_reg_a.cu", "omni_fft_reg_b.cu")),
                 ("direct", ("omni_fft_direct.cu",))]


def kernel_source_hash(pass_name):
    """Hash of the sources that define the kernel of a pass (by its stat name)."""
    from paper_0909_0001_gb300.build import CSRC
    kind = pass_name.split()[2] if len(pass_name.split()) > 2 else ""
    files = ["omni_fft_common.cuh", "omni_internal.h"]
    for key, srcs in _PASS_SOURCES:
        if kind.startswith(key):
            files += list(srcs)
            break
    h = hashlib.sha256()
    for f in files:
        path = os.path.join(CSRC, f)
        if os.path.exists(path):
            with open(path, "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel_name, workload, precision, units_per_launch):
    """DRAM bytes per launch from a committed ncu summary while the kernel's
    sources match; scaled by the channel-samples per launch when the bench's
    launches are a different size (the traffic grows in proportion to them)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None, None
    want = kernel_source_hash(kernel_name)
    with open(path) as f:
        for line in f:
            p = line.strip().split("|")
            if len(p) >= 6 and p[0].strip() == workload and p[1].strip() == precision \
                    and p[2].strip() == kernel_name and p[3].strip() == want:
                try:
                    b, u = float(p[4]), float(p[5])
                except ValueError:
                    return None, None
                if abs(u - units_per_launch) <= 0.01 * u:
                    return b, "ncu, same launch size"
                return b * units_per_launch / u, "ncu at %g channel-samples per launch, scaled" % u
    return None, None


def hbm_peak_gbs():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return float(json.load(f).get("hbm_gbs", 6800.0))
    return 6800.0


def alu_peak_tflops(sm_mhz):
    """FP32 CUDA-core peak: 152 SMs x 128 FP32 lanes x 2 flops (FMA) x clock."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


def units_per_launch(stat, profiled_units):
    """Channel-samples one launch of a forward pass processes (profiled_units:
    channels x samples over all the profiled steps)."""
    return profiled_units / max(1, stat["launches"])


def roofline(stats, workload, path_precision, profiled_units=0, serial_shares=None, serial_stats=None):
    """Roofline of the dominant kernel (largest share of the event-timed region).
    serial_stats: the same kernels timed with the two-stream chunk overlap off,
    where a launch's event span is that kernel alone (reported beside the main
    figure, which comes from the headline's own configuration)."""
    timed = [s for s in stats if s["launches"] > 0 and s["total_ms"] > 0]
    if not timed:
        return None
    top = max(timed, key=lambda s: s["total_ms"])
    peaks = {}
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            peaks = json.load(f)
    kind = "measured" if peaks else "fallback"
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    # the kernel runs inside a long step: sustained tensor peak; fp16 dense = bf16 dense
    tensor_peak = peaks.get("bf16_tflops_sustained", 1700.0)
    alu_peak = alu_peak_tflops(peaks.get("sm_max_mhz", 2070.0))
    avg_s = top["total_ms"] / top["launches"] * 1e-3
    bytes_per_launch = top["bytes"] / top["launches"]
    flops_per_launch = top["flops"] / top["launches"]
    gbs = bytes_per_launch / avg_s / 1e9
    tfs = flops_per_launch / avg_s / 1e12
    total = sum(s["total_ms"] for s in timed)
    hbm = {"achieved": round(gbs, 1), "peak": hbm_peak, "unit": "GB/s",
           "frac": round(gbs / hbm_peak, 4), "bytes_per_launch": bytes_per_launch}
    if top["tensor"]:
        main = {"bound": "tensor", "achieved": round(tfs, 2), "peak": tensor_peak,
                "unit": "TFLOP/s", "frac": round(tfs / tensor_peak, 4),
                "peak_note": "bf16_tflops_sustained of %s (fp16 dense = bf16 dense)" % kind}
    else:
        main = {"bound": "alu", "achieved": round(tfs, 2), "peak": round(alu_peak, 1),
                "unit": "TFLOP/s", "frac": round(tfs / alu_peak, 4),
                "peak_note": "FP32 FMA: 152 SMs x 128 lanes x 2 x max SM clock"}
    traffic, traffic_note = recorded_traffic(top["name"], workload, path_precision,
                                             units_per_launch(top, profiled_units))
    serial = None
    for st in serial_stats or []:
        if st["name"] == top["name"] and st["launches"] > 0 and st["total_ms"] > 0:
            s_avg = st["total_ms"] / st["launches"] * 1e-3
            s_b, s_f = st["bytes"] / st["launches"], st["flops"] / st["launches"]
            peak = main["peak"]
            serial = {"avg_launch_ms": s_avg * 1e3, "achieved": round(s_f / s_avg / 1e12, 2),
                      "frac": round(s_f / s_avg / 1e12 / peak, 4),
                      "hbm_achieved": round(s_b / s_avg / 1e9, 1),
                      "hbm_frac": round(s_b / s_avg / 1e9 / hbm_peak, 4)}
    main.update({"traffic": traffic, "traffic_note": traffic_note,
                 "kernel": top["name"], "flops_per_launch": flops_per_launch,
                 "avg_launch_ms": avg_s * 1e3,
                 "share_of_kernel_time": round(top["total_ms"] / total, 4),
                 "share_serial": (serial_shares or {}).get(top["name"]),
                 "hbm": hbm, "serial": serial})
    return main


def step_hbm(stats, ms_per_step):
    """Algorithmic bytes of every pass of one step (from the profiled steps) over
    the step time: the step-level fraction of the HBM roofline."""
    timed = [s for s in stats if s["launches"] > 0]
    if not timed or not ms_per_step:
        return None
    peaks = {}
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            peaks = json.load(f)
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    per_step = sum(s["bytes"] for s in timed) / PROFILED_STEPS
    gbs = per_step / (ms_per_step * 1e-3) / 1e9
    return {"bytes_per_step": per_step, "achieved": round(gbs, 1), "peak": hbm_peak, "unit": "GB/s",
            "frac": round(gbs / hbm_peak, 4),
            "note": "algorithmic bytes (voltages in, spectra out and back in, accumulator folds) "
                    "of all passes per step / ms_per_step; peak %s" %
                    ("of measured" if peaks else "of fallback")}


# ------------------------------------------------------------------ CPU oracle

def oracle_rate(w, x_host, target_s=15.0, max_samples=64, with_seconds=False):
    """Time the oracle as it stands on channel 0's first samples; antenna-samples/s."""
    from oracle import oracle
    dims = w.dims
    lib = oracle.lib()
    try:
        import ctypes
        lib.oracle_num_threads.restype = ctypes.c_int
        cores = int(lib.oracle_num_threads())
    except AttributeError:
        cores = os.cpu_count()
    ts = 1
    t0 = time.perf_counter()
    oracle.correlate(dims, x_host[0:1, 0:ts])
    dt = time.perf_counter() - t0
    ts = int(max(1, min(max_samples, x_host.shape[1], target_s / max(dt, 1e-3))))
    t0 = time.perf_counter()
    oracle.correlate(dims, x_host[0:1, 0:ts])
    dt = time.perf_counter() - t0
    units = w.n_antennas * ts
    sample = f"channel 0, first {ts} samples ({units} antenna-samples), {dt:.1f} s"
    if with_seconds:
        return units / dt, cores, sample, dt
    return units / dt, cores, sample


# ------------------------------------------------------------------ direct N^2 context

def direct_n2(w, x_chan, vis_chan):
    """The N^2 correlator the hypercube avoids, for context: for one channel,
    V_ij = sum_t x_t(i) conj(x_t(j)) as two real TF32 tensor-core GEMMs
    (int8 voltages are exact in TF32), then summed per 2n-D lag.  The lag index
    is linear in the lattice index, q(i, j) = a_i - a_j + const.  Returns
    (antenna-samples/s, relative difference from the hypercube's visibilities)."""
    import torch
    dims = w.dims
    T = x_chan.shape[0]
    strides, s = [], 1
    for n in dims:
        strides.append(s)
        s *= 2 * n - 1
    m = torch.from_numpy(synth_indices(w)).to(x_chan.device)          # [N][D]
    a = (m * torch.tensor(strides, device=m.device)).sum(dim=1)        # [N]
    const = sum((n - 1) * st for n, st in zip(dims, strides))
    q = (a[:, None] - a[None, :] + const).reshape(-1)                  # [N*N]
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        def run():
            xf = x_chan.float()                                        # [T][N][2]
            xr, xi = xf[..., 0], xf[..., 1]
            top = torch.cat([xr, xi], dim=0)                           # [2T][N]
            vr = top.t() @ top                                         # Xr'Xr + Xi'Xi
            vi = torch.cat([xi, -xr], dim=0).t() @ top                 # Xi'Xr - Xr'Xi
            out = torch.zeros(2, s, dtype=torch.float64, device=x_chan.device)
            out[0].index_add_(0, q, vr.reshape(-1).double())
            out[1].index_add_(0, q, vi.reshape(-1).double())
            return torch.complex(out[0], out[1])
        run()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        v = run()
        e1.record()
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) * 1e-3
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    diff = float((v - vis_chan).abs().norm() / vis_chan.abs().norm())
    return w.n_antennas * T / sec, diff, sec


def synth_indices(w):
    from paper_0909_0001_gb300 import synth
    return synth.antenna_indices(w.levels).astype("int64")


# ------------------------------------------------------------------ arms

def run_reference(args):
    """The oracle as it stands, timed on this host's cores on a bounded sample of
    the workload each step (the oracle's cost is exactly linear in samples x
    channels, so the rate of the sample is the rate of the workload)."""
    from paper_0909_0001_gb300.multirank import rank_env
    rank, _, world = rank_env()
    if rank != 0:
        return
    from paper_0909_0001_gb300 import synth
    w = synth.workload(args.workload)
    x = synth.voltages(w, channels=1, samples=64)
    per_step = max(4.0, 120.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        oracle_rate(w, x, target_s=per_step)
    rates, secs, cores, sample = [], [], None, ""
    for _ in range(args.steps):
        r, cores, sample, sec = oracle_rate(w, x, target_s=per_step, with_seconds=True)
        rates.append(r)
        secs.append(sec)
    value = statistics.mean(rates)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.mean(secs) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": line_config(w, args.precision, world),
            "extrapolated": True,
            "extrapolation": ("each step times the oracle on the bounded sample named in "
                              "cpu_baseline.sample; ms_per_step is that measured time, and value "
                              "is the measured rate, which holds for the whole workload because "
                              "the oracle's cost is linear in samples x channels (full step: "
                              "%.0f s)" % (w.n_antennas * w.samples * w.channels / value)),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample + " per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def timed_steps(plan, x, vis, steps, warmup, stream, barrier, profile):
    """Warm up, then time `steps` steps (correlate + visibilities) with CUDA events."""
    import torch

    def step():
        plan.correlate(x)
        plan.visibilities(reset=True, out=vis)

    for _ in range(max(3, warmup)):
        step()
    torch.cuda.synchronize()
    plan.kernel_stats(clear=True)
    plan.profile(profile)
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    plan.profile(False)
    return e0.elapsed_time(e1) / steps, plan.kernel_stats(clear=True)


PROFILED_STEPS = 2


def measure(plan, x, vis, steps, warmup, stream, barrier, units_per_step):
    """Timed steps with per-launch events off (the number reported), clocks
    sampled during them; then PROFILED_STEPS more steps with per-launch CUDA
    events for the kernel shares and the dominant kernel's launch duration.
    Returns (ms per step, clocks, kernel stats, channel-samples profiled); the
    stats carry "timed_launches", the launches of the timed (unprofiled) steps."""
    import torch
    with ClockSampler(torch.cuda.current_device()) as clk:
        ms, hstats = timed_steps(plan, x, vis, steps, warmup, stream, barrier, False)
    _, stats = timed_steps(plan, x, vis, PROFILED_STEPS, 0, stream, lambda: None, True)
    launches = sum(st["launches"] for st in hstats)
    for st in stats:
        st["timed_launches"] = launches
    return ms, clk.summary(), stats, units_per_step * PROFILED_STEPS


def kernel_list(stats):
    return [{k: s[k] for k in ("name", "launches", "total_ms")} for s in stats if s["launches"]]


def other_workloads(args, stream):
    """The benchmark's other configurations, each timed like the headline and
    reported as a sub-record: 1-level 16x16 (1 x 64), 3-level (16 x 256),
    1024x1024 (16 x 64) on every path the library supports for them, and the
    48 uneven arrays of a batch plan (128 x 512) against 48 separate plans."""
    import torch
    from paper_0909_0001_gb300 import omni, synth
    out = []
    for name in ("grid16", "hier3", "grid1024"):
        w = synth.workload(name)
        x = synth.voltages(w, device="cuda")
        units = w.n_antennas * w.samples * w.channels
        rec = {"workload": name, "config": workload_config(w, "see paths"), "paths": {}}
        for prec in ("mixed", "mixed_bf16", "fp32"):
            try:
                plan = omni.Plan(w.levels, w.channels, dtype=w.dtype, precision=prec)
            except omni.OmniError as e:
                rec["paths"][prec] = {"unsupported": str(e)}
                continue
            vis = torch.empty((w.channels, plan.n_lags), dtype=torch.complex128, device="cuda")
            steps = max(3, min(args.steps, 10))
            ms, clocks, stats, prof_units = measure(plan, x, vis, steps, 3, stream, lambda: None,
                                                    w.channels * w.samples)
            rec["paths"][prec] = {"value": units / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
                                  "steps": steps, "warmup": 3, "clocks": clocks,
                                  "roofline": roofline(stats, name, prec, prof_units),
                                  "kernels": kernel_list(stats)}
            plan.close()
            del vis
        del x
        torch.cuda.empty_cache()
        out.append(rec)
    out.append(batch_record(args, stream))
    return out


def batch_record(args, stream, rank=0, barrier=lambda: None, dev=None):
    """48 uneven arrays in one batch plan, and the same arrays as 48 plans."""
    import torch
    from paper_0909_0001_gb300 import multirank, omni, synth
    arrays = synth.batch_arrays()
    C, T = 128, 512
    volts = synth.batch_voltages(arrays, C, T, device="cuda", seed=9090004 + 1000 * rank)
    plan = omni.BatchPlan(arrays, C, dtype="ci8")
    flat = plan.pack(volts)
    del volts
    units = plan.n_antennas * C * T
    vis = torch.empty(C * plan.n_lags, dtype=torch.complex128, device="cuda")
    steps = max(3, min(args.steps, 10))
    ms, clocks, stats, prof_units = measure(plan, flat, vis, steps, 3, stream, barrier, C * T)
    rate, slowest = multirank.job_rate(units, ms * 1e-3, device=dev)
    # the same step replayed from one CUDA graph (every member's launches, both
    # streams of each member's overlapped chunk passes, captured once)
    graph_rec = None
    try:
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            plan.correlate(flat)
        plan.visibilities(reset=True, out=vis)  # discard the capture-time state
        for _ in range(3):
            g.replay()
            plan.visibilities(reset=True, out=vis)
        barrier()
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for _ in range(steps):
            g.replay()
            plan.visibilities(reset=True, out=vis)
        g1.record(stream)
        torch.cuda.synchronize()
        g_ms = g0.elapsed_time(g1) / steps
        g_rate, g_s = multirank.job_rate(units, g_ms * 1e-3, device=dev)
        graph_rec = {"value": g_rate, "unit": UNIT, "ms_per_step": g_s * 1e3, "steps": steps,
                     "note": "omni_correlate of the batch plan captured once in a CUDA graph and "
                             "replayed each step; omni_visibilities(reset) outside the graph"}
        del g
    except (RuntimeError, omni.OmniError) as e:
        graph_rec = {"unavailable": str(e).splitlines()[0][:200]}
    singles, offs, off = [], [], 0
    for levels, N in zip(arrays, plan.antennas):
        singles.append(omni.Plan(levels, C, dtype="ci8"))
        offs.append(off)
        off += C * T * N * 2
    views = [flat[o:o + C * T * N * 2].view(C, T, N, 2) for o, N in zip(offs, plan.antennas)]
    outs = [torch.empty((C, q), dtype=torch.complex128, device="cuda") for q in plan.lags]

    def step_all():
        for sp, v, o in zip(singles, views, outs):
            sp.correlate(v)
            sp.visibilities(reset=True, out=o)

    for _ in range(3):
        step_all()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step_all()
    e1.record(stream)
    torch.cuda.synchronize()
    sep_ms = e0.elapsed_time(e1) / steps
    sep_rate, sep_s = multirank.job_rate(units, sep_ms * 1e-3, device=dev)
    for sp in singles:
        sp.close()
    plan.close()
    del flat, vis, outs
    torch.cuda.empty_cache()
    return {"workload": "batch48",
            "config": {"workload": f"{len(arrays)} uneven arrays (single-level 8x8..64x64, "
                                   "2-level 4x4 tiles on 8x8/16x16 grids), batch plan",
                       "arrays": len(arrays), "antennas_total": plan.n_antennas,
                       "channels": C, "samples": T, "input": "ci8", "precision": "fp32",
                       "shape_groups": len(set(tuple((l.n1, l.n2) for l in a) for a in arrays)),
                       "l2": "inputs larger than L2 (%.1f GB per step); no flush"
                             % (units * 2 / 1e9)},
            "paths": {"fp32": {"value": rate, "unit": UNIT, "ms_per_step": slowest * 1e3,
                               "steps": steps, "warmup": 3, "clocks": clocks,
                               "roofline": roofline(stats, "batch48", "fp32", prof_units),
                               "kernels": kernel_list(stats),
                               "separate_plans": {"value": sep_rate, "ms_per_step": sep_s * 1e3,
                                                  "plans": len(singles)},
                               "graph_replay": graph_rec}}}


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_0909_0001_gb300 import multirank, omni, synth

    rank, local_rank, world = multirank.rank_env()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    w = synth.workload(args.workload)
    if args.channels:
        w.channels = args.channels
    if args.samples:
        w.samples = args.samples
    units = w.n_antennas * w.samples * w.channels
    # weak scaling: every rank correlates its own channels (no data-path collective)
    x = synth.voltages(w, device="cuda", channel_offset=rank * w.channels)
    stream = torch.cuda.current_stream()
    results = {}
    precisions = [args.precision] + ([] if args.precision == "fp32" or args.no_compare
                                     else ["fp32"] + (["mixed_bf16"] if args.precision == "mixed" else []))
    for prec in precisions:
        plan = omni.Plan(w.levels, w.channels, dtype=w.dtype, precision=prec)
        vis = torch.empty((w.channels, plan.n_lags), dtype=torch.complex128, device="cuda")
        # both paths are timed the same way: per-launch events off, clocks sampled;
        # then a short second run with per-launch events gives the kernel shares
        ms, clocks_p, stats, prof_units = measure(plan, x, vis, args.steps, args.warmup, stream,
                                                  barrier, w.channels * w.samples)
        if prec == args.precision:
            clocks = clocks_p
        rate, slowest = multirank.job_rate(units, ms * 1e-3, device=dev)
        results[prec] = {"plan": plan, "vis": vis, "ms": slowest * 1e3, "value": rate,
                         "stats": stats, "prof_units": prof_units, "clocks": clocks_p}
        if prec != args.precision:
            plan.close()
    head = results[args.precision]
    plan, vis = head["plan"], head["vis"]

    # kernel shares without the two-stream chunk overlap (event spans of
    # concurrent kernels overlap, so the headline run's shares are not serial
    # shares; these are the ones an ncu launch list, serialised, can confirm)
    serial = None
    sstats = None
    serial_ms = None
    if rank == 0:
        os.environ["OMNI_OVERLAP"] = "0"
        try:
            sp = omni.Plan(w.levels, w.channels, dtype=w.dtype, precision=args.precision)
        finally:
            del os.environ["OMNI_OVERLAP"]
        svis = torch.empty_like(vis)
        serial_ms, sstats = timed_steps(sp, x, svis, 2, 3, stream, lambda: None, True)
        sp.close()
        del svis
        tot = sum(st["total_ms"] for st in sstats if st["launches"])
        serial = {st["name"]: round(st["total_ms"] / tot, 4) for st in sstats if st["launches"]}

    # physical-baseline epilogue: radial profile of the step's visibilities
    epilogue = None
    if rank == 0:
        n_bins = 256
        rmax = max(float(np.hypot(*omni.baselines(w.levels)[2].T).max()), 1.0)
        bins, _ = omni.radial_bins(w.levels, rmax / n_bins * 1.0001, n_bins)
        gbins = torch.from_numpy(bins).cuda()
        prof = torch.empty((w.channels, n_bins), dtype=torch.complex128, device="cuda")
        omni.sum_groups(vis, gbins, n_bins, out=prof)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 10
        e0.record(stream)
        for _ in range(reps):
            omni.sum_groups(vis, gbins, n_bins, out=prof)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_e = e0.elapsed_time(e1) / reps
        nbytes = vis.numel() * 16 + bins.size * 4 + prof.numel() * 16
        epilogue = {"radial_profile_ms": ms_e, "bins": n_bins, "lags": int(vis.shape[1]),
                    "GB_per_s": nbytes / (ms_e * 1e-3) / 1e9}

    # end to end through the host-buffer entry points
    e2e = None
    if not args.no_e2e:
        xh = x.cpu().pin_memory()
        vh = torch.empty((w.channels, plan.n_lags), dtype=torch.complex128).pin_memory()
        for _ in range(2):
            plan.correlate_host(xh)
            plan.visibilities_host(reset=True, out=vh)
        # per-step wall times, median (single host-side outliers of 2-3x were
        # seen on the first steps after a large pinned allocation)
        n_e2e = max(3, min(args.steps, 5))
        times = []
        for _ in range(n_e2e):
            barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            plan.correlate_host(xh)
            plan.visibilities_host(reset=True, out=vh)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        dt = statistics.median(times)
        e2e_rate, e2e_s = multirank.job_rate(units, dt, device=dev)
        e2e = {"value": e2e_rate, "unit": UNIT,
               "h2d_bytes_per_step": xh.numel() * xh.element_size(),
               "d2h_bytes_per_step": vh.numel() * vh.element_size(),
               "ms_per_step": e2e_s * 1e3, "steps": n_e2e}
        del xh, vh

    # beam-space variant (Appendix A steps 4-5) on the same voltages, FP32 path
    beams = None
    if rank == 0 and len(w.levels) >= 2 and not args.no_beams:
        bp = omni.BeamPlan(w.levels, w.channels, dtype=w.dtype)
        bvis = torch.empty((w.channels, bp.n_lags), dtype=torch.complex128, device="cuda")
        ms_b, bstats = timed_steps(bp, x, bvis, max(2, min(args.steps, 5)), 3, stream,
                                   lambda: None, True)
        beams = {"value": units / (ms_b * 1e-3), "unit": UNIT, "ms_per_step": ms_b,
                 "pointings": bp.n_beams, "coarse_lags": bp.n_coarse_lags,
                 "kernels": [{k: st[k] for k in ("name", "launches", "total_ms")}
                             for st in bstats if st["launches"]]}
        bp.close()
        del bvis

    # F-engine (Appendix A step 2) producing this workload's voltages from raw
    # int8 samples: F = the channel count, 4-tap polyphase frames, T frames
    fe = None
    if rank == 0 and not args.no_fengine:
        F, P, T = w.channels, 4, w.samples
        S = (T + P - 1) * 2 * F
        gen = torch.Generator(device="cuda").manual_seed(9090007)
        raw = torch.randint(-128, 128, (w.n_antennas, S), generator=gen, device="cuda",
                            dtype=torch.int16).to(torch.int8)
        n = torch.arange(P * 2 * F, dtype=torch.float64)
        win = (torch.hann_window(P * 2 * F, periodic=False, dtype=torch.float64)
               * torch.sinc((n - (P * 2 * F - 1) / 2) / (2 * F))).float().cuda()
        fout = torch.empty((F, T, w.n_antennas, 2), dtype=torch.int8, device="cuda")
        need = omni.load().omni_fengine_scratch_bytes(w.n_antennas, S, F, P)
        fscr = torch.empty(need // 8, dtype=torch.float64, device="cuda")
        for _ in range(3):
            omni.fengine(raw, F, P, window=win, scale=0.05, out=fout, scratch=fscr)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 3
        e0.record(stream)
        for _ in range(reps):
            omni.fengine(raw, F, P, window=win, scale=0.05, out=fout, scratch=fscr)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_f = e0.elapsed_time(e1) / reps
        alg = raw.numel() + fout.numel()                  # raw in, int8 voltages out
        design = alg + 2 * need                           # plus the FP32 spectra round trip
        fe = {"value": w.n_antennas * T * F / (ms_f * 1e-3), "unit": UNIT, "ms_per_step": ms_f,
              "channels": F, "taps": P, "frames": T, "antennas": w.n_antennas,
              "hbm": {"algorithmic_bytes": alg, "design_bytes": design,
                      "achieved_GBs_design": design / (ms_f * 1e-3) / 1e9,
                      "frac_design": design / (ms_f * 1e-3) / 1e9 / hbm_peak_gbs()}}
        del raw, fout, fscr

    # tile hybrid (Sec. III) on the same voltages: the level-1 blocks as tiles at
    # their level-2 positions, correlated pairwise by brute force; on this
    # lattice, summing tile pairs with equal grid offsets must give back the
    # hypercube's visibilities
    tiles = None
    if rank == 0 and len(w.levels) == 2 and not args.no_tiles:
        lv1, lv2 = w.levels
        A2 = np.array(lv2.A, dtype=np.float64).reshape(2, 2)
        grid = np.array([(j1, j2) for j2 in range(lv2.n2) for j1 in range(lv2.n1)], dtype=np.float64)
        offs = grid @ A2.T
        N1, N2 = lv2.n1, lv2.n2
        tiles = {"tiles": N1 * N2, "pairs": (N1 * N2) ** 2}
        for tprec in ("mixed", "fp32"):
            try:
                tp = omni.TilePlan(lv1, offs, w.channels, dtype=w.dtype, precision=tprec)
            except omni.OmniError as e:
                tiles[tprec] = {"unsupported": str(e)}
                continue
            tvis = torch.empty((w.channels, tp.n_lags), dtype=torch.complex128, device="cuda")
            ms_t, clk_t, tstats, tunits = measure(tp, x, tvis, max(2, min(args.steps, 5)), 3, stream,
                                                  lambda: None, w.channels * w.samples)
            # regroup channel 0 by (intra-tile lag, tile-grid lag) and compare
            Vt = tp.split(tvis)[0]                                   # [i][j][Q1 Q2]
            gi = torch.arange(tp.n_tiles, device="cuda")
            d1 = (gi % N1)[:, None] - (gi % N1)[None, :] + (N1 - 1)
            d2 = (gi // N1)[:, None] - (gi // N1)[None, :] + (N2 - 1)
            dg = (d1 + (2 * N1 - 1) * d2).reshape(-1)                # tile-grid lag index
            acc = torch.zeros(((2 * N1 - 1) * (2 * N2 - 1), tp.n_tile_lags), dtype=torch.complex128,
                              device="cuda")
            acc.index_add_(0, dg, Vt.reshape(-1, tp.n_tile_lags))
            hyp = vis[0]
            diff = float((acc.reshape(-1) - hyp).abs().norm() / hyp.abs().norm())
            tiles[tprec] = {"value": units / (ms_t * 1e-3), "unit": UNIT, "ms_per_step": ms_t,
                            "clocks": clk_t, "rel_diff_vs_hypercube_ch0": diff,
                            "roofline": roofline(tstats, "tiles64", tprec, tunits),
                            "kernels": kernel_list(tstats)}
            tp.close()
            del tvis, acc

    n2 = None
    if rank == 0 and not args.no_direct and w.n_antennas <= 16384:
        # one channel of the same step's voltages (its visibilities are vis[0])
        rate_n2, diff_n2, sec_n2 = direct_n2(w, x[0], vis[0])
        n2 = {"value": rate_n2, "unit": UNIT, "seconds": sec_n2, "rel_diff_vs_hypercube": diff_n2,
              "sample": f"channel 0, {w.samples} samples, TF32 tensor-core GEMMs + lag binning"}

    others = None
    if rank == 0 and world == 1 and not args.no_others:
        others = other_workloads(args, stream)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r, cores, sample = oracle_rate(w, x[0:1, 0:64].cpu())
        cpu = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}

    if rank == 0:
        stats = head["stats"]
        line = {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": head["ms"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": {"mixed": "f16x3+f32", "mixed_bf16": "bf16x6+f32"}.get(args.precision, "f32"),
                "data": "synthetic",
                "config": line_config(w, args.precision, world),
                "timing": ("ms_per_step and value from CUDA events around the timed steps with "
                           "per-launch events off; roofline and kernels from %d further steps "
                           "with per-launch CUDA events" % PROFILED_STEPS),
                "roofline": roofline(stats, args.workload, args.precision, head["prof_units"],
                                     serial, sstats),
                "step_hbm": step_hbm(stats, head["ms"]),
                "serial_profiled_ms_per_step": serial_ms,
                "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": stats[0]["timed_launches"] if stats else 0,
                "clocks": clocks, "epilogue": epilogue, "direct_n2": n2, "beam_space": beams,
                "tile_hybrid": tiles, "fengine": fe, "other_workloads": others,
                "kernels": kernel_list(stats)}
        if "fp32" in results and args.precision != "fp32":
            f = results["fp32"]
            line["fp32_path"] = {"value": f["value"], "ms_per_step": f["ms"],
                                 "speedup_of_headline": head["value"] / f["value"]}
        if "mixed_bf16" in results and args.precision != "mixed_bf16":
            f = results["mixed_bf16"]
            line["mixed_bf16_path"] = {"value": f["value"], "ms_per_step": f["ms"], "clocks": f["clocks"],
                                       "note": "level 1 FP32 FFT, level 2 lag-space GEMM with BF16 "
                                               "operands split three ways (6 products)",
                                       "roofline": roofline(f["stats"], args.workload, "mixed_bf16",
                                                            f["prof_units"]),
                                       "kernels": kernel_list(f["stats"])}
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.destroy_process_group()


def run_batch(args):
    """Uneven independent arrays in one batch plan vs one plan per array (FP32 path)."""
    import torch
    import torch.distributed as dist
    from paper_0909_0001_gb300 import multirank

    rank, local_rank, world = multirank.rank_env()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    rec = batch_record(args, torch.cuda.current_stream(), rank=rank, barrier=barrier, dev=dev)
    if rank == 0:
        f = rec["paths"]["fp32"]
        line = {"metric": METRIC, "value": f["value"], "unit": UNIT, "n_gpus": world,
                "steps": f["steps"], "warmup": f["warmup"], "ms_per_step": f["ms_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic", "config": rec["config"], "roofline": f["roofline"],
                "gpu_launches": sum(k["launches"] for k in f["kernels"]) * f["steps"] // PROFILED_STEPS,
                "clocks": f["clocks"], "separate_plans": f["separate_plans"],
                "graph_replay": f["graph_replay"]}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch48":
        run_batch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
