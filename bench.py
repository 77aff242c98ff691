#!/usr/bin/env python3
"""Benchmark of the X-engine hot path on the 512-input, 128-channel workload.

One step = one pass of the whole hot path over one batch: 16 corr_accumulate calls of 8192-sample
blocks (N = 512 inputs = 256 dual-pol stations, C = 128 channels, 4+4-bit Gaussian-plus-tone samples;
unpack -> cross-multiply -> flush to int64, autos from the diagonal) followed by a dump of the cross
and auto accumulators with reset (the integrate-and-dump step). Inputs (16 distinct blocks, 8 GiB)
are resident in HBM before timing; they exceed L2, so no flush is needed between steps.

Prints ONE JSON line (rank 0). Metric: useful Tera-CMAC/s = N (N + 1) / 2 * C * T / time / 1e12, plus
the real-time factor at the 24.0 kHz channel rate. `--impl reference` times the CPU oracle instead.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--path fp8tc|i8mma|fp32] [--impl reference]
Multi-GPU: launched by torch.distributed.run; channels are independent, so rank r correlates its own
contiguous 128-channel range (replicas.channel_shards) of a band of 128 x n_gpus channels (weak
scaling), with no data-path collective.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Tera-CMAC/s + real-time factor, 512-input 4-bit X-engine: int8-TC vs FP32 path"
N_IN, N_CHAN, T_BLOCK, N_BLOCKS, N_POL = 512, 128, 8192, 16, 2
CHANNEL_RATE_HZ = 24000.0  # 98.304 MHz / 4096 (Sec. 2)
SEED = 0x14113751 + 2
WORKLOAD = "N=512 inputs (256 dual-pol stations), 128 channels, 16 blocks x 8192 samples per step, 4+4-bit Gaussian sigma=2.5 + common tone rho=0.1"


def useful_cmacs(N, C, T):
    return N * (N + 1) // 2 * C * T


def source_hash(kernel_files):
    import hashlib

    h = hashlib.sha256()
    for f in kernel_files:
        h.update(open(os.path.join(ROOT, "paper_1411_3751_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel_files, profile_md, blocks_per_launch, tile_plan=None):
    """DRAM bytes per launch recorded by an ncu capture (profiles/), if the kernel sources still match
    and the capture covered launches of the same size (and tile plan, where it records one)."""
    try:
        text = open(os.path.join(ROOT, "profiles", profile_md)).read()
        keys = ("traffic_bytes_per_launch:", "source_sha256:", "blocks_per_launch:", "tile_plan:")
        vals = dict(l.split(": ", 1) for l in text.splitlines() if l.startswith(keys))
        if vals.get("source_sha256", "").strip() != source_hash(kernel_files):
            return None
        if abs(float(vals.get("blocks_per_launch", "1")) - blocks_per_launch) > 1e-9:
            return None
        if tile_plan is not None and "tile_plan" in vals and int(vals["tile_plan"]) != tile_plan:
            return None
        return int(vals["traffic_bytes_per_launch"])
    except Exception:
        return None


XENG_SOURCES = ["xeng_fp8tc.cu", "f8_common.cuh", "ptx_sm100.cuh"]
PAIR_SOURCES = ["xeng_pair.cu", "f8_common.cuh", "ptx_sm100.cuh"]
PREP_SOURCES = ["f8_prep.cu", "f8_common.cuh"]


def xeng_profile(tile_plan):
    """(kernel name, its sources, its ncu summary in profiles/) for the X-engine of a tile plan."""
    if tile_plan == 3:
        return "f8_xeng_pair_kernel", PAIR_SOURCES, "f8_xeng_pair_512in_128ch_8192.md"
    return "f8_xeng_kernel", XENG_SOURCES, "f8_xeng_512in_128ch_8192.md"


def step_traffic(xeng_launches, prep_launches, blocks_per_launch, tile_plan, ms_step=None, hbm_gbs=None):
    """DRAM bytes of one step from the ncu captures summarised in profiles/ (per launch, source-hash
    checked) against the algorithmic bytes of the step: the input read once, the int64 cross
    accumulators read and written once per X-engine launch, and the dumped visibilities written once;
    with the step time, the rate those bytes imply as a share of the measured HBM copy bandwidth (the
    builds beside the multiply move the same bytes as in sequence)."""
    from paper_1411_3751_gb300 import corr

    acc = N_CHAN * corr.corr_n_baselines(N_IN, N_POL) * N_POL * N_POL * 2 * 8
    inp = T_BLOCK * N_BLOCKS * N_CHAN * N_IN
    alg = inp + xeng_launches * 2 * acc + acc
    _, x_src, x_md = xeng_profile(tile_plan)
    x = profiled_traffic(x_src, x_md, blocks_per_launch, tile_plan)
    pr = profiled_traffic(PREP_SOURCES, "f8_prep_512in_128ch_8192.md", 1)
    out = {"algorithmic_bytes": alg, "xeng_bytes_per_launch": x, "prep_bytes_per_launch": pr,
           "xeng_launches": xeng_launches, "prep_launches": prep_launches}
    if x is not None and pr is not None:
        dump = 3 * acc  # dump kernels (not captured) at their own algorithmic bytes: read, write, reset
        meas = x * xeng_launches + pr * prep_launches + dump
        out.update({"measured_bytes": meas, "ratio": meas / alg})
        if ms_step and hbm_gbs:
            out["step_gbs"] = meas / (ms_step / 1e3) / 1e9
            out["step_frac_of_hbm"] = out["step_gbs"] / hbm_gbs
    return out


def run_extras():
    """The other workloads of the metric, shortened so the whole benchmark stays within minutes:
    flush overhead at 512 inputs x 256 channels x 65536 samples (saturating inputs), five uneven
    sub-arrays in one grouped graph-replayed launch vs separate launches, the streaming loop over
    18 s of data (two 9 s cross dumps and eighteen 1 s total-power dumps per stream), and the 32- and
    64-input arrays against the HBM copy bandwidth."""
    import torch

    from paper_1411_3751_gb300 import corr, measure_configs, synth

    out = {}
    for name, fn in (("precision", lambda: measure_configs.precision(corr, synth, torch, reps=2)),
                     ("group", lambda: measure_configs.group(corr, synth, torch, reps=5)),
                     ("stream", lambda: measure_configs.stream_loop(corr, synth, torch, n_blocks=1800)),
                     ("small", lambda: measure_configs.small(corr, synth, torch, reps=3))):
        t0 = time.perf_counter()
        try:
            out[name] = fn()
        except Exception as e:  # a failing extra must not cost the headline line
            out[name] = {"error": "%s: %s" % (type(e).__name__, e)}
        out[name]["wall_s"] = time.perf_counter() - t0
        torch.cuda.empty_cache()
    return out


def issued_flops_per_sample(n_inputs, n_chans, plan=0):
    """MMA flops the tensor path issues per sample under a tile plan (M = 128 instructions of N = nb
    columns; plan 2 items carry a second half of nb1 = extra & 0xFFFF columns), split into wide
    (N = 256) and narrow (N <= 128) instructions. A plan-3 item is one M = 256, N = 256 instruction on
    an SM pair: per SM the work of an M = 128, N = 256 one, counted as two wide instructions."""
    from paper_1411_3751_gb300 import corr

    wide = narrow = 0
    if plan == 3:
        return 2 * 256 * 256 * n_chans * len(corr.corr_tile_plan(n_inputs, 3)), 0
    for _c0, _a0, nb, extra in corr.corr_tile_plan(n_inputs, plan):
        for n in (nb, (extra & 0xFFFF) if plan == 2 else 0):
            if n > 128:
                wide += 2 * 128 * n * n_chans
            elif n > 0:
                narrow += 2 * 128 * n * n_chans
    return wide, narrow


def roofline_peak(peaks, clk, timed_s):
    """FP8 tensor peak from the measured bf16 GEMM rate (x 2, the nominal fp8/bf16 ratio): the burst
    figure when the kernel ran at the maximum SM clock with no power cap over a short timed region
    (under a second), else the sustained figure (a seconds-long loop under the power cap)."""
    at_max = bool(clk.get("sm_mhz") and clk.get("sm_max_mhz") and clk["sm_mhz"] >= 0.98 * clk["sm_max_mhz"])
    capped = "sw_power_cap" in (clk.get("reasons") or [])
    burst = at_max and not capped and timed_s < 1.0
    key = "bf16_tflops" if burst else "bf16_tflops_sustained"
    val = peaks.get(key, peaks.get("bf16_tflops"))
    why = ("SM clock at its maximum, no power cap, %.2f s timed" % timed_s if burst else
           "SM clock %s of %s MHz, power cap %s, %.2f s timed" % (clk.get("sm_mhz"), clk.get("sm_max_mhz"),
                                                                 "active" if capped else "inactive", timed_s))
    return 2.0 * float(val), ("burst" if burst else "sustained"), why


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(n_gpus):
    from paper_1411_3751_gb300 import replicas

    # a replica that dies makes the others' next barrier fail within 10 minutes instead of hanging
    return replicas.init("nccl", timeout_s=600)


def barrier(world):
    from paper_1411_3751_gb300 import replicas

    replicas.barrier(world)


def max_over_ranks(x, world):
    from paper_1411_3751_gb300 import replicas

    return replicas.max_over_ranks(x, world, "cuda")


def cpu_baseline(seconds_target=15.0):
    """Time the CPU oracle on a bounded sample of the workload (all host cores, channels in parallel)."""
    import numpy as np

    from oracle import oracle
    from paper_1411_3751_gb300 import synth

    cores = os.cpu_count() or 1
    spec = synth.Spec(kind="gauss_tone", seed=SEED)
    # calibration: one channel x 1024 samples on one thread
    x = synth.generate_host(spec, 1024, 1, N_IN)
    t0 = time.perf_counter()
    oracle.correlate(x, N_POL, threads=1)
    per_cmac = (time.perf_counter() - t0) / useful_cmacs(N_IN, 1, 1024)
    # one thread on one channel, about 2 s
    T1 = int(2.0 / (per_cmac * useful_cmacs(N_IN, 1, 1))) if per_cmac > 0 else 1024
    T1 = max(256, min(T_BLOCK, (T1 // 256) * 256))
    x = synth.generate_host(spec, T1, 1, N_IN)
    t0 = time.perf_counter()
    oracle.correlate(x, N_POL, threads=1)
    dt1 = time.perf_counter() - t0
    single = {"value": useful_cmacs(N_IN, 1, T1) / dt1 / 1e12, "cores": 1,
              "sample": "1 channel x %d samples x %d inputs, %.1f s" % (T1, N_IN, dt1)}
    chans = cores
    T = int(seconds_target / (per_cmac * useful_cmacs(N_IN, 1, 1)) / 1.0) if per_cmac > 0 else 1024
    T = max(256, min(T_BLOCK, (T // 256) * 256))
    x = synth.generate_host(spec, T, chans, N_IN)
    t0 = time.perf_counter()
    oracle.correlate(x, N_POL, threads=cores)
    dt = time.perf_counter() - t0
    cm = useful_cmacs(N_IN, chans, T)
    return {"value": cm / dt / 1e12, "unit": "Tera-CMAC/s", "cores": cores, "kind": "oracle",
            "sample": "%d channels x %d samples x %d inputs (of 128 x 131072 x 512), %.1f s, threads across channels"
                      % (chans, T, N_IN, dt),
            "real_time_factor": (T / CHANNEL_RATE_HZ) / dt * (chans / N_CHAN), "single_thread": single}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import __graft_entry__

    __graft_entry__.build()
    import numpy as np

    from oracle import oracle
    from paper_1411_3751_gb300 import synth

    cores = os.cpu_count() or 1
    spec = synth.Spec(kind="gauss_tone", seed=SEED)
    chans, T = cores, 512
    x = synth.generate_host(spec, T, chans, N_IN)
    for _ in range(max(0, args.warmup)):
        oracle.correlate(x[:64], N_POL, threads=cores)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.correlate(x, N_POL, threads=cores)
        times.append(time.perf_counter() - t0)
    dt = sum(times)
    cm = useful_cmacs(N_IN, chans, T) * args.steps
    value = cm / dt / 1e12
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Tera-CMAC/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "n_inputs": N_IN, "n_chans": N_CHAN,
                                            "n_time_per_step": T_BLOCK * N_BLOCKS, "n_pol": N_POL},
            "cpu_baseline": {"value": value, "unit": "Tera-CMAC/s", "cores": cores, "kind": "oracle",
                             "sample": "each step: %d channels x %d samples x %d inputs on %d threads" % (chans, T, N_IN, cores)},
            "e2e": {"value": value, "unit": "Tera-CMAC/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--path", default="fp8tc", choices=["fp8tc", "fp8tc_fused", "i8mma", "fp32"])
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=-1,
                    help="steps of the end-to-end leg (default: as many as --steps; 0 skips it)")
    ap.add_argument("--fp32-steps", type=int, default=2)
    ap.add_argument("--i8-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the flush-overhead, grouped-launch, streaming and small-array measurements")
    ap.add_argument("--no-probe", action="store_true", help="skip the tcgen05 issue-rate probe")
    ap.add_argument("--no-autotune", action="store_true", help="keep the library's default batch schedule")
    ap.add_argument("--tile-plan", type=int, default=-1,
                    help="tile plan of the tensor path (0-3; -1: the library default, then the autotuner)")
    ap.add_argument("--prep-sms", type=int, default=-1,
                    help="SMs building the next launch's operand beside the X-engine (-1 library default, 0 none)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.e2e_steps < 0:
        args.e2e_steps = args.steps
    if args.impl == "reference":
        return run_reference(args)

    import torch

    import __graft_entry__

    world, rank, local = dist_setup(args.gpus)
    if rank == 0 or not os.path.exists(os.path.join(ROOT, "paper_1411_3751_gb300", "_build", "libcorr.so")):
        __graft_entry__.build()
    barrier(world)
    from paper_1411_3751_gb300 import corr, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    # rank r correlates its own contiguous channel range of a band of N_CHAN x world channels (the
    # paper's partition: each GPU its own channels, no exchange in the X stage); at one GPU the band
    # is the 128-channel workload itself
    from paper_1411_3751_gb300 import replicas

    band = N_CHAN * world
    c0, c1 = replicas.channel_shards(band, world)[rank]
    spec = synth.Spec(kind="gauss_tone", seed=SEED)
    blocks = [synth.generate_device(spec, T_BLOCK, band, N_IN, t0=b * T_BLOCK, c_range=(c0, c1))
              for b in range(N_BLOCKS)]
    torch.cuda.synchronize()
    xc = corr.Correlator(N_IN, N_CHAN, T_BLOCK, N_POL, path=args.path)
    xc.set_prep_sms(args.prep_sms)
    if args.tile_plan >= 0 and args.path.startswith("fp8tc"):
        xc.set_tile_plan(args.tile_plan)
    tuning = None
    if args.path == "fp8tc" and not args.no_autotune and args.prep_sms == -1 and args.tile_plan < 0:
        # the batch schedule (tile plan, blocks per launch, concurrent build SMs) timed on these blocks
        tuning = xc.autotune(blocks, reps=2)
    xc_plan = xc.tile_plan if args.path.startswith("fp8tc") else 0
    cross_out = torch.empty(xc.out_shape(corr.CORR_WHAT_CROSS), dtype=torch.int64, device=dev)
    autos_out = torch.empty(xc.out_shape(corr.CORR_WHAT_AUTO), dtype=torch.int64, device=dev)

    def step():
        xc.accumulate_batch(blocks)
        xc.dump(corr.CORR_WHAT_CROSS, reset=True, out=cross_out)
        xc.dump(corr.CORR_WHAT_AUTO, reset=True, out=autos_out)

    for _ in range(args.warmup):
        step()
    xc.sync()
    # the tcgen05 issue rate of this GPU at its current clock, just before the timed region
    probe = None
    if args.path.startswith("fp8tc") and not args.no_probe:
        r256 = corr.corr_probe_mma_rate(16384, 256, stream.cuda_stream)
        r128 = corr.corr_probe_mma_rate(16384, 128, stream.cuda_stream)
        probe = {"tflops_n256": r256[0], "cycles_per_mma_n256": r256[1], "tflops_n128": r128[0],
                 "cycles_per_mma_n128": r128[1], "mma_per_sm": 16384,
                 "what": "tcgen05.mma kind::f8f6f4 M=128 K=32 back to back from unchanging shared memory, one CTA per SM"}
    # timed region
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    xc.profile(True)
    barrier(world)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms_total = ev0.elapsed_time(ev1)
    xeng_ms, xeng_n = xc.profile_read(corr.CORR_KERNEL_XENG)
    unpack_ms, unpack_n = xc.profile_read(corr.CORR_KERNEL_UNPACK)
    dump_ms, dump_n = xc.profile_read(corr.CORR_KERNEL_DUMP)
    autos_ms, autos_n = xc.profile_read(corr.CORR_KERNEL_AUTOS)
    xc.profile(False)
    clk = clocks.stop()
    xc.sync()
    ms_total = max_over_ranks(ms_total, world)
    ms_step = ms_total / args.steps
    cm_step = useful_cmacs(N_IN, N_CHAN, T_BLOCK * N_BLOCKS)
    value = cm_step * args.steps * world / (ms_total / 1e3) / 1e12
    rtf = (T_BLOCK * N_BLOCKS / CHANNEL_RATE_HZ) / (ms_step / 1e3)

    # roofline of the dominant kernel (the X-engine), from its live event timings
    peaks, peak_src = load_peaks()
    per_launch_ms = xeng_ms / max(1, xeng_n)
    # algorithmic flops of one X-engine launch: a batch launch covers several 8192-sample blocks
    blocks_per_launch = N_BLOCKS * args.steps / max(1, xeng_n)
    flops_launch = 8.0 * useful_cmacs(N_IN, N_CHAN, T_BLOCK) * blocks_per_launch
    if args.path.startswith("fp8tc"):
        peak, which, why = roofline_peak(peaks, clk, ms_total / 1e3)
        peak_note = "%s bf16 %s x 2 (nominal fp8/bf16 ratio): %s" % (peak_src, which, why)
        bound = "tensor"
    elif args.path == "i8mma":
        peak = 158.0  # mma.sync m16n8k32 s8 throughput measured by a microbenchmark on this GPU
        peak_note = "mma.sync s8 microbenchmark (TOP/s)"
        bound = "tensor"
    else:
        peak = 77.9  # FP32 FMA peak measured by a microbenchmark on this GPU at 1.95 GHz
        peak_note = "FP32 FMA microbenchmark (152 SMs x 128 lanes x 2 flop)"
        bound = "alu"
    achieved = flops_launch / (per_launch_ms / 1e3) / 1e12
    # with overlapped batches the X-engine shares the GPU with the operand build: all launches but
    # the last of each batch run on SMs - prep_sms SMs
    n_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    prep_sms = xc.prep_sms if args.path == "fp8tc" else 0
    launches_per_batch = max(1, round(xeng_n / args.steps))
    if prep_sms > 0 and launches_per_batch > 1:
        sm_share = ((launches_per_batch - 1) * (n_sms - prep_sms) + n_sms) / (launches_per_batch * n_sms)
    else:
        sm_share = 1.0
    traffic = None
    x_kernel, x_src, x_md = xeng_profile(xc_plan)
    if args.path == "fp8tc":
        traffic = profiled_traffic(x_src, x_md, blocks_per_launch, xc_plan)
    roof = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": traffic, "kernel": {"fp8tc": x_kernel, "fp8tc_fused": "f8_fused_kernel",
                                           "i8mma": "xeng_i8mma_kernel"}.get(args.path, "xeng_fp32_kernel"),
            "peak_source": peak_note, "launch_ms": per_launch_ms,
            "algorithmic": "8 flop x N(N+1)/2 x C x T per launch = %.3e flop (%.0f blocks of 8192 samples per launch)"
                           % (flops_launch, blocks_per_launch),
            "sm_share": sm_share, "frac_of_sms_held": achieved / peak / sm_share}
    if args.path.startswith("fp8tc") and probe:
        # the same kernel against the tcgen05 issue rate measured on this GPU just before the timed
        # region: the ideal launch time of the MMAs the tile plan issues, and the useful rate's share
        wide, narrow = issued_flops_per_sample(N_IN, N_CHAN, xc_plan)
        samples = T_BLOCK * blocks_per_launch
        ideal_ms = (wide * samples / (probe["tflops_n256"] * 1e12) + narrow * samples / (probe["tflops_n128"] * 1e12)) * 1e3
        roof["issue_probe"] = dict(probe)
        roof["issued_flop_per_launch"] = (wide + narrow) * samples
        roof["frac_issue"] = ideal_ms / per_launch_ms
        roof["frac_useful_of_issue_peak"] = achieved / probe["tflops_n256"]
    if args.path == "fp8tc":
        roof["step_traffic"] = step_traffic(xeng_n / args.steps, unpack_n / args.steps, blocks_per_launch, xc_plan,
                                            ms_step, peaks.get("hbm_gbs") if peaks else None)
    if args.path == "fp8tc" and prep_sms > 0 and launches_per_batch > 1:
        # the step overlaps the operand build with the multiply, so the X-engine launches above ran on
        # fewer SMs beside a build; the same kernel on the same launches with the passes in sequence
        # (the whole GPU, nothing beside it), timed after the step's timed region
        xc.set_prep_sms(0)
        step()
        xc.sync()
        xc.profile(True)
        for _ in range(5):
            step()
        xc.sync()
        iso_ms, iso_n = xc.profile_read(corr.CORR_KERNEL_XENG)
        xc.profile(False)
        xc.set_prep_sms(prep_sms)
        iso_launch = iso_ms / max(1, iso_n)
        # a few launches on the whole GPU with nothing beside them: against the burst peak
        iso_peak = 2.0 * peaks["bf16_tflops"] if peaks and "bf16_tflops" in peaks else peak
        iso = {"launch_ms": iso_launch, "achieved": flops_launch / (iso_launch / 1e3) / 1e12, "peak": iso_peak,
               "peak_source": "%s bf16 burst x 2 (20 launches on the whole GPU, nothing beside them)" % peak_src,
               "what": "the same kernel and launches with the batch's two passes in sequence (whole GPU, no "
                       "concurrent build), 5 steps after the timed region"}
        iso["frac"] = iso["achieved"] / iso_peak
        if probe:
            iso["frac_issue"] = ideal_ms / iso_launch
        roof["isolated"] = iso

    # end-to-end through the public API from pinned host buffers
    e2e = None
    if args.e2e_steps > 0:
        # pinned buffers filled straight from the device (no pageable intermediate copies)
        host_blocks = [torch.empty(tuple(blocks[b].shape), dtype=torch.uint8, pin_memory=True) for b in range(N_BLOCKS)]
        for b in range(N_BLOCKS):
            host_blocks[b].copy_(blocks[b])
        torch.cuda.synchronize()
        cross_h = torch.empty(xc.out_shape(corr.CORR_WHAT_CROSS), dtype=torch.int64).pin_memory()
        autos_h = torch.empty(xc.out_shape(corr.CORR_WHAT_AUTO), dtype=torch.int64).pin_memory()

        def e2e_step():
            for b in range(N_BLOCKS):
                xc.accumulate_host(host_blocks[b])
            xc.dump(corr.CORR_WHAT_CROSS, reset=True, out=cross_h)
            xc.dump(corr.CORR_WHAT_AUTO, reset=True, out=autos_h)

        e2e_step()
        torch.cuda.synchronize()
        barrier(world)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        marks = []
        e0.record(stream)
        for _ in range(args.e2e_steps):
            e2e_step()
            marks.append(torch.cuda.Event(enable_timing=True))
            marks[-1].record(stream)
        e1.record(stream)
        torch.cuda.synchronize()
        e_ms = max_over_ranks(e0.elapsed_time(e1), world)
        # per-step times, so that a sporadic stall of the host link shows as such
        per_step = sorted([e0.elapsed_time(marks[0])] + [marks[k - 1].elapsed_time(marks[k])
                                                          for k in range(1, len(marks))])
        # the host link on this machine: plain pinned copies of the same blocks, same process
        scratch = torch.empty_like(blocks[0])
        scratch.copy_(host_blocks[0], non_blocking=True)
        torch.cuda.synchronize()
        l0, l1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0.record()
        for b in range(N_BLOCKS):
            scratch.copy_(host_blocks[b], non_blocking=True)
        l1.record()
        torch.cuda.synchronize()
        h2d = N_BLOCKS * T_BLOCK * N_CHAN * N_IN
        link_gbs = h2d / (l0.elapsed_time(l1) / 1e3) / 1e9
        e2e = {"value": cm_step * args.e2e_steps * world / (e_ms / 1e3) / 1e12, "unit": "Tera-CMAC/s",
               "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": cross_h.numel() * 8 + autos_h.numel() * 8,
               "ms_per_step": e_ms / args.e2e_steps,
               "ms_per_step_median": per_step[len(per_step) // 2], "ms_per_step_max": per_step[-1],
               "link_h2d_gbs": link_gbs, "link_bound_ms_per_step": h2d / link_gbs / 1e6}
        del host_blocks, scratch

    # same-GPU comparison legs of the metric on the same workload: the integer tensor path
    # (mma.sync s8) and the FP32 CUDA-core path (the paper's arithmetic)
    def path_leg(path, n_steps):
        if not args.path.startswith("fp8tc") or n_steps <= 0:
            return None
        xc.set_path(path)
        step()
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(n_steps):
            step()
        f1.record(stream)
        torch.cuda.synchronize()
        f_ms = max_over_ranks(f0.elapsed_time(f1), world) / n_steps
        xc.set_path(args.path)
        return {"value": cm_step * world / (f_ms / 1e3) / 1e12, "unit": "Tera-CMAC/s", "ms_per_step": f_ms,
                "real_time_factor": (T_BLOCK * N_BLOCKS / CHANNEL_RATE_HZ) / (f_ms / 1e3), "steps": n_steps}

    i8 = path_leg("i8mma", args.i8_steps)
    fp32 = path_leg("fp32", args.fp32_steps)
    xc.sync()
    xc.close()
    extras = None
    if rank == 0 and world == 1 and not args.no_extras:
        del blocks, cross_out, autos_out
        torch.cuda.empty_cache()
        extras = run_extras()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline()

    if rank == 0:
        launches_per_step = (xeng_n + unpack_n + dump_n + autos_n) / args.steps
        line = {
            "metric": METRIC, "value": value, "unit": "Tera-CMAC/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"i8mma": "s8", "fp32": "f32"}.get(args.path, "e4m3"), "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_inputs": N_IN, "n_chans": N_CHAN, "n_time_per_block": T_BLOCK,
                       "blocks_per_step": N_BLOCKS, "n_pol": N_POL, "path": args.path,
                       "prep_sms": prep_sms, "tile_plan": xc_plan,
                       "blocks_per_launch": blocks_per_launch, "autotune": tuning,
                       "l2": "inputs 8 GiB > L2, no flush needed",
                       "parallelism": "channel shards: each GPU a contiguous 128-channel range of a 128 x n_gpus-channel band",
                       "band_channels": N_CHAN * world},
            "real_time_factor": rtf,
            "roofline": roof,
            "kernel_ms_per_step": {"xeng": xeng_ms / args.steps, "unpack": unpack_ms / args.steps,
                                   "autos": autos_ms / args.steps, "dump": dump_ms / args.steps},
            "gpu_launches": (xeng_n + unpack_n + dump_n + autos_n),
            "gpu_launches_per_step": launches_per_step,
            "clocks": clk,
            "e2e": e2e,
            "i8mma_path": i8,
            "fp32_path": fp32,
            "cpu_baseline": cpu,
        }
        if extras is not None:
            line["configs"] = extras
        print(json.dumps(line))
    from paper_1411_3751_gb300 import replicas

    replicas.finalize(world)
    return 0


if __name__ == "__main__":
    sys.exit(main())
