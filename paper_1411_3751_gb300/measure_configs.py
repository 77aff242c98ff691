"""Measurements of the secondary workloads (one JSON line each):

* tiny: 32 inputs x 8 channels x 1024 samples (uniform components), each arithmetic path; a launch-
  bound case (the FP32 path is the paper's arithmetic);

* small: 32 and 64 inputs (LWA1's 64-input system) x 2400 channels x 4 blocks of 8192 samples, FP8
  tensor path: Tera-CMAC/s and the HBM traffic of the two passes (input read once, operand written
  and read back) against the measured copy bandwidth, the bound for these small arrays;
* precision: 512 inputs x 256 channels x 65536 samples with saturation-heavy segments; X-engine time
  with in-chip partial sums flushed to int64 every 4096 / 16384 / 65536 samples on the FP8 tcgen05
  path and every 16384 / 65536 samples on the int8 mma.sync path (the flush overhead is the
  difference to the 65536 case);
* group: sub-arrays of 32, 64, 200, 256 and 512 inputs with 2400, 600, 300, 150 and 109 channels of
  4096 samples: one autotuned grouped launch replayed from a CUDA graph vs separate per-array launches;
* stream: one 512-input x 2400-channel stream and three 64-input streams in 10 ms blocks with 9 s
  cross-power and 1 s total-power dumps over >= 100 s-equivalent; real-time factor and dump latency;
* requant: the F-engine tail at the paper's sizes: 512 inputs x 1024 spectra of a 4096-channel PFB
  (18+18-bit integers), 2398 channels selected, requantised to 4+4 bits and corner-turned; bytes moved
  per second against the measured HBM copy bandwidth;
* pfb: the PFB F-engine at the paper's sizes: 512 inputs, 4 taps, 8192-point real FFT, 64 spectra
  (int8 ADC samples -> float32 channels); spectra per second against the 24 000 per second per input
  a 196.608 MHz ADC produces;
* fastdump: the 512-input x 2400-channel stream at the paper's minimum dump time (0.33 s = 8000
  samples, float32 visibilities) with 1 s total power of ten outrigger stations (selective dumps).

    python -m paper_1411_3751_gb300.measure_configs [--only tiny|small|precision|group|stream|fastdump|requant|pfb]
"""
from __future__ import annotations

import argparse
import json
import os
import sys


def _useful(N, C, T):
    return N * (N + 1) // 2 * C * T


def tiny(corr, synth, torch, reps=200):
    N, C, T, npol = 32, 8, 1024, 2
    x = synth.generate_device(synth.Spec(kind="uniform", seed=0x14113751 + 1), T, C, N)
    out = {"config": "tiny: N=32, C=8, T=1024, uniform"}
    for path in ("fp32", "i8mma", "fp8tc"):
        with corr.Correlator(N, C, T, npol, path=path) as xc:
            for _ in range(3):
                xc.accumulate(x)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                xc.accumulate(x)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
        out[path] = {"ms_per_block": ms, "tcmac_s": _useful(N, C, T) / (ms / 1e3) / 1e12,
                     "real_time_factor": (T / 24000.0) / (ms / 1e3)}
    return out


def small(corr, synth, torch, reps=5, path="fp8tc"):
    import json as _json

    try:
        hbm = float(_json.load(open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                                                 "MEASURED_PEAKS.json")))["hbm_gbs"])
    except Exception:
        hbm = 6800.0
    out = {"config": "small: N=32 and 64, C=2400, 4 x 8192 samples, %s" % path, "hbm_gbs_peak": hbm}
    T, C, B, npol = 8192, 2400, 4, 2
    for N in (32, 64):
        blocks = [synth.generate_device(synth.Spec(kind="gauss_tone", seed=0x14113751 + 60 + b), T, C, N)
                  for b in range(B)]
        with corr.Correlator(N, C, T, npol, path=path) as xc:
            xc.accumulate_batch(blocks)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                xc.accumulate_batch(blocks)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
        r_buf = ((2 * N + 31) // 32) * 32
        samples = T * B * C
        moved = samples * N + 2 * samples * r_buf  # input once, operand written and read back
        out[str(N)] = {"ms_per_step": ms, "tcmac_s": _useful(N, C, T * B) / (ms / 1e3) / 1e12,
                       "hbm_gbs": moved / (ms / 1e3) / 1e9, "hbm_frac": moved / (ms / 1e3) / 1e9 / hbm,
                       "real_time_factor": (T * B / 24000.0) / (ms / 1e3)}
        del blocks
    return out


def precision(corr, synth, torch, reps=3):
    N, C, T, npol = 512, 256, 65536, 2
    spec = synth.Spec(kind="saturate", seed=0x14113751 + 3, seg_len=4096, m8_segment=5)
    x = synth.generate_device(spec, T, C, N)
    out = {"config": "precision: N=512, C=256, T=65536, saturating segments"}
    for path, flushes in (("fp8tc", (4096, 16384, 65536)), ("i8mma", (16384, 65536))):
        res = {}
        with corr.Correlator(N, C, T, npol, path=path) as xc:
            for flush in flushes:
                xc.set_flush_period(flush)
                xc.accumulate(x)  # warm-up
                xc.sync()
                xc.profile(True)
                for _ in range(reps):
                    xc.accumulate(x)
                ms, n = xc.profile_read(corr.CORR_KERNEL_XENG)
                pms, _ = xc.profile_read(corr.CORR_KERNEL_UNPACK)
                xc.profile(False)
                xc.reset()
                res[str(flush)] = {"xeng_ms": ms / n, "prep_ms": pms / n,
                                   "tcmac_s": _useful(N, C, T) / (ms / n / 1e3) / 1e12}
        base = res["65536"]["xeng_ms"]
        out[path] = {"flush": res,
                     "flush_overhead_pct": {k: 100.0 * (v["xeng_ms"] - base) / base for k, v in res.items()}}
    return out


def group(corr, synth, torch, reps=5):
    shapes = [(32, 2400), (64, 600), (200, 300), (256, 150), (512, 109)]
    T, npol = 4096, 2
    blocks = [synth.generate_device(synth.Spec(kind="gauss_tone", seed=0x14113751 + 4 + 100 * i), T, c, n)
              for i, (n, c) in enumerate(shapes)]
    useful = sum(_useful(n, c, T) for n, c in shapes)
    st = torch.cuda.Stream()
    res = {"config": "group: N=%s C=%s T=4096" % ([s[0] for s in shapes], [s[1] for s in shapes])}
    with torch.cuda.stream(st), corr.Group(shapes, T, npol) as g:
        res["tile_plans"] = g.autotune(blocks)
        g.capture(blocks, st)
        for name, fn in (("grouped_graph", lambda: g.launch(st)), ("grouped", lambda: g.accumulate(blocks)),
                         ("separate", lambda: g.accumulate(blocks, separate=True))):
            fn()
            st.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(reps):
                fn()
            e1.record(st)
            st.synchronize()
            ms = e0.elapsed_time(e1) / reps
            res[name] = {"ms": ms, "tcmac_s": useful / (ms / 1e3) / 1e12}
    res["speedup_graph_vs_separate"] = res["separate"]["ms"] / res["grouped_graph"]["ms"]
    return res


def stream_loop(corr, synth, torch, n_blocks=10000):
    from . import stream

    specs = [stream.StreamSpec("leda512", 512, 2400, gulp_blocks=25, seed=0x14113751 + 5)]
    specs += [stream.StreamSpec("lwa64_%d" % k, 64, 2400, gulp_blocks=25, seed=0x14113751 + 50 + k) for k in range(3)]
    srv = stream.Server(hbm_budget_bytes=sum(s.footprint() for s in specs) + (1 << 30), keep_dumps=0)
    try:
        for s in specs:
            srv.admit(s)
        srv.admit(stream.StreamSpec("extra512", 512, 2400, gulp_blocks=25))
        out = srv.run(n_blocks)
    finally:
        srv.close()
    out["config"] = "stream: 512x2400 + 3 x 64x2400 inputs x channels, 10 ms blocks, %d blocks" % n_blocks
    return out


def fast_dump(corr, synth, torch, n_blocks=60):
    from . import stream

    outr = (251, 252, 253, 254, 255, 3, 77, 128, 200, 9)
    sp = stream.StreamSpec("leda512_fast", 512, 2400, block_samples=8000, gulp_blocks=1, cross_every=1,
                           auto_every=3, seed=0x14113751 + 6, outriggers=outr, cross_fmt=corr.CORR_FMT_CF32)
    srv = stream.Server(hbm_budget_bytes=sp.footprint() + (1 << 30), keep_dumps=0)
    try:
        srv.admit(sp)
        out = srv.run(n_blocks)
    finally:
        srv.close()
    out["config"] = ("fastdump: 512 x 2400 inputs x channels, 8000-sample blocks (0.33 s), float32 cross dump "
                     "every block, outrigger total power every 3 blocks, %d blocks" % n_blocks)
    out["cross_bytes_per_dump"] = 2400 * 32896 * 4 * 2 * 4
    return out


def requant(corr, synth, torch, reps=5):
    import json as _json

    N, T, F, chan0, C = 512, 1024, 4096, 1229, 2398
    g = torch.Generator(device="cuda")
    g.manual_seed(0x14113751 + 7)
    x = (torch.randn((N, T, F, 2), device="cuda", generator=g) * 3000.0).round_().clamp_(-(1 << 17), (1 << 17) - 1)
    x = x.to(torch.int32)
    out = torch.empty((T, C, N), dtype=torch.uint8, device="cuda")
    gain = 2.5 / 3000.0
    corr.requantize(x, chan0, C, gain=gain, out=out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        corr.requantize(x, chan0, C, gain=gain, out=out)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    moved = N * T * C * (8 + 1)  # read the selected int32 pairs, write one byte per sample
    try:
        peaks = _json.load(open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                                             "MEASURED_PEAKS.json")))
        hbm = float(peaks["hbm_gbs"])
    except Exception:
        hbm = 6800.0
    return {"config": "requant: N=512, T=1024, F=4096, chan0=1229, C=2398, int32 in", "ms": ms,
            "gbs": moved / (ms / 1e3) / 1e9, "frac_of_hbm": moved / (ms / 1e3) / 1e9 / hbm,
            "samples_per_s": N * T * C / (ms / 1e3),
            "real_time_factor": (T / 24000.0) / (ms / 1e3)}


def pfb(corr, synth, torch, reps=5):
    N, T, P = 512, 64, 4
    g = torch.Generator(device="cuda")
    g.manual_seed(0x14113751 + 8)
    adc = (torch.randn((N, (T + P - 1) * 8192), device="cuda", generator=g) * 20.0).round_().clamp_(-128, 127)
    adc = adc.to(torch.int8)
    out = torch.empty((N, T, 4096, 2), dtype=torch.float32, device="cuda")
    corr.pfb(adc, P, out=out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        corr.pfb(adc, P, out=out)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    spectra = N * T
    # nominal flops of one spectrum: FIR 2 P M, complex FFT 5 (M/2) log2(M/2), split step ~ 10 (M/2)
    flops = spectra * (2 * P * 8192 + 5 * 4096 * 12 + 10 * 4096)
    moved = spectra * (8192 + 4096 * 8)  # one new ADC frame in, 4096 float32 complex channels out
    return {"config": "pfb: N=512 inputs, 4 taps, 8192-point real FFT, 64 spectra", "ms": ms,
            "spectra_per_s": spectra / (ms / 1e3), "tflops_nominal": flops / (ms / 1e3) / 1e12,
            "gbs": moved / (ms / 1e3) / 1e9, "real_time_factor": (T / 24000.0) / (ms / 1e3)}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", default="")
    ap.add_argument("--stream-blocks", type=int, default=10000)
    a = ap.parse_args(argv)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1411_3751_gb300 import corr, synth

    todo = [a.only] if a.only else ["tiny", "small", "precision", "group", "stream", "fastdump", "requant", "pfb"]
    for name in todo:
        if name == "tiny":
            r = tiny(corr, synth, torch)
        elif name == "small":
            r = small(corr, synth, torch)
            print(json.dumps({"measure": name, **r}))
            r = small(corr, synth, torch, path="fp8tc_fused")
        elif name == "precision":
            r = precision(corr, synth, torch)
        elif name == "group":
            r = group(corr, synth, torch)
        elif name == "fastdump":
            r = fast_dump(corr, synth, torch)
        elif name == "requant":
            r = requant(corr, synth, torch)
        elif name == "pfb":
            r = pfb(corr, synth, torch)
        else:
            r = stream_loop(corr, synth, torch, a.stream_blocks)
        print(json.dumps({"measure": name, **r}))
        sys.stdout.flush()


if __name__ == "__main__":
    main()
