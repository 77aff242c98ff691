"""Streaming serving loop over the C ABI: device-resident accumulators per stream, admission by HBM
footprint, a cross-power dump every `cross_every` blocks and a total-power dump every `auto_every`
blocks (the paper's 9 s and 1 s cadences, Sec. 2.5 and Sec. 2.6, with 10 ms blocks of 240 samples at
the 24.0 kHz channel rate), dump latency statistics.

The samples of each stream are produced on the device by the seeded generator (the paper's live
F-engine data are not available) one gulp of `gulp_blocks` blocks at a time; each gulp is one
`corr_accumulate` of gulp_blocks x block_samples samples. A dump's latency is measured with CUDA
events from the moment the last block of its window has been generated to the moment its host copy
is complete. The real-time factor is reported for the whole loop (the input generator shares the GPU)
and for the correlator's own work (accumulate and dump calls, timed with events).

With `outriggers` set, the total-power dump covers only those stations (selective dump and reset of
their cells, Sec. 2.6); the cross dump then carries the full visibilities. `cross_fmt` selects the
cross dump format (CF32 is exact while a dump's sums stay below 2^24, e.g. the paper's 0.33 s
minimum dump time of Table 1: 8000 samples x 128 < 2^24).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

from . import corr, synth

CHANNEL_RATE_HZ = 24000.0


@dataclass
class StreamSpec:
    name: str
    n_inputs: int
    n_chans: int
    n_pol: int = 2
    block_samples: int = 240     # 10 ms at 24.0 kHz
    gulp_blocks: int = 50        # blocks per accumulate call
    cross_every: int = 900       # blocks per cross-power dump (9 s)
    auto_every: int = 100        # blocks per total-power dump (1 s)
    seed: int = 0x14113751 + 5
    kind: str = "gauss_tone"
    outriggers: tuple = ()       # stations whose total power alone is dumped at the auto cadence (Sec. 2.6)
    cross_fmt: int = corr.CORR_FMT_CI64

    def gulp_samples(self) -> int:
        return self.block_samples * self.gulp_blocks

    def input_bytes(self) -> int:
        return self.gulp_samples() * self.n_chans * self.n_inputs

    def footprint(self) -> int:
        """Device bytes of the stream: the context plus its gulp buffer."""
        return corr.corr_footprint_bytes(self.n_inputs, self.n_chans, self.gulp_samples(), self.n_pol,
                                         corr.CORR_PATH_FP8TC) + self.input_bytes()


@dataclass
class _Live:
    spec: StreamSpec
    xc: object
    buf: object
    cross_host: object
    autos_host: object
    blocks_done: int = 0
    cross_lat: list = field(default_factory=list)
    auto_lat: list = field(default_factory=list)
    cross_dumps: list = field(default_factory=list)   # (first block, host array) of kept dumps
    auto_dumps: list = field(default_factory=list)


class Server:
    """Admits streams by footprint against an HBM budget and runs them block by block."""

    def __init__(self, hbm_budget_bytes: int, keep_dumps: int = 1):
        self.budget = int(hbm_budget_bytes)
        self.used = 0
        self.streams: list[_Live] = []
        self.rejected: list[str] = []
        self.keep_dumps = keep_dumps

    def admit(self, spec: StreamSpec) -> bool:
        import torch

        if spec.auto_every % spec.gulp_blocks or spec.cross_every % spec.gulp_blocks:
            raise ValueError("dump cadences must be multiples of the gulp")
        fp = spec.footprint()
        free, _ = torch.cuda.mem_get_info()
        if self.used + fp > self.budget or fp > free:
            self.rejected.append(spec.name)
            return False
        xc = corr.Correlator(spec.n_inputs, spec.n_chans, spec.gulp_samples(), spec.n_pol, path="fp8tc")
        buf = torch.empty((spec.gulp_samples(), spec.n_chans, spec.n_inputs), dtype=torch.uint8, device="cuda")
        cdt = torch.int64 if spec.cross_fmt == corr.CORR_FMT_CI64 else torch.float32
        cross_h = torch.empty(xc.out_shape(corr.CORR_WHAT_CROSS), dtype=cdt).pin_memory()
        ashape = (xc.station_out_shape(corr.CORR_WHAT_AUTO, len(spec.outriggers)) if spec.outriggers
                  else xc.out_shape(corr.CORR_WHAT_AUTO))
        autos_h = torch.empty(ashape, dtype=torch.int64).pin_memory()
        self.streams.append(_Live(spec, xc, buf, cross_h, autos_h))
        self.used += fp
        return True

    def run(self, n_blocks: int) -> dict:
        """Run every admitted stream for n_blocks blocks; returns real-time factors and dump latencies.
        All streams share the block length and the gulp; n_blocks must be a multiple of the gulp."""
        import torch

        if not self.streams:
            raise ValueError("no stream admitted")
        gulp = self.streams[0].spec.gulp_blocks
        if any(l.spec.gulp_blocks != gulp or l.spec.block_samples != self.streams[0].spec.block_samples
               for l in self.streams):
            raise ValueError("streams must share the block length and the gulp")
        if n_blocks % gulp:
            raise ValueError("n_blocks must be a multiple of the gulp")
        ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
        t_start, t_end = ev(), ev()
        torch.cuda.synchronize()
        t_start.record()
        pending = []  # (live, kind, ready_event, done_event)
        busy = []     # (start, end) events around the correlator's own work (accumulate + dumps)
        for _ in range(n_blocks // gulp):
            for live in self.streams:
                sp = live.spec
                synth.generate_device(synth.Spec(kind=sp.kind, seed=sp.seed), sp.gulp_samples(), sp.n_chans,
                                      sp.n_inputs, t0=live.blocks_done * sp.block_samples, out=live.buf,
                                      sync=False)
                ready = ev()
                ready.record()
                live.xc.accumulate(live.buf)
                live.blocks_done += gulp
                for kind, every, what, host in (("auto", sp.auto_every, corr.CORR_WHAT_AUTO, live.autos_host),
                                                ("cross", sp.cross_every, corr.CORR_WHAT_CROSS, live.cross_host)):
                    if live.blocks_done % every == 0:
                        if kind == "auto" and sp.outriggers:
                            live.xc.dump_stations(sp.outriggers, what, reset=True, out=host)
                        elif kind == "cross":
                            live.xc.dump(what, fmt=sp.cross_fmt, reset=True, out=host)
                        else:
                            live.xc.dump(what, reset=True, out=host)
                        done = ev()
                        done.record()
                        pending.append((live, kind, ready, done))
                        self._keep(live, kind, done, live.blocks_done - every)
                end = ev()
                end.record()
                busy.append((ready, end))
        t_end.record()
        torch.cuda.synchronize()
        wall_s = t_start.elapsed_time(t_end) / 1e3
        for live, kind, ready, done in pending:
            (live.auto_lat if kind == "auto" else live.cross_lat).append(ready.elapsed_time(done))
        out = {"wall_s": wall_s, "streams": {}}
        for live in self.streams:
            sp = live.spec
            sim_s = live.blocks_done * sp.block_samples / CHANNEL_RATE_HZ
            out["streams"][sp.name] = {
                "n_inputs": sp.n_inputs, "n_chans": sp.n_chans, "blocks": live.blocks_done,
                "samples_per_s": live.blocks_done * sp.block_samples * sp.n_chans * sp.n_inputs / wall_s,
                "cross_dumps": len(live.cross_lat), "auto_dumps": len(live.auto_lat),
                "cross_latency_ms": _pct(live.cross_lat), "auto_latency_ms": _pct(live.auto_lat),
            }
        sim = max(l.blocks_done * l.spec.block_samples for l in self.streams) / CHANNEL_RATE_HZ
        corr_s = sum(a.elapsed_time(b) for a, b in busy) / 1e3
        out["simulated_s"] = sim
        out["correlator_s"] = corr_s
        # whole loop (input generation on the same GPU included) and the correlator alone
        out["real_time_factor"] = sim / wall_s
        out["real_time_factor_correlator"] = sim / corr_s
        out["rejected"] = list(self.rejected)
        return out

    def _keep(self, live, kind, done, first_block):
        """Keep host copies of the first `keep_dumps` dumps of each kind (the host buffers are reused)."""
        store = live.auto_dumps if kind == "auto" else live.cross_dumps
        if len(store) < self.keep_dumps:
            done.synchronize()
            src = live.autos_host if kind == "auto" else live.cross_host
            store.append((first_block, src.numpy().copy()))


    def close(self):
        for live in self.streams:
            live.xc.close()
        self.streams = []


def _pct(lat):
    if not lat:
        return {"p50": None, "p99": None, "n": 0}
    s = sorted(lat)
    p = lambda q: s[min(len(s) - 1, max(0, int(math.ceil(q * len(s))) - 1))]  # noqa: E731
    return {"p50": p(0.50), "p99": p(0.99), "n": len(s)}
