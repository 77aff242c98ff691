"""Profiling driver: a few accumulate calls on one synthetic workload, for `ncu -k <kernel> -s/-c`.

    python -m paper_1411_3751_gb300.profile_case --n 512 --c 128 --t 8192 --blocks 3 --path fp8tc
    python -m paper_1411_3751_gb300.profile_case --n 512 --c 32 --t 8192 --blocks 8 --batch --prep-sms 30
    python -m paper_1411_3751_gb300.profile_case --requant --n 512 --c 2398 --t 256 --blocks 3
    python -m paper_1411_3751_gb300.profile_case --pfb --n 512 --t 16 --blocks 3

Holds a single input block on the device (the same block is accumulated --blocks times), so the
device footprint stays at a few GB for the 512-input, 128-channel case.
"""
from __future__ import annotations

import argparse
import os
import sys


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--c", type=int, default=128)
    ap.add_argument("--t", type=int, default=8192)
    ap.add_argument("--npol", type=int, default=2)
    ap.add_argument("--blocks", type=int, default=3)
    ap.add_argument("--path", default="fp8tc")
    ap.add_argument("--seed", type=int, default=0x14113751 + 2)
    ap.add_argument("--batch", action="store_true",
                    help="accumulate the block --blocks times in one corr_accumulate_batch call (the blocks "
                         "then share tensor-core launches, as in the benchmark)")
    ap.add_argument("--prep-sms", type=int, default=-1,
                    help="SMs of the overlapped operand build in batches (-1 library default, 0 sequential)")
    ap.add_argument("--pfb", action="store_true",
                    help="profile the PFB instead: --n inputs x --t spectra, 4 taps")
    ap.add_argument("--requant", action="store_true",
                    help="profile the requantiser instead: --n inputs x --t spectra of a 4096-channel PFB, "
                         "--c channels selected (int32 input)")
    a = ap.parse_args(argv)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1411_3751_gb300 import corr, synth

    if a.pfb:
        g = torch.Generator(device="cuda")
        g.manual_seed(a.seed)
        adc = (torch.randn((a.n, (a.t + 3) * 8192), device="cuda", generator=g) * 20.0).round_().clamp_(-128, 127)
        adc = adc.to(torch.int8)
        out = torch.empty((a.n, a.t, 4096, 2), dtype=torch.float32, device="cuda")
        for _ in range(a.blocks):
            corr.pfb(adc, 4, out=out)
        torch.cuda.synchronize()
        print("profile_case ok: pfb N=%d T=%d blocks=%d" % (a.n, a.t, a.blocks))
        return
    if a.requant:
        g = torch.Generator(device="cuda")
        g.manual_seed(a.seed)
        pfb = (torch.randn((a.n, a.t, 4096, 2), device="cuda", generator=g) * 3000.0).round_().to(torch.int32)
        out = torch.empty((a.t, a.c, a.n), dtype=torch.uint8, device="cuda")
        for _ in range(a.blocks):
            corr.requantize(pfb, 1229, a.c, gain=2.5 / 3000.0, out=out)
        torch.cuda.synchronize()
        print("profile_case ok: requant N=%d T=%d C=%d blocks=%d" % (a.n, a.t, a.c, a.blocks))
        return
    x = synth.generate_device(synth.Spec(kind="gauss_tone", seed=a.seed), a.t, a.c, a.n)
    with corr.Correlator(a.n, a.c, a.t, a.npol, path=a.path) as xc:
        xc.set_prep_sms(a.prep_sms)
        if a.batch:
            xc.accumulate_batch([x] * a.blocks)
        else:
            for _ in range(a.blocks):
                xc.accumulate(x)
        xc.dump(corr.CORR_WHAT_CROSS)
        xc.sync()
    torch.cuda.synchronize()
    print("profile_case ok: N=%d C=%d T=%d blocks=%d path=%s" % (a.n, a.c, a.t, a.blocks, a.path))


if __name__ == "__main__":
    main()
