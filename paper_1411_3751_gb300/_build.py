"""Compile the native parts in-tree: libcorr.so (CUDA, sm_103a) and the input generator libraries.

Outputs go to ``paper_1411_3751_gb300/_build/``. Sources compile in parallel, one ``-gencode``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
SYNTH = os.path.join(PKG, "synth")
INCLUDE = os.path.join(ROOT, "include")
OUT = os.path.join(PKG, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall"] + ARCH

CORR_SOURCES = ["corr_api.cu", "xeng_fp32.cu", "xeng_i8mma.cu", "xeng_fp8tc.cu", "f8_prep.cu", "xeng_f8fused.cu", "autos_dump.cu", "requant.cu", "pfb.cu", "corr_static.cu", "selftest.cu", "corr_group.cu", "probe.cu", "corner_turn.cu", "prep_tma.cu", "xeng_pair.cu"]

LIBCORR = os.path.join(OUT, "libcorr.so")
LIBSYNTH_CUDA = os.path.join(OUT, "libcorrsynth_cuda.so")
LIBSYNTH_HOST = os.path.join(OUT, "libcorrsynth_host.so")


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return exe


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed: %s\n%s" % (" ".join(cmd), r.stdout))
    return r.stdout


def _newer(target, deps):
    if not os.path.exists(target):
        return False
    t = os.path.getmtime(target)
    return all(os.path.getmtime(d) <= t for d in deps)


def _headers():
    hs = [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    hs += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    return hs


def build(force: bool = False, verbose: bool = False) -> dict:
    """Build all native libraries; returns {name: path}. Raises RuntimeError on a compiler error."""
    os.makedirs(OUT, exist_ok=True)
    jobs = []
    hdrs = _headers()
    objs = []
    for src in CORR_SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OUT, src.replace(".cu", ".o"))
        objs.append(o)
        if force or not _newer(o, [s] + hdrs):
            jobs.append([nvcc()] + NVCC_FLAGS + ["-I", INCLUDE, "-I", CSRC, "-c", s, "-o", o])
    synth_h = os.path.join(SYNTH, "synth.h")
    synth_cu = os.path.join(SYNTH, "synth.cu")
    synth_c = os.path.join(SYNTH, "synth_host.c")
    if force or not _newer(LIBSYNTH_CUDA, [synth_cu, synth_h]):
        jobs.append([nvcc()] + NVCC_FLAGS + ["-I", SYNTH, "-shared", synth_cu, "-o", LIBSYNTH_CUDA])
    if force or not _newer(LIBSYNTH_HOST, [synth_c, synth_h]):
        jobs.append(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-I", SYNTH, synth_c, "-o", LIBSYNTH_HOST])
    logs = []
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
            for out in ex.map(_run, jobs):
                logs.append(out)
    if force or not _newer(LIBCORR, objs):
        logs.append(_run([nvcc()] + ARCH + ["-shared", "-o", LIBCORR] + objs))
    if verbose:
        for l in logs:
            if l.strip():
                print(l)
    return {"libcorr": LIBCORR, "synth_cuda": LIBSYNTH_CUDA, "synth_host": LIBSYNTH_HOST}


if __name__ == "__main__":
    print(build(verbose=True))
