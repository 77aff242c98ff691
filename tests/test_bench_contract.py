"""The benchmark's one-line JSON contract.

* reference arm (`--impl reference`, the CPU oracle; runs here without a GPU): the keys, the units
  and the e2e block with zero host-link bytes;
* native arm (GPU): one short run of the default workload with the comparison legs switched off,
  checking every key the line promises and the internal consistency of the numbers (whole-job value
  from ms_per_step, the roofline fraction, launches per step).
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BASE_KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
             "vs_baseline", "dtype", "data", "config", "e2e", "cpu_baseline"}


def _run(args, timeout):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT, capture_output=True,
                         text=True, timeout=timeout)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    return json.loads(lines[0])


def test_reference_arm_line():
    line = _run(["--impl", "reference", "--steps", "1", "--warmup", "3"], timeout=600)
    assert BASE_KEYS <= set(line)
    assert line["impl"] == "reference" and line["unit"] == "Tera-CMAC/s" and line["higher_is_better"] is True
    assert line["value"] > 0 and line["steps"] == 1 and line["warmup"] == 3
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["n_inputs"] == 512 and line["config"]["n_chans"] == 128


def test_reference_arm_other_ranks_exit_quietly():
    """Launched as rank 1 of 2 (as torchrun would), the reference arm does no work, prints nothing
    and exits 0; rank 0 alone prints the line."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1", MASTER_PORT="29599")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                          "--steps", "1", "--warmup", "3"], cwd=ROOT, capture_output=True, text=True, timeout=300,
                         env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    assert not [l for l in out.stdout.splitlines() if l.startswith("{")]


@pytest.mark.gpu
def test_native_arm_line():
    line = _run(["--steps", "2", "--warmup", "3", "--e2e-steps", "1", "--fp32-steps", "0", "--i8-steps", "0",
                 "--no-cpu-baseline", "--no-extras"], timeout=900)
    assert BASE_KEYS | {"roofline", "clocks", "gpu_launches"} <= set(line)
    assert line["n_gpus"] == 1 and line["scaling"] == "weak" and line["dtype"] == "e4m3"
    cfg = line["config"]
    cmac = cfg["n_inputs"] * (cfg["n_inputs"] + 1) // 2 * cfg["n_chans"] * cfg["n_time_per_block"] * cfg["blocks_per_step"]
    assert abs(line["value"] - cmac / (line["ms_per_step"] / 1e3) / 1e12) < 1e-6 * line["value"]
    roof = line["roofline"]
    assert roof["bound"] == "tensor" and roof["unit"] == "TFLOP/s" and 0 < roof["frac"] < 1.3
    assert abs(roof["frac"] - roof["achieved"] / roof["peak"]) < 1e-9
    # the issue-rate probe: a positive rate, the kernel's share of it below 1 (it cannot beat the
    # instruction it issues), and the wide instruction at least as fast per flop as the narrow one
    probe = roof["issue_probe"]
    assert probe["tflops_n256"] > 0 and probe["tflops_n128"] > 0
    assert 0 < roof["frac_issue"] < 1.05 and 0 < roof["frac_useful_of_issue_peak"] < roof["frac_issue"]
    assert probe["tflops_n256"] >= 0.95 * probe["tflops_n128"]
    assert line["gpu_launches"] > 0 and line["gpu_launches_per_step"] == line["gpu_launches"] / 2
    e2e = line["e2e"]
    assert e2e["unit"] == "Tera-CMAC/s" and 0 < e2e["value"] <= line["value"]
    # one byte per (input, channel, sample) crosses the host link every step
    assert e2e["h2d_bytes_per_step"] == cfg["n_inputs"] * cfg["n_chans"] * cfg["n_time_per_block"] * cfg["blocks_per_step"]
    assert set(line["clocks"]) >= {"sm_mhz", "sm_max_mhz", "reasons"}
