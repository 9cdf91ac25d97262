"""Host-side checks of the product path and the benchmark contract (no GPU).

* Without a CUDA device the library refuses to create a context: the path has
  no CPU fallback.
* `bench.py --impl reference` (the FP64 oracle timed on the host cores)
  prints one JSON line with the contract's keys.
* The roofline bookkeeping names the nearer roof (HBM against the tensor pipe
  or FP32 FMA) from the kernel's own counts, and scales captured DRAM
  traffic multiples by the algorithmic bytes."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_no_device_fails_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    import paper_2012_13173_gb300 as H
    H.load()
    with pytest.raises(H.HcgError):
        H.Gridder(0)


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3",
                        "--scale", "0.1"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "contributions/s"
    for k in ("metric", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling", "vs_baseline",
              "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["steps"] == 1 and d["warmup"] == 3 and d["higher_is_better"] is True
    assert d["config"]["workload"] == "drift-16M-c256-x3"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


class _Field:
    """The parts of a synthetic field that the roofline bookkeeping reads."""
    name = "drift-16M-c256"
    nchan = 256
    cells = 1000 * 1000


def test_roofline_takes_the_nearer_roof():
    import bench
    peaks = (6651.7, 1897.2, 78.6, "measured")
    n, pairs = 15_960_000, 4_152_714_715
    # tensor path, FP32 storage: 2.136e13 issued MMA flops in 41.1 ms is
    # 0.56 of the TF32 rate (BF16 x 1.1/2.25), far above the HBM fraction
    info = {"samples_kept": n, "contributions": pairs * 256, "path": 2, "tensor_flops": 21_363_972_636_672}
    e = bench.roofline_entry(_Field, "f32", info, 41.1, peaks)
    assert e["bound"] == "tensor" and e["unit"] == "TFLOP/s" and e["kernel"] == "k_tc_gather_f32"
    assert abs(e["peak"] - 1897.2 * 1.1 / 2.25) < 0.1
    assert abs(e["frac"] - 21_363_972_636_672 / 0.0411 / 1e12 / (1897.2 * 1.1 / 2.25)) < 1e-3
    assert e["frac"] > e["hbm_frac"]
    # the same bytes in far less time: the HBM roof is the nearer one
    info_fast = dict(info, tensor_flops=1)
    e2 = bench.roofline_entry(_Field, "bf16", info_fast, 1.0, peaks)
    assert e2["bound"] == "hbm" and e2["unit"] == "GB/s"
    alg = n * 256 * 2 + 24 * n + 4 * _Field.cells * 257
    assert e2["alg_bytes"] == alg and abs(e2["achieved"] - alg / 1e-3 / 1e9) < 0.1
    # CUDA-core path: FP32 FMA roof (2 flops per contribution) vs HBM
    info_cc = {"samples_kept": n, "contributions": pairs * 256, "path": 1}
    e3 = bench.roofline_entry(_Field, "f32", info_cc, 158.4, peaks)
    assert e3["bound"] == "alu" and abs(e3["frac"] - 2 * pairs * 256 / 0.1584 / 1e12 / 78.6) < 1e-3


def test_traffic_is_the_captured_multiple_of_the_algorithmic_bytes():
    import bench
    assert bench.traffic_of("drift-16M-c256", "f32", "k_tc_gather_f32", 1_000_000) == round(
        bench.TRAFFIC_RATIO[("drift-16M-c256", "f32", "k_tc_gather_f32")] * 1_000_000)
    assert bench.traffic_of("no-such-workload", "f32", "k_tc_gather_f32", 1_000_000) is None
