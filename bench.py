#!/usr/bin/env python3
"""Throughput of the GB300 gridding path (HCGrid, arXiv 2012.13173).

One step = one full pass of the path over the workload's inputs, already
resident in HBM: HEALPix pixel of every sample, radix sort, both lookup
tables, the table-driven gather of Eq. (1) and the normalisation (plus the
device quantisation when a reduced storage type is asked for).

Metric: gridded sample-channel contributions per second; a contribution is
one (cell, sample, channel) triple with the sample inside the cell's kernel
support, counted exactly by the kernels.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

The default workload, drift-16M-c256-x3, is the 16M-sample, 256-channel
drift scan (1000 x 1000 cells of 0.6', FWHM 3', support 4 sigma) stored as
FP32, BF16 and E4M3 side by side and gridded in one batched, captured
launch, each form with the autotuner's choice; the line also carries the
plain FP32 gather on the same inputs, each kernel's roofline and the error
of each form against the FP64 oracle on sampled cells.  Other workloads:
drift-1M-c1024, drift-4M-c4096, uniform-20k (one field, --storage), any of
them with -x3, and batch-64.

Under torchrun each rank grids its own replica of the workload (the path
needs no data exchange); value = all ranks' contributions / max rank time.
``--impl reference`` times the FP64 CPU oracle on a bounded sample of the
same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "gridded sample·channel contributions/s + %HBM/tensor peak, tuned vs plain FP32"
UNIT = "contributions/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p.get("bf16_tflops", 1964.4)), "measured"
    except Exception:
        return 6800.0, 1900.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.25)
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            return None
        sm, mx, reasons = [], 0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _device_spectra(f, torch, dev, chunk=1 << 16):
    out = torch.empty((f.n, f.nchan), dtype=torch.float32, device=dev)
    for a in range(0, f.n, chunk):
        b = min(f.n, a + chunk)
        out[a:b] = f.spectra(np.arange(a, b), device=dev)
    return out


def device_inputs(f, storage, torch, dev):
    """The benchmark's inputs on the device: lon, lat (FP64), the spectra made
    on the device and stored as `storage` (BF16: FP32 rounded to nearest even;
    E4M3: per channel the scale amax / 448, the scaled values rounded to
    e4m3), and the E4M3 scales (None otherwise).  Made once, before timing."""
    lon_d = torch.from_numpy(f.lon).to(dev)
    lat_d = torch.from_numpy(f.lat).to(dev)
    spec_d, scale_d = stored(_device_spectra(f, torch, dev), storage, torch)
    torch.cuda.empty_cache()
    return lon_d, lat_d, spec_d, scale_d


def stored(spec32, storage, torch):
    """FP32 spectra as the benchmark stores them: unchanged, BF16 (round to
    nearest even), or E4M3 with per-channel scales amax / 448.  Returns
    (spectra, scales or None)."""
    if storage == "bf16":
        return spec32.to(torch.bfloat16), None
    if storage == "e4m3":
        amax = spec32.abs().amax(dim=0)
        scale = torch.where(amax > 0, amax / 448.0, torch.ones_like(amax)).to(torch.float32)
        return (spec32 / scale[None, :]).to(torch.float8_e4m3fn), scale
    return spec32, None


PATHS = ("auto", "gather", "tensor", "scatter", "staged")


def make_gridder(H, f, storage, index, stream, path="auto", tuning=(0, 0, 0)):
    """A Gridder for field f as the benchmark runs it: the field's kernel and
    grid, `storage`, and the library's own path choice unless `path` pins
    one, with `tuning` = (cells per block, channels per thread, tile depth)."""
    g = H.Gridder(index, stream)
    g.set_kernel(f.fwhm, f.support)
    g.set_grid(f.lon0, f.lat0, f.pix, f.nx, f.ny)
    g.set_storage(storage)
    if path != "auto" or any(tuning):
        code = {"auto": H.PATH_AUTO, "gather": H.PATH_GATHER, "tensor": H.PATH_TENSOR, "scatter": H.PATH_SCATTER,
                "staged": H.PATH_STAGED}
        g.set_tuning(cells_per_block=tuning[0], chans_per_thread=tuning[1], tile_depth=tuning[2], path=code[path])
    return g


def _alg_bytes(n_kept, nchan, cells, esize):
    """Algorithmic bytes of one pass: spectra read once, FP64 lon/lat, cube and
    weights written, the per-channel scales."""
    return n_kept * nchan * esize + 16 * n_kept + 4 * cells * (nchan + 1) + 4 * nchan


def _gather_bytes(n_kept, nchan, cells, esize):
    """Algorithmic bytes of the gather kernel: spectra read once, the 24 B of
    sorted per-sample data (offsets, cos lat, row), cube and weights written."""
    return n_kept * nchan * esize + 24 * n_kept + 4 * cells * (nchan + 1)


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch
# of a gather kernel, as a multiple of its algorithmic bytes, from one ncu
# capture of the current kernel code on a reduced-side case of the same
# workload (same density, a few GB on the device); the line reports that
# multiple times the launch's algorithmic bytes.  Keys: (workload without
# any -x3 suffix, storage, kernel).  Absent entries report null.
TRAFFIC_RATIO = {
    # drift-16M-c256 at half side (4.1M samples, 500 x 500 cells), one launch each
    ("drift-16M-c256", "f32", "k_tc_gather_f32"): 2.261,
    ("drift-16M-c256", "bf16", "k_tc_gather"): 1.457,
    ("drift-16M-c256", "e4m3", "k_tc_gather"): 1.018,
    # drift-1M-c1024 at full size (4.5 GB of algorithmic bytes)
    ("drift-1M-c1024", "f32", "k_gather_list"): 1.120,
    # drift-4M-c4096 at 0.35 side (0.48M samples, 210 x 210 cells)
    ("drift-4M-c4096", "bf16", "k_tc_gather"): 1.458,
    ("drift-4M-c4096", "e4m3", "k_tc_gather"): 1.151,
}


def traffic_of(name, storage, kernel, alg_bytes):
    r = TRAFFIC_RATIO.get((name, storage, kernel))
    return None if r is None else round(r * alg_bytes)


def gpu_local_cpus(index):
    """The CPUs sysfs lists as local to CUDA device `index` (its NUMA node),
    or None when that cannot be read."""
    try:
        import torch
        p = torch.cuda.get_device_properties(index)
        bus = "%04x:%02x:%02x.0" % (p.pci_domain_id, p.pci_bus_id, p.pci_device_id)
        with open("/sys/bus/pci/devices/%s/local_cpulist" % bus) as fh:
            text = fh.read().strip()
        cpus = set()
        for part in text.split(","):
            lo, _, hi = part.partition("-")
            cpus.update(range(int(lo), int(hi or lo) + 1))
        return cpus & os.sched_getaffinity(0) or None
    except Exception:
        return None


def job_rate(units_per_rank, ms_local, dist=None, device=None):
    """Whole-job rate of N replicas: every rank processed `units_per_rank` in
    `ms_local` ms; the job takes as long as its slowest rank (the max over
    ranks, an all-reduce when distributed).  Returns (units per second summed
    over the ranks, the job's ms)."""
    ms, world = float(ms_local), 1
    if dist is not None and dist.is_initialized():
        import torch
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms, world = float(t.item()), dist.get_world_size()
    return units_per_rank * world / (ms / 1e3), ms


def cpu_oracle_rate(f, target_s=12.0, seed=0):
    """The FP64 oracle timed on the host cores on a square block of cells at a
    seeded random position, grown until it takes about a third of target_s
    (a compact block needs only the samples around it)."""
    import oracle
    geom = np.array(f.geom())
    rng = np.random.default_rng(seed)
    side = 8
    while True:
        sx, sy = min(side, f.nx), min(side, f.ny)
        i0 = int(rng.integers(0, f.nx - sx + 1))
        j0 = int(rng.integers(0, f.ny - sy + 1))
        jj, ii = np.meshgrid(np.arange(j0, j0 + sy), np.arange(i0, i0 + sx), indexing="ij")
        cells = (jj * f.nx + ii).ravel().astype(np.int64)
        off, ids, _ = oracle.neighbours_band(geom, f.lon, f.lat, cells)
        rows = np.unique(ids)
        spec = f.spectra_np(rows)
        t0 = time.perf_counter()
        v, w, ab, cnt = oracle.grid_cells(geom, f.lon[rows], f.lat[rows], spec, cells)
        dt = time.perf_counter() - t0
        if dt >= target_s / 3 or (sx == f.nx and sy == f.ny):
            contrib = float(cnt.sum()) * f.nchan
            return {"value": contrib / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                    "sample": f"a {sx}x{sy} block of {f.cells} cells (all their contributors, all {f.nchan} "
                              f"channels), {dt:.1f} s"}, dt
        side = int(side * min(4.0, max(1.5, math.sqrt(target_s / 3 / max(dt, 1e-3)))))


def run_reference(args, f, world, rank):
    if rank != 0:
        return
    steps = []
    meta = None
    for k in range(args.warmup + args.steps):
        meta, dt = cpu_oracle_rate(f, target_s=max(2.0, 30.0 / (args.warmup + args.steps)), seed=k)
        if k >= args.warmup:
            steps.append(meta["value"])
    value = statistics.median(steps)
    meta["value"] = value
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "samples": f.n, "nchan": f.nchan, "grid": f"{f.nx}x{f.ny}"},
            "cpu_baseline": meta,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def batch_setup(fields, H, torch, dev, index, stream):
    """The benchmark's batch: one Gridder per field (inputs made on the
    device, BF16 fields rounded to nearest even), all added to one Batch.
    Returns (batch, gridders, the device inputs the gridders borrow)."""
    keep, gs = [], []
    for f in fields:
        lon_d = torch.from_numpy(f.lon).to(dev)
        lat_d = torch.from_numpy(f.lat).to(dev)
        spec = _device_spectra(f, torch, dev)
        if f.dtype == "bf16":
            spec = spec.to(torch.bfloat16)
        g = H.Gridder(index, stream)
        g.set_kernel(f.fwhm, f.support)
        g.set_grid(f.lon0, f.lat0, f.pix, f.nx, f.ny)
        g.set_storage(f.dtype)
        g.load_samples(lon_d, lat_d, spec, borrow=True)
        keep.append((lon_d, lat_d, spec))
        gs.append(g)
    torch.cuda.empty_cache()
    b = H.Batch(index, stream)
    for g in gs:
        b.add(g)
    return b, gs, keep


def run_batch(args, torch, H, dev, local, world, dist):
    """Uneven fields gridded by one captured graph (hcg_batch)."""
    from paper_2012_13173_gb300 import synth
    count = int(args.workload.split("-")[1])
    fields = synth.batch_fields(seed=4, count=count, scale=args.scale)
    stream = torch.cuda.Stream(dev)
    b, gs, keep = batch_setup(fields, H, torch, dev, local, stream)
    torch.cuda.synchronize(dev)
    for _ in range(args.warmup):
        b.grid()
    b.sync()
    contrib = sum(g.info()["contributions"] for g in gs)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clk = Clocks(local)
    clk.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        b.grid()
    t1.record(stream)
    torch.cuda.synchronize(dev)
    clocks = clk.stop()
    if dist:
        dist.barrier()
    ms = t0.elapsed_time(t1) / args.steps
    value, ms = job_rate(contrib, ms, dist, dev)
    esz = {"f32": 4, "bf16": 2}
    alg = sum(_alg_bytes(g.info()["samples_kept"], f.nchan, f.cells, esz[f.dtype]) for f, g in zip(fields, gs))
    hbm, _, peak_kind = _peaks()
    achieved = alg / (ms / 1e3) / 1e9
    paths = [g.info()["path"] for g in gs]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+bf16", "data": "synthetic",
            "config": {"workload": args.workload, "fields": count, "samples": int(sum(f.n for f in fields)),
                       "channels": sorted({f.nchan for f in fields}), "tensor_fields": paths.count(2),
                       "l2": "inputs larger than L2", "parallelism": f"replicas x{world}"},
            "contributions_per_step": contrib,
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                         "frac": round(achieved / hbm, 4), "traffic": None, "kernel": "whole graph",
                         "alg_bytes": alg, "peak_kind": peak_kind},
            "cpu_baseline": None, "e2e": None, "gpu_launches": b.info()["launches"] * args.steps,
            "batch": b.info(), "clocks": clocks}
    return line


ESIZE = {"f32": 4, "bf16": 2, "e4m3": 1}
L2_BYTES = 129 * 2 ** 20          # the GB300's L2
TRIPLE = ("f32", "bf16", "e4m3")
PATH_NAME = {1: "gather", 2: "tensor", 3: "scatter", 4: "staged"}


def triple_setup(f, H, torch, dev, index, stream, tune=True, path="auto"):
    """One field stored three ways -- FP32, BF16 and E4M3 -- as three Gridders
    (device inputs borrowed, outputs bound to device buffers), each tuned by
    the library's autotuner (cached per key) unless tune is False (then on
    `path`), added to one Batch: gridded side by side by one captured graph.
    Returns (batch, [(storage, gridder, cube, weights, scale, tuned choice)],
    inputs kept)."""
    lon_d = torch.from_numpy(f.lon).to(dev)
    lat_d = torch.from_numpy(f.lat).to(dev)
    spec32 = _device_spectra(f, torch, dev)
    keep = [lon_d, lat_d]
    fields = []
    for st in TRIPLE:
        spec, scale = stored(spec32, st, torch)
        cube = torch.empty((f.ny, f.nx, f.nchan), dtype=torch.float32, device=dev)
        w = torch.empty((f.ny, f.nx), dtype=torch.float32, device=dev)
        g = make_gridder(H, f, st, index, stream, "auto" if tune else path)
        g.load_samples(lon_d, lat_d, spec, chan_scale=scale, borrow=True)
        g.bind_output(cube, w)
        choice = g.autotune() if tune else None
        keep += [spec, scale]
        fields.append((st, g, cube, w, scale, choice))
    torch.cuda.synchronize(dev)
    torch.cuda.empty_cache()
    b = H.Batch(index, stream)
    for fl in fields:
        b.add(fl[1])
    return b, fields, keep


def patch_cells(f, seed=7, patches=10, side=32, corner=16):
    """A seeded sample of cells for the error against the FP64 oracle:
    `patches` random side x side blocks plus a corner x corner block at each
    corner of the grid (edge cells with one-sided support)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(patches):
        i0 = int(rng.integers(0, max(1, f.nx - side + 1)))
        j0 = int(rng.integers(0, max(1, f.ny - side + 1)))
        jj, ii = np.meshgrid(np.arange(j0, min(f.ny, j0 + side)), np.arange(i0, min(f.nx, i0 + side)), indexing="ij")
        out.append((jj * f.nx + ii).ravel())
    for j0 in (0, max(0, f.ny - corner)):
        for i0 in (0, max(0, f.nx - corner)):
            jj, ii = np.meshgrid(np.arange(j0, min(f.ny, j0 + corner)), np.arange(i0, min(f.nx, i0 + corner)),
                                 indexing="ij")
            out.append((jj * f.nx + ii).ravel())
    return np.unique(np.concatenate(out)).astype(np.int64)


def err_vs_fp64(f, results, cells):
    """Error of each stored form against the FP64 oracle (Eq. 1) on `cells`:
    results = [(storage, values[ncell, C] float64, weights[ncell], scale or
    None)].  Per form: the maximum condition-aware error |V - V64| /
    (|V64| + sum w |s| / W) and the largest per-channel normwise error
    ||V_c - V64_c||_2 / ||V64_c||_2, both against the oracle on the FP32
    spectra (end to end) and, for BF16 / E4M3, against the oracle on the
    stored (rounded) values; plus the largest per-cell weight error."""
    import oracle
    from oracle import quant as Q
    geom = np.array(f.geom())
    _, ids, _ = oracle.neighbours_band(geom, f.lon, f.lat, cells)
    rows = np.unique(ids)
    x = f.spectra_np(rows)
    lon, lat = f.lon[rows], f.lat[rows]
    v, wr, ab, cnt = oracle.grid_cells(geom, lon, lat, x, cells)
    ok = cnt > 0

    def stats(got, vref, abref):
        cond = np.abs(got[ok] - vref[ok]) / (np.abs(vref[ok]) + abref[ok])
        norm = np.linalg.norm(got[ok] - vref[ok], axis=0) / np.maximum(np.linalg.norm(vref[ok], axis=0), 1e-300)
        return float(cond.max()), float(norm.max())

    out = {}
    for st, got, gw, scale in results:
        e = {"tol": {"f32": 1e-5, "bf16": 4e-3, "e4m3": 3e-2}[st]}
        e["max_cond"], e["max_normwise"] = stats(got, v, ab)
        e["weights_max_rel"] = float((np.abs(gw[ok] - wr[ok]) / wr[ok]).max())
        e["empty_cells_nan"] = bool(np.all(np.isnan(got[~ok])) and np.all(gw[~ok] == 0))
        if st != "f32":
            if st == "bf16":
                deq = Q.bf16_bits_to_f32(Q.bf16_round_bits(x)).astype(np.float64)
            else:
                sc = np.asarray(scale, np.float32)
                y = (x / sc[None, :]).astype(np.float32)
                deq = Q.e4m3_dequantise(Q.e4m3_encode(y).reshape(x.shape), sc)
            v2, _, ab2, _ = oracle.grid_cells(geom, lon, lat, deq, cells)
            e["vs_stored_max_cond"], e["vs_stored_max_normwise"] = stats(got, v2, ab2)
        e["within_tol"] = e["max_cond"] <= e["tol"] and e["empty_cells_nan"]
        out[st] = e
    out["_sample"] = (f"{cells.size} cells ({int(ok.sum())} non-empty): 10 random 32x32 blocks and 16x16 corner "
                      f"blocks, all {f.nchan} channels, {rows.size} contributing samples")
    return out


def gather_ms(g, steps):
    """Mean device time of the gather kernel of hcg_grid on g over `steps`
    passes (the library's stage timers: CUDA events on its stream)."""
    g.set_profiling(True)
    for _ in range(steps):
        g.grid()
    g.sync()
    ms = g.stage_times()["gather"]
    g.set_profiling(False)
    return ms


# Nominal dense tensor rates relative to BF16 (2.25 PFLOP/s): kind::tf32 1.1,
# kind::f16 (BF16, and FP16 operands after E4M3 widening) 2.25.
TENSOR_RATIO = {"f32": 1.1 / 2.25, "bf16": 1.0, "e4m3": 1.0}


def roofline_entry(f, storage, info, kernel_ms, peaks):
    """Roofline of one gather kernel.  CUDA-core paths spend one FP32 FMA per
    contribution: bound "alu", achieved = 2 x contributions / kernel time
    against the measured FP32 FMA peak.  The tensor path has two roofs: HBM
    (algorithmic bytes: spectra once, the sorted sample data, cube and
    weights) and the tensor pipe (the MMA work the kernel issued, counted by
    the kernel: dense blocks of 128 cells x candidates x channels, three
    split-TF32 products for FP32 storage) against the measured BF16 peak
    times the nominal ratio of the operand kind; the bound reported is the
    roof the kernel is closer to."""
    hbm, bf16, fp32, kind = peaks
    s = kernel_ms / 1e3
    alg = _gather_bytes(info["samples_kept"], f.nchan, f.cells, ESIZE[storage])
    flops = 2.0 * info["contributions"]
    kname = {2: "k_tc_gather_f32" if storage == "f32" else "k_tc_gather", 4: "k_gather_staged"}.get(
        info["path"], "k_gather_list" if f.nchan >= 256 else "k_gather")
    e = {"kernel": kname, "storage": storage, "path": PATH_NAME.get(info["path"]), "kernel_ms": round(kernel_ms, 4),
         "alg_bytes": alg, "useful_tflops": round(flops / s / 1e12, 2), "hbm_gbs": round(alg / s / 1e9, 1),
         "hbm_frac": round(alg / s / 1e9 / hbm, 4)}
    if info["path"] == 2:
        tpeak = bf16 * TENSOR_RATIO[storage]
        tach = info.get("tensor_flops", 0) / s / 1e12
        e.update({"tensor_tflops": round(tach, 1), "tensor_peak": round(tpeak, 1),
                  "tensor_frac": round(tach / tpeak, 4), "tensor_frac_useful": round(flops / s / 1e12 / tpeak, 4),
                  "tensor_flops_per_launch": info.get("tensor_flops", 0)})
        if e["tensor_frac"] >= e["hbm_frac"]:
            e.update({"bound": "tensor", "achieved": e["tensor_tflops"], "peak": round(tpeak, 1), "unit": "TFLOP/s",
                      "frac": e["tensor_frac"],
                      "peak_kind": f"{kind} BF16 x {TENSOR_RATIO[storage]:.3f} (nominal ratio of the operand kind)"})
        else:
            e.update({"bound": "hbm", "achieved": e["hbm_gbs"], "peak": hbm, "unit": "GB/s", "frac": e["hbm_frac"],
                      "peak_kind": kind})
    else:
        e["alu_frac"] = round(flops / s / 1e12 / fp32, 4)
        if e["alu_frac"] >= e["hbm_frac"]:
            e.update({"bound": "alu", "achieved": e["useful_tflops"], "peak": round(fp32, 1), "unit": "TFLOP/s",
                      "frac": e["alu_frac"], "peak_kind": "measured (hcg_measure_fp32_peak)"})
        else:
            e.update({"bound": "hbm", "achieved": e["hbm_gbs"], "peak": hbm, "unit": "GB/s", "frac": e["hbm_frac"],
                      "peak_kind": kind})
    return e


def run_triple(args, torch, H, dev, local, world, dist):
    """The workload stored as FP32, BF16 and E4M3 side by side in one batched,
    captured launch (the tuned form), against the plain FP32 gather alone."""
    from paper_2012_13173_gb300 import synth
    base = args.workload[:-3]
    f = synth.workload(base, scale=args.scale) if args.scale != 1.0 else synth.workload(base)
    stream = torch.cuda.Stream(dev)
    fp32_peak = H.measure_fp32_peak(local)
    hbm, bf16, peak_kind = _peaks()
    peaks = (hbm, bf16, fp32_peak, peak_kind)
    b, fields, keep = triple_setup(f, H, torch, dev, local, stream, tune=not args.no_tune, path=args.path)
    for _ in range(args.warmup):
        b.grid()
    b.sync()
    infos = [fl[1].info() for fl in fields]
    contrib = sum(i["contributions"] for i in infos)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clk = Clocks(local)
    clk.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        b.grid()
    t1.record(stream)
    torch.cuda.synchronize(dev)
    clocks = clk.stop()
    if dist:
        dist.barrier()
    ms = t0.elapsed_time(t1) / args.steps
    value, ms = job_rate(contrib, ms, dist, dev)
    batch_info = b.info()

    # each kernel of the batch timed on its own (same kernel, same stream)
    ksteps = max(3, min(args.steps, 10))
    per = []
    for (st, g, cube, w, scale, choice), info in zip(fields, infos):
        per.append(roofline_entry(f, st, info, gather_ms(g, ksteps), peaks))
    dom = max(per, key=lambda e: e["kernel_ms"])

    # the plain FP32 gather (CUDA cores, default layout) on the same inputs
    spec32 = keep[2]
    gp = make_gridder(H, f, "f32", local, stream, "gather")
    gp.load_samples(keep[0], keep[1], spec32, borrow=True)
    for _ in range(2):
        gp.grid()
    gp.sync()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(ksteps):
        gp.grid()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    p_ms = e0.elapsed_time(e1) / ksteps
    pinfo = gp.info()
    p_roof = roofline_entry(f, "f32", pinfo, gather_ms(gp, ksteps), peaks)
    plain = {"path": "gather (CUDA cores, default layout)", "ms_per_step": round(p_ms, 3),
             "contributions_per_step": pinfo["contributions"], "value": pinfo["contributions"] / (p_ms / 1e3),
             "kernel_ms": p_roof["kernel_ms"], "frac": p_roof["frac"], "bound": p_roof["bound"],
             "useful_tflops": p_roof["useful_tflops"], "hbm_frac": p_roof["hbm_frac"]}
    gp.close()

    # error against the FP64 oracle, per stored form, on sampled cells
    err = None
    if rank0(dist) and not args.no_err:
        cells = patch_cells(f)
        idx = torch.from_numpy(cells).to(dev)
        res = []
        for st, g, cube, w, scale, choice in fields:
            got = cube.view(f.cells, f.nchan)[idx].double().cpu().numpy()
            gw = w.view(-1)[idx].double().cpu().numpy()
            res.append((st, got, gw, None if scale is None else scale.cpu().numpy()))
        err = err_vs_fp64(f, res, cells)

    # end to end through the public API: every step loads the three forms
    # from pinned host memory (copied by the library), grids the batch and
    # copies the three cubes and weights back to pinned host memory
    e2e = None
    if args.e2e_steps > 0:
        e2e = triple_e2e(args, f, fields, keep, H, torch, dev, local, stream, contrib, dist)

    cpu = None
    if rank0(dist) and world == 1 and not args.no_cpu:
        cpu, _ = cpu_oracle_rate(f)

    alg_all = sum(_alg_bytes(i["samples_kept"], f.nchan, f.cells, ESIZE[st]) for (st, *_), i in zip(fields, infos))
    roof = {k: dom[k] for k in ("bound", "achieved", "peak", "unit", "frac", "kernel", "kernel_ms", "alg_bytes",
                                "peak_kind", "hbm_frac")}
    for k in ("tensor_frac", "tensor_flops_per_launch", "alu_frac"):
        if k in dom:
            roof[k] = dom[k]
    roof["traffic"] = traffic_of(f.name, dom["storage"], dom["kernel"], dom["alg_bytes"])
    roof["storage"] = dom["storage"]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+bf16+e4m3", "data": "synthetic",
            "config": {"workload": args.workload, "samples": f.n, "nchan": f.nchan, "grid": f"{f.nx}x{f.ny}",
                       "fwhm_arcmin": round(f.fwhm * 60, 4), "support_sigma": round(f.support / (f.fwhm / 2.3548200450309493), 3),
                       "forms": {st: {"path": PATH_NAME.get(i["path"]), "tuning": choice}
                                 for (st, g, c, w, sc, choice), i in zip(fields, infos)},
                       "l2": f"inputs larger than L2 ({f.n * f.nchan * 7 / 1e9:.1f} GB spectra)",
                       "parallelism": f"replicas x{world}"},
            "contributions_per_step": contrib, "pairs_per_step": infos[0]["pairs"],
            "whole_step_hbm_gbs": round(alg_all / (ms / 1e3) / 1e9, 1),
            "roofline": roof, "roofline_by_kernel": per, "plain_fp32": plain,
            "tuned_vs_plain_fp32": {e["storage"]: round(plain["kernel_ms"] / e["kernel_ms"], 3) for e in per},
            "err_vs_fp64": err, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": batch_info["launches"] * args.steps, "batch": batch_info,
            "peaks": {"hbm_gbs": hbm, "bf16_tflops": bf16, "fp32_fma_tflops_measured": round(fp32_peak, 1),
                      "fp8_tflops": round(2 * bf16, 1), "fp8_note": "measured BF16 x 2 (nominal FP8:BF16 ratio)"},
            "clocks": clocks}
    b.close()
    for fl in fields:
        fl[1].close()
    return line


def rank0(dist):
    return dist is None or not dist.is_initialized() or dist.get_rank() == 0


def triple_e2e(args, f, fields, keep, H, torch, dev, local, stream, contrib, dist):
    """End to end through the public API, the three stored forms' spectra in
    pinned host memory.  stream (default): each form has its own Gridder and
    stream, its spectra streamed from the host inside its hcg_grid and its
    cube delivered to pinned host memory (hcg_bind_host_output), so the copies
    of one form overlap the gathers of the others; copy: every form copied
    whole at load, one batch, cubes fetched."""
    saved_cpus = os.sched_getaffinity(0)
    local_cpus = gpu_local_cpus(local)
    if local_cpus:
        os.sched_setaffinity(0, local_cpus)
    streamed = args.e2e_mode == "stream"
    lon_h = torch.from_numpy(f.lon).pin_memory()
    lat_h = torch.from_numpy(f.lat).pin_memory()
    hosts, gs, streams = [], [], []
    be = None if streamed else H.Batch(local, stream)
    for k, (st, g, cube, w, scale, choice) in enumerate(fields):
        spec_d = keep[2 + 2 * k]
        spec_h = torch.empty(spec_d.shape, dtype=spec_d.dtype).pin_memory()
        spec_h.copy_(spec_d)
        scale_h = scale.cpu() if scale is not None else None
        cube_h = torch.empty((f.ny, f.nx, f.nchan), dtype=torch.float32).pin_memory()
        w_h = torch.empty((f.ny, f.nx), dtype=torch.float32).pin_memory()
        sk = torch.cuda.Stream(dev) if streamed else stream
        ge = make_gridder(H, f, st, local, sk)
        if choice:
            ge.set_tuning(cells_per_block=choice["cells_per_block"], chans_per_thread=choice["chans_per_thread"],
                          tile_depth=choice["tile_depth"], path=choice["path"])
        if streamed:
            ge.bind_host_output(cube_h, w_h)
        hosts.append((spec_h, scale_h, cube_h, w_h))
        gs.append(ge)
        streams.append(sk)

    def step():
        for ge, (spec_h, scale_h, cube_h, w_h) in zip(gs, hosts):
            ge.load_samples(lon_h, lat_h, spec_h, chan_scale=scale_h, stream=streamed)
        if streamed:
            for ge in gs:
                ge.grid()
            for ge in gs:
                ge.sync()
        else:
            be.grid()
            for ge, (spec_h, scale_h, cube_h, w_h) in zip(gs, hosts):
                ge.fetch(cube_h, w_h)

    if not streamed:
        for ge, (spec_h, scale_h, cube_h, w_h) in zip(gs, hosts):
            ge.load_samples(lon_h, lat_h, spec_h, chan_scale=scale_h)
            be.add(ge)
    step()
    torch.cuda.synchronize(dev)
    a = time.perf_counter()
    for _ in range(args.e2e_steps):
        step()
    torch.cuda.synchronize(dev)
    e_ms = (time.perf_counter() - a) * 1e3 / args.e2e_steps
    e_value, e_ms = job_rate(contrib, e_ms, dist, dev)
    h2d = sum(16 * f.n + f.n * f.nchan * ESIZE[st] + (4 * f.nchan if st == "e4m3" else 0) for st in TRIPLE)
    d2h = 3 * f.cells * (f.nchan + 1) * 4
    if be is not None:
        be.close()
    for ge in gs:
        ge.close()
    del hosts
    os.sched_setaffinity(0, saved_cpus)
    mode = ("three stored forms streamed from pinned host memory, one Gridder and stream per form (the copies "
            "of one form overlap the gathers of the others), cubes delivered to pinned host memory"
            if streamed else "three stored forms copied from pinned host memory at load, one batch, cubes copied back")
    return {"value": e_value, "unit": UNIT, "ms_per_step": round(e_ms, 3), "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "mode": mode,
            "host_cpus": "GPU-local (%d)" % len(local_cpus) if local_cpus else "any"}


def run_sweep(args, torch, H, dev):
    """Scaling sweeps after Sec. 4.2 (Figs. of the sample-count and field-size
    experiments): uniformly random positions in a square field centred at
    (180, +30) deg, one N(0, 1) value per sample (C = 1), FWHM 300 arcsec,
    support 3 sigma, cells of 200 arcsec.  'samples': a 5 x 5 deg field (90 x 90
    cells) with N from 1e3 to 3.6e8; 'field': fields of 0.1 to 60 deg at 1e5
    samples per square degree.  Inputs are made on the device (seeded); each
    point prints one JSON line: device time of hcg_grid (events), its stages,
    and the end-to-end time with host inputs and host results."""
    fwhm, pix = 300.0 / 3600.0, 200.0 / 3600.0
    if args.sweep == "samples":
        points = [(5.0, n) for n in (1_000, 10_000, 100_000, 1_000_000, 10_000_000, 100_000_000, 360_000_000)]
    else:
        points = [(side, int(round(1e5 * side * side))) for side in (0.1, 0.5, 1.0, 5.0, 10.0, 30.0, 60.0)]
    gen = torch.Generator(device=dev)
    for side, n in points:
        gen.manual_seed(1000 + n)
        lat0 = 30.0
        # uniform on the sphere inside the field: lon uniform, sin(lat) uniform
        lon = 180.0 + side * (torch.rand(n, generator=gen, device=dev, dtype=torch.float64) - 0.5)
        s0, s1 = np.sin(np.radians(lat0 - side / 2)), np.sin(np.radians(lat0 + side / 2))
        lat = torch.rad2deg(torch.asin(s0 + (s1 - s0) * torch.rand(n, generator=gen, device=dev,
                                                                        dtype=torch.float64)))
        spec = torch.randn((n, 1), generator=gen, device=dev, dtype=torch.float32)
        nx = max(1, int(round(side / pix)))
        g = H.Gridder(dev.index, torch.cuda.current_stream(dev))
        g.set_kernel(fwhm, 3.0 * fwhm / 2.3548200450309493)
        g.set_grid(180.0, lat0, pix, nx, nx)
        g.load_samples(lon, lat, spec, borrow=True)
        for _ in range(args.warmup):
            g.grid()
        g.sync()
        g.set_profiling(True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            g.grid()
        e1.record()
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / args.steps
        stages = g.stage_times()
        g.set_profiling(False)
        info = g.info()
        # end to end: host inputs copied in, result copied out
        lon_h, lat_h, spec_h = lon.cpu().pin_memory(), lat.cpu().pin_memory(), spec.cpu().pin_memory()
        cube_h = torch.empty((nx, nx, 1), dtype=torch.float32).pin_memory()
        w_h = torch.empty((nx, nx), dtype=torch.float32).pin_memory()
        ge = H.Gridder(dev.index, torch.cuda.current_stream(dev))
        ge.set_kernel(fwhm, 3.0 * fwhm / 2.3548200450309493)
        ge.set_grid(180.0, lat0, pix, nx, nx)
        ge.load_samples(lon_h, lat_h, spec_h)
        ge.grid()
        ge.fetch(cube_h, w_h)
        torch.cuda.synchronize(dev)
        a = time.perf_counter()
        for _ in range(max(1, args.e2e_steps)):
            ge.load_samples(lon_h, lat_h, spec_h)
            ge.grid()
            ge.fetch(cube_h, w_h)
        e2e_ms = (time.perf_counter() - a) * 1e3 / max(1, args.e2e_steps)
        print(json.dumps({"sweep": args.sweep, "field_deg": side, "samples": n, "grid": f"{nx}x{nx}",
                          "ms_per_pass": round(ms, 4), "stage_ms": {k: round(v, 4) for k, v in stages.items()},
                          "pairs": info["pairs"], "contributions_per_s": info["contributions"] / (ms / 1e3),
                          "e2e_ms": round(e2e_ms, 3)}), flush=True)
        g.close()
        ge.close()
        del lon, lat, spec, lon_h, lat_h, spec_h
        torch.cuda.empty_cache()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="drift-16M-c256-x3",
                    help="a named workload, NAME-x3 for its FP32, BF16 and E4M3 forms in one batch, or batch-64")
    ap.add_argument("--storage", default="f32", choices=["f32", "bf16", "e4m3"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--sweep", default="", choices=["", "samples", "field"],
                    help="scaling sweep (one JSON line per point) instead of the benchmark line")
    ap.add_argument("--e2e-mode", default="stream", choices=["stream", "copy"],
                    help="end-to-end leg: host spectra streamed by channel windows, or copied whole at load")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-err", action="store_true", help="skip the error against the FP64 oracle (x3 workloads)")
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the autotuner (x3 workloads: every form then runs --path)")
    ap.add_argument("--tuning", default="0,0,0",
                    help="cells per block, channels per thread, tile depth (0 = automatic)")
    ap.add_argument("--path", default="auto", choices=list(PATHS),
                    help="gridding path (scatter: the Sec. 2.2 atomic-add comparison)")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="shrink the field side by this factor at the same density (profiling runs)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    from paper_2012_13173_gb300 import synth
    if args.workload.startswith("batch-"):
        f = None
    else:
        base = args.workload[:-3] if args.workload.endswith("-x3") else args.workload
        f = synth.workload(base, scale=args.scale) if args.scale != 1.0 else synth.workload(base)

    if args.impl == "reference":
        run_reference(args, f, world, rank)
        return

    import torch
    import paper_2012_13173_gb300 as H
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    if args.sweep:
        run_sweep(args, torch, H, dev)
        return

    if args.workload.endswith("-x3"):
        del f
        line = run_triple(args, torch, H, dev, local, world, dist)
        if rank == 0:
            print(json.dumps(line), flush=True)
        if dist:
            dist.destroy_process_group()
        return

    if args.workload.startswith("batch-"):
        line = run_batch(args, torch, H, dev, local, world, dist)
        if rank == 0:
            print(json.dumps(line), flush=True)
        if dist:
            dist.destroy_process_group()
        return

    stream = torch.cuda.current_stream(dev)
    lon_d, lat_d, spec_d, scale_d = device_inputs(f, args.storage, torch, dev)
    cube = torch.empty((f.ny, f.nx, f.nchan), dtype=torch.float32, device=dev)
    wts = torch.empty((f.ny, f.nx), dtype=torch.float32, device=dev)

    tuning = tuple(int(x) for x in args.tuning.split(","))
    g = make_gridder(H, f, args.storage, local, stream, args.path, tuning)
    g.load_samples(lon_d, lat_d, spec_d, chan_scale=scale_d, borrow=True)
    g.bind_output(cube, wts)

    for _ in range(args.warmup):
        g.grid()
    g.sync()
    info = g.info()
    g.set_profiling(True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clk = Clocks(local)
    clk.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        g.grid()
    t1.record(stream)
    torch.cuda.synchronize(dev)
    clocks = clk.stop()
    if dist:
        dist.barrier()
    ms = t0.elapsed_time(t1) / args.steps
    g.sync()
    stages = g.stage_times()
    g.set_profiling(False)
    contrib = info["contributions"]
    value, ms = job_rate(contrib, ms, dist, dev)
    esize = {"f32": 4, "bf16": 2, "e4m3": 1}[args.storage]
    hbm, bf16, peak_kind = _peaks()
    gb = _gather_bytes(info["samples_kept"], f.nchan, f.cells, esize)
    g_ms = stages["gather"]
    achieved = gb / (g_ms / 1e3) / 1e9
    if info["path"] == 3:
        kname = "k_scatter"
        roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(achieved / hbm, 4), "kernel": kname, "kernel_ms": round(g_ms, 4), "alg_bytes": gb,
                "peak_kind": peak_kind}
    else:
        ent = roofline_entry(f, args.storage, info, g_ms, (hbm, bf16, H.measure_fp32_peak(local), peak_kind))
        kname = ent["kernel"]
        roof = {k: ent[k] for k in ("bound", "achieved", "peak", "unit", "frac", "kernel", "kernel_ms", "alg_bytes",
                                    "peak_kind", "hbm_frac")}
        for k in ("tensor_frac", "tensor_flops_per_launch", "alu_frac"):
            if k in ent:
                roof[k] = ent[k]
    roof["traffic"] = traffic_of(f.name, args.storage, kname, roof["alg_bytes"]) if not any(tuning) else None

    # end to end through the public API with host buffers (pinned)
    e2e = None
    if args.e2e_steps > 0:
        # host buffers in the GPU's own NUMA node: run on its local CPUs while
        # they are allocated and used (the oracle below gets every core back)
        saved_cpus = os.sched_getaffinity(0)
        local_cpus = gpu_local_cpus(local)
        if local_cpus:
            os.sched_setaffinity(0, local_cpus)
        lon_h = torch.from_numpy(f.lon).pin_memory()
        lat_h = torch.from_numpy(f.lat).pin_memory()
        spec_h = torch.empty((f.n, f.nchan), dtype=spec_d.dtype).pin_memory()
        spec_h.copy_(spec_d)
        scale_h = scale_d.cpu() if scale_d is not None else None
        cube_h = torch.empty((f.ny, f.nx, f.nchan), dtype=torch.float32).pin_memory()
        w_h = torch.empty((f.ny, f.nx), dtype=torch.float32).pin_memory()
        ge = make_gridder(H, f, args.storage, local, stream, args.path, tuning)

        streamed = args.e2e_mode == "stream"

        if streamed:
            ge.bind_host_output(cube_h, w_h)

        def e2e_step():
            # stream: the spectra stay in pinned host memory and hcg_grid copies
            # them in window by window of channels and the cube back out the
            # same way, both overlapping the gather; copy: one whole copy at
            # load time, the pass, then one whole copy back
            ge.load_samples(lon_h, lat_h, spec_h, chan_scale=scale_h, stream=streamed)
            ge.grid()
            if streamed:
                ge.sync()
            else:
                ge.fetch(cube_h, w_h)

        e2e_step()
        torch.cuda.synchronize(dev)
        ge_window = ge.info()["stream_window"]
        a = time.perf_counter()
        for _ in range(args.e2e_steps):
            e2e_step()
        torch.cuda.synchronize(dev)
        e_ms = (time.perf_counter() - a) * 1e3 / args.e2e_steps
        e_value, e_ms = job_rate(contrib, e_ms, dist, dev)
        h2d = f.n * 16 + f.n * f.nchan * esize + (f.nchan * 4 if scale_d is not None else 0)
        d2h = f.cells * (f.nchan + 1) * 4
        e2e = {"value": e_value, "unit": UNIT, "ms_per_step": round(e_ms, 3),
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "mode": ("host spectra streamed in windows of %d channels" % ge_window) if streamed
               else "whole copy at load",
               "host_cpus": "GPU-local (%d)" % len(local_cpus) if local_cpus else "any"}
        ge.close()
        del lon_h, lat_h, spec_h, cube_h, w_h
        os.sched_setaffinity(0, saved_cpus)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu, _ = cpu_oracle_rate(f)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.storage, "data": "synthetic",
            "config": {"workload": f.name, "samples": f.n, "nchan": f.nchan, "grid": f"{f.nx}x{f.ny}",
                       "fwhm_arcmin": round(f.fwhm * 60, 4), "support_sigma": round(f.support / (f.fwhm / 2.3548200450309493), 3),
                       "path": {1: "gather", 2: "tensor", 3: "scatter", 4: "staged"}.get(info["path"], info["path"]),
                       "l2": (f"inputs larger than L2 ({f.n * f.nchan * esize / 1e9:.2f} GB spectra)"
                              if f.n * f.nchan * esize > L2_BYTES else
                              f"inputs fit in L2 ({f.n * f.nchan * esize / 1e6:.2f} MB spectra, no flush): a "
                              "latency-bound small field, timed warm"),
                       "parallelism": f"replicas x{world}"},
            "contributions_per_step": contrib, "pairs_per_step": info["pairs"],
            "stage_ms": {k: round(v, 4) for k, v in stages.items()},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": info["launches"] * args.steps, "clocks": clocks}
    if rank == 0:
        print(json.dumps(line), flush=True)
    g.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
