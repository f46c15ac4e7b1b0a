"""Benchmark of the box-sum Gaussian filter on one GB300 (or N replicas).

Default workload: one 4096 x 4096 single-channel uint8 1/f image (seed 2),
sigma = 8, K = 4 (radii 4, 9, 14, 20), replicate boundary, FP32 output.  A
step is one full filter pass (rows + columns) of that image.  L2 is flushed
(a write of twice the L2 size) before every timed step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload headline|f32|config1|precision]

Prints one JSON line (rank 0).  Under torchrun each rank filters its own copy
(replicas: the images are independent, no collective on the data path).
"""
import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (H, W, C, in dtype, out dtype, sigma, K, boundary, seed, offset)
    "headline": (4096, 4096, 1, "u8", "f32", 8.0, 4, "replicate", 2, 0.0),
    "f32": (4096, 4096, 1, "f32", "f32", 8.0, 4, "replicate", 2, 0.0),
    "config1": (512, 512, 1, "f32", "f32", 5.0, 3, "replicate", 1, 0.0),
    "precision": (8192, 8192, 1, "f32", "f32", 100.0, 5, "replicate", 4, 1.0e4),
}
BYTES = {"u8": 1, "u16": 2, "f32": 4, "bf16": 2, "f16": 2}
KERNEL_SOURCES = ["paper_1107_4958_gb300/csrc/strip_kernel.cuh", "paper_1107_4958_gb300/csrc/filter_host.cu",
                  "paper_1107_4958_gb300/csrc/internal.h"]


def kernel_hash():
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def recorded_traffic(workload):
    """DRAM bytes per launch from a committed ncu summary, if taken on this kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        d = json.load(fh)
    rec = d.get(workload)
    if not rec or rec.get("kernel_hash") != kernel_hash():
        return None
    return rec.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        if not self.samples:
            return None
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        smax = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[3 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(self.samples)}


def oracle_rate(H, W, C, in_name, sigma, K, boundary, seed, offset, budget_s=10.0):
    """CPU oracle throughput (output pixels / s) on a bounded sample of the workload:
    whole output rows computed by the FP64 oracle until `budget_s` has elapsed."""
    from oracle import filter as of
    from oracle import fit as ofit
    from paper_1107_4958_gb300 import synth
    rng = np.random.default_rng(0)
    f = synth.image(H, W, seed=seed, dtype="u8" if in_name == "u8" else "f32", c=C, offset=offset)
    r, w = ofit.fit_gaussian_boxes(sigma, K)
    done = 0
    t0 = time.perf_counter()
    rows = 0
    while time.perf_counter() - t0 < budget_s:
        ys = [int(rng.integers(0, H))]
        of.filter_rows_at(f.astype(np.float64), r, w, boundary, ys)
        done += W * C
        rows += 1
    dt = time.perf_counter() - t0
    return done / dt, "%d random output rows of %dx%dx%d (%.1f s)" % (rows, H, W, C, dt)


def run_reference(args, wl):
    H, W, C, in_name, out_name, sigma, K, boundary, seed, offset = wl
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    budget = max(1.0, 20.0 / max(1, args.steps + args.warmup))
    rates = []
    samples = []
    for i in range(args.warmup + args.steps):
        rate, sample = oracle_rate(H, W, C, in_name, sigma, K, boundary, seed, offset, budget_s=budget)
        if i >= args.warmup:
            rates.append(rate)
            samples.append(sample)
    gpx = float(np.mean(rates)) / 1e9
    line = {"impl": "reference", "metric": "Gpixel/s", "value": gpx, "unit": "Gpixel/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": H * W * C / (gpx * 1e9) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "H": H, "W": W, "C": C, "in": in_name,
                       "out": out_name, "sigma": sigma, "K": K, "boundary": boundary,
                       "l2": "oracle on host cores"},
            "cpu_baseline": {"value": gpx, "unit": "Gpixel/s", "cores": 1, "kind": "oracle",
                             "sample": samples[0] if samples else ""},
            "e2e": {"value": gpx, "unit": "Gpixel/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="headline", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, wl)
        return
    H, W, C, in_name, out_name, sigma, K, boundary, seed, offset = wl

    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)

    import __graft_entry__
    __graft_entry__.build()
    from paper_1107_4958_gb300 import gaussbox, synth
    from paper_1107_4958_gb300.abi_types import BOUNDARY_CODE, dtype_code

    tdt = {"u8": torch.uint8, "f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}
    f = synth.image(H, W, seed=seed, dtype="u8" if in_name == "u8" else "f32", c=C, offset=offset)
    host_in = torch.from_numpy(f).to(tdt[in_name]).pin_memory()
    x = host_in.to(dev)
    y = torch.empty(x.shape, dtype=tdt[out_name], device=dev)
    host_out = torch.empty(y.shape, dtype=y.dtype).pin_memory()
    stream = torch.cuda.current_stream(dev)
    sh = stream.cuda_stream
    pitch_in = W * C * BYTES[in_name]
    pitch_out = W * C * BYTES[out_name]
    bcode = BOUNDARY_CODE[boundary]

    def step():
        gaussbox.gauss_filter(x.data_ptr(), pitch_in, y.data_ptr(), pitch_out, H, W, C, dtype_code(x.dtype),
                              dtype_code(y.dtype), sigma, K, bcode, sh)

    l2 = torch.cuda.get_device_properties(dev).L2_cache_size
    flush = torch.empty(max(4 * l2, 512 << 20), dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        flush.fill_(1)
        step()
    torch.cuda.synchronize()

    clocks = ClockSampler(dev.index) if rank == 0 else None
    if clocks:
        clocks.start()
        time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    for i in range(args.steps):
        flush.fill_(1)
        evs[i][0].record(stream)
        step()
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = [a.elapsed_time(b) for a, b in evs]
    ms_step = float(np.mean(ms))

    # end to end through the public call with host buffers: H2D, filter, D2H per step
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_steps = max(3, min(args.steps, 20))
    e0.record(stream)
    for _ in range(e2e_steps):
        x.copy_(host_in, non_blocking=True)
        step()
        host_out.copy_(y, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    csamp = clocks.stop() if clocks else None

    t = torch.tensor([ms_step, e2e_ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_step, e2e_ms = float(t[0]), float(t[1])
    assert gaussbox.gf_get_device_status() == 0
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    px = H * W * C
    gpx = px * world / (ms_step * 1e-3) / 1e9
    alg_bytes = px * (BYTES[in_name] + BYTES[out_name])
    peak, peak_kind = measured_peaks()
    achieved = alg_bytes / (ms_step * 1e-3) / 1e9
    line = {
        "metric": "Gpixel/s", "value": gpx, "unit": "Gpixel/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if in_name != "u8" else "i32+f32", "data": "synthetic",
        "config": {"workload": args.workload, "H": H, "W": W, "C": C, "in": in_name, "out": out_name,
                   "sigma": sigma, "K": K, "boundary": boundary, "parallelism": "replicas",
                   "l2": "flushed before each step (%d MB write, > 2x L2)" % (flush.numel() >> 20)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind,
                     "traffic": recorded_traffic(args.workload),
                     "alg_bytes_per_launch": alg_bytes, "kernel": "strip_filter_kernel"},
        "e2e": {"value": px * world / (e2e_ms * 1e-3) / 1e9, "unit": "Gpixel/s",
                "h2d_bytes_per_step": host_in.numel() * host_in.element_size(),
                "d2h_bytes_per_step": host_out.numel() * host_out.element_size()},
        "gpu_launches": args.steps,
        "clocks": csamp,
        "ms_per_step_min": float(np.min(ms)), "ms_per_step_median": float(np.median(ms)),
    }
    if not args.no_cpu_baseline:
        rate, sample = oracle_rate(H, W, C, in_name, sigma, K, boundary, seed, offset, budget_s=10.0)
        line["cpu_baseline"] = {"value": rate / 1e9, "unit": "Gpixel/s", "cores": 1, "kind": "oracle",
                                "sample": sample}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
