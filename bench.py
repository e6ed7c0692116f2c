#!/usr/bin/env python
"""Benchmark of the CCC hot path on GB300: elementwise comparisons per second.

A step is one pass of the whole 2-way hot path through the C ABI
(ccc2_tally_metric): per-SNP allele counts, the e4m3 count-operand unpack, and
the tcgen05 tally kernel with the fused CCC epilogue writing all tallies and
CCC values of the upper triangle to HBM.  A comparison is one (pair, individual)
element pair producing four tallies (Sec. 6).

Default workload (one GPU): 2-way CCC at scale, n_v = 20,000 SNP vectors x
n_f = 16,384 individuals, Hardy-Weinberg genotypes with Beta(1/2,1/2) minor
allele frequencies floored at 0.01, 1% missing entries, seed 1; synthetic
(the counter-based generator in synth/).

Prints ONE JSON line (rank 0).  Under torchrun with N ranks every rank runs an
independent panel of the same shape (seed 1 + rank); there is no data-path
collective (weak scaling), only a barrier around the timed region.

--impl reference times the CPU oracle (oracle/, all host cores) on a bounded
random sample of pairs of the same workload in every step.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "2-way CCC elementwise comparisons/sec on 1 GB300"
UNIT = "comparisons/s"
WORKLOAD = ("2-way CCC at scale: n_v=20000 SNP vectors x n_f=16384 individuals, Hardy-Weinberg "
            "genotypes, Beta(1/2,1/2) MAF floored at 0.01, 1% missing, seed 1; all 199,990,000 "
            "unique pairs, 4 int32 tallies + 4 fp32 CCC per pair")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n-v", type=int, default=20000)
    ap.add_argument("--n-f", type=int, default=16384)
    ap.add_argument("--path", default="tc", choices=["tc", "popc"])
    ap.add_argument("--skip-cpu", action="store_true", help="no oracle CPU baseline")
    ap.add_argument("--skip-e2e", action="store_true", help="no host-buffer end-to-end timing")
    ap.add_argument("--skip-popc", action="store_true", help="no popcount-path comparison")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU time of the oracle baseline sample")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["bf16_tflops"]), float(d["hbm_gbs"]), "measured"
    except Exception:
        return 1900.0, 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_id), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        time.sleep(0.3)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
                pw.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "power_w_max": max(pw) if pw else None, "reasons": sorted(reasons)}


def gpu_id_for(torch, dev):
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return str(dev)


def cpu_baseline(geno, n_f, n_v, seconds, seed=7):
    """Oracle on host cores over random pairs of the same panel, ~`seconds` of CPU work."""
    import oracle
    rng = np.random.default_rng(seed)
    batch = 8192
    done = 0
    t0 = time.perf_counter()
    while True:
        i = rng.integers(0, n_v - 1, size=batch)
        j = i + 1 + (rng.random(batch) * (n_v - 1 - i)).astype(np.int64)
        oracle.ccc2_pairs(geno, n_f, i, j)
        done += batch
        el = time.perf_counter() - t0
        if el >= seconds or done >= 64 * batch:
            break
    return {"value": done * n_f / el, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
            "sample": f"{done} uniformly random pairs (i<j) of the same panel, all {n_f} "
                      f"individuals each, {el:.1f} s on the host cores"}


def run_reference(args):
    """The CPU oracle timed on this workload (rank 0 only)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    n_v, n_f = args.n_v, args.n_f
    geno = synth.panel_hwe(n_v, n_f, seed=1, p_missing=0.01)
    rng = np.random.default_rng(11)
    pairs_per_step = 4096

    def step():
        i = rng.integers(0, n_v - 1, size=pairs_per_step)
        j = i + 1 + (rng.random(pairs_per_step) * (n_v - 1 - i)).astype(np.int64)
        oracle.ccc2_pairs(geno, n_f, i, j)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    el = time.perf_counter() - t0
    value = args.steps * pairs_per_step * n_f / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64/f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_v": n_v, "n_f": n_f,
                   "sample_per_step": f"{pairs_per_step} random pairs x {n_f} individuals"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                         "sample": f"{pairs_per_step} uniformly random pairs per step, "
                                   f"{args.steps} timed steps"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)

    import torch

    import paper_1705_08213_gb300 as ccc
    from paper_1705_08213_gb300 import build as cbuild

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl", device_id=dev)
        pg = dist
    if rank == 0:
        cbuild.build()
    if pg is not None:
        pg.barrier()
    ccc.load()

    n_v, n_f = args.n_v, args.n_f
    npairs = n_v * (n_v - 1) // 2
    cmp_per_step = npairs * n_f
    path = ccc.CCC_PATH_TC if args.path == "tc" else ccc.CCC_PATH_POPC

    geno_np = synth.panel_hwe(n_v, n_f, seed=1 + rank, p_missing=0.01)
    host_geno = torch.from_numpy(geno_np.view(np.int64)).pin_memory()
    geno = host_geno.to(dev)
    opts0 = ccc.ccc_opts_default(path=path)
    ws = torch.empty(ccc.ccc_workspace_size(geno, n_f, opts0, ccc.CCC_OP_2WAY), dtype=torch.uint8,
                     device=dev)
    opts = ccc.ccc_opts_default(path=path, workspace=ws)
    tally = torch.empty((npairs, 4), dtype=torch.int32, device=dev)
    out = torch.empty((npairs, 4), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        ccc.ccc2_tally_metric(geno, n_f, tally, out, opts, stream)

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize(dev)
    if ccc.ccc_status(opts) != ccc.CCC_OK:
        raise RuntimeError("device status not ok after warm-up")

    # ---------------------------------------------------------------- timed region
    sampler = ClockSampler(gpu_id_for(torch, dev)) if local == 0 else None
    if sampler:
        sampler.start()
    if pg is not None:
        pg.barrier()
    torch.cuda.synchronize(dev)
    ccc.ccc_timing_enable(True)
    ccc.ccc_timing_read()
    launches0 = ccc.ccc_launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    if pg is not None:
        pg.barrier()
    launches = ccc.ccc_launch_count() - launches0
    kernel_ms, kernel_n = ccc.ccc_timing_read()
    ccc.ccc_timing_enable(False)
    clocks = sampler.stop() if sampler else None
    elapsed_ms = ev0.elapsed_time(ev1)
    ms_per_step = elapsed_ms / args.steps
    if pg is not None:
        t = torch.tensor([ms_per_step], device=dev)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        ms_per_step = float(t.item())
    if ccc.ccc_status(opts) != ccc.CCC_OK:
        raise RuntimeError("device status not ok after the timed region")
    value = world * cmp_per_step / (ms_per_step * 1e-3)

    # Roofline of the dominant kernel (the tally kernel), from its own events.
    bf16_peak, hbm_peak, peak_src = measured_peaks()
    kernel_avg_ms = kernel_ms / max(kernel_n, 1)
    if path == ccc.CCC_PATH_TC:
        flops = 8.0 * cmp_per_step  # 4 MAC per comparison, 2 flops per MAC
        achieved = flops / (kernel_avg_ms * 1e-3) / 1e12
        peak = 2.0 * bf16_peak  # e4m3 dense = 2x bf16 dense (nominal 4.5 / 2.25 PFLOP/s)
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None,
                "kernel": "k_tally2_tc", "kernel_ms": kernel_avg_ms,
                "peak_note": f"e4m3 dense peak = 2 x {peak_src} bf16 burst {bf16_peak:.0f} TFLOP/s "
                             "(kind::i8 is not available on sm_103a)"}
    else:
        popc = 9.0 * cmp_per_step / 64.0  # nine 64-bit AND+POPC per 64 comparisons
        achieved = popc / (kernel_avg_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": None, "unit": "Tpopc64/s",
                "frac": None, "traffic": None, "kernel": "k_tally2_popc",
                "kernel_ms": kernel_avg_ms}

    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "e4m3 operands, fp32 accumulate" if path == ccc.CCC_PATH_TC else "u64 bit planes",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_v": n_v, "n_f": n_f, "path": args.path,
                   "parallelism": f"{world} independent panels (one per GPU)" if world > 1 else "1 GPU",
                   "l2": "inputs larger than L2: 655 MB e4m3 operand matrix read and 6.4 GB of "
                         "tallies+CCC written per step (L2 129 MB)"},
        "gpu_launches": int(launches),
        "roofline": roof,
        "clocks": clocks,
    }

    # ---------------------------------------------------------------- end to end
    if not args.skip_e2e and rank == 0:
        host_tally = torch.empty((npairs, 4), dtype=torch.int32, pin_memory=True)
        host_ccc = torch.empty((npairs, 4), dtype=torch.float32, pin_memory=True)
        e2e_steps = max(1, min(args.steps, 5))

        def e2e_step():
            geno.copy_(host_geno, non_blocking=True)
            ccc.ccc2_tally_metric(geno, n_f, tally, out, opts, stream)
            host_tally.copy_(tally, non_blocking=True)
            host_ccc.copy_(out, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(e2e_steps):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        e2e_ms = e0.elapsed_time(e1) / e2e_steps
        result["e2e"] = {"value": cmp_per_step / (e2e_ms * 1e-3), "unit": UNIT,
                         "h2d_bytes_per_step": host_geno.numel() * 8,
                         "d2h_bytes_per_step": npairs * 32, "ms_per_step": e2e_ms,
                         "note": "pinned host panel -> device, ccc2_tally_metric, all tallies and "
                                 "CCC values -> pinned host, one stream"}
        del host_tally, host_ccc

    # ---------------------------------------------------------------- popcount path
    if not args.skip_popc and rank == 0 and path == ccc.CCC_PATH_TC:
        del ws
        opts_p0 = ccc.ccc_opts_default(path=ccc.CCC_PATH_POPC)
        wsp = torch.empty(ccc.ccc_workspace_size(geno, n_f, opts_p0, ccc.CCC_OP_2WAY),
                          dtype=torch.uint8, device=dev)
        opts_p = ccc.ccc_opts_default(path=ccc.CCC_PATH_POPC, workspace=wsp)
        ccc.ccc2_tally_metric(geno, n_f, tally, out, opts_p, stream)
        torch.cuda.synchronize(dev)
        ccc.ccc_timing_enable(True)
        ccc.ccc_timing_read()
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        nps = 2
        p0.record(stream)
        for _ in range(nps):
            ccc.ccc2_tally_metric(geno, n_f, tally, out, opts_p, stream)
        p1.record(stream)
        torch.cuda.synchronize(dev)
        pk_ms, pk_n = ccc.ccc_timing_read()
        ccc.ccc_timing_enable(False)
        pms = p0.elapsed_time(p1) / nps
        result["popc_path"] = {"value": cmp_per_step / (pms * 1e-3), "unit": UNIT,
                               "ms_per_step": pms, "kernel_ms": pk_ms / max(pk_n, 1),
                               "tc_speedup": pms / ms_per_step}

    # ---------------------------------------------------------------- CPU baseline
    if not args.skip_cpu and rank == 0 and world == 1:
        result["cpu_baseline"] = cpu_baseline(geno_np, n_f, n_v, args.cpu_seconds)

    if rank == 0:
        print(json.dumps(result), flush=True)
    if pg is not None:
        pg.barrier()
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
