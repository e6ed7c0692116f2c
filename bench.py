#!/usr/bin/env python
"""Benchmark of the CCC hot path on GB300: elementwise comparisons per second.

A comparison is one element pair (2-way) or triple (3-way) of one individual,
producing four (eight) tallies (Sec. 6).  A step is one pass of the whole hot
path through the C ABI over one synthetic panel resident in HBM.

Workloads (``--workload``):
  2way    default; 2-way CCC at scale: n_v = 20,000 SNP vectors x n_f = 16,384
          individuals, Hardy-Weinberg genotypes, Beta(1/2,1/2) minor-allele
          frequencies floored at 0.01, 1% missing, seed 1.  Step =
          ccc2_tally_metric: the count-operand unpack (e2m1 rows and the
          per-SNP factors from one read of the codes), the tcgen05 tally
          kernel with the fused CCC epilogue writing every tally and CCC value
          of the upper triangle (6.4 GB).
  3way    3-way CCC: n_v = 1,536 x n_f = 8,192, same genotype model, seed 4;
          step = ccc3_tally_metric over all slabs (602,800,640 triples, 38.6 GB).
  filter  2-way with thresholded output: n_v = 200,000 x n_f = 4,096, same
          model, seed 5, plus 1,000 planted near-duplicate pairs (1% of entries
          redrawn); step = ccc2_filter keeping pairs with max CCC > 0.16.
  small   2-way, n_v = 256 x n_f = 1,024, uniform genotypes, 2% missing, seed 0.
  batched 64 independent 2-way panels, n_v ~ U{500..8000}, n_f ~ U{2000..50000}
          (shape draws seed 2), Hardy-Weinberg model (seed 2, panel index k);
          step = ccc2_batched with the schedule chosen by ccc2_batched_tune,
          captured once in a CUDA graph and replayed; compared with all panels
          in one persistent launch and with 64 sequential ccc2_tally_metric calls.
  multi   2-way CCC of markers with s = 4 allele states, 10,000 x 16,384, seed
          6; step = ccc2_multi_tally_metric (16 tallies + 16 CCC per pair).
  long    2-way, 512 SNPs x 1,000,000 individuals, seed 7: few tiles with long
          vectors, computed in K parts (ccc_opts.split automatic).

Panels whose inputs fit the 129 MB L2 (3way, small) get a 256 MB write before
every timed step, outside that step's CUDA events; the others are larger than L2.

Prints ONE JSON line (rank 0).  Under torchrun with N ranks every rank runs an
independent panel of the same shape (seed + rank); there is no data-path
collective (weak scaling), only a barrier around the timed region.  With
--scaling strong every rank holds the same panel and computes its own range of
rows (2-way) or slabs (3-way) from paper_1705_08213_gb300.shard; value = the
whole panel's comparisons / the slowest rank's time.

--impl reference times the CPU oracle (oracle/, all host cores) on a bounded
random sample of the same workload in every step.
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

UNIT = "comparisons/s"

WORKLOADS = {
    "2way": dict(
        kind=2, n_v=20000, n_f=16384, seed=1, model="hwe", p_missing=0.01,
        metric="2-way CCC elementwise comparisons/sec on 1 GB300",
        text=("2-way CCC at scale: n_v=20000 SNP vectors x n_f=16384 individuals, Hardy-Weinberg "
              "genotypes, Beta(1/2,1/2) MAF floored at 0.01, 1% missing, seed 1; all 199,990,000 "
              "unique pairs, 4 int32 tallies + 4 fp32 CCC per pair")),
    "3way": dict(
        kind=3, n_v=1536, n_f=8192, seed=4, model="hwe", p_missing=0.01,
        metric="3-way CCC elementwise comparisons/sec on 1 GB300",
        text=("3-way CCC: n_v=1536 x n_f=8192, Hardy-Weinberg genotypes, Beta(1/2,1/2) MAF floored "
              "at 0.01, 1% missing, seed 4; all 602,800,640 unique triples i<j<k (slabs of fixed j), "
              "8 int32 tallies + 8 fp32 CCC per triple")),
    "filter": dict(
        kind=2, n_v=200000, n_f=4096, seed=5, model="hwe", p_missing=0.01, planted=1000,
        threshold=0.16, metric="2-way CCC elementwise comparisons/sec on 1 GB300",
        text=("2-way CCC large, thresholded output: n_v=200000 x n_f=4096, Hardy-Weinberg genotypes, "
              "Beta(1/2,1/2) MAF floored at 0.01, 1% missing, seed 5, 1000 planted near-duplicate "
              "pairs (1% of entries redrawn); 19,999,900,000 pairs, kept if max CCC > 0.16")),
    "batched": dict(
        kind=2, n_panels=64, seed=2, model="hwe", p_missing=0.01,
        metric="2-way CCC elementwise comparisons/sec on 1 GB300",
        text=("2-way CCC batched: 64 independent panels, n_v uniform in [500,8000], n_f uniform in "
              "[2000,50000] (shape seed 2), Hardy-Weinberg genotypes, Beta(1/2,1/2) MAF floored at "
              "0.01, 1% missing; one persistent launch over all panels' tiles, CUDA-graph replay")),
    "multi": dict(
        kind=2, states=4, n_v=10000, n_f=16384, seed=6, model="multi", p_missing=0.01,
        metric="2-way multi-allelic CCC elementwise comparisons/sec on 1 GB300",
        text=("2-way CCC of markers with s=4 allele states: n_v=10000 markers x n_f=16384 "
              "individuals, per-marker state weights Beta(1/2,1/2) floored at 0.01 and normalised, "
              "two alleles drawn independently, 1% missing, seed 6; all 49,995,000 unique pairs, "
              "16 int32 tallies + 16 fp32 CCC per pair")),
    "long": dict(
        kind=2, n_v=512, n_f=1000000, seed=7, model="hwe", p_missing=0.01, split_compare=True,
        metric="2-way CCC elementwise comparisons/sec on 1 GB300",
        text=("2-way CCC, few SNPs with long vectors: n_v=512 x n_f=1,000,000, Hardy-Weinberg "
              "genotypes, Beta(1/2,1/2) MAF floored at 0.01, 1% missing, seed 7; all 130,816 pairs "
              "(10 SM-pair tiles: the individuals are split into K parts, ccc_opts.split automatic)")),
    "small": dict(
        kind=2, n_v=256, n_f=1024, seed=0, model="uniform", p_missing=0.02,
        metric="2-way CCC elementwise comparisons/sec on 1 GB300",
        text=("2-way CCC plain: n_v=256 x n_f=1024, genotypes uniform on {0,1,2}, 2% missing, "
              "seed 0; all 32,640 unique pairs")),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="2way", choices=sorted(WORKLOADS))
    ap.add_argument("--n-v", type=int, default=None)
    ap.add_argument("--n-f", type=int, default=None)
    ap.add_argument("--path", default="tc", choices=["tc", "popc"])
    ap.add_argument("--tile", type=int, default=0, choices=[0, 1, 2, 3],
                    help="tensor-core variant (0 automatic). 2-way: 1 one SM, 2 SM pairs; 3-way: "
                         "1 masked operands in HBM, 2 masked operands in shared memory, "
                         "3 genotype classes of v_j")
    ap.add_argument("--operand", default="auto", choices=["auto", "e4m3", "e2m1"],
                    help="tensor-core count operands (ccc_opts.operand): auto = e2m1 (FP4) on the "
                         "2-way SM-pair tiles, e4m3 elsewhere")
    ap.add_argument("--scaling", default="weak", choices=["weak", "strong"],
                    help="weak: an independent panel per rank; strong: one panel split by rows/slabs")
    ap.add_argument("--skip-cpu", action="store_true", help="no oracle CPU baseline")
    ap.add_argument("--skip-e2e", action="store_true", help="no host-buffer end-to-end timing")
    ap.add_argument("--skip-popc", action="store_true", help="no popcount-path comparison")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU time of the oracle baseline sample")
    ap.add_argument("--e2e-mode", default="auto", choices=["auto", "stream", "direct", "copy"],
                    help="e2e leg: ccc2_stream phases (stream), results stored by the kernels "
                         "straight into pinned host memory (direct), or one copy per output "
                         "after the call (copy); auto = stream for 2-way, copy otherwise")
    ap.add_argument("--panels", type=int, default=None,
                    help="batched workload: only the first N of its 64 panels (a reduced case)")
    ap.add_argument("--no-sub", action="store_true",
                    help="default 2-way line only: no 3way / batched / filter sub-records")
    ap.add_argument("--source-hash", action="store_true",
                    help="print the hash of the CUDA sources (for profiles/ncu_traffic.json) and exit")
    a = ap.parse_args()
    if a.source_hash:
        for k in KERNEL_SOURCES:
            print(k, source_hash(k))
        raise SystemExit(0)
    w = workload_dict(a.workload, a.n_v, a.n_f)
    if a.panels is not None and a.workload == "batched":
        w["shapes"] = w["shapes"][:max(1, a.panels)]
        w["text"] = (f"reduced case of the batched workload: its first {len(w['shapes'])} panels "
                     "(not the bench line's configuration)")
        w["reduced"] = True
    if a.steps is None:
        a.steps = DEFAULT_STEPS[a.workload]
    return a, w


DEFAULT_STEPS = {"2way": 60, "3way": 12, "filter": 3, "small": 200, "batched": 10, "multi": 60,
                 "long": 20}
# Workloads attached to the default 2-way line as sub-records (one GPU): timed steps and
# warm-up of each, and the seconds of oracle time for its cpu_baseline.
SUB_WORKLOADS = {"3way": (8, 3), "batched": (5, 3), "filter": (3, 3)}
SUB_CPU_SECONDS = 8.0


def workload_dict(name, n_v=None, n_f=None):
    """The workload's description, with the optional reduced sizes and the batched shapes."""
    w = dict(WORKLOADS[name])
    w["name"] = name
    if n_v is not None or n_f is not None:
        w["n_v"] = n_v if n_v is not None else w["n_v"]
        w["n_f"] = n_f if n_f is not None else w["n_f"]
        w["text"] = (f"reduced case of the {name} workload: n_v={w['n_v']} x n_f={w['n_f']}, "
                     f"same generator and seed (not the bench line's configuration)")
        w["reduced"] = True
    if name == "batched":
        rng = np.random.default_rng(w["seed"])
        w["shapes"] = [(int(rng.integers(500, 8001)), int(rng.integers(2000, 50001)))
                       for _ in range(w["n_panels"])]
        w["n_v"], w["n_f"] = max(v for v, _ in w["shapes"]), max(f for _, f in w["shapes"])
    return w


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def make_panel(w, rank=0):
    seed = w["seed"] + rank
    if w["model"] == "multi":
        return synth.panel_multi(w["n_v"], w["n_f"], w["states"], seed=seed, p_missing=w["p_missing"])
    if w["model"] == "uniform":
        g = synth.panel_uniform(w["n_v"], w["n_f"], seed=seed, p_missing=w["p_missing"])
    else:
        g = synth.panel_hwe(w["n_v"], w["n_f"], seed=seed, p_missing=w["p_missing"])
    if w.get("planted"):
        synth.plant_near_duplicates(g, w["n_f"], w["planted"], seed=seed + 1000)
    return g


def inputs_fit_l2(w):
    """Whether a single-panel workload's operand rows fit the 129 MB L2."""
    return "shapes" not in w and w["n_v"] * w["n_f"] * 2 <= 129e6


def l2_flush_buffer(w, torch, dev):
    """A 256 MB device buffer to overwrite between timed steps (twice the L2), or None."""
    return torch.empty(256 << 20, dtype=torch.uint8, device=dev) if inputs_fit_l2(w) else None


def comparisons(w):
    if "shapes" in w:
        return sum(v * (v - 1) // 2 * f for v, f in w["shapes"])
    n_v, n_f = w["n_v"], w["n_f"]
    if w["kind"] == 2:
        return n_v * (n_v - 1) // 2 * n_f
    return n_v * (n_v - 1) * (n_v - 2) // 6 * n_f


# Device-code files of each tally kernel: a traffic figure stays valid while they are unchanged.
KERNEL_SOURCES = {
    "k_tally2_tc_pair": ["k_tc2.cu", "tc_pipeline_pair.cuh", "tc_pipeline.cuh", "tc_sched.cuh",
                         "ccc_dev.cuh", "ccc_metric.cuh", "ccc_launch.h"],
    "k_tally2_tc_pair_fp4": ["k_tc2.cu", "tc_pipeline_pair.cuh", "tc_pipeline.cuh", "tc_sched.cuh",
                             "ccc_dev.cuh", "ccc_metric.cuh", "ccc_launch.h"],
    "k_tally2_tc_pair_fp4w": ["k_tc2.cu", "tc_pipeline_pair.cuh", "tc_pipeline.cuh", "tc_sched.cuh",
                              "ccc_dev.cuh", "ccc_metric.cuh", "ccc_launch.h"],
    "k_tally2_tc_pair_split_fp4": ["k_tc2.cu", "tc_pipeline_pair.cuh", "tc_pipeline.cuh",
                                   "tc_sched.cuh", "ccc_dev.cuh", "ccc_metric.cuh", "ccc_launch.h"],
    "k_tally2_tc_pair_batched_fp4": ["k_tc2.cu", "tc_pipeline_pair.cuh", "tc_pipeline.cuh",
                                     "tc_sched.cuh", "ccc_dev.cuh", "ccc_metric.cuh",
                                     "ccc_launch.h"],
    "k_tally2_tc_pair_split": ["k_tc2.cu", "tc_pipeline_pair.cuh", "tc_pipeline.cuh", "tc_sched.cuh",
                               "ccc_dev.cuh", "ccc_metric.cuh", "ccc_launch.h"],
    "k_tally2_tc_pair_packed": ["k_tc2.cu", "tc_pipeline_pair.cuh", "tc_pipeline.cuh", "tc_sched.cuh",
                                "ccc_dev.cuh", "ccc_metric.cuh", "ccc_launch.h"],
    "k_tally2_tc_pair_split_packed": ["k_tc2.cu", "tc_pipeline_pair.cuh", "tc_pipeline.cuh",
                                      "tc_sched.cuh", "ccc_dev.cuh", "ccc_metric.cuh", "ccc_launch.h"],
    "k_tally2_multi_fp4": ["k_multi.cuh", "k_multi.cu", "tc_pipeline_pair.cuh", "tc_pipeline.cuh",
                           "tc_sched.cuh", "ccc_dev.cuh", "ccc_metric.cuh", "ccc_launch.h"],
    "k_tally2_multi": ["k_multi.cuh", "k_multi.cu", "tc_pipeline_pair.cuh", "tc_pipeline.cuh",
                       "tc_sched.cuh", "ccc_dev.cuh", "ccc_metric.cuh", "ccc_launch.h"],
    "k_tally2_tc": ["k_tc2.cu", "tc_pipeline.cuh", "tc_sched.cuh", "ccc_dev.cuh", "ccc_metric.cuh",
                    "ccc_launch.h"],
    "k_tally3_tc": ["k_tc3.cu", "tc_pipeline.cuh", "ccc_dev.cuh", "ccc_metric.cuh", "ccc_launch.h"],
    "k_tally3_class": ["k_tc3c.cu", "tc_pipeline_pair.cuh", "tc_pipeline.cuh", "ccc_dev.cuh",
                       "ccc_metric.cuh", "ccc_launch.h"],
    "k_tally3_class_w": ["k_tc3c.cu", "tc_pipeline_pair.cuh", "tc_pipeline.cuh", "ccc_dev.cuh",
                         "ccc_metric.cuh", "ccc_launch.h"],
}


def source_hash(kernel="k_tally2_tc_pair"):
    """SHA-256 of the device-code files of a tally kernel, identifying what an ncu capture measured."""
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES.get(kernel, []):
        h.update(name.encode())
        with open(os.path.join(ROOT, "paper_1705_08213_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_record(kernel, workload):
    """The profiles/ncu_traffic.json record of `kernel` on `workload`, or None when there is
    none or it was captured on different CUDA sources."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            rec = json.load(f).get(f"{kernel}@{workload}")
    except (OSError, ValueError):
        return None
    if not rec or rec.get("source_hash") != source_hash(kernel):
        return None
    return rec


def ncu_traffic(kernel, workload):
    """DRAM bytes per launch (per step for the 3-way class route) of `kernel` on `workload`
    from profiles/ncu_traffic.json, or None when that capture was taken on different CUDA
    sources."""
    rec = ncu_record(kernel, workload)
    if rec is None:
        return None
    return float(rec.get("dram_bytes_per_step", rec.get("dram_bytes_per_launch")))


# 64-bit AND+POPC per second: 16 32-bit POPC per SM per clock (measured: 7.5 64-bit
# AND+POPC per SM per clock in a register-only loop), 152 SMs at 2,070 MHz.
POPC64_PEAK_T = 152 * 2.070e9 * 16 / 2 / 1e12


_RATES = {}


def probe_rates(ccc, torch, dev):
    """Work per SM clock cycle of the tally kernels' execution units on this GPU, measured once
    per process with the library's rate probes (ccc_mma_rate, ccc_popc_rate): back-to-back
    M = 256 x N = 256 cta_group::2 MMAs on every SM pair, and register-only 64-bit AND+POPC."""
    if _RATES:
        return _RATES
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    _RATES["sms"] = sms
    n_mma = 8192
    for kind, name, k in ((ccc.CCC_MMA_E4M3, "e4m3", 32), (ccc.CCC_MMA_E2M1, "e2m1", 64)):
        ccc.ccc_mma_rate(kind, 256, 256, sms // 2)
        cycles, bad = ccc.ccc_mma_rate(kind, 256, n_mma, sms // 2)
        med = statistics.median(cycles)
        _RATES[name] = {"flops_per_sm_per_clock": 2.0 * 256 * 256 * k * n_mma / med / 2.0,
                        "cycles_per_mma": med / n_mma, "bad": bad}
    ccc.ccc_popc_rate(256, sms)
    cyc = statistics.median(ccc.ccc_popc_rate(4096, sms))
    _RATES["popc64_per_sm_per_clock"] = 8.0 * 1024 * 4096 / cyc
    return _RATES


def clock_normalised(achieved, per_clock, clocks, sms, what):
    """Fraction of the peak at the SM clock the kernel ran at: achieved / (work per SM per
    cycle x SMs x median SM MHz sampled during the timed region)."""
    mhz = (clocks or {}).get("sm_mhz")
    src = "median SM clock sampled during the timed region"
    if not mhz:
        mhz, src = 2070.0, "no clock samples: maximum SM clock 2,070 MHz"
    peak = per_clock * sms * mhz * 1e6 / 1e12
    return {"peak": peak, "frac": achieved / peak, "per_sm_per_clock": per_clock, "sms": sms,
            "sm_mhz": mhz, "note": f"{what} x {sms} SMs x {mhz:.0f} MHz ({src})"}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["bf16_tflops"]), float(d["hbm_gbs"]), "measured"
    except Exception:
        return 1900.0, 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling around the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []
        self.thread = None
        self.t_on = self.t_off = None

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

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def mark_on(self):
        self.t_on = time.monotonic()

    def mark_off(self):
        self.t_off = time.monotonic()

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
        lo = (self.t_on or 0) - 0.11
        hi = (self.t_off or 1e30) + 0.11
        for t, line in self.lines:
            if not (lo <= t <= hi):
                continue
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
            return {"sm_mhz": None, "sm_max_mhz": None, "samples": 0,
                    "reasons": ["no samples inside the timed region"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "power_w_max": max(pw) if pw else None, "reasons": sorted(reasons)}


def gpu_id_for(torch, dev):
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return str(dev)


def oracle_sample(geno, w, rng, n_sample):
    """One oracle call on a random sample of the workload; returns comparisons done."""
    import oracle
    n_v, n_f = w["n_v"], w["n_f"]
    if w["kind"] == 2:
        i = rng.integers(0, n_v - 1, size=n_sample)
        j = i + 1 + (rng.random(n_sample) * (n_v - 1 - i)).astype(np.int64)
        if w.get("states"):
            oracle.ccc2_multi_pairs(geno, n_f, w["states"], i, j)
        else:
            oracle.ccc2_pairs(geno, n_f, i, j)
        return n_sample * n_f
    j = rng.integers(1, n_v - 1, size=n_sample)
    i = (rng.random(n_sample) * j).astype(np.int64)
    k = j + 1 + (rng.random(n_sample) * (n_v - 1 - j)).astype(np.int64)
    oracle.ccc3_triples(geno, n_f, i, j, k)
    return n_sample * n_f


def cpu_baseline(geno, w, seconds, seed=7):
    """The oracle on host cores over random pairs (triples) of the same panel."""
    import oracle
    rng = np.random.default_rng(seed)
    n_sample = max(64, int(4e8 // w["n_f"]))
    done, calls = 0, 0
    t0 = time.perf_counter()
    while True:
        done += oracle_sample(geno, w, rng, n_sample)
        calls += 1
        el = time.perf_counter() - t0
        if el >= seconds or calls >= 200:
            break
    what = "pairs (i<j)" if w["kind"] == 2 else "triples (i<j<k)"
    return {"value": done / el, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
            "sample": f"{calls * n_sample} uniformly random {what} of the same panel, all "
                      f"{w['n_f']} individuals each, {el:.1f} s on the host cores"}


def run_reference(args, w):
    """The CPU oracle timed on this workload (rank 0 only)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    geno = make_panel(w)
    rng = np.random.default_rng(11)
    n_sample = max(64, int(6e7 // w["n_f"]))
    for _ in range(args.warmup):
        oracle_sample(geno, w, rng, n_sample)
    t0 = time.perf_counter()
    done = 0
    for _ in range(args.steps):
        done += oracle_sample(geno, w, rng, n_sample)
    el = time.perf_counter() - t0
    value = done / el
    what = "pairs" if w["kind"] == 2 else "triples"
    line = {
        "impl": "reference", "metric": w["metric"], "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64/f64", "data": "synthetic",
        "config": {"workload": w["text"], "n_v": w["n_v"], "n_f": w["n_f"],
                   "sample_per_step": f"{n_sample} random {what} x {w['n_f']} individuals"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                         "sample": f"{n_sample} uniformly random {what} per step, {args.steps} "
                                   "timed steps"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


class Runner:
    """Device buffers and one step of the chosen workload through the C ABI."""

    def __init__(self, ccc, torch, dev, w, path, geno_np, tile=0, shard=None, operand=0):
        self.ccc, self.torch, self.dev, self.w, self.path = ccc, torch, dev, w, path
        self.tile = tile
        self.operand = operand
        n_v, n_f = w["n_v"], w["n_f"]
        # Rows (2-way) or slabs (3-way) [lo, hi) of this rank; None = the whole panel.
        self.shard = shard
        self.states = w.get("states")
        self.host_geno = torch.from_numpy(geno_np if self.states else geno_np.view(np.int64))
        self.host_geno = self.host_geno.pin_memory()
        self.geno = self.host_geno.to(dev)
        op = ccc.CCC_OP_2WAY if w["kind"] == 2 else ccc.CCC_OP_3WAY
        o0 = ccc.ccc_opts_default(path=path, tile=tile, operand=operand)
        size = (ccc.ccc_multi_workspace_size(self.geno, n_f, self.states, o0) if self.states else
                ccc.ccc_workspace_size(self.geno, n_f, o0, op))
        self.ws = torch.empty(size, dtype=torch.uint8, device=dev)
        self.opts = ccc.ccc_opts_default(path=path, workspace=self.ws, tile=tile, operand=operand)
        self.filter = "threshold" in w
        if self.filter:
            self.cap = 1 << 20
            self.hits = torch.zeros(self.cap * 40, dtype=torch.uint8, device=dev)
            self.n_hits = torch.zeros(1, dtype=torch.int64, device=dev)
            self.out_bytes = 8
        else:
            lo, hi = shard if shard is not None else (0, n_v)
            rows = ccc.ccc2_rows_count(n_v, lo, hi) if w["kind"] == 2 else ccc.ccc3_count(n_v, lo, hi)
            rows = max(rows, 1)
            width = (self.states ** 2 if self.states else 4) if w["kind"] == 2 else 8
            self.tally = torch.empty((rows, width), dtype=torch.int32, device=dev)
            self.out = torch.empty((rows, width), dtype=torch.float32, device=dev)
            self.out_bytes = rows * width * 8

    def step(self, stream):
        ccc, w = self.ccc, self.w
        if self.filter:
            ccc.ccc2_filter(self.geno, w["n_f"], w["threshold"], self.hits, self.cap, self.n_hits,
                            self.opts, stream)
        elif self.shard is not None and w["kind"] == 2:
            lo, hi = self.shard
            if self.states:
                ccc.ccc2_multi_tally_metric_rows(self.geno, w["n_f"], self.states, lo, hi, self.tally,
                                                 self.out, self.opts, stream)
            else:
                ccc.ccc2_tally_metric_rows(self.geno, w["n_f"], lo, hi, self.tally, self.out,
                                           self.opts, stream)
        elif self.states:
            ccc.ccc2_multi_tally_metric(self.geno, w["n_f"], self.states, self.tally, self.out,
                                        self.opts, stream)
        elif w["kind"] == 2:
            ccc.ccc2_tally_metric(self.geno, w["n_f"], self.tally, self.out, self.opts, stream)
        else:
            lo, hi = self.shard if self.shard is not None else (0, w["n_v"])
            ccc.ccc3_tally_metric(self.geno, w["n_f"], lo, hi, self.tally, self.out, self.opts,
                                  stream)

    def e2e(self, stream, steps, phases=8, mode="auto"):
        """Host panel -> device, the step, results -> pinned host memory, per step.

        stream (2-way): ccc2_stream, whose phases copy finished results to the
        host while later phases compute.  direct: the same call with the output
        arrays in pinned host memory, so the kernels' epilogues store the results
        over the host link themselves.  copy: the call, then one copy per output.
        Filter: the hit count comes back (the hits stay on the device).
        """
        torch, ccc, w = self.torch, self.ccc, self.w
        if mode == "auto":
            # Phases split the rows; a panel of few tiles is better served by one
            # K-split call and a copy of its small output.
            mode = "stream" if not (self.filter or w.get("split_compare")) else "copy"
        self.e2e_mode = mode if not self.filter else "copy"
        streamed = mode == "stream" and not self.filter
        direct = mode == "direct" and not self.filter
        if direct:
            host = [torch.empty(self.tally.shape, dtype=torch.int32, pin_memory=True),
                    torch.empty(self.out.shape, dtype=torch.float32, pin_memory=True)]
            dev = []
            self.tally, self.out = host  # the kernels write these host arrays directly
        elif self.filter:
            host = [torch.empty(1, dtype=torch.int64, pin_memory=True)]
            dev = [self.n_hits]
        elif streamed:
            host = [torch.empty(self.tally.shape, dtype=torch.int32, pin_memory=True),
                    torch.empty(self.out.shape, dtype=torch.float32, pin_memory=True)]
            dev = []
            del self.tally, self.out, self.ws
            o0 = ccc.ccc_opts_default(path=self.path, tile=self.tile, operand=self.operand)
            if self.states:
                size = ccc.ccc2_multi_stream_workspace_size(self.geno, w["n_f"], self.states, phases, o0)
            else:
                size = (ccc.ccc2_stream_workspace_size if w["kind"] == 2 else
                        ccc.ccc3_stream_workspace_size)(self.geno, w["n_f"], phases, o0)
            self.ws_stream = torch.empty(size, dtype=torch.uint8, device=self.dev)
            self.opts = ccc.ccc_opts_default(path=self.path, workspace=self.ws_stream,
                                             tile=self.tile, operand=self.operand)
        else:
            host = [torch.empty(self.tally.shape, dtype=torch.int32, pin_memory=True),
                    torch.empty(self.out.shape, dtype=torch.float32, pin_memory=True)]
            dev = [self.tally, self.out]

        def one():
            self.geno.copy_(self.host_geno, non_blocking=True)
            if streamed and self.states:
                ccc.ccc2_multi_stream(self.geno, w["n_f"], self.states, phases, host[0], host[1],
                                      self.opts, stream)
            elif streamed:
                (ccc.ccc2_stream if w["kind"] == 2 else ccc.ccc3_stream)(
                    self.geno, w["n_f"], phases, host[0], host[1], self.opts, stream)
            else:
                self.step(stream)
            for h, d in zip(host, dev):
                h.copy_(d, non_blocking=True)

        one()
        torch.cuda.synchronize(self.dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            one()
        e1.record(stream)
        torch.cuda.synchronize(self.dev)
        if self.filter:
            self.hit_count = int(host[0].item())
        return (e0.elapsed_time(e1) / steps,
                self.host_geno.numel() * self.host_geno.element_size(), self.out_bytes)


def run_batched(args, w, ccc, torch, dev, stream, rank, world, pg):
    """The batched workload: autotune, capture one CUDA graph, replay it."""
    shapes = w["shapes"]
    genos_np = [synth.panel_hwe(v, f, seed=w["seed"] + 1000 * rank, panel=k,
                                p_missing=w["p_missing"]) for k, (v, f) in enumerate(shapes)]
    genos = [torch.from_numpy(g.view(np.int64)).to(dev) for g in genos_np]
    n_fs = [f for _, f in shapes]
    tallies = [torch.empty((ccc.ccc2_count(v), 4), dtype=torch.int32, device=dev) for v, _ in shapes]
    cccs = [torch.empty((ccc.ccc2_count(v), 4), dtype=torch.float32, device=dev) for v, _ in shapes]
    opts = ccc.ccc_opts_default()
    ws = torch.empty(ccc.ccc2_batched_workspace_size(genos, n_fs, opts), dtype=torch.uint8,
                     device=dev)
    opts = ccc.ccc_opts_default(workspace=ws)
    cmp_per_step = comparisons(w)
    with torch.cuda.stream(stream):
        group, order = ccc.ccc2_batched_tune(genos, n_fs, tallies, cccs, opts, stream)
        for _ in range(max(args.warmup, 1)):
            ccc.ccc2_batched(genos, n_fs, tallies, cccs, opts, stream)
    torch.cuda.synchronize(dev)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        ccc.ccc2_batched(genos, n_fs, tallies, cccs, opts, stream)
    graph.replay()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(gpu_id_for(torch, dev))
    sampler.start()
    time.sleep(0.5)
    launches0 = ccc.ccc_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler.mark_on()
    e0.record(stream)
    for _ in range(args.steps):
        graph.replay()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    sampler.mark_off()
    ms_graph = e0.elapsed_time(e1) / args.steps
    # Same steps through the C ABI directly, with the library's kernel events.
    ccc.ccc_timing_enable(True)
    ccc.ccc_timing_read()
    d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    d0.record(stream)
    for _ in range(args.steps):
        ccc.ccc2_batched(genos, n_fs, tallies, cccs, opts, stream)
    d1.record(stream)
    torch.cuda.synchronize(dev)
    kernel_ms, kernel_n = ccc.ccc_timing_read()
    ccc.ccc_timing_enable(False)
    direct_launches = ccc.ccc_launch_count() - launches0
    ms_direct = d0.elapsed_time(d1) / args.steps
    clocks = sampler.stop()
    # The same step with every panel's tiles in the one persistent tally launch
    # (no panel launched on its own: ccc_opts.solo < 0), graph-captured as above.
    o1 = ccc.ccc_opts_default(workspace=ws)
    for name, _ in type(opts)._fields_:
        setattr(o1, name, getattr(opts, name))
    o1.solo = -1
    with torch.cuda.stream(stream):
        ccc.ccc2_batched(genos, n_fs, tallies, cccs, o1, stream)
    torch.cuda.synchronize(dev)
    graph1 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph1, stream=stream):
        ccc.ccc2_batched(genos, n_fs, tallies, cccs, o1, stream)
    graph1.replay()
    torch.cuda.synchronize(dev)
    launches1 = ccc.ccc_launch_count()
    with torch.cuda.stream(stream):
        ccc.ccc2_batched(genos, n_fs, tallies, cccs, o1, stream)
    launches1 = ccc.ccc_launch_count() - launches1
    torch.cuda.synchronize(dev)
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    for _ in range(args.steps):
        graph1.replay()
    g1.record(stream)
    torch.cuda.synchronize(dev)
    ms_one = g0.elapsed_time(g1) / args.steps
    del graph1
    # 64 sequential single-panel calls, one shared workspace.
    o0 = ccc.ccc_opts_default()
    wss = torch.empty(max(ccc.ccc_workspace_size(g, f, o0, ccc.CCC_OP_2WAY)
                          for g, f in zip(genos, n_fs)), dtype=torch.uint8, device=dev)
    os_ = ccc.ccc_opts_default(workspace=wss)
    for g, f, t, c in zip(genos, n_fs, tallies, cccs):
        ccc.ccc2_tally_metric(g, f, t, c, os_, stream)
    torch.cuda.synchronize(dev)
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nseq = max(1, min(args.steps, 3))
    s0.record(stream)
    for _ in range(nseq):
        for g, f, t, c in zip(genos, n_fs, tallies, cccs):
            ccc.ccc2_tally_metric(g, f, t, c, os_, stream)
    s1.record(stream)
    torch.cuda.synchronize(dev)
    ms_seq = s0.elapsed_time(s1) / nseq
    # End to end through the same C ABI call: every panel copied from pinned
    # host memory, the batched call, every tally and CCC array copied back to
    # pinned host memory, per step.
    e2e = None
    if not args.skip_e2e:
        host_in = [torch.from_numpy(g.view(np.int64)).pin_memory() for g in genos_np]
        host_out = [torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in tallies + cccs]
        bi = sum(h.numel() * h.element_size() for h in host_in)
        bo = sum(h.numel() * h.element_size() for h in host_out)

        def e2e_step():
            with torch.cuda.stream(stream):
                for d, h in zip(genos, host_in):
                    d.copy_(h, non_blocking=True)
                ccc.ccc2_batched(genos, n_fs, tallies, cccs, opts, stream)
                for h, d in zip(host_out, tallies + cccs):
                    h.copy_(d, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize(dev)
        x0, x1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        nx = max(1, min(args.steps, 5))
        x0.record(stream)
        for _ in range(nx):
            e2e_step()
        x1.record(stream)
        torch.cuda.synchronize(dev)
        ms_e2e = x0.elapsed_time(x1) / nx
        e2e = {"value": cmp_per_step / (ms_e2e * 1e-3), "unit": UNIT, "h2d_bytes_per_step": bi,
               "d2h_bytes_per_step": bo, "ms_per_step": ms_e2e, "steps": nx, "mode": "copy",
               "note": "pinned host panels -> device, ccc2_batched, every output -> pinned host "
                       "memory (one stream, no overlap)"}
        del host_in, host_out
    bf16_peak, _, peak_src = measured_peaks()
    kstep = kernel_ms / args.steps
    achieved = 8.0 * cmp_per_step / (kstep * 1e-3) / 1e12
    # The tuned schedule: SM-pair tiles run e2m1 operands (automatic), one-SM tiles e4m3.
    fp4 = opts.tile != 1
    ratio = 6.0 if fp4 else 2.0
    peak = ratio * bf16_peak
    kind = "e2m1" if fp4 else "e4m3"
    result = {
        "metric": w["metric"], "value": cmp_per_step / (ms_graph * 1e-3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_graph,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": ("e2m1 operands (kind::mxf4, unit scale factors), fp32 accumulate" if fp4 else
                  "e4m3 operands, fp32 accumulate"), "data": "synthetic",
        "config": {"workload": w["text"], "panels": len(shapes), "comparisons": cmp_per_step,
                   "schedule": {"group": group, "order": order, "tile": int(opts.tile),
                                "split": int(opts.split), "solo": int(opts.solo),
                                "tuned_by": "ccc2_batched_tune"},
                   "l2": "inputs larger than L2"},
        "gpu_launches": int(direct_launches // args.steps),
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None,
                     "kernel": "k_tally2_tc_pair_batched_fp4" if fp4 else "k_tally2_tc_batched",
                     "kernel_ms_per_step": kstep, "kernel_launches": kernel_n,
                     "note": "kernel time: summed duration of the tally launches (the shared "
                             "persistent launch and any solo launches), from the library's events "
                             "over the same number of direct (not graph) steps right after the "
                             "graph replays",
                     "peak_note": f"{kind} dense = {ratio:.0f} x {peak_src} bf16 burst "
                                  f"{bf16_peak:.0f} (nominal dense ratio)"},
        "clocks": clocks,
        "direct_calls": {"ms_per_step": ms_direct, "value": cmp_per_step / (ms_direct * 1e-3)},
        "one_persistent_launch": {"ms_per_step": ms_one, "value": cmp_per_step / (ms_one * 1e-3),
                                  "gpu_launches": int(launches1),
                                  "note": "ccc_opts.solo = -1: all 64 panels' tiles (and their K "
                                          "split units) in one persistent tally launch, the "
                                          "operand unpacks on a side stream; graph replay"},
        "sequential_64_calls": {"ms_per_step": ms_seq, "value": cmp_per_step / (ms_seq * 1e-3),
                                "batched_speedup": ms_seq / ms_graph},
    }
    rates = probe_rates(ccc, torch, dev)
    result["roofline"]["clock_normalised"] = clock_normalised(
        achieved, rates[kind]["flops_per_sm_per_clock"], clocks, rates["sms"],
        f"{kind} flops per SM per clock of the ccc_mma_rate probe")
    if e2e is not None:
        result["e2e"] = e2e
    if not args.skip_cpu:
        k = int(np.argmax([v for v, _ in shapes]))
        wk = dict(kind=2, n_v=shapes[k][0], n_f=shapes[k][1])
        result["cpu_baseline"] = cpu_baseline(genos_np[k], wk, args.cpu_seconds)
        result["cpu_baseline"]["sample"] += f" (panel {k}, the largest)"
    return result


def main():
    args, w = parse()
    if args.impl == "reference":
        if args.workload == "batched":
            k = int(np.argmax([v for v, _ in w["shapes"]]))
            w = dict(w, n_v=w["shapes"][k][0], n_f=w["shapes"][k][1], seed=w["seed"])
        return run_reference(args, w)

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

    result = run_workload(args, w, ccc, torch, dev, rank, world, local, pg)
    if (rank == 0 and world == 1 and args.workload == "2way" and not w.get("reduced")
            and not args.no_sub and args.path == "tc" and args.tile == 0):
        # The other at-scale workloads, each timed in full as its own record.
        result["workloads"] = {}
        for name, (steps, warmup) in SUB_WORKLOADS.items():
            torch.cuda.synchronize(dev)
            torch.cuda.empty_cache()
            sub = argparse.Namespace(**vars(args))
            sub.workload, sub.steps, sub.warmup = name, steps, warmup
            sub.cpu_seconds = SUB_CPU_SECONDS
            sub.scaling = "weak"
            try:
                rec = run_workload(sub, workload_dict(name), ccc, torch, dev, rank, world, local,
                                   pg)
            except Exception as e:  # recorded, so one failing workload does not hide the others
                rec = {"error": f"{type(e).__name__}: {e}"}
            result["workloads"][name] = rec
        torch.cuda.empty_cache()
    if rank == 0:
        print(json.dumps(result), flush=True)
    if pg is not None:
        pg.barrier()
        pg.destroy_process_group()
    return 0


def run_workload(args, w, ccc, torch, dev, rank, world, local, pg):
    """One workload's record (the bench line's keys) on this rank."""
    if args.workload == "batched":
        if world > 1:
            raise SystemExit("the batched workload runs on one GPU")
        side = torch.cuda.Stream(dev)  # CUDA graphs are captured on a non-default stream
        with torch.cuda.stream(side):
            return run_batched(args, w, ccc, torch, dev, side, rank, world, pg)
    path = ccc.CCC_PATH_TC if args.path == "tc" else ccc.CCC_PATH_POPC
    cmp_per_step = comparisons(w)
    strong = args.scaling == "strong"
    shard_range = None
    cmp_rank = cmp_per_step  # comparisons this rank computes per step
    if strong:
        if "threshold" in w:
            raise SystemExit("--scaling strong covers the 2way, 3way, small and multi workloads")
        from paper_1705_08213_gb300 import shard as sh
        n_v = w["n_v"]
        if w["kind"] == 3:
            shard_range = sh.slab_range(n_v, world, rank)
            cmp_rank = ccc.ccc3_count(n_v, *shard_range) * w["n_f"]
        else:
            shard_range = (sh.multi_pair_range(n_v, w["states"], world, rank) if w.get("states")
                           else sh.pair_range(n_v, world, rank))
            cmp_rank = ccc.ccc2_rows_count(n_v, *shard_range) * w["n_f"]
    geno_np = make_panel(w, 0 if strong else rank)
    operand = {"auto": ccc.CCC_OPERAND_AUTO, "e4m3": ccc.CCC_OPERAND_E4M3,
               "e2m1": ccc.CCC_OPERAND_E2M1}[args.operand]
    # The library's automatic choice: e2m1 on the 2-way SM-pair tiles, for markers with at
    # most 8 states (no K split at these sizes), and on the 3-way genotype-class route's wide
    # tiles (n_f <= 16,383).
    fp4 = (path == ccc.CCC_PATH_TC and operand != ccc.CCC_OPERAND_E4M3 and
           ((w["kind"] == 2 and not w.get("states") and args.tile in (0, 2)) or
            (w["kind"] == 2 and w.get("states") and w["states"] <= 8 and args.tile in (0, 2)) or
            (w["kind"] == 3 and args.tile in (0, 3) and w["n_f"] <= 16383)))
    run = Runner(ccc, torch, dev, w, path, geno_np, tile=args.tile,
                 shard=shard_range if strong else None, operand=operand)
    stream = torch.cuda.current_stream(dev)

    sampler = ClockSampler(gpu_id_for(torch, dev)) if local == 0 else None
    if sampler:
        sampler.start()  # its start-up overlaps the warm-up, never the timed region
    for _ in range(max(args.warmup, 0)):
        run.step(stream)
    torch.cuda.synchronize(dev)
    if ccc.ccc_status(run.opts) != ccc.CCC_OK:
        raise RuntimeError("device status not ok after warm-up")

    # ---------------------------------------------------------------- timed region
    if pg is not None:
        pg.barrier()
    torch.cuda.synchronize(dev)
    ccc.ccc_timing_enable(True)
    ccc.ccc_timing_read()
    launches0 = ccc.ccc_launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    # Inputs that fit the 129 MB L2: a 256 MB write before every timed step,
    # outside that step's own events, so that no step finds its inputs in L2.
    flush = l2_flush_buffer(w, torch, dev)
    step_events = []
    if sampler:
        sampler.mark_on()
    ev0.record(stream)
    for _ in range(args.steps):
        if flush is not None:
            flush.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            run.step(stream)
            b.record(stream)
            step_events.append((a, b))
        else:
            run.step(stream)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    if sampler:
        sampler.mark_off()
    if pg is not None:
        pg.barrier()
    launches = ccc.ccc_launch_count() - launches0
    kernel_ms, kernel_n = ccc.ccc_timing_read()
    ccc.ccc_timing_enable(False)
    clocks = sampler.stop() if sampler else None
    ms_per_step = (sum(a.elapsed_time(b) for a, b in step_events) if step_events else
                   ev0.elapsed_time(ev1)) / args.steps
    del flush
    if pg is not None:
        t = torch.tensor([ms_per_step], device=dev)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        ms_per_step = float(t.item())
    if ccc.ccc_status(run.opts) != ccc.CCC_OK:
        raise RuntimeError("device status not ok after the timed region")
    value = (1 if strong else world) * cmp_per_step / (ms_per_step * 1e-3)
    # The launch-bound small panel: the same step captured once in a CUDA graph
    # and replayed, so that the host's per-call work leaves the loop.
    graph_rec = None
    if args.workload == "small" and not strong:
        side = torch.cuda.Stream(dev)  # graphs are captured on a non-default stream
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            run.step(side)
            torch.cuda.synchronize(dev)
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=side):
                run.step(side)
            graph.replay()
            torch.cuda.synchronize(dev)
            gr0, gr1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            gr0.record(side)
            for _ in range(args.steps):
                graph.replay()
            gr1.record(side)
            torch.cuda.synchronize(dev)
        ms_graph = gr0.elapsed_time(gr1) / args.steps
        del graph
        graph_rec = {"ms_per_step": ms_graph, "value": cmp_per_step / (ms_graph * 1e-3),
                     "note": "the step captured once in a CUDA graph and replayed back to back "
                             "(the C ABI call's host checks and launches leave the timed loop; "
                             "no L2 flush between replays)"}

    # Roofline of the dominant kernel (the tally kernel), from its own events:
    # summed duration of its launches in the timed region / steps.
    bf16_peak, hbm_peak, peak_src = measured_peaks()
    kernel_step_ms = kernel_ms / args.steps
    packed = "_packed" if args.tile == 3 else "_fp4" if fp4 else ""
    if w["kind"] == 3:
        packed = ""
    kname = {(2, True): ("k_tally2_multi" + ("_fp4" if fp4 else "") if w.get("states") else
                         "k_tally2_tc_pair_split" + packed if w.get("split_compare") else
                         "k_tally2_tc_pair" + packed + ("w" if fp4 and w.get("threshold") is not None
                                                        else "")
                         if args.tile != 1 else "k_tally2_tc"),
             (3, True): {1: "k_tally3_tc", 2: "k_tally3_fused"}.get(
                 args.tile, "k_tally3_class_w" if w["n_f"] <= 16383 else "k_tally3_class"),
             (2, False): "k_tally2_popc", (3, False): "k_tally3_popc"}[(w["kind"],
                                                                       path == ccc.CCC_PATH_TC)]
    if path == ccc.CCC_PATH_TC:
        # Credited work: 4 MAC (8 flops) per 2-way comparison and 8 MAC (16 flops) per
        # 3-way comparison, the tensor work of the masked-operand formulation; padding
        # and diagonal-tile waste are not credited.  The genotype-class 3-way route
        # executes 4 MAC per comparison (plus the product over the individuals with v_j
        # missing), so its credited rate reads twice its executed one.
        per_cmp = 8.0 if w["kind"] == 2 else 16.0
        if w.get("states"):
            per_cmp = 2.0 * w["states"] ** 2  # s^2 MAC per comparison
        flops = per_cmp * cmp_rank
        achieved = flops / (kernel_step_ms * 1e-3) / 1e12
        # The peak of the kernel's own operand type: the measured bf16 burst times the nominal
        # dense ratio (e4m3 4.5 / 2.25 PFLOP/s; e2m1 13.5 / 2.25).
        ratio = 6.0 if fp4 else 2.0
        peak = ratio * bf16_peak
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": ncu_traffic(kname, args.workload)
                if (args.n_v is None and args.n_f is None) else None, "kernel": kname,
                "kernel_ms_per_step": kernel_step_ms, "kernel_launches": kernel_n,
                "per_unit": f"{per_cmp:.0f} flops per comparison",
                "peak_note": (f"{'e2m1' if fp4 else 'e4m3'} dense peak = {ratio:.0f} x {peak_src} "
                              f"bf16 burst {bf16_peak:.0f} TFLOP/s (nominal dense ratio; "
                              "kind::i8 is not available on sm_103a)")}
        rates = probe_rates(ccc, torch, dev)
        kind = "e2m1" if fp4 else "e4m3"
        roof["clock_normalised"] = clock_normalised(
            achieved, rates[kind]["flops_per_sm_per_clock"], clocks, rates["sms"],
            f"{kind} flops per SM per clock of the ccc_mma_rate probe")
        if kname.startswith("k_tally3_class"):
            ex = 8.0 * cmp_rank / (kernel_step_ms * 1e-3) / 1e12
            roof["executed"] = {"per_unit": "8 flops per comparison (T product; the D product "
                                            "over individuals with v_j missing not counted)",
                                "achieved": ex, "frac": ex / peak,
                                "frac_clock_normalised": ex / roof["clock_normalised"]["peak"]}
            if fp4:
                # The same executed rate against the e4m3 operand peak (2 x the bf16
                # burst), the denominator the class route was first read against.
                e4m3_peak = 2.0 * bf16_peak
                roof["executed"]["frac_of_e4m3_peak"] = ex / e4m3_peak
                roof["executed"]["e4m3_peak"] = e4m3_peak
    else:
        per = 8.0 / 64.0 if w["kind"] == 2 else 24.0 / 64.0
        achieved = per * cmp_rank / (kernel_step_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": POPC64_PEAK_T, "unit": "T popc64/s",
                "frac": achieved / POPC64_PEAK_T, "traffic": None, "kernel": kname,
                "kernel_ms_per_step": kernel_step_ms, "kernel_launches": kernel_n,
                "per_unit": f"{per * 64:.0f} 64-bit POPC per 64 comparisons",
                "peak_note": "16 32-bit POPC per SM per clock x 152 SMs x 2,070 MHz / 2"}
        rates = probe_rates(ccc, torch, dev)
        roof["clock_normalised"] = clock_normalised(
            achieved, rates["popc64_per_sm_per_clock"], clocks, rates["sms"],
            "64-bit AND+POPC per SM per clock of the ccc_popc_rate probe")

    # Output bytes of one step: int32 tallies + fp32 CCC values (the hit list when thresholded).
    if w.get("threshold") is not None:
        out_bytes = 0.0
    elif w["kind"] == 3:
        out_bytes = 64.0 * cmp_rank / w["n_f"]
    else:
        out_bytes = 8.0 * (w.get("states") or 2) ** 2 * cmp_rank / w["n_f"]
    # The tally kernel against the HBM roofline as well (context; the bound above is the
    # tensor pipe): algorithmic bytes = operand rows read once + outputs written once (the
    # capture's own figure where one matches these sources), and the captured DRAM traffic.
    if path == ccc.CCC_PATH_TC and not strong:
        full = args.n_v is None and args.n_f is None
        rec = ncu_record(kname, args.workload) if full else None
        alg = None
        if rec is not None:
            alg = rec.get("algorithmic_bytes_per_step", rec.get("algorithmic_bytes_per_launch"))
        if alg is None:
            rows = (w.get("states") or 2) * w["n_v"] if w["kind"] == 2 else 0
            alg = out_bytes + rows * w["n_f"] * (0.5 if fp4 else 1.0)
        ks = kernel_step_ms * 1e-3
        traffic = roof.get("traffic")
        roof["hbm_context"] = {
            "unit": "GB/s", "peak": hbm_peak, "peak_note": f"{peak_src} copy bandwidth",
            "algorithmic_bytes": float(alg), "achieved": alg / ks / 1e9,
            "frac": alg / ks / 1e9 / hbm_peak,
            "dram_achieved": traffic / ks / 1e9 if traffic else None,
            "dram_frac": traffic / ks / 1e9 / hbm_peak if traffic else None}
    result = {
        "metric": w["metric"], "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": args.scaling, "vs_baseline": None,
        "dtype": ("e2m1 operands (kind::mxf4, unit scale factors), fp32 accumulate" if fp4 else
                  "e4m3 operands, fp32 accumulate" if path == ccc.CCC_PATH_TC else "u64 bit planes"),
        "data": "synthetic",
        "config": {"workload": w["text"], "n_v": w["n_v"], "n_f": w["n_f"], "path": args.path,
                   "tile": ({0: "automatic (256x256 on an SM pair)", 1: "128x256 on one SM",
                             2: "256x256 on an SM pair",
                             3: "256x256 on an SM pair, 2-bit codes expanded in shared memory"}
                            if w["kind"] == 2 else
                            {0: "automatic (genotype classes of v_j on SM pairs)",
                             1: "masked operands L_j formed in HBM", 2: "L_j formed in shared memory",
                             3: "genotype classes of v_j on SM pairs"})[args.tile],
                   "parallelism": ((f"one panel over {world} GPUs, rank 0 computing "
                                    f"{'slabs' if w['kind'] == 3 else 'rows'} {list(shard_range)}")
                                   if strong and world > 1 else
                                   f"{world} independent panels (one per GPU)" if world > 1
                                   else "1 GPU"),
                   "l2": ("inputs larger than L2 (operand matrix and outputs exceed the 129 MB L2)"
                          if not inputs_fit_l2(w) else
                          "inputs fit the 129 MB L2: flushed before every timed step by a 256 MB "
                          "write outside the step's events (ms_per_step sums the steps' own "
                          f"events; each step also writes {out_bytes / 1e9:.3g} GB of outputs)")},
        "gpu_launches": int(launches),
        "roofline": roof,
        "clocks": clocks,
    }
    if graph_rec is not None:
        result["graph_replay"] = graph_rec

    if w.get("split_compare") and rank == 0:
        # The same call with the K split turned off (ccc_opts.split = 1).
        run.opts.split = 1
        run.step(stream)
        torch.cuda.synchronize(dev)
        u0 = torch.cuda.Event(enable_timing=True)
        u1 = torch.cuda.Event(enable_timing=True)
        u0.record(stream)
        for _ in range(3):
            run.step(stream)
        u1.record(stream)
        torch.cuda.synchronize(dev)
        ums = u0.elapsed_time(u1) / 3
        run.opts.split = 0
        result["unsplit"] = {"value": cmp_per_step / (ums * 1e-3), "unit": UNIT, "ms_per_step": ums,
                             "split_speedup": ums / ms_per_step,
                             "note": "ccc_opts.split = 1: one K part per tile"}

    if not args.skip_e2e and rank == 0 and not (strong and world > 1):
        e2e_ms, bi, bo = run.e2e(stream, max(1, min(args.steps, 5)), mode=args.e2e_mode)
        result["e2e"] = {"value": cmp_per_step / (e2e_ms * 1e-3), "unit": UNIT,
                         "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo, "ms_per_step": e2e_ms,
                         "mode": run.e2e_mode,
                         "note": {"stream": "pinned host panel -> device, "
                                            + ("ccc2_multi_stream" if w.get("states") else
                                               f"ccc{w['kind']}_stream")
                                            + " (8 phases: results of each phase copied to pinned "
                                              "host memory while the next computes)",
                                  "direct": "pinned host panel -> device, the same C ABI call with "
                                            "its output arrays in pinned host memory (the kernel "
                                            "epilogues store over the host link)",
                                  "copy": "pinned host panel -> device, the same C ABI call, "
                                          "results -> pinned host memory"}[run.e2e_mode]}
        if run.filter:
            result["config"]["hits_per_step"] = run.hit_count

    if fp4 and rank == 0 and not (strong and world > 1):
        # The same call with e4m3 operands (ccc_opts.operand = E4M3), kernel time included.
        for name in ("ws", "ws_stream"):
            if hasattr(run, name):
                delattr(run, name)
        if not run.filter and not hasattr(run, "tally"):
            lo, hi = run.shard if run.shard is not None else (0, w["n_v"])
            rows = (ccc.ccc2_rows_count(w["n_v"], lo, hi) if w["kind"] == 2 else
                    ccc.ccc3_count(w["n_v"], lo, hi))
            width = ((w["states"] ** 2 if w.get("states") else 4) if w["kind"] == 2 else 8)
            run.tally = torch.empty((rows, width), dtype=torch.int32, device=dev)
            run.out = torch.empty((rows, width), dtype=torch.float32, device=dev)
        o8 = ccc.ccc_opts_default(operand=ccc.CCC_OPERAND_E4M3)
        op8 = ccc.CCC_OP_2WAY if w["kind"] == 2 else ccc.CCC_OP_3WAY
        size8 = (ccc.ccc_multi_workspace_size(run.geno, w["n_f"], w["states"], o8)
                 if w.get("states") else ccc.ccc_workspace_size(run.geno, w["n_f"], o8, op8))
        ws8 = torch.empty(size8, dtype=torch.uint8, device=dev)
        run.opts = ccc.ccc_opts_default(operand=ccc.CCC_OPERAND_E4M3, workspace=ws8)
        run.step(stream)
        torch.cuda.synchronize(dev)
        n8 = max(1, min(args.steps, 10 if w["kind"] == 2 else 4))
        ccc.ccc_timing_enable(True)
        ccc.ccc_timing_read()
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        q0.record(stream)
        for _ in range(n8):
            run.step(stream)
        q1.record(stream)
        torch.cuda.synchronize(dev)
        k8, _ = ccc.ccc_timing_read()
        ccc.ccc_timing_enable(False)
        ms8 = q0.elapsed_time(q1) / n8
        result["e4m3_path"] = {"value": cmp_per_step / (ms8 * 1e-3), "unit": UNIT,
                               "ms_per_step": ms8, "kernel_ms_per_step": k8 / n8,
                               "fp4_speedup": ms8 / ms_per_step,
                               "kernel_fp4_speedup": (k8 / n8) / kernel_step_ms,
                               "note": "the same step with e4m3 count operands (kind::f8f6f4)"}
        del ws8

    if (not args.skip_popc and rank == 0 and path == ccc.CCC_PATH_TC and w["kind"] == 2
            and not run.filter and not w.get("states")):
        for name in ("ws", "ws_stream"):
            if hasattr(run, name):
                delattr(run, name)
        if not hasattr(run, "tally"):
            rows = ccc.ccc2_count(w["n_v"])
            run.tally = torch.empty((rows, 4), dtype=torch.int32, device=dev)
            run.out = torch.empty((rows, 4), dtype=torch.float32, device=dev)
        o0 = ccc.ccc_opts_default(path=ccc.CCC_PATH_POPC)
        wsp = torch.empty(ccc.ccc_workspace_size(run.geno, w["n_f"], o0, ccc.CCC_OP_2WAY),
                          dtype=torch.uint8, device=dev)
        run.opts = ccc.ccc_opts_default(path=ccc.CCC_PATH_POPC, workspace=wsp)
        run.step(stream)
        torch.cuda.synchronize(dev)
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        nps = 2
        p0.record(stream)
        for _ in range(nps):
            run.step(stream)
        p1.record(stream)
        torch.cuda.synchronize(dev)
        pms = p0.elapsed_time(p1) / nps
        popc_t = 8.0 / 64.0 * cmp_per_step / (pms * 1e-3) / 1e12
        result["popc_path"] = {"value": cmp_per_step / (pms * 1e-3), "unit": UNIT,
                               "ms_per_step": pms, "tc_speedup": pms / ms_per_step,
                               "alu_frac": popc_t / POPC64_PEAK_T,
                               "alu_note": "8 64-bit POPC per 64 comparisons against "
                                           f"{POPC64_PEAK_T:.2f} T/s (16 POPC per SM per clock)"}

    if not args.skip_cpu and rank == 0 and world == 1:
        result["cpu_baseline"] = cpu_baseline(geno_np, w, args.cpu_seconds)

    return result


if __name__ == "__main__":
    sys.exit(main())
