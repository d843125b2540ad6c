#!/usr/bin/env python3
"""Throughput benchmark: jammed RSA samples per second on one GB300.

Workload (default): L = 1024 periodic lattice, k = 32, 1000 samples with
seeds 1..1000 per step (per rank under torchrun; rank r uses seeds
r*1000 + 1 ..).  One step runs the whole path for the batch: the parallel
greedy rounds to jamming (n_j), the contact graph, and the first-wrap
bisection (n_c).  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

`--impl reference` times the CPU oracle (a plain sequential scan plus
union-find in C) on the host cores, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    "L1024_k32_x1000": dict(L=1024, k=32, n=1000),
    "L64_k4_x100": dict(L=64, k=4, n=100),
    # small cases for ncu captures (a few GB on the device)
    "L1024_k32_x64": dict(L=1024, k=32, n=64),
    "L8192_k512_x2": dict(L=8192, k=512, n=2),
    # large k held on the device: 8 samples of L = 32768 (1 G cells each)
    "L32768_k4096_x8": dict(L=32768, k=4096, n=8),
}
METRIC = "jammed samples/s (n_j and n_c per sample, bit-exact to the oracle)"
# Algorithmic work of the round kernels.  Byte-type kernels (the general
# line path): bytes per lattice cell per launch -- the cell-minimum passes
# read occupancy (1 B) and write or read-modify-write the 8-byte cell
# minimum, the acceptance passes read it.
BYTES_PER_CELL = {"k_row_cmin": 9, "k_col_cmin": 17, "k_row_accept": 8, "k_col_accept": 8,
                  # long-k line path: window minima write the 8-byte minimum of
                  # one orientation and read occupancy bits; the combine reads
                  # both minima and writes two 2-byte argmin codes; acceptance
                  # reads one code per cell and occupancy bits
                  "k_line_cmin_h": 8.125, "k_line_cmin_v": 8.125, "k_line_codes": 20,
                  "k_line_accept_h": 2.125, "k_line_accept_v": 2.125}
# Integer-ALU kernels (the 32x32 tile path), counted in 32-bit lane
# operations: a 64-bit minimum is 4 ops (two compares, two selects) plus 1
# when the argmin is tracked, a width-k window minimum by van Herk /
# Gil-Werman is 3 minima per cell, a liveness test of a candidate's k cells
# is 4 ops (shift, mask, compare of a 64-bit word), a splitmix64 priority is
# 20 ops (64-bit add 2, three 64-bit xor-shifts at 4, two 64-bit constant
# multiplies at 3).
OPS_PER_KEY = 20
OPS_PER_CELL = {
    # horizontal and vertical argmin window minima, their combination into a
    # one-byte code (min + select), two liveness tests
    "k_tile_cmin": 2 * 3 * 5 + 6 + 2 * 4,
    # per direction: "code is the start value" and "next code is this + 1"
    # (two byte compares and an add); keys only for accepted candidates
    "k_tile_accept": 2 * 3,
}
# long-k path: work counter holding each kernel's processed cells, and the
# share of it that kernel did (the two acceptance passes share one counter)
LINE_WORK = {"k_line_cmin_h": (0, 1.0), "k_line_cmin_v": (1, 1.0), "k_line_accept_h": (2, 0.5),
             "k_line_accept_v": (2, 0.5), "k_line_codes": (3, 1.0)}
TILE_WORK = {"k_tile_cmin": ("cmin_cells", "cmin_keys"),
             "k_tile_accept": ("accept_cells", "accept_keys")}
ALU_LANES_PER_SM = 128  # 4 schedulers x 32 lanes, one integer op per lane per clock


# The source file that holds each kernel: a DRAM-traffic figure measured by
# ncu is used only while that file is unchanged.
KERNEL_FILE = {"k_tile_cmin": "rsa_tile.cuh", "k_tile_accept": "rsa_tile.cuh",
               "k_line_cmin_h": "rsa_line.cuh", "k_line_cmin_v": "rsa_line.cuh",
               "k_line_codes": "rsa_line.cuh", "k_line_accept_h": "rsa_line.cuh",
               "k_line_accept_v": "rsa_line.cuh", "k_row_cmin": "rsa_kernels.cuh",
               "k_col_cmin": "rsa_kernels.cuh", "k_row_accept": "rsa_kernels.cuh",
               "k_col_accept": "rsa_kernels.cuh"}


def src_digest(kernel: str) -> str:
    """First 16 hex digits of the SHA-256 of the code in the file that holds
    `kernel`: // comments and blank lines are left out, so documentation
    edits keep a measurement valid while any code change voids it."""
    import re
    f = os.path.join(ROOT, "paper_1810_06800_gb300", "csrc", KERNEL_FILE.get(kernel, "rsa.cu"))
    with open(f) as fh:
        lines = [re.sub(r"//.*$", "", ln).rstrip() for ln in fh]
    code = "\n".join(ln for ln in lines if ln)
    return hashlib.sha256(code.encode()).hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.idx)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def shard_seeds(rank: int, n: int):
    """Seeds of rank r: r*n + 1 .. r*n + n (weak scaling, disjoint across ranks)."""
    import numpy as np
    return np.arange(rank * n + 1, rank * n + n + 1, dtype=np.uint64)


def max_over_ranks(value: float, pg, device=None) -> float:
    """Slowest rank's time; `pg` is torch.distributed (or None for one rank)."""
    if pg is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def cpu_oracle_rate(L, k, seeds, budget_s, threads):
    """Samples/s of the oracle on `threads` host threads over a bounded
    prefix of the seeds (grown until it takes at least budget_s)."""
    import oracle
    done, t_total, m = 0, 0.0, max(1, threads)
    while True:
        chunk = seeds[done:done + m]
        if not chunk:
            break
        t0 = time.perf_counter()
        oracle.samples(L, k, chunk, threads=threads)
        t_total += time.perf_counter() - t0
        done += len(chunk)
        if t_total >= budget_s:
            break
        m = min(2 * m, len(seeds) - done) or m
    return done / t_total, done, t_total


def run_reference(args, wl, world, rank):
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    L, k, n = wl["L"], wl["k"], wl["n"]
    cores = os.cpu_count() or 1
    seeds = list(range(1, n + 1))
    per_step = min(n, 2 * cores)
    for w in range(args.warmup):
        oracle.samples(L, k, seeds[:per_step], threads=cores)
    t0 = time.perf_counter()
    for s in range(args.steps):
        lo = (s * per_step) % n
        oracle.samples(L, k, (seeds + seeds)[lo:lo + per_step], threads=cores)
    dt = time.perf_counter() - t0
    rate = per_step * args.steps / dt
    sample = f"{per_step} seeds of {args.workload} per step on {cores} threads"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": rate, "unit": "samples/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": args.workload, "L": L, "k": k, "samples_per_step": per_step},
        "cpu_baseline": {"value": rate, "unit": "samples/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": rate, "unit": "samples/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="L1024_k32_x1000", choices=sorted(WORKLOADS))
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    wl = WORKLOADS[args.workload]
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, wl, world, rank)

    import numpy as np
    import torch

    from paper_1810_06800_gb300 import rsa

    assert args.warmup >= 3, "at least 3 warm-up steps"
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    L, k, n = wl["L"], wl["k"], wl["n"]
    seeds = shard_seeds(rank, n)
    stream = torch.cuda.current_stream()
    lat = rsa.Lattice(L, k)
    h = lat.h

    def barrier():
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        rsa.rsa_run_seeds(h, seeds, stream)
    torch.cuda.synchronize()
    rsa.rsa_kernel_stats(h)  # reset counters
    rsa.rsa_work_stats(h)

    # ---- device-timed region (inputs resident: seeds + workspace) ----
    clocks = ClockSampler(int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0])
                          if os.environ.get("CUDA_VISIBLE_DEVICES", "").isdigit() else local)
    rsa.rsa_profile(h, True)
    barrier()
    clocks.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        rsa.rsa_run_seeds(h, seeds, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ck = clocks.stop()
    ms = e0.elapsed_time(e1)
    kstats = rsa.rsa_kernel_stats(h)
    work = rsa.rsa_work_stats(h)
    rsa.rsa_profile(h, False)
    st = rsa.rsa_sample_stats(h, n)
    nj, nc = rsa.rsa_results(h, n)
    ms = max_over_ranks(ms, pg, "cuda")
    value = n * world * args.steps / (ms / 1e3)

    # ---- end-to-end through the C ABI with host buffers ----
    nj_h = np.zeros(n, dtype=np.uint32)
    nc_h = np.zeros(n, dtype=np.uint32)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        seeds_h = np.ascontiguousarray(seeds)  # host input, copied to HBM in the call
        rsa.rsa_run_seeds(h, seeds_h, stream)
        nj_h, nc_h = rsa.rsa_results(h, n)     # device -> host results
    barrier()
    wall = time.perf_counter() - t0
    wall = max_over_ranks(wall, pg, "cuda")
    e2e = n * world * args.steps / wall
    assert np.array_equal(nj_h, nj) and np.array_equal(nc_h, nc)

    # ---- the plain path: one sample per run call, for comparison ----
    plain_n = min(16, n)
    barrier()
    t0 = time.perf_counter()
    for i in range(plain_n):
        rsa.rsa_run_seeds(h, seeds[i:i + 1], stream)
        rsa.rsa_results(h, 1)
    plain_rate = plain_n / (time.perf_counter() - t0)

    if rank != 0:
        lat.close()
        if pg is not None:
            pg.destroy_process_group()
        return 0

    # ---- roofline of the dominant kernel (CUDA events over the timed region) ----
    ours = {name: v for name, v in kstats.items() if v[1] > 0}
    dom = max(ours, key=lambda nm: ours[nm][0])
    dom_ms, dom_launches = ours[dom]
    passes = int(np.sum(st["rounds"].astype(np.int64) + 1)) * args.steps
    hbm_peak, peak_kind = measured_peaks()
    traffic_db = {}
    tp = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if os.path.exists(tp):
        with open(tp) as f:
            traffic_db = json.load(f)
    ent = traffic_db.get(dom)
    fresh = bool(ent) and ent.get("src") == src_digest(dom)
    if dom in TILE_WORK:
        cells_key, keys_key = TILE_WORK[dom]
        cells, keys = work[cells_key], work[keys_key]
        ops = cells * OPS_PER_CELL[dom] + keys * OPS_PER_KEY
        sm_count = torch.cuda.get_device_properties(local).multi_processor_count
        sm_mhz = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["sm_max_mhz"]) \
            if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 2070.0
        peak = sm_count * ALU_LANES_PER_SM * sm_mhz * 1e6 / 1e9  # Gop/s
        achieved = ops / (dom_ms / 1e3) / 1e9
        roof = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak,
                "unit": "Gop/s", "frac": achieved / peak,
                "traffic": (ent["bytes_per_cell"] * cells / dom_launches) if fresh else None,
                "peak_source": f"{sm_count} SMs x {ALU_LANES_PER_SM} int lanes x {sm_mhz:.0f} MHz",
                "alg_ops_per_launch": ops / dom_launches,
                "cells_per_launch": cells / dom_launches,
                # one argmin code byte per cell written (cmin) or read (accept)
                "hbm_view": {"alg_bytes_per_launch": 1.0 * cells / dom_launches,
                             "achieved_gbs": 1.0 * cells / (dom_ms / 1e3) / 1e9,
                             "peak_gbs": hbm_peak,
                             "frac": 1.0 * cells / (dom_ms / 1e3) / 1e9 / hbm_peak}}
    elif dom in BYTES_PER_CELL:
        if dom in LINE_WORK:   # cells of segments / tiles not skipped as dead
            ctr, share = LINE_WORK[dom]
            cells = work["raw"][ctr] * share
        else:
            cells = passes * L * L
        alg_bytes = BYTES_PER_CELL[dom] * cells
        achieved = alg_bytes / (dom_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm_peak,
                "unit": "GB/s", "frac": achieved / hbm_peak,
                "traffic": (ent["bytes_per_cell"] * cells / dom_launches) if fresh else None,
                "peak_source": f"{peak_kind} hbm_gbs",
                "alg_bytes_per_launch": alg_bytes / dom_launches}
    else:
        roof = {"bound": "latency", "kernel": dom, "achieved": None, "peak": hbm_peak,
                "unit": "GB/s", "frac": None, "traffic": None}
    kernel_table = {nm: {"ms": round(v[0], 3), "launches": v[1],
                         "share": round(v[0] / sum(x[0] for x in ours.values()), 4)}
                    for nm, v in ours.items()}

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cores = os.cpu_count() or 1
        rate, m, secs = cpu_oracle_rate(L, k, [int(s) for s in seeds], args.cpu_seconds, cores)
        # the same oracle on one core, over a shorter prefix of the seeds
        rate1, m1, secs1 = cpu_oracle_rate(L, k, [int(s) for s in seeds],
                                           max(1.0, args.cpu_seconds / 5), 1)
        cpu = {"value": rate, "unit": "samples/s", "cores": cores, "kind": "oracle",
               "sample": f"first {m} seeds of {args.workload} ({secs:.1f} s on {cores} threads)",
               "single_core": {"value": rate1, "unit": "samples/s",
                               "sample": f"first {m1} seeds ({secs1:.1f} s on 1 thread)"}}

    out = {
        "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic",
        "config": {"workload": args.workload, "L": L, "k": k, "samples_per_step": n,
                   "seeds": f"rank*{n}+1..rank*{n}+{n}",
                   "l2": "working set %.1f GB per step > 129 MB L2" % (
                       rsa.rsa_workspace_bytes(L, k, n) / 1e9),
                   "parallelism": f"samples sharded over {world} GPU(s), no collective"},
        "sites_per_s": value * L * L,
        "e2e": {"value": e2e, "unit": "samples/s", "h2d_bytes_per_step": int(8 * n),
                "d2h_bytes_per_step": int(128 * n)},
        "plain_one_sample_per_launch": {"value": plain_rate, "unit": "samples/s",
                                        "samples": plain_n},
        "gpu_launches": int(sum(v[1] for v in ours.values())),
        "roofline": roof,
        "kernels": kernel_table,
        "clocks": ck,
        "cpu_baseline": cpu,
        "stats": {"rounds_mean": float(st["rounds"].mean()),
                  "probes_mean": float(st["probes"].mean()),
                  "edges_mean": float(st["edges"].mean()),
                  "p_j_mean": float((k * nj / L / L).mean()),
                  "p_c_mean": float((k * nc / L / L).mean())},
    }
    print(json.dumps(out), flush=True)
    lat.close()
    if pg is not None:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
