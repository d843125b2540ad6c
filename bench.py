#!/usr/bin/env python3
"""Throughput benchmark: jammed RSA samples per second on one GB300.

Workload (default): the large-k batch, L = 32768 periodic lattice, k = 4096,
8 samples with seeds 1..8 per step (per rank under torchrun; rank r uses
seeds r*8 + 1 ..), 78 GB held on the device.  One step runs the whole path
for the batch: the parallel greedy rounds to jamming (n_j), the contact
graph, and the first-wrap bisection (n_c).  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME]

`value` is timed on the product path (graph-replayed round and probe loops,
no per-kernel events).  A separate profiled pass of the same steps records a
CUDA event pair around every launch for the per-kernel shares and the
roofline of the dominant kernel.  `--impl reference` times the CPU oracle (a
plain sequential scan plus union-find in C) on the host cores, on a bounded
sample of the same workload.
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
    # the largest single-GPU configuration: the default
    "L32768_k4096_x8": dict(L=32768, k=4096, n=8),
    "L1024_k32_x1000": dict(L=1024, k=32, n=1000),
    "L64_k4_x100": dict(L=64, k=4, n=100),
    # small cases for ncu captures (a few GB on the device)
    "L1024_k32_x64": dict(L=1024, k=32, n=64),
    "L8192_k512_x2": dict(L=8192, k=512, n=2),
    "L8192_k512_x8": dict(L=8192, k=512, n=8),
    "L16384_k4096_x1": dict(L=16384, k=4096, n=1),
}
DEFAULT_WORKLOAD = "L32768_k4096_x8"
# Batches of uneven shapes, run through rsa_run_mix (each shape the way the
# autotuner picks): groups of (L, k, samples); rank r takes seeds
# r*n + 1 .. r*n + n of every group.
MIX_WORKLOADS = {
    "uneven_k2-8-64-512_x256": [(32, 2, 256), (128, 8, 256), (1024, 64, 256), (8192, 512, 256)],
    "L64_k4_x100_mix": [(64, 4, 100)],
}
METRIC = "jammed samples/s (n_j and n_c per sample, bit-exact to the oracle)"

# Algorithmic bytes per processed lattice cell of each round kernel, from
# the byte model of the method's unfused steps: rowmin reads a priority and
# writes a cell minimum (8 + 8); colmin reads a priority and the row minimum
# and writes their minimum (8 + 8 + 8); accept reads the cell minimum along
# both orientations and both priorities (2 x 8 + 16); kill reads occupancy
# (1).  A kernel that carries out several of these steps is credited with
# their sum over the cells it processed; where two kernels split one step,
# each is credited with the part it does.  Priorities are recomputed rather
# than stored and minima are kept as short argmin codes, so the kernels move
# far fewer DRAM bytes than this (ncu "traffic").
STEP_BYTES = {"rowmin": 16.0, "colmin": 24.0, "accept": 32.0, "kill": 1.0}
KERNEL_STEPS = {
    # 32 x 32 tile path: one pass both window minima, one pass acceptance
    "k_tile_cmin": (("rowmin", "colmin"), 40.0),
    "k_tile_accept": (("accept", "kill"), 33.0),
    # long-k line path: horizontal windows (rowmin); vertical windows (the
    # window part of colmin, 16 of its 24 bytes); the per-cell combine of
    # the two minima (the remaining 8); acceptance along rows / columns (half
    # of accept + kill each)
    "k_line_cmin_h": (("rowmin",), 16.0),
    "k_line_cmin_v": (("colmin",), 16.0),
    "k_line_codes": (("colmin",), 8.0),
    "k_line_combine": (("colmin",), 8.0),
    "k_line_accept_h": (("accept", "kill"), 16.5),
    "k_line_accept_v": (("accept", "kill"), 16.5),
    # long-k lines of whole k-blocks: the same split with argmin offsets
    "k_lwin_h": (("rowmin",), 16.0),
    "k_lwin_v": (("colmin",), 16.0),
    "k_lcomb": (("colmin",), 8.0),
    "k_lacc_h": (("accept", "kill"), 16.5),
    "k_lacc_v": (("accept", "kill"), 16.5),
    # general path
    "k_row_cmin": (("rowmin",), 16.0),
    "k_col_cmin": (("colmin",), 24.0),
    "k_row_accept": (("accept", "kill"), 16.5),
    "k_col_accept": (("accept", "kill"), 16.5),
}
# Processed cells per kernel: (work counter, share of it).  Tile path
# counters: 0 cmin cells, 1 cmin keys, 2 accept cells, 3 accept keys; long-k
# path: 0 / 1 horizontal / vertical window cells, 2 acceptance cells (both
# orientations), 3 combine cells.  The general path has no counters: every
# cell of every round.
WORK_CELLS = {"k_tile_cmin": (0, 1.0), "k_tile_accept": (2, 1.0),
              "k_line_cmin_h": (0, 1.0), "k_line_cmin_v": (1, 1.0),
              "k_line_codes": (3, 1.0), "k_line_combine": (3, 1.0),
              "k_line_accept_h": (2, 0.5), "k_line_accept_v": (2, 0.5),
              "k_lwin_h": (0, 1.0), "k_lwin_v": (1, 1.0), "k_lcomb": (3, 1.0),
              "k_lacc_h": (2, 0.5), "k_lacc_v": (2, 0.5)}
# A second view of the tile kernels, which are bound by integer issue:
# algorithmic 32-bit lane operations (a 64-bit minimum is 4 ops plus 1 when
# the argmin is tracked, a window minimum is 3 minima per cell, a liveness
# test 4 ops, a splitmix64 priority 20 ops) against 128 integer lanes per SM
# per clock.
OPS_PER_KEY = 20
OPS_PER_CELL = {"k_tile_cmin": 2 * 3 * 5 + 6 + 2 * 4, "k_tile_accept": 2 * 3}
TILE_KEYS = {"k_tile_cmin": 1, "k_tile_accept": 3}
ALU_LANES_PER_SM = 128

# The source file that holds each kernel: a DRAM-traffic figure measured by
# ncu is used only while that file is unchanged.
KERNEL_FILE = {"k_tile_cmin": "rsa_tile.cuh", "k_tile_accept": "rsa_tile.cuh",
               "k_line_cmin_h": "rsa_line.cuh", "k_line_cmin_v": "rsa_line.cuh",
               "k_line_codes": "rsa_line.cuh", "k_line_accept_h": "rsa_line.cuh",
               "k_line_accept_v": "rsa_line.cuh", "k_lwin_h": "rsa_lwin.cuh",
               "k_lwin_v": "rsa_lwin.cuh", "k_lcomb": "rsa_lwin.cuh",
               "k_lacc_h": "rsa_lwin.cuh", "k_lacc_v": "rsa_lwin.cuh",
               "k_row_cmin": "rsa_kernels.cuh",
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


def oracle_case(L: int, k: int):
    """(L', k', scale) on which the CPU oracle is timed for workload (L, k).
    One oracle sample of L >= 4096 takes minutes (about half an hour at
    L = 32768: a sort of 2 L^2 priorities and a scan), far beyond a bounded
    baseline, so the oracle then runs the same model at L' = L / 2^j <= 2048
    with the same L/k, and its rate is scaled to samples of the workload by
    the lattice sites, scale = (L / L')^2.  The sort costs O(log L) more per
    site at L than at L', so the scaled rate overstates the oracle's speed
    at the workload's own size (by about 1.3x at L = 32768)."""
    j = 0
    while (L >> j) > 2048 and L % (2 << j) == 0 and k % (2 << j) == 0:
        j += 1
    return L >> j, k >> j, float(1 << (2 * j))


def cpu_oracle_rate(L, k, seeds, budget_s, threads):
    """Samples/s of the oracle on `threads` host threads over a bounded
    prefix of the seeds (grown until it takes at least budget_s), on the
    (possibly scaled-down) case of oracle_case."""
    import oracle
    Lo, ko, scale = oracle_case(L, k)
    done, t_total, m = 0, 0.0, max(1, threads)
    while True:
        chunk = seeds[done:done + m]
        if not chunk:
            break
        t0 = time.perf_counter()
        oracle.samples(Lo, ko, chunk, threads=threads)
        t_total += time.perf_counter() - t0
        done += len(chunk)
        if t_total >= budget_s:
            break
        m = min(2 * m, len(seeds) - done) or m
    return done / t_total / scale, done, t_total, (Lo, ko, scale)


def sample_text(wl_name, L, k, m, secs, threads):
    Lo, ko, scale = oracle_case(L, k)
    if scale == 1.0:
        return f"first {m} seeds of {wl_name} ({secs:.1f} s on {threads} threads)"
    return (f"{m} seeded samples of L={Lo}, k={ko} (the same L/k) in {secs:.1f} s on "
            f"{threads} threads, scaled by the sites ratio ({L}/{Lo})^2 = {scale:.0f} to "
            f"samples of L={L}, k={k}; one oracle sample of the workload itself takes "
            f"minutes (4017-6247 s on one x86 core at L=32768, k=4096), so the scaled rate "
            f"overstates the oracle's full-size speed")


def run_reference(args, wl, world, rank):
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    L, k, n = wl["L"], wl["k"], wl["n"]
    Lo, ko, scale = oracle_case(L, k)
    cores = os.cpu_count() or 1
    seeds = list(range(1, max(n, 2 * cores) + 1))
    # samples per step: one per core on a scaled-down case, else a bounded
    # prefix of the workload's own seeds
    per_step = cores if scale > 1.0 else min(n, 2 * cores)
    for w in range(args.warmup):
        oracle.samples(Lo, ko, seeds[:per_step], threads=cores)
    t0 = time.perf_counter()
    for s in range(args.steps):
        lo = (s * per_step) % len(seeds)
        oracle.samples(Lo, ko, (seeds + seeds)[lo:lo + per_step], threads=cores)
    dt = time.perf_counter() - t0
    rate = per_step * args.steps / dt / scale
    sample = sample_text(args.workload, L, k, per_step, dt / args.steps, cores) + " (per step)"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": rate, "unit": "samples/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": args.workload, "L": L, "k": k, "samples_per_step": per_step,
                   "oracle_case": {"L": Lo, "k": ko, "sites_scale": scale}},
        "cpu_baseline": {"value": rate, "unit": "samples/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": rate, "unit": "samples/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)
    return 0


def roofline(dom, kstats, work, passes, L, n_cells_round, hbm_peak, peak_kind, sm_count, sm_mhz,
             window_threads=0):
    """Roofline of kernel `dom` over the profiled pass: algorithmic bytes per
    processed cell (KERNEL_STEPS) times the cells its launches processed,
    over its summed CUDA-event time, against the measured copy bandwidth.
    `window_threads` is the window-pass CTA size the run asked for (0: the
    library's default, not known here)."""
    dom_ms, dom_launches = kstats[dom]
    if dom in WORK_CELLS:
        ctr, share = WORK_CELLS[dom]
        cells = work["raw"][ctr] * share
    else:
        cells = passes * n_cells_round
    steps, bpc = KERNEL_STEPS.get(dom, ((), None))
    out = {"bound": "hbm", "kernel": dom, "unit": "GB/s", "peak": hbm_peak,
           "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)"}
    if bpc is None or dom_ms <= 0:
        out.update(achieved=None, frac=None, traffic=None, note="no byte model for this kernel")
        return out
    alg = bpc * cells
    achieved = alg / (dom_ms / 1e3) / 1e9
    out.update(achieved=achieved, frac=achieved / hbm_peak,
               alg_bytes_per_cell=bpc, steps=list(steps),
               cells_per_launch=cells / dom_launches,
               alg_bytes_per_launch=alg / dom_launches,
               avg_launch_ms=dom_ms / dom_launches)
    # measured DRAM bytes per launch, scaled from the ncu capture's bytes per
    # cell; null once the kernel's source file has changed since the capture,
    # or when the capture names a window-pass CTA size the run did not ask for
    traffic_db = {}
    tp = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if os.path.exists(tp):
        with open(tp) as f:
            traffic_db = json.load(f)
    ent = traffic_db.get(dom)
    fresh = bool(ent) and ent.get("src") == src_digest(dom)
    if fresh and "window_threads" in ent:
        fresh = ent["window_threads"] == window_threads
    out["traffic"] = (ent["bytes_per_cell"] * cells / dom_launches) if fresh else None
    if dom in OPS_PER_CELL:
        keys = work["raw"][TILE_KEYS[dom]]
        ops = cells * OPS_PER_CELL[dom] + keys * OPS_PER_KEY
        peak = sm_count * ALU_LANES_PER_SM * sm_mhz * 1e6 / 1e9
        got = ops / (dom_ms / 1e3) / 1e9
        out["alu_view"] = {"bound": "alu", "achieved": got, "peak": peak, "unit": "Gop/s",
                           "frac": got / peak,
                           "peak_source": f"{sm_count} SMs x {ALU_LANES_PER_SM} int lanes x "
                                          f"{sm_mhz:.0f} MHz"}
    return out


def mix_arrays(groups, rank):
    import numpy as np
    L, k, sd = [], [], []
    for (gl, gk, gn) in groups:
        L += [gl] * gn
        k += [gk] * gn
        sd += list(range(rank * gn + 1, rank * gn + gn + 1))
    return np.array(L, np.uint32), np.array(k, np.uint32), np.array(sd, np.uint64)


def mix_oracle_rate(groups, threads, reps=1):
    """Samples/s of the oracle on the whole mix: per group, `threads`
    samples of its (possibly scaled-down) oracle case on `threads` host
    threads give its time per sample; the mix takes the sum over groups of
    samples x time per sample."""
    import oracle
    total_t, total_n, secs, parts = 0.0, 0, 0.0, []
    for (gl, gk, gn) in groups:
        Lo, ko, scale = oracle_case(gl, gk)
        t0 = time.perf_counter()
        for r in range(reps):
            oracle.samples(Lo, ko, list(range(1 + r * threads, 1 + (r + 1) * threads)),
                           threads=threads)
        dt = time.perf_counter() - t0
        secs += dt
        per_sample = dt / (reps * threads) * scale
        total_t += gn * per_sample
        total_n += gn
        parts.append(f"L={Lo} k={ko} x{reps * threads}" + (f" (x{scale:.0f} sites)" if scale > 1 else ""))
    return total_n / total_t, secs, "; ".join(parts)


def run_reference_mix(args, groups, rank):
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        mix_oracle_rate(groups, cores)
    rates, t0 = [], time.perf_counter()
    for _ in range(args.steps):
        r, _, parts = mix_oracle_rate(groups, cores)
        rates.append(r)
    dt = time.perf_counter() - t0
    rate = sum(rates) / len(rates)
    n = sum(g[2] for g in groups)
    sample = (f"per step, {cores} samples per shape on {cores} threads ({parts}); the mix's "
              f"{n} samples take the sum of samples x time per sample")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": rate, "unit": "samples/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": args.workload, "groups": groups},
        "cpu_baseline": {"value": rate, "unit": "samples/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": rate, "unit": "samples/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)
    return 0


def run_mix(args, groups, world, rank, local):
    """A batch of uneven shapes through rsa_run_mix: one step = every group's
    samples in one call.  Compared with the plain form: each shape's batch on
    its own handle, one after another."""
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
    L, k, sd = mix_arrays(groups, rank)
    n = int(sd.size)
    stream = torch.cuda.current_stream()

    def barrier():
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):          # the first call also tunes each shape
        nj, nc = rsa.rsa_run_mix(L, k, sd, stream)
    choices = {f"L{gl}_k{gk}": rsa.rsa_tune(gl, gk, gn, measure=False) for (gl, gk, gn) in groups}
    # ---- device-timed: events on the caller's stream bracket every call
    clocks = ClockSampler(local)
    barrier()
    rsa.rsa_mix_launches()   # reset the launch count
    clocks.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record(stream)
    for _ in range(args.steps):
        nj2, nc2 = rsa.rsa_run_mix(L, k, sd, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    barrier()
    ck = clocks.stop()
    gpu_launches = rsa.rsa_mix_launches()   # kernels of the timed calls
    ms = max_over_ranks(e0.elapsed_time(e1), pg, "cuda")
    wall = max_over_ranks(wall, pg, "cuda")
    assert np.array_equal(nj, nj2) and np.array_equal(nc, nc2)
    value = n * world * args.steps / (ms / 1e3)
    # host arrays in, host results out: the same calls are end to end
    e2e = n * world * args.steps / wall
    # ---- plain: each shape's batch on its own handle, one after another
    rsa.rsa_mix_release()   # the mix's cached handles hold their workspaces
    barrier()
    t0 = time.perf_counter()
    per_shape = {}
    for (gl, gk, gn) in groups:
        sel = (L == gl) & (k == gk)
        lat = rsa.Lattice(gl, gk)
        t1 = time.perf_counter()
        pj, pc = lat.run(sd[sel])
        per_shape[f"L{gl}_k{gk}"] = gn / (time.perf_counter() - t1)
        lat.close()
        assert np.array_equal(pj, nj[sel]) and np.array_equal(pc, nc[sel])
    plain = n / (time.perf_counter() - t0)
    if rank != 0:
        if pg is not None:
            pg.destroy_process_group()
        return 0
    # ---- roofline: a profiled pass of the shape with the most cells on its
    #      own handle (the global path's kernels); the small-lattice groups run
    #      from shared memory and move no DRAM bytes per cell
    big = max(groups, key=lambda g: g[0] * g[0] * g[2])
    sel = (L == big[0]) & (k == big[1])
    lat = rsa.Lattice(big[0], big[1])
    lat.run(sd[sel])
    rsa.rsa_kernel_stats(lat.h)
    rsa.rsa_work_stats(lat.h)
    rsa.rsa_profile(lat.h, True)
    lat.run(sd[sel])
    kst = {nm: v for nm, v in rsa.rsa_kernel_stats(lat.h).items() if v[1] > 0}
    work = rsa.rsa_work_stats(lat.h)
    st = rsa.rsa_sample_stats(lat.h, int(sel.sum()))
    lat.close()
    dom = max(kst, key=lambda nm: kst[nm][0])
    hbm_peak, peak_kind = measured_peaks()
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    passes = int(np.sum(st["rounds"].astype(np.int64) + 1))
    roof = roofline(dom, kst, work, passes, big[0], big[0] ** 2, hbm_peak, peak_kind, sm_count,
                    2070.0)
    roof["shape"] = f"L={big[0]} k={big[1]}, {big[2]} samples, one profiled pass on its handle"
    total = sum(v[0] for v in kst.values())
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cores = os.cpu_count() or 1
        rate, secs, parts = mix_oracle_rate(groups, cores)
        cpu = {"value": rate, "unit": "samples/s", "cores": cores, "kind": "oracle",
               "sample": f"{cores} samples per shape on {cores} threads ({parts}), {secs:.1f} s"}
    out = {
        "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic",
        "config": {"workload": args.workload, "groups": groups, "samples_per_step": n,
                   "api": "rsa_run_mix (one call per step)",
                   "l2": "no flush: working set above 129 MB L2",
                   "parallelism": f"samples sharded over {world} GPU(s), no collective",
                   "tuned": choices},
        "sites_per_s": value * float(np.mean(L.astype(np.float64) ** 2)),
        "e2e": {"value": e2e, "unit": "samples/s", "h2d_bytes_per_step": 16 * n,
                "d2h_bytes_per_step": 8 * n},
        "plain_per_shape_handles": {"value": plain, "unit": "samples/s",
                                    "per_shape": per_shape},
        "gpu_launches": gpu_launches,
        "roofline": roof,
        "kernels": {nm: {"ms": round(v[0], 3), "launches": v[1], "share": round(v[0] / total, 4)}
                    for nm, v in kst.items()},
        "clocks": ck,
        "cpu_baseline": cpu,
    }
    print(json.dumps(out), flush=True)
    if pg is not None:
        pg.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD,
                    choices=sorted(WORKLOADS) + sorted(MIX_WORKLOADS))
    ap.add_argument("--profile-steps", type=int, default=2,
                    help="steps of the separate pass with per-kernel CUDA events")
    ap.add_argument("--window-threads", type=int, default=0,
                    help="CTA size of the long-k window pass (128 or 256; 0 = the library default)")
    ap.add_argument("--rounds-per-check", type=int, default=0,
                    help="greedy rounds per captured chunk (0 = the library default)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    world, rank, local = dist_setup()
    if args.workload in MIX_WORKLOADS:
        if args.impl == "reference":
            return run_reference_mix(args, MIX_WORKLOADS[args.workload], rank)
        return run_mix(args, MIX_WORKLOADS[args.workload], world, rank, local)
    wl = WORKLOADS[args.workload]
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
    if args.window_threads:
        rsa.rsa_set_window_threads(h, args.window_threads)
    if args.rounds_per_check:
        rsa.rsa_set_rounds_per_check(h, args.rounds_per_check)

    def barrier():
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        rsa.rsa_run_seeds(h, seeds, stream)
    torch.cuda.synchronize()
    rsa.rsa_kernel_stats(h)  # reset counters
    rsa.rsa_work_stats(h)

    # ---- device-timed region: the product path (graph replay, no events);
    #      inputs resident (seeds, workspace) ----
    clocks = ClockSampler(int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0])
                          if os.environ.get("CUDA_VISIBLE_DEVICES", "").isdigit() else local)
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
    launches = rsa.rsa_kernel_stats(h)   # launch counts of the timed region
    rsa.rsa_work_stats(h)
    gpu_launches = int(sum(v[1] for v in launches.values()))
    st = rsa.rsa_sample_stats(h, n)
    nj, nc = rsa.rsa_results(h, n)
    ms = max_over_ranks(ms, pg, "cuda")
    value = n * world * args.steps / (ms / 1e3)

    # ---- profiled pass: the same steps with an event pair per launch ----
    psteps = max(1, args.profile_steps)
    rsa.rsa_profile(h, True)
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for _ in range(psteps):
        rsa.rsa_run_seeds(h, seeds, stream)
    p1.record(stream)
    torch.cuda.synchronize()
    prof_ms = p0.elapsed_time(p1)
    kstats = rsa.rsa_kernel_stats(h)
    work = rsa.rsa_work_stats(h)
    rsa.rsa_profile(h, False)
    pst = rsa.rsa_sample_stats(h, n)
    pj, pc = rsa.rsa_results(h, n)
    assert np.array_equal(pj, nj) and np.array_equal(pc, nc)

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

    # ---- roofline of the dominant kernel (profiled pass, CUDA events) ----
    ours = {name: v for name, v in kstats.items() if v[1] > 0}
    dom = max(ours, key=lambda nm: ours[nm][0])
    passes = int(np.sum(pst["rounds"].astype(np.int64) + 1)) * psteps
    hbm_peak, peak_kind = measured_peaks()
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    sm_mhz = float(json.load(open(pk))["sm_max_mhz"]) if os.path.exists(pk) else 2070.0
    roof = roofline(dom, ours, work, passes, L, L * L, hbm_peak, peak_kind, sm_count, sm_mhz,
                    args.window_threads)
    # the same figures for every round kernel with a byte model
    roof_all = {}
    for nm in ours:
        if nm in KERNEL_STEPS:
            r = roofline(nm, ours, work, passes, L, L * L, hbm_peak, peak_kind, sm_count, sm_mhz,
                         args.window_threads)
            roof_all[nm] = {k2: r.get(k2) for k2 in ("achieved", "frac", "alg_bytes_per_cell",
                                                      "avg_launch_ms", "traffic")}
    total_ms = sum(x[0] for x in ours.values())
    kernel_table = {nm: {"ms": round(v[0], 3), "launches": v[1],
                         "share": round(v[0] / total_ms, 4)} for nm, v in ours.items()}

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cores = os.cpu_count() or 1
        sd = [int(s) for s in seeds] + list(range(n + 1, n + 2 * cores + 1))
        rate, m, secs, _ = cpu_oracle_rate(L, k, sd, args.cpu_seconds, cores)
        rate1, m1, secs1, _ = cpu_oracle_rate(L, k, sd, max(1.0, args.cpu_seconds / 5), 1)
        cpu = {"value": rate, "unit": "samples/s", "cores": cores, "kind": "oracle",
               "sample": sample_text(args.workload, L, k, m, secs, cores),
               "single_core": {"value": rate1, "unit": "samples/s",
                               "sample": sample_text(args.workload, L, k, m1, secs1, 1)}}

    out = {
        "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic",
        "config": {"workload": args.workload, "L": L, "k": k, "samples_per_step": n,
                   "seeds": f"rank*{n}+1..rank*{n}+{n}",
                   "l2": "no flush: working set %.1f GB per step > 129 MB L2" % (
                       rsa.rsa_workspace_bytes(L, k, n) / 1e9),
                   "parallelism": f"samples sharded over {world} GPU(s), no collective",
                   "window_threads": args.window_threads or None,
                   "rounds_per_check": args.rounds_per_check or None},
        "sites_per_s": value * L * L,
        "e2e": {"value": e2e, "unit": "samples/s", "h2d_bytes_per_step": int(8 * n),
                "d2h_bytes_per_step": int(128 * n)},
        "plain_one_sample_per_launch": {"value": plain_rate, "unit": "samples/s",
                                        "samples": plain_n},
        "gpu_launches": gpu_launches,
        "roofline": roof,
        "rooflines": roof_all,
        "profiled_pass": {"steps": psteps, "ms_per_step": prof_ms / psteps,
                          "note": "per-kernel shares and the roofline come from this pass; "
                                  "value is timed without per-launch events"},
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
