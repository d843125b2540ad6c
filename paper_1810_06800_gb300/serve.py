"""Continuous-batching server for RSA jobs on one GPU.

A job asks for ``n`` samples of an (L, k) lattice with seeds seed .. seed+n-1.
Jobs are split into batches; a batch is admitted as soon as its device
workspace (``rsa_workspace_bytes``) fits in the free-HBM budget and a worker
is idle.  Workers are host threads, each with its own CUDA stream and its
own handles (one per lattice shape); the library call releases the GIL, so
batches of different jobs run on the GPU at the same time and jobs that
arrive while others run are admitted as memory and workers free up.  The
per-batch workspace is a torch tensor bound to the handle, returned to
torch's caching allocator when the batch ends, so lattice state stays on the
device and nothing is copied back but n_j and n_c.

Every sample's result depends only on (L, k, seed), so a job's results are
the same alone and in any mix.

``python -m paper_1810_06800_gb300.serve`` replays the seeded Poisson job
stream of ``workloads.served_jobs`` and prints one JSON line with latency
percentiles and throughput.
"""
from __future__ import annotations

import argparse
import json
import threading
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Job:
    job: int
    L: int
    k: int
    n: int
    seed: int
    t_arrival: float = 0.0
    nj: np.ndarray = None
    nc: np.ndarray = None
    remaining: int = 0
    t_done: float = None
    error: str = None
    done_event: threading.Event = field(default_factory=threading.Event)


@dataclass
class Batch:
    job: Job
    offset: int
    n: int
    bytes: int


class Scheduler:
    """Admission control and bookkeeping; the device work is done by a
    ``runner(L, k, seeds, nbytes, worker) -> (n_j, n_c)`` callable, so the
    policy can be tested without a GPU."""

    def __init__(self, runner, workspace_bytes, budget_bytes: int, workers: int = 4,
                 max_batch: int = 256, clock=time.perf_counter, max_wait_s: float = 2.0):
        self.runner = runner
        self.max_wait_s = max_wait_s
        self.ws_bytes = workspace_bytes
        self.budget = int(budget_bytes)
        self.max_batch = max_batch
        self.clock = clock
        self.cv = threading.Condition()
        self.pending = deque()
        self.in_flight_bytes = 0
        self.peak_bytes = 0
        self.running = 0
        self.peak_running = 0
        self.closed = False
        self.jobs = []
        self.threads = [threading.Thread(target=self._work, args=(w,), daemon=True)
                        for w in range(workers)]
        for t in self.threads:
            t.start()

    def batch_size(self, L: int, k: int, n: int) -> int:
        """Largest batch (<= max_batch, <= n) whose workspace fits a worker's
        share of the budget (budget / workers, so that every worker can hold a
        batch at once and no single allocation claims all free HBM); a batch
        of one sample may use the whole budget."""
        share = max(1, self.budget // max(1, len(self.threads)))
        b = min(n, self.max_batch)
        while b > 1 and self.ws_bytes(L, k, b) > share:
            b = (b + 1) // 2
        if self.ws_bytes(L, k, b) > self.budget:
            raise MemoryError(f"one sample of L={L} k={k} needs {self.ws_bytes(L, k, 1)} bytes, "
                              f"budget is {self.budget}")
        return b

    def submit(self, job: Job) -> Job:
        job.t_arrival = job.t_arrival or self.clock()
        job.nj = np.zeros(job.n, dtype=np.uint32)
        job.nc = np.zeros(job.n, dtype=np.uint32)
        b = self.batch_size(job.L, job.k, job.n)
        batches = [Batch(job, o, min(b, job.n - o), self.ws_bytes(job.L, job.k, min(b, job.n - o)))
                   for o in range(0, job.n, b)]
        job.remaining = len(batches)
        with self.cv:
            self.jobs.append(job)
            self.pending.extend(batches)
            self.cv.notify_all()
        return job

    def _take(self):
        """Next batch to run: the oldest pending batch if it fits the free
        budget; otherwise the oldest later batch that fits (first fit), unless
        the head has already waited max_wait_s, in which case nothing
        overtakes it until memory frees up for it."""
        with self.cv:
            while True:
                if self.closed and not self.pending:
                    return None
                pick = None
                if self.pending:
                    head = self.pending[0]
                    if self.in_flight_bytes + head.bytes <= self.budget:
                        pick = 0
                    elif self.clock() - head.job.t_arrival < self.max_wait_s:
                        for i in range(1, len(self.pending)):
                            if self.in_flight_bytes + self.pending[i].bytes <= self.budget:
                                pick = i
                                break
                if pick is not None:
                    b = self.pending[pick]
                    del self.pending[pick]
                    self.in_flight_bytes += b.bytes
                    self.running += 1
                    self.peak_bytes = max(self.peak_bytes, self.in_flight_bytes)
                    self.peak_running = max(self.peak_running, self.running)
                    return b
                self.cv.wait(timeout=0.05)

    def _work(self, w: int):
        while True:
            b = self._take()
            if b is None:
                return
            job = b.job
            seeds = np.arange(job.seed + b.offset, job.seed + b.offset + b.n, dtype=np.uint64)
            err = None
            try:
                nj, nc = self.runner(job.L, job.k, seeds, b.bytes, w)
            except Exception as e:  # keep serving; the job reports the error
                err = f"{type(e).__name__}: {e}"
                nj = nc = None
            with self.cv:
                self.in_flight_bytes -= b.bytes
                self.running -= 1
                if err:
                    job.error = job.error or err
                else:
                    job.nj[b.offset:b.offset + b.n] = nj
                    job.nc[b.offset:b.offset + b.n] = nc
                job.remaining -= 1
                if job.remaining == 0:
                    job.t_done = self.clock()
                    job.done_event.set()
                self.cv.notify_all()

    def close(self, wait: bool = True):
        with self.cv:
            self.closed = True
            self.cv.notify_all()
        if wait:
            for t in self.threads:
                t.join()

    def stats(self):
        lat = np.array([j.t_done - j.t_arrival for j in self.jobs if j.t_done is not None])
        return dict(jobs=len(self.jobs), done=int(len(lat)),
                    p50_s=float(np.percentile(lat, 50)) if len(lat) else None,
                    p99_s=float(np.percentile(lat, 99)) if len(lat) else None,
                    peak_in_flight_bytes=int(self.peak_bytes),
                    peak_concurrent_batches=int(self.peak_running))


class GpuRunner:
    """Runs a batch through the C ABI on the worker's own stream with a
    torch-allocated workspace bound to a cached handle."""

    def __init__(self, workers: int, device: int = 0):
        import torch

        from . import rsa
        self.torch, self.rsa = torch, rsa
        self.device = device
        self.streams = [torch.cuda.Stream(device=device) for _ in range(workers)]
        self.handles = [dict() for _ in range(workers)]

    def __call__(self, L, k, seeds, nbytes, w):
        torch, rsa = self.torch, self.rsa
        torch.cuda.set_device(self.device)
        st = self.streams[w]
        with torch.cuda.stream(st):
            h = self.handles[w].get((L, k))
            if h is None:
                h = self.handles[w][(L, k)] = rsa.rsa_create(L, k, 1)
            try:
                buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=f"cuda:{self.device}")
            except torch.cuda.OutOfMemoryError:
                # the free budget counted memory that torch's cache holds in
                # blocks too small for this workspace: return them and retry
                torch.cuda.empty_cache()
                buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=f"cuda:{self.device}")
            ptr = (buf.data_ptr() + 255) // 256 * 256
            try:
                rsa.rsa_bind_workspace(h, ptr, nbytes)
                rsa.rsa_run_seeds(h, seeds, st)
                nj, nc = rsa.rsa_results(h, len(seeds))
            finally:
                rsa.rsa_bind_workspace(h, None)
                del buf
        return nj, nc

    def close(self):
        for hs in self.handles:
            for h in hs.values():
                self.rsa.rsa_destroy(h)
            hs.clear()


def gpu_budget(reserve_frac: float = 0.1, device: int = 0) -> int:
    """Free HBM now, less a reserve for torch, the library and other users."""
    import torch
    free, total = torch.cuda.mem_get_info(device)
    return int(free - reserve_frac * total)


def make_server(workers: int = 4, budget_bytes: int | None = None, max_batch: int = 256,
                device: int = 0):
    from . import rsa
    runner = GpuRunner(workers, device)
    budget = gpu_budget(device=device) if budget_bytes is None else budget_bytes
    sch = Scheduler(runner, rsa.rsa_workspace_bytes, budget, workers, max_batch)
    sch.gpu_runner = runner
    return sch


def replay(jobs, workers: int = 4, budget_bytes: int | None = None, time_scale: float = 1.0,
           max_batch: int = 256):
    """Submit jobs at their arrival times (seconds x time_scale) and wait."""
    sch = make_server(workers, budget_bytes, max_batch)
    t0 = time.perf_counter()
    subs = []
    for j in jobs:
        delay = t0 + j["t"] * time_scale - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        subs.append(sch.submit(Job(j["job"], j["L"], j["k"], j["n"], j["seed"],
                                   t_arrival=time.perf_counter())))
    for job in subs:
        job.done_event.wait()
    wall = time.perf_counter() - t0
    sch.close()
    sch.gpu_runner.close()
    st = sch.stats()
    samples = sum(j.n for j in subs)
    sites = sum(j.n * j.L * j.L for j in subs)
    st.update(wall_s=wall, samples=samples, samples_per_s=samples / wall, sites_per_s=sites / wall,
              errors=[j.error for j in subs if j.error])
    return st, subs


def main():
    from . import workloads
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--jobs", type=int, default=40)
    ap.add_argument("--rate", type=float, default=4.0, help="mean arrivals per second")
    ap.add_argument("--max-k", type=int, default=1024)
    ap.add_argument("--workers", type=int, default=4)
    ap.add_argument("--max-batch", type=int, default=256)
    ap.add_argument("--master-seed", type=int, default=1810)
    ap.add_argument("--uneven", action="store_true",
                    help="the batched uneven-size workload: k in {2, 8, 64, 512}, L = 16k, "
                         "256 samples each (seeds 1..256), all submitted at once")
    args = ap.parse_args()
    if args.uneven:
        jobs = [dict(job=i, t=0.0, L=w["L"], k=w["k"], n=len(w["seeds"]), seed=w["seeds"][0])
                for i, w in enumerate(workloads.BATCHED_UNEVEN)]
        st, subs = replay(jobs, args.workers, max_batch=args.max_batch)
        st.update(metric="batched uneven (L, k) groups: samples/s and sites/s",
                  groups=[dict(L=j.L, k=j.k, n=j.n, latency_s=j.t_done - j.t_arrival,
                               p_j=float((j.k * j.nj / j.L**2).mean()),
                               p_c=float((j.k * j.nc / j.L**2).mean())) for j in subs])
        print(json.dumps(st))
        return
    jobs = workloads.served_jobs(args.jobs, args.rate, args.master_seed, max_k=args.max_k)
    st, _ = replay(jobs, args.workers, max_batch=args.max_batch)
    st.update(metric="served RSA jobs: latency percentiles and throughput", jobs_spec=dict(
        n=args.jobs, rate_per_s=args.rate, max_k=args.max_k, master_seed=args.master_seed,
        workers=args.workers))
    print(json.dumps(st))


if __name__ == "__main__":
    main()
