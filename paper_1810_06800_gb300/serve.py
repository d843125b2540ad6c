"""Continuous-batching server for RSA jobs on one GPU.

A job asks for ``n`` samples of an (L, k) lattice with seeds seed .. seed+n-1.
Jobs are split into batches; a batch is admitted as soon as its device
workspace (``rsa_workspace_bytes``) fits in the free-HBM budget and a worker
is idle, the job that has received the least service so far first.  Workers
are host threads, each with its own CUDA stream and its own handles (one
per lattice shape); the library call releases the GIL, so batches of
different jobs run on the GPU at the same time and jobs that arrive while
others run are admitted as memory and workers free up.  The
per-batch workspace is a torch tensor bound to the handle, returned to
torch's caching allocator when the batch ends, so lattice state stays on the
device and nothing is copied back but n_j and n_c.

Every sample's result depends only on (L, k, seed), so a job's results are
the same alone and in any mix.

A job can be cancelled from the host (``Scheduler.cancel``): its batches not
yet started are dropped, the ones on the GPU finish and are discarded, and
the job ends with error "cancelled".  With a journal file, every finished
batch is appended to it as one JSON line; a scheduler started later with the
same journal fills a resubmitted job's finished samples from it and runs
only the rest (restart after a crash or a cancel).

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
    t_start: float = None  # its first batch started on a worker
    error: str = None
    cancelled: bool = False
    attained: int = 0      # lattice sites of its batches started so far
    from_journal: int = 0  # samples filled from the journal
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
                 max_batch: int = 256, clock=time.perf_counter, max_wait_s: float = 2.0,
                 journal: str | None = None):
        self.runner = runner
        self.journal = journal
        self.journal_lock = threading.Lock()
        self.journal_done = {}  # (job, L, k, seed) -> {sample: (n_j, n_c)}
        if journal:
            self._load_journal()
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

    def _load_journal(self):
        import os
        if not os.path.exists(self.journal):
            return
        with open(self.journal) as f:
            for line in f:
                try:
                    r = json.loads(line)
                except ValueError:
                    continue  # a line cut short by a crash
                done = self.journal_done.setdefault((r["job"], r["L"], r["k"], r["seed"]), {})
                for i, (a, b) in enumerate(zip(r["nj"], r["nc"])):
                    done[r["offset"] + i] = (a, b)

    def _journal_batch(self, job: Job, offset: int, nj, nc):
        line = json.dumps(dict(job=job.job, L=job.L, k=job.k, seed=job.seed, offset=offset,
                               nj=[int(v) for v in nj], nc=[int(v) for v in nc]))
        with self.journal_lock, open(self.journal, "a") as f:
            f.write(line + "\n")
            f.flush()

    def submit(self, job: Job) -> Job:
        job.t_arrival = job.t_arrival or self.clock()
        job.nj = np.zeros(job.n, dtype=np.uint32)
        job.nc = np.zeros(job.n, dtype=np.uint32)
        b = self.batch_size(job.L, job.k, job.n)
        # samples already in the journal are filled, the rest run in batches
        # over the contiguous ranges still missing
        known = self.journal_done.get((job.job, job.L, job.k, job.seed), {})
        todo = []
        for i in range(job.n):
            if i in known:
                job.nj[i], job.nc[i] = known[i]
            else:
                todo.append(i)
        job.from_journal = job.n - len(todo)
        batches = []
        i = 0
        while i < len(todo):
            j = i
            while j + 1 < len(todo) and todo[j + 1] == todo[j] + 1 and j + 1 - i < b:
                j += 1
            o, m = todo[i], j - i + 1
            batches.append(Batch(job, o, m, self.ws_bytes(job.L, job.k, m)))
            i = j + 1
        job.remaining = len(batches)
        with self.cv:
            self.jobs.append(job)
            if not batches:
                job.t_done = self.clock()
                job.done_event.set()
            self.pending.extend(batches)
            self.cv.notify_all()
        return job

    def cancel(self, job: Job) -> None:
        """Drop the job's batches not yet started; the ones on the GPU finish
        and are discarded.  The job ends with error "cancelled"."""
        with self.cv:
            if job.done_event.is_set():
                return
            job.cancelled = True
            job.error = "cancelled"
            keep = deque(b for b in self.pending if b.job is not job)
            job.remaining -= len(self.pending) - len(keep)
            self.pending = keep
            if job.remaining == 0:
                job.t_done = self.clock()
                job.done_event.set()
            self.cv.notify_all()

    def _take(self):
        """Next batch to run.  Among the jobs with a pending batch, the one
        that has received the least service so far (lattice sites of its
        batches already started) goes first, then the earliest arrival: a
        short job that arrives behind a long one waits for a worker to finish
        one batch, not for the long job, and jobs of equal service take turns.
        A batch runs only if its workspace fits the free budget.  The oldest
        job's next batch, once it has waited max_wait_s without fitting, is
        not overtaken until memory frees up for it."""
        with self.cv:
            while True:
                if self.closed and not self.pending:
                    return None
                pick = None
                if self.pending:
                    heads = {}  # job -> index of its next batch (pending is in submit order)
                    for i, b in enumerate(self.pending):
                        heads.setdefault(id(b.job), i)
                    head = self.pending[0]
                    if (self.in_flight_bytes + head.bytes > self.budget
                            and self.clock() - head.job.t_arrival >= self.max_wait_s):
                        order = [0]
                    else:
                        order = sorted(heads.values(),
                                       key=lambda i: (self.pending[i].job.attained, i))
                    for i in order:
                        if self.in_flight_bytes + self.pending[i].bytes <= self.budget:
                            pick = i
                            break
                if pick is not None:
                    b = self.pending[pick]
                    del self.pending[pick]
                    b.job.attained += b.job.L * b.job.L * b.n
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
            if job.t_start is None:
                job.t_start = self.clock()
            seeds = np.arange(job.seed + b.offset, job.seed + b.offset + b.n, dtype=np.uint64)
            err = None
            try:
                nj, nc = self.runner(job.L, job.k, seeds, b.bytes, w)
            except Exception as e:  # keep serving; the job reports the error
                err = f"{type(e).__name__}: {e}"
                nj = nc = None
            if not err and self.journal and not job.cancelled:
                self._journal_batch(job, b.offset, nj, nc)
            with self.cv:
                self.in_flight_bytes -= b.bytes
                self.running -= 1
                if job.cancelled:
                    pass  # its results are discarded
                elif err:
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
        done = [j for j in self.jobs if j.t_done is not None and not j.cancelled]
        lat = np.array([j.t_done - j.t_arrival for j in done])
        # latency = queue wait (arrival to first batch start) + service
        wait = np.array([(j.t_start if j.t_start is not None else j.t_done) - j.t_arrival
                         for j in done])

        def pct(a, q):
            return float(np.percentile(a, q)) if len(a) else None
        return dict(jobs=len(self.jobs), done=int(len(lat)),
                    p50_s=pct(lat, 50), p99_s=pct(lat, 99),
                    wait_p50_s=pct(wait, 50), wait_p99_s=pct(wait, 99),
                    service_p50_s=pct(lat - wait, 50), service_p99_s=pct(lat - wait, 99),
                    peak_in_flight_bytes=int(self.peak_bytes),
                    peak_concurrent_batches=int(self.peak_running))


class DeviceRunner:
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
        if rsa.rsa_tune(L, k, len(seeds), measure=False)["mode"] == "small":
            # small lattices: one CTA per sample, no workspace to bind
            return rsa.rsa_run_small(L, k, seeds, stream=st)
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
        for st in self.streams:
            st.synchronize()
        self.torch.cuda.empty_cache()


def gpu_budget(reserve_frac: float = 0.1, device: int = 0) -> int:
    """Free HBM now, less a reserve for torch, the library and other users.
    Blocks that torch's caching allocator holds but no tensor uses (an earlier
    server's workspaces) are returned to the device first."""
    import torch
    torch.cuda.empty_cache()
    free, total = torch.cuda.mem_get_info(device)
    return int(free - reserve_frac * total)


def make_server(workers: int = 4, budget_bytes: int | None = None, max_batch: int = 256,
                device: int = 0, journal: str | None = None):
    from . import rsa
    runner = DeviceRunner(workers, device)
    budget = gpu_budget(device=device) if budget_bytes is None else budget_bytes
    sch = Scheduler(runner, rsa.rsa_workspace_bytes, budget, workers, max_batch, journal=journal)
    sch.device_runner = runner
    return sch


def replay(jobs, workers: int = 4, budget_bytes: int | None = None, time_scale: float = 1.0,
           max_batch: int = 256, journal: str | None = None):
    """Submit jobs at their arrival times (seconds x time_scale) and wait."""
    sch = make_server(workers, budget_bytes, max_batch, journal=journal)
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
    sch.device_runner.close()
    st = sch.stats()
    samples = sum(j.n for j in subs)
    sites = sum(j.n * j.L * j.L for j in subs)
    st.update(wall_s=wall, samples=samples, samples_per_s=samples / wall, sites_per_s=sites / wall,
              errors=[j.error for j in subs if j.error])
    return st, subs


def _job_table(subs):
    return [dict(job=j.job, L=j.L, k=j.k, n=j.n, latency_s=round(j.t_done - j.t_arrival, 4),
                 wait_s=round((j.t_start or j.t_done) - j.t_arrival, 4)) for j in subs]


def main():
    from . import workloads
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--jobs", type=int, default=500)
    ap.add_argument("--rate", type=float, default=4.0, help="mean arrivals per second")
    ap.add_argument("--max-k", type=int, default=1024)
    ap.add_argument("--workers", type=int, default=4)
    ap.add_argument("--max-batch", type=int, default=256)
    ap.add_argument("--master-seed", type=int, default=1810)
    ap.add_argument("--capacity", action="store_true",
                    help="first replay every job at once to measure the capacity (jobs/s), "
                         "then replay the same jobs as a Poisson stream at --load x capacity")
    ap.add_argument("--load", type=float, default=0.7)
    ap.add_argument("--journal", default=None, help="JSON-lines journal of finished batches")
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
    spec = dict(n=args.jobs, max_k=args.max_k, master_seed=args.master_seed,
                workers=args.workers, max_batch=args.max_batch,
                job_mix="k uniform over powers of two in 1..max_k, L/k uniform over "
                        "{8, 16, 32} (L <= 32768), samples uniform in 16..256")
    if args.capacity:
        # closed loop: every job at t = 0; capacity = jobs / wall time
        jobs0 = workloads.served_jobs(args.jobs, 1.0, args.master_seed, max_k=args.max_k)
        burst = [dict(j, t=0.0) for j in jobs0]
        cap_st, _ = replay(burst, args.workers, max_batch=args.max_batch)
        capacity = args.jobs / cap_st["wall_s"]
        rate = args.load * capacity
        jobs = workloads.served_jobs(args.jobs, rate, args.master_seed, max_k=args.max_k)
        st, subs = replay(jobs, args.workers, max_batch=args.max_batch)
        st.update(metric="served RSA jobs: latency percentiles and throughput",
                  capacity=dict(jobs_per_s=capacity, samples_per_s=cap_st["samples_per_s"],
                                wall_s=cap_st["wall_s"]),
                  load=args.load, rate_per_s=rate, jobs_spec=spec,
                  slowest=sorted(_job_table(subs), key=lambda r: -r["latency_s"])[:10])
        print(json.dumps(st))
        return
    jobs = workloads.served_jobs(args.jobs, args.rate, args.master_seed, max_k=args.max_k)
    st, subs = replay(jobs, args.workers, max_batch=args.max_batch, journal=args.journal)
    spec.update(rate_per_s=args.rate)
    st.update(metric="served RSA jobs: latency percentiles and throughput", jobs_spec=spec)
    print(json.dumps(st))


if __name__ == "__main__":
    main()
