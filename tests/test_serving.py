"""Continuous-batching scheduler (host logic on CPU with a fake runner) and
the served path on the GPU: every job's results are identical alone and in
a mix, and match the oracle."""
import itertools
import threading
import time

import numpy as np
import pytest

from paper_1810_06800_gb300 import serve


def _fake_ws(L, k, n):
    return L * L * n


def _fake_runner(log, lock, delay=0.002):
    def run(L, k, seeds, nbytes, w):
        with lock:
            log.append(("start", w, nbytes))
        time.sleep(delay)
        # deterministic stand-in results: functions of (L, k, seed) only
        s = seeds.astype(np.uint64)
        nj = ((s * np.uint64(2654435761) + np.uint64(L * 131 + k)) % np.uint64(1000)).astype(np.uint32)
        nc = (nj // 2).astype(np.uint32)
        with lock:
            log.append(("end", w, nbytes))
        return nj, nc
    return run


def _expected(L, k, seed, n):
    s = np.arange(seed, seed + n, dtype=np.uint64)
    nj = ((s * np.uint64(2654435761) + np.uint64(L * 131 + k)) % np.uint64(1000)).astype(np.uint32)
    return nj, (nj // 2).astype(np.uint32)


def test_scheduler_splits_batches_and_respects_the_budget():
    log, lock = [], threading.Lock()
    budget = 64 * 64 * 10          # ten 64x64 samples in flight at most
    sch = serve.Scheduler(_fake_runner(log, lock), _fake_ws, budget, workers=3, max_batch=8)
    jobs = [sch.submit(serve.Job(i, L, k, n, seed))
            for i, (L, k, n, seed) in enumerate([(64, 4, 30, 1), (32, 2, 5, 100), (64, 8, 17, 7),
                                                 (16, 1, 40, 3)])]
    for j in jobs:
        assert j.done_event.wait(10)
    sch.close()
    for j in jobs:
        wj, wc = _expected(j.L, j.k, j.seed, j.n)
        assert np.array_equal(j.nj, wj) and np.array_equal(j.nc, wc)
    # in-flight workspace never exceeded the budget, and batches overlapped
    inflight = peak = 0
    for ev, _, b in log:
        inflight += b if ev == "start" else -b
        peak = max(peak, inflight)
    assert peak <= budget
    st = sch.stats()
    assert st["done"] == 4 and st["peak_in_flight_bytes"] <= budget
    assert st["peak_concurrent_batches"] >= 2


def test_batches_fit_a_workers_share_of_the_budget():
    # 4 workers share an 8 MiB budget: a batch takes at most 2 MiB, so every
    # worker can hold one at once; a single sample may still use it all
    sch = serve.Scheduler(lambda *a: None, _fake_ws, budget_bytes=8 * 1024 * 1024, workers=4,
                          max_batch=256)
    assert sch.batch_size(1024, 32, 100) == 2
    assert sch.batch_size(2048, 32, 100) == 1
    sch.close()


def test_batch_size_shrinks_to_fit_the_budget():
    sch = serve.Scheduler(lambda *a: None, _fake_ws, budget_bytes=1024 * 1024 * 3, workers=1,
                          max_batch=256)
    assert sch.batch_size(1024, 32, 100) == 2   # 1 MiB per sample, 3 MiB budget
    with pytest.raises(MemoryError):
        sch.batch_size(4096, 32, 1)
    sch.close()


def test_job_alone_and_in_a_mix_agree_fake():
    log, lock = [], threading.Lock()
    specs = [(64, 4, 12, 5), (32, 2, 9, 50), (128, 8, 6, 9)]
    alone = []
    for i, (L, k, n, seed) in enumerate(specs):
        sch = serve.Scheduler(_fake_runner(log, lock), _fake_ws, 10**9, workers=1, max_batch=4)
        j = sch.submit(serve.Job(i, L, k, n, seed))
        j.done_event.wait(10)
        sch.close()
        alone.append((j.nj.copy(), j.nc.copy()))
    sch = serve.Scheduler(_fake_runner(log, lock), _fake_ws, 10**9, workers=3, max_batch=4)
    mixed = [sch.submit(serve.Job(i, *sp)) for i, sp in enumerate(specs)]
    for j in mixed:
        j.done_event.wait(10)
    sch.close()
    for (aj, ac), j in zip(alone, mixed):
        assert np.array_equal(aj, j.nj) and np.array_equal(ac, j.nc)


@pytest.mark.gpu
def test_served_jobs_alone_and_in_a_mix_match():
    import oracle
    from paper_1810_06800_gb300 import rsa
    specs = [(64, 4, 24, 1), (96, 16, 10, 300), (128, 64, 6, 77), (100, 3, 8, 9), (32, 2, 40, 5)]
    alone = []
    for L, k, n, seed in specs:
        lat = rsa.Lattice(L, k)
        alone.append(lat.run(np.arange(seed, seed + n, dtype=np.uint64)))
        lat.close()
    sch = serve.make_server(workers=3, budget_bytes=256 << 20, max_batch=8)
    jobs = [sch.submit(serve.Job(i, *sp)) for i, sp in enumerate(specs)]
    for j in jobs:
        assert j.done_event.wait(120)
    sch.close()
    sch.device_runner.close()
    for (aj, ac), j in zip(alone, jobs):
        assert j.error is None
        assert np.array_equal(aj, j.nj) and np.array_equal(ac, j.nc)
    assert sch.stats()["peak_concurrent_batches"] >= 2
    # and the oracle agrees on a few samples of each job
    for j in jobs:
        for i in range(min(3, j.n)):
            wj, wc, _ = oracle.sample(j.L, j.k, j.seed + i)
            assert (int(j.nj[i]), int(j.nc[i])) == (wj, wc)


def test_cancel_drops_pending_batches_and_keeps_serving_the_rest():
    log, lock = [], threading.Lock()
    sch = serve.Scheduler(_fake_runner(log, lock, delay=0.02), _fake_ws, 64 * 64 * 4, workers=2,
                          max_batch=2)
    big = sch.submit(serve.Job(0, 64, 4, 40, 1))       # 20 batches of 2
    small = sch.submit(serve.Job(1, 32, 2, 6, 50))
    time.sleep(0.05)                                    # a few batches have started
    sch.cancel(big)
    assert big.done_event.wait(10) and small.done_event.wait(10)
    sch.close()
    assert big.cancelled and big.error == "cancelled"
    started = sum(1 for ev, _, b in log if ev == "start" and b == 64 * 64 * 2)
    assert 1 <= started < 20                            # the rest never ran
    wj, wc = _expected(32, 2, 50, 6)
    assert small.error is None and np.array_equal(small.nj, wj) and np.array_equal(small.nc, wc)
    assert sch.in_flight_bytes == 0 and sch.running == 0
    assert sch.stats()["done"] == 1                     # latency stats leave the cancelled job out


def test_journal_restart_runs_only_the_missing_samples(tmp_path):
    journal = str(tmp_path / "served.jsonl")
    log, lock = [], threading.Lock()
    sch = serve.Scheduler(_fake_runner(log, lock, delay=0.02), _fake_ws, 64 * 64 * 2, workers=1,
                          max_batch=4, journal=journal)
    a = sch.submit(serve.Job(0, 64, 4, 24, 1))
    b = sch.submit(serve.Job(1, 32, 2, 8, 9))
    time.sleep(0.07)
    sch.cancel(a)                                       # the "crash": part of job 0 is journaled
    assert a.done_event.wait(10) and b.done_event.wait(10)
    sch.close()
    first_batches = sum(1 for ev, _, _ in log if ev == "start")
    # restart with the same journal: finished samples come from it
    log2 = []
    sch2 = serve.Scheduler(_fake_runner(log2, lock), _fake_ws, 64 * 64 * 2, workers=1,
                           max_batch=4, journal=journal)
    a2 = sch2.submit(serve.Job(0, 64, 4, 24, 1))
    b2 = sch2.submit(serve.Job(1, 32, 2, 8, 9))
    assert a2.done_event.wait(10) and b2.done_event.wait(10)
    sch2.close()
    for j in (a2, b2):
        wj, wc = _expected(j.L, j.k, j.seed, j.n)
        assert j.error is None and np.array_equal(j.nj, wj) and np.array_equal(j.nc, wc)
    assert b2.from_journal == 8 and 0 < a2.from_journal < 24
    ran = sum(n for ev, _, n in log2 if ev == "start") // (64 * 64)
    assert ran == 24 - a2.from_journal                  # only the missing samples ran
    assert first_batches >= 1


@pytest.mark.gpu
def test_served_large_k_jobs_alone_and_in_a_mix_match():
    # shapes of the served stream's upper range (k up to 1024, L/k in
    # {8, 16, 32}) next to small-lattice jobs run one CTA per sample
    import oracle
    from paper_1810_06800_gb300 import rsa
    specs = [(8192, 1024, 2, 1), (2048, 256, 3, 5), (1024, 64, 4, 7), (64, 4, 20, 3),
             (32, 1, 10, 9), (16, 2, 12, 4)]
    alone = []
    for L, k, n, seed in specs:
        lat = rsa.Lattice(L, k)
        alone.append(lat.run(np.arange(seed, seed + n, dtype=np.uint64)))
        lat.close()
    sch = serve.make_server(workers=4, budget_bytes=16 << 30, max_batch=4)
    jobs = [sch.submit(serve.Job(i, *sp)) for i, sp in enumerate(specs)]
    for j in jobs:
        assert j.done_event.wait(300)
    sch.close()
    sch.device_runner.close()
    for (aj, ac), j in zip(alone, jobs):
        assert j.error is None
        assert np.array_equal(aj, j.nj) and np.array_equal(ac, j.nc)
    for j in jobs:
        if j.L <= 1024:
            wj, wc = oracle.samples(j.L, j.k, list(range(j.seed, j.seed + j.n)))
            assert np.array_equal(j.nj, wj.astype(np.uint32)) and np.array_equal(j.nc, wc.astype(np.uint32))


def test_short_job_does_not_wait_behind_a_long_one():
    # one worker; a 20-batch job arrives first, a one-batch job just after:
    # the short job runs after at most two of the long job's batches
    log, lock = [], threading.Lock()
    sch = serve.Scheduler(_fake_runner(log, lock, delay=0.02), _fake_ws, 10**9, workers=1,
                          max_batch=2)
    long_job = sch.submit(serve.Job(0, 64, 4, 40, 1))
    short = sch.submit(serve.Job(1, 32, 2, 2, 50))
    assert short.done_event.wait(10) and long_job.done_event.wait(10)
    sch.close()
    starts = [b for ev, _, b in log if ev == "start"]
    assert starts.index(32 * 32 * 2) <= 2
    assert short.t_done < long_job.t_done
    wj, wc = _expected(32, 2, 50, 2)
    assert np.array_equal(short.nj, wj) and np.array_equal(short.nc, wc)
    wj, wc = _expected(64, 4, 1, 40)
    assert np.array_equal(long_job.nj, wj) and np.array_equal(long_job.nc, wc)


def test_jobs_of_equal_service_take_turns():
    # two equal jobs on one worker alternate batch by batch
    log, lock = [], threading.Lock()
    sch = serve.Scheduler(_fake_runner(log, lock, delay=0.005), _fake_ws, 10**9, workers=1,
                          max_batch=1)
    a = sch.submit(serve.Job(0, 16, 2, 6, 1))
    b = sch.submit(serve.Job(1, 17, 2, 6, 1))
    assert a.done_event.wait(10) and b.done_event.wait(10)
    sch.close()
    sizes = [n for ev, _, n in log if ev == "start"]
    # after the first batch (taken before job b existed, or a's by arrival)
    # neither job runs three batches in a row
    runs = max(len(list(g)) for _, g in itertools.groupby(sizes))
    assert runs <= 2
