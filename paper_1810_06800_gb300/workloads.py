"""Seeded synthetic inputs shared by the tests, the benchmark and the
serving driver.  This module holds no arithmetic of the method: it only
names sample seeds, job streams and caller-supplied priority orders.

The paper's runs use L = 100k lattices (Sec. II.A); the workloads below are
the same model at sizes one GPU holds, with L/k between 8 and 32."""
from __future__ import annotations

import numpy as np

# (name, L, k, seeds) -- seeds are the per-sample splitmix64 seeds
PLAIN_SMALL = dict(name="L64_k4_x100", L=64, k=4, seeds=list(range(1, 101)))
PLAIN_SCALE = dict(name="L1024_k32_x1000", L=1024, k=32, seeds=list(range(1, 1001)))
BATCHED_UNEVEN = [dict(name=f"L{16 * k}_k{k}_x256", L=16 * k, k=k, seeds=list(range(1, 257)))
                  for k in (2, 8, 64, 512)]
LARGE_K = dict(name="L32768_k4096_x8", L=32768, k=4096, seeds=list(range(1, 9)))


def served_jobs(n_jobs: int = 500, rate_per_s: float = 50.0, master_seed: int = 1810,
                max_k: int = 1024, samples_lo: int = 16, samples_hi: int = 256):
    """Poisson stream of jobs: k uniform over powers of two in [1, max_k],
    L/k uniform over {8, 16, 32} (L capped at 32768), samples uniform in
    [samples_lo, samples_hi], a 63-bit random seed; exponential gaps of mean
    1/rate_per_s.  Returns a list of dicts with arrival times in seconds."""
    rng = np.random.default_rng(master_seed)
    ks = [1 << i for i in range(int(np.log2(max_k)) + 1)]
    t = 0.0
    jobs = []
    for j in range(n_jobs):
        t += float(rng.exponential(1.0 / rate_per_s))
        k = int(rng.choice(ks))
        L = min(int(rng.choice([8, 16, 32])) * k, 32768)
        n = int(rng.integers(samples_lo, samples_hi + 1))
        seed = int(rng.integers(0, 2**62))
        jobs.append(dict(job=j, t=t, L=L, k=k, n=n, seed=seed))
    return jobs


def permutation_keys(L: int, rng_seed: int) -> np.ndarray:
    """2 L^2 distinct priorities: a uniformly random permutation of 1..2L^2."""
    rng = np.random.default_rng(rng_seed)
    return (rng.permutation(2 * L * L) + 1).astype(np.uint64)


def monotone_keys(L: int, descending: bool = False) -> np.ndarray:
    """Adversarial order: priority increases with the candidate index
    (row-major scan of horizontal then vertical candidates)."""
    n = 2 * L * L
    k = np.arange(1, n + 1, dtype=np.uint64)
    return k[::-1].copy() if descending else k


def wide_keys(L: int, rng_seed: int) -> np.ndarray:
    """2 L^2 distinct priorities spread over the full 64-bit range, including
    0, 1, 2^63 - 1, 2^63 and 2^64 - 2 (never 2^64 - 1)."""
    rng = np.random.default_rng(rng_seed)
    n = 2 * L * L
    special = [0, 1, 2**63 - 1, 2**63, 2**64 - 2][:n]
    v = set(special)
    rest = []
    while len(special) + len(rest) < n:
        for x in rng.integers(0, 2**64 - 1, size=n, dtype=np.uint64):
            x = int(x)
            if x not in v:
                v.add(x)
                rest.append(x)
    arr = np.array(special + rest[:n - len(special)], dtype=np.uint64)
    rng.shuffle(arr)
    return arr


def two_band_packing() -> np.ndarray:
    """A jammed packing of k = 4 mers on an L = 40 = 10k torus made of two
    clusters, the size of the paper's example of a jammed state with several
    clusters (Sec. III.C).  Returned as horizontal candidate indices y*L + x.

    Along every row the cells with (x - y) mod 40 in {0, 20} stay empty: two
    diagonal lines that no 4-neighbour step crosses, so they cut the torus
    into two diagonal bands of 19 cells per row.  In each band an even row
    holds 4-mers at offsets 1-4, 6-9, 11-14, 16-19 from its diagonal and an
    odd row at 2-5, 7-10, 12-15, 16-19.  The odd-row 4-mers span the gaps
    between the even-row 4-mers above and below them, so each band is one
    cluster, winding once in x and once in y.  No row or column holds more than two free cells in a
    row, so no 4-mer fits anywhere."""
    L = 40
    out = []
    for y in range(L):
        starts = (1, 6, 11, 16) if y % 2 == 0 else (2, 7, 12, 16)
        for band in (0, 20):
            out.extend(y * L + (y + band + s) % L for s in starts)
    return np.array(out, dtype=np.uint32)


def packing_first_keys(L: int, first: np.ndarray, rng_seed: int) -> np.ndarray:
    """2 L^2 distinct priorities in which the candidates `first` take the
    smallest ones (1 .. len(first), in random order) and every other
    candidate a larger one (random order).  When `first` is a jammed packing
    the greedy scan accepts exactly it."""
    rng = np.random.default_rng(rng_seed)
    n = 2 * L * L
    first = np.asarray(first, dtype=np.int64)
    rest = np.setdiff1d(np.arange(n), first)
    keys = np.empty(n, dtype=np.uint64)
    keys[first] = rng.permutation(first.size) + 1
    keys[rest] = rng.permutation(rest.size) + 1 + first.size
    return keys
