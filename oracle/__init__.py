"""CPU oracle for RSA of linear k-mers on an L x L torus -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its
``cpu_baseline`` leg and ``--impl reference`` arm) may import this package.
The product path (``paper_1810_06800_gb300``) never imports it, and this
package never imports the product path; the two share no code.

What it computes (arXiv:1810.06800):
  * RSA deposition to jamming (Sec. II.A, II.B) as the sequential scan of all
    2 L^2 (orientation, y, x) candidates in ascending splitmix64-priority
    order, accepting a candidate iff its k cells are free  -> n_j.
  * The number of k-mers on the lattice when a cluster first wraps the torus
    in one or both directions (Sec. II.C, II.D), by union-find over k-mers
    with displacement vectors and an exact "disagreeing lift" rule  -> n_c.
    The paper's own |x1-x2|+|y1-y2| > 2k test is evaluated alongside.
  * The configuration of the first m accepted k-mers: its cluster-size
    histogram (Sec. II.A Eq. CSD, Sec. III) and the directions in which its
    clusters wind round the torus  -> :func:`configuration`.

The C code lives in ``rsa_oracle.c``; :func:`build` compiles it with gcc.
The brute-force checkers in :mod:`oracle.brute` are independent pure-Python
restatements used to pin this code (BFS on the lifted lattice, the exact RSA
Markov chain, exhaustive jammed packings).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rsa_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "librsa_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle's C code into ``oracle/_build/librsa_oracle.so``."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or (
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
        tmp = _LIB_PATH + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    u32, u64, i64p = ctypes.c_uint32, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int64)
    vp = ctypes.c_void_p
    lib.oracle_mix64.restype = u64
    lib.oracle_mix64.argtypes = [u64]
    lib.oracle_base.restype = u64
    lib.oracle_base.argtypes = [u64]
    lib.oracle_key.restype = u64
    lib.oracle_key.argtypes = [u64, u64]
    lib.oracle_keys.restype = None
    lib.oracle_keys.argtypes = [u32, u64, vp]
    lib.oracle_scan.restype = ctypes.c_int64
    lib.oracle_scan.argtypes = [u32, u32, vp, vp, vp]
    lib.oracle_scan_seed.restype = ctypes.c_int64
    lib.oracle_scan_seed.argtypes = [u32, u32, u64, u32, vp, vp]
    lib.oracle_percolation.restype = ctypes.c_int64
    lib.oracle_percolation.argtypes = [u32, u32, vp, ctypes.c_int64, i64p]
    lib.oracle_sample.restype = ctypes.c_int
    lib.oracle_sample.argtypes = [u32, u32, u64, i64p, i64p, i64p]
    lib.oracle_sample_keys.restype = ctypes.c_int
    lib.oracle_sample_keys.argtypes = [u32, u32, vp, i64p, i64p, i64p, vp]
    lib.oracle_is_jammed.restype = ctypes.c_int
    lib.oracle_is_jammed.argtypes = [u32, u32, vp]
    lib.oracle_contacts.restype = ctypes.c_int
    lib.oracle_contacts.argtypes = [u32, u32, vp, ctypes.c_int64, i64p, i64p, i64p]
    lib.oracle_configuration.restype = ctypes.c_int
    lib.oracle_configuration.argtypes = [u32, u32, vp, ctypes.c_int64, vp, ctypes.c_int64,
                                         ctypes.POINTER(ctypes.c_int32)]
    lib.oracle_max_free_runs.restype = None
    lib.oracle_max_free_runs.argtypes = [u32, vp, ctypes.POINTER(u32), ctypes.POINTER(u32)]
    _lib = lib
    return lib


def _check_lk(L: int, k: int) -> None:
    if not (1 <= k <= L <= 32768):
        raise ValueError(f"need 1 <= k <= L <= 32768, got L={L} k={k}")


def mix64(z: int) -> int:
    """splitmix64 output finaliser (Stafford Mix13)."""
    return int(_load().oracle_mix64(z & (2**64 - 1)))


def base(seed: int) -> int:
    return int(_load().oracle_base(seed & (2**64 - 1)))


def keys(L: int, seed: int) -> np.ndarray:
    """All 2 L^2 candidate priorities of one sample, indexed (o*L + y)*L + x."""
    out = np.empty(2 * L * L, dtype=np.uint64)
    _load().oracle_keys(L, seed & (2**64 - 1), out.ctypes.data)
    return out


def scan(L: int, k: int, key_arr: np.ndarray):
    """Greedy scan.  Returns (accepted idx in scan order, occupancy uint8[L,L])."""
    _check_lk(L, k)
    key_arr = np.ascontiguousarray(key_arr, dtype=np.uint64)
    assert key_arr.size == 2 * L * L
    acc = np.empty(L * L // k + 1, dtype=np.uint32)
    occ = np.empty((L, L), dtype=np.uint8)
    nj = _load().oracle_scan(L, k, key_arr.ctypes.data, acc.ctypes.data, occ.ctypes.data)
    if nj == -1:
        raise ValueError("keys are not distinct")
    if nj < 0:
        raise MemoryError("oracle_scan failed")
    return acc[:nj].copy(), occ


def scan_seed(L: int, k: int, seed: int, parts: int = 1):
    """scan(L, k, keys(L, seed)) without holding the key array: the largest
    lattices need only the sort pairs, and with parts > 1 only those of one
    key range at a time (about 32 GB / parts at L = 32768, every key hashed
    parts + 1 times).  Returns (accepted idx, occupancy)."""
    _check_lk(L, k)
    acc = np.empty(L * L // k + 1, dtype=np.uint32)
    occ = np.empty((L, L), dtype=np.uint8)
    nj = _load().oracle_scan_seed(L, k, seed & (2**64 - 1), max(1, int(parts)), acc.ctypes.data,
                                  occ.ctypes.data)
    if nj < 0:
        raise MemoryError("oracle_scan_seed failed")
    return acc[:nj].copy(), occ


def percolation(L: int, k: int, accepted: np.ndarray):
    """(n_c exact, n_c by the paper's > 2k test) for accepted k-mers in order."""
    accepted = np.ascontiguousarray(accepted, dtype=np.uint32)
    ncp = ctypes.c_int64(0)
    nc = _load().oracle_percolation(L, k, accepted.ctypes.data, accepted.size,
                                    ctypes.byref(ncp))
    if nc < 0:
        raise MemoryError("oracle_percolation failed")
    return int(nc), int(ncp.value)


def sample(L: int, k: int, seed: int):
    """One seeded sample: (n_j, n_c, n_c by the paper's > 2k test)."""
    _check_lk(L, k)
    nj, nc, ncp = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    rc = _load().oracle_sample(L, k, seed & (2**64 - 1), ctypes.byref(nj),
                               ctypes.byref(nc), ctypes.byref(ncp))
    if rc != 0:
        raise RuntimeError(f"oracle_sample failed rc={rc}")
    return int(nj.value), int(nc.value), int(ncp.value)


def sample_keys(L: int, k: int, key_arr: np.ndarray):
    """Caller-supplied priorities: (n_j, n_c, n_c paper, accepted idx)."""
    _check_lk(L, k)
    key_arr = np.ascontiguousarray(key_arr, dtype=np.uint64)
    assert key_arr.size == 2 * L * L
    acc = np.empty(L * L // k + 1, dtype=np.uint32)
    nj, nc, ncp = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    rc = _load().oracle_sample_keys(L, k, key_arr.ctypes.data, ctypes.byref(nj),
                                    ctypes.byref(nc), ctypes.byref(ncp), acc.ctypes.data)
    if rc == -1:
        raise ValueError("keys are not distinct")
    if rc != 0:
        raise RuntimeError(f"oracle_sample_keys failed rc={rc}")
    return int(nj.value), int(nc.value), int(ncp.value), acc[:nj.value].copy()


def is_jammed(L: int, k: int, occ: np.ndarray) -> bool:
    occ = np.ascontiguousarray(occ, dtype=np.uint8)
    return bool(_load().oracle_is_jammed(L, k, occ.ctypes.data))


def contacts(L: int, k: int, accepted):
    """Interspecific contacts (n_x, n_y, n_xy) of a configuration (Sec. II.A)."""
    acc = np.ascontiguousarray(accepted, dtype=np.uint32)
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    rc = _load().oracle_contacts(L, k, acc.ctypes.data, acc.size, ctypes.byref(a),
                                 ctypes.byref(b), ctypes.byref(c))
    if rc != 0:
        raise MemoryError("oracle_contacts failed")
    return int(a.value), int(b.value), int(c.value)


def configuration(L: int, k: int, accepted, m: int):
    """The first m accepted k-mers (scan order) as a configuration
    (Sec. II.C, II.D): (counts, wrap_x, wrap_y) where counts[s] is the number
    of clusters of exactly s k-mers (length m + 1) and wrap_x / wrap_y say
    whether some cluster winds round the torus along x / y."""
    acc = np.ascontiguousarray(accepted, dtype=np.uint32)
    if not 0 <= m <= acc.size:
        raise ValueError("m out of range")
    counts = np.zeros(m + 1, dtype=np.int64)
    w = ctypes.c_int32(0)
    rc = _load().oracle_configuration(L, k, acc.ctypes.data, m, counts.ctypes.data, m + 1,
                                      ctypes.byref(w))
    if rc != 0:
        raise MemoryError("oracle_configuration failed rc=%d" % rc)
    return counts, bool(w.value & 1), bool(w.value & 2)


def max_free_runs(occ: np.ndarray):
    """(longest free run along rows, along columns), circular; the lattice is
    jammed for k-mers iff both are < k.  O(L^2), usable at any size."""
    occ = np.ascontiguousarray(occ, dtype=np.uint8)
    L = occ.shape[0]
    h, v = ctypes.c_uint32(), ctypes.c_uint32()
    _load().oracle_max_free_runs(L, occ.ctypes.data, ctypes.byref(h), ctypes.byref(v))
    return int(h.value), int(v.value)


def occupancy_from_accepted(L: int, k: int, accepted) -> np.ndarray:
    """uint8[L, L] occupancy of the given accepted candidates (idx)."""
    occ = np.zeros((L, L), dtype=np.uint8)
    acc = np.asarray(accepted, dtype=np.int64)
    o, r = np.divmod(acc, L * L)
    y, x = np.divmod(r, L)
    for i in range(k):
        h = o == 0
        occ[y[h], (x[h] + i) % L] += 1
        occ[(y[~h] + i) % L, x[~h]] += 1
    return occ


def samples(L: int, k: int, seeds, threads: int = 1):
    """Many seeded samples -> int64 arrays (n_j, n_c).  ctypes releases the
    GIL during each call, so ``threads`` > 1 runs samples on several cores."""
    seeds = [int(s) for s in seeds]
    _load()
    if threads <= 1:
        res = [sample(L, k, s) for s in seeds]
    else:
        with ThreadPoolExecutor(max_workers=threads) as ex:
            res = list(ex.map(lambda s: sample(L, k, s), seeds))
    nj = np.array([r[0] for r in res], dtype=np.int64)
    nc = np.array([r[1] for r in res], dtype=np.int64)
    return nj, nc
