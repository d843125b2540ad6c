"""Python binding of the C ABI in ``include/rsa.h`` (argument marshalling only).

Every step of the method runs in the CUDA library ``_lib/librsa_gb300.so``;
this module never computes any part of it.  If the library is missing the
first call raises, so nothing can silently fall back to the CPU.
PyTorch is used only for the CUDA stream and, optionally, for device memory
bound as the library's workspace.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

RSA_OK, RSA_EINVAL, RSA_ENOMEM, RSA_ECUDA, RSA_ETIMEOUT, RSA_ENOWRAP, RSA_ESTATE = (
    0, -1, -2, -3, -4, -5, -6)
_NAMES = {RSA_EINVAL: "RSA_EINVAL", RSA_ENOMEM: "RSA_ENOMEM", RSA_ECUDA: "RSA_ECUDA",
          RSA_ETIMEOUT: "RSA_ETIMEOUT", RSA_ENOWRAP: "RSA_ENOWRAP", RSA_ESTATE: "RSA_ESTATE"}
SYMBOLS = ["rsa_create", "rsa_run_batch", "rsa_run_seeds", "rsa_run_keys", "rsa_run_static",
           "rsa_results",
           "rsa_sample_stats", "rsa_contacts", "rsa_cluster_sizes", "rsa_wrap_dirs", "rsa_accepted",
           "rsa_workspace_bytes", "rsa_bind_workspace", "rsa_test_caps",
           "rsa_run_small", "rsa_run_mix", "rsa_tune", "rsa_set_rounds_per_check",
           "rsa_set_window_threads",
           "rsa_mix_release", "rsa_mix_launches", "rsa_profile", "rsa_kernel_stats", "rsa_work_stats", "rsa_destroy", "rsa_kernel_name",
           "rsa_last_error"]

_lib = None


RSA_MODE_GLOBAL, RSA_MODE_SMALL = 0, 1


class TuneT(ctypes.Structure):
    """rsa_tune_t: how a shape runs (see include/rsa.h)."""
    _fields_ = [("mode", ctypes.c_uint32), ("threads", ctypes.c_uint32),
                ("rounds_per_check", ctypes.c_uint32), ("window_threads", ctypes.c_uint32),
                ("ms_per_sample", ctypes.c_double)]


class RSAError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


def library_path() -> str:
    return _build.LIB


def load():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"CUDA library {_build.LIB} is missing: run "
                           "paper_1810_06800_gb300.build.build() (or __graft_entry__.build())")
    lib = ctypes.CDLL(_build.LIB)
    u32, u64, vp, ip = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int
    lib.rsa_create.argtypes = [u32, u32, u64, ctypes.POINTER(vp)]
    lib.rsa_run_batch.argtypes = [vp, u32, vp]
    lib.rsa_run_seeds.argtypes = [vp, vp, u32, vp]
    lib.rsa_run_keys.argtypes = [vp, vp, vp]
    lib.rsa_run_static.argtypes = [u32, u32, vp, u32, vp, vp, vp]
    lib.rsa_results.argtypes = [vp, vp, vp, u32]
    lib.rsa_sample_stats.argtypes = [vp, vp, vp, vp, vp, u32]
    lib.rsa_contacts.argtypes = [vp, vp, vp, vp, u32]
    lib.rsa_cluster_sizes.argtypes = [vp, u32, u32, vp, u32]
    lib.rsa_wrap_dirs.argtypes = [vp, u32, u32, ctypes.POINTER(u32), ctypes.POINTER(u32)]
    lib.rsa_accepted.argtypes = [vp, u32, vp, u32, ctypes.POINTER(u32)]
    lib.rsa_workspace_bytes.argtypes = [u32, u32, u32, ctypes.POINTER(u64)]
    lib.rsa_bind_workspace.argtypes = [vp, vp, u64]
    lib.rsa_test_caps.argtypes = [vp, u32, u32, u32, u32]
    lib.rsa_run_small.argtypes = [vp, vp, vp, u32, u32, vp, vp, vp]
    lib.rsa_run_mix.argtypes = [vp, vp, vp, u32, vp, vp, vp]
    lib.rsa_tune.argtypes = [u32, u32, u32, ip, ctypes.POINTER(TuneT)]
    lib.rsa_set_rounds_per_check.argtypes = [vp, u32]
    lib.rsa_set_window_threads.argtypes = [vp, u32]
    lib.rsa_mix_release.argtypes = []
    lib.rsa_mix_launches.argtypes = []
    lib.rsa_destroy.argtypes = [vp]
    lib.rsa_destroy.restype = None
    lib.rsa_profile.argtypes = [vp, ip]
    lib.rsa_kernel_stats.argtypes = [vp, vp, vp, u32]
    lib.rsa_work_stats.argtypes = [vp, vp, u32]
    lib.rsa_kernel_name.argtypes = [u32]
    lib.rsa_kernel_name.restype = ctypes.c_char_p
    lib.rsa_last_error.argtypes = []
    lib.rsa_last_error.restype = ctypes.c_char_p
    for name in SYMBOLS[:-3]:
        getattr(lib, name).restype = ip
    lib.rsa_mix_release.restype = None
    lib.rsa_mix_launches.restype = ctypes.c_ulonglong
    _lib = lib
    return lib


def _check(rc):
    if rc != 0:
        raise RSAError(rc, load().rsa_last_error().decode())
    return rc


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            return ctypes.c_void_p(0)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def rsa_create(L: int, k: int, seed: int = 1):
    h = ctypes.c_void_p()
    _check(load().rsa_create(L, k, seed & (2**64 - 1), ctypes.byref(h)))
    return h


def rsa_run_batch(h, n_samples: int, stream=None):
    return _check(load().rsa_run_batch(h, n_samples, _stream_ptr(stream)))


def rsa_run_seeds(h, seeds, stream=None):
    a = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint64))
    return _check(load().rsa_run_seeds(h, a.ctypes.data, a.size, _stream_ptr(stream)))


def rsa_run_keys(h, keys, stream=None):
    a = np.ascontiguousarray(np.asarray(keys, dtype=np.uint64))
    return _check(load().rsa_run_keys(h, a.ctypes.data, _stream_ptr(stream)))


def rsa_run_static(L: int, k: int, seeds, stream=None):
    """Workspace-free run: no handle, no device allocation (for callers that
    cannot allocate device memory); same results as rsa_run_seeds +
    rsa_results.  Returns (n_j, n_c)."""
    a = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint64))
    nj = np.zeros(a.size, dtype=np.uint32)
    nc = np.zeros(a.size, dtype=np.uint32)
    _check(load().rsa_run_static(L, k, a.ctypes.data, a.size, nj.ctypes.data, nc.ctypes.data,
                                 _stream_ptr(stream)))
    return nj, nc


def _shape_arrays(L, k, seeds):
    seeds = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint64))
    n = seeds.size
    Ls = np.ascontiguousarray(np.broadcast_to(np.asarray(L, dtype=np.uint32), (n,)))
    ks = np.ascontiguousarray(np.broadcast_to(np.asarray(k, dtype=np.uint32), (n,)))
    return Ls, ks, seeds


def rsa_run_small(L, k, seeds, threads: int = 0, stream=None):
    """Small lattices, one CTA per sample, any mix of shapes in one launch.
    L and k are scalars or per-sample arrays.  Returns (n_j, n_c)."""
    Ls, ks, sd = _shape_arrays(L, k, seeds)
    nj = np.zeros(sd.size, dtype=np.uint32)
    nc = np.zeros(sd.size, dtype=np.uint32)
    _check(load().rsa_run_small(Ls.ctypes.data, ks.ctypes.data, sd.ctypes.data, sd.size, threads,
                                nj.ctypes.data, nc.ctypes.data, _stream_ptr(stream)))
    return nj, nc


def rsa_run_mix(L, k, seeds, stream=None):
    """A batch of samples of uneven shapes (per-sample L, k, seed arrays),
    each shape run the way rsa_tune picks.  Returns (n_j, n_c)."""
    Ls, ks, sd = _shape_arrays(L, k, seeds)
    nj = np.zeros(sd.size, dtype=np.uint32)
    nc = np.zeros(sd.size, dtype=np.uint32)
    _check(load().rsa_run_mix(Ls.ctypes.data, ks.ctypes.data, sd.ctypes.data, sd.size,
                              nj.ctypes.data, nc.ctypes.data, _stream_ptr(stream)))
    return nj, nc


def rsa_mix_release():
    load().rsa_mix_release()


def rsa_mix_launches() -> int:
    """Kernel launches of rsa_run_small and rsa_run_mix since the last call."""
    return int(load().rsa_mix_launches())


def rsa_tune(L: int, k: int, n: int, measure: bool = True) -> dict:
    t = TuneT()
    _check(load().rsa_tune(L, k, n, 1 if measure else 0, ctypes.byref(t)))
    return dict(mode="small" if t.mode == RSA_MODE_SMALL else "global", threads=t.threads,
                rounds_per_check=t.rounds_per_check, window_threads=t.window_threads,
                ms_per_sample=t.ms_per_sample)


def rsa_set_rounds_per_check(h, rounds: int):
    return _check(load().rsa_set_rounds_per_check(h, rounds))


def rsa_set_window_threads(h, threads: int):
    return _check(load().rsa_set_window_threads(h, threads))


def rsa_results(h, n: int, check: bool = True):
    nj = np.zeros(n, dtype=np.uint32)
    nc = np.zeros(n, dtype=np.uint32)
    rc = load().rsa_results(h, nj.ctypes.data, nc.ctypes.data, n)
    if check:
        _check(rc)
    return nj, nc


def rsa_sample_stats(h, n: int):
    r = np.zeros(n, dtype=np.uint32)
    p = np.zeros(n, dtype=np.uint32)
    e = np.zeros(n, dtype=np.uint32)
    s = np.zeros(n, dtype=np.int32)
    _check(load().rsa_sample_stats(h, r.ctypes.data, p.ctypes.data, e.ctypes.data,
                                   s.ctypes.data, n))
    return dict(rounds=r, probes=p, edges=e, status=s)


def rsa_contacts(h, n: int):
    """(n_x, n_y, n_xy) uint32 arrays of the last run's first n samples."""
    a = np.zeros(n, dtype=np.uint32)
    b = np.zeros(n, dtype=np.uint32)
    c = np.zeros(n, dtype=np.uint32)
    _check(load().rsa_contacts(h, a.ctypes.data, b.ctypes.data, c.ctypes.data, n))
    return a, b, c


def rsa_cluster_sizes(h, sample: int, m: int):
    """counts[s] = clusters of exactly s k-mers among the first m accepted
    k-mers of `sample` (uint32, length m + 1)."""
    out = np.zeros(m + 1, dtype=np.uint32)
    _check(load().rsa_cluster_sizes(h, sample, m, out.ctypes.data, m + 1))
    return out


def rsa_wrap_dirs(h, sample: int, m: int):
    """(winds along x, winds along y) for the first m accepted k-mers."""
    wx, wy = ctypes.c_uint32(), ctypes.c_uint32()
    _check(load().rsa_wrap_dirs(h, sample, m, ctypes.byref(wx), ctypes.byref(wy)))
    return bool(wx.value), bool(wy.value)


def rsa_accepted(h, sample: int):
    cnt = ctypes.c_uint32()
    _check(load().rsa_accepted(h, sample, None, 0, ctypes.byref(cnt)))
    out = np.zeros(max(cnt.value, 1), dtype=np.uint32)
    _check(load().rsa_accepted(h, sample, out.ctypes.data, cnt.value, ctypes.byref(cnt)))
    return out[:cnt.value]


def rsa_workspace_bytes(L: int, k: int, n_samples: int) -> int:
    b = ctypes.c_uint64()
    _check(load().rsa_workspace_bytes(L, k, n_samples, ctypes.byref(b)))
    return int(b.value)


def rsa_bind_workspace(h, tensor_or_ptr, nbytes: int | None = None):
    if tensor_or_ptr is None:
        return _check(load().rsa_bind_workspace(h, None, 0))
    if hasattr(tensor_or_ptr, "data_ptr"):
        ptr = tensor_or_ptr.data_ptr()
        nbytes = tensor_or_ptr.numel() * tensor_or_ptr.element_size()
    else:
        ptr = int(tensor_or_ptr)
    return _check(load().rsa_bind_workspace(h, ctypes.c_void_p(ptr), int(nbytes)))


def rsa_test_caps(h, round_cap: int = 0, uf_steps: int = 0, probe_cap: int = 0,
                  edge_cap: int = 0):
    """TEST ONLY: lower the device loop caps of later runs (0 = default)."""
    return _check(load().rsa_test_caps(h, round_cap, uf_steps, probe_cap, edge_cap))


def rsa_profile(h, enable: bool = True):
    return _check(load().rsa_profile(h, 1 if enable else 0))


def rsa_kernel_name(kind: int) -> str:
    return load().rsa_kernel_name(kind).decode()


def rsa_kernel_stats(h):
    """{kernel name: (total ms, launches)} since the previous call."""
    n = 0
    while rsa_kernel_name(n):
        n += 1
    ms = np.zeros(n, dtype=np.float64)
    cnt = np.zeros(n, dtype=np.uint64)
    _check(load().rsa_kernel_stats(h, ms.ctypes.data, cnt.ctypes.data, n))
    return {rsa_kernel_name(i): (float(ms[i]), int(cnt[i])) for i in range(n)}


def rsa_work_stats(h):
    """Round-pass work since the previous call: the four counters under their
    tile-path names, and as ``raw`` (their long-k path meaning differs; see
    include/rsa.h)."""
    out = np.zeros(4, dtype=np.uint64)
    _check(load().rsa_work_stats(h, out.ctypes.data, 4))
    return dict(cmin_cells=int(out[0]), cmin_keys=int(out[1]), accept_cells=int(out[2]),
                accept_keys=int(out[3]), raw=[int(v) for v in out])


def rsa_destroy(h):
    if h is not None and h.value:
        load().rsa_destroy(h)


def rsa_last_error() -> str:
    return load().rsa_last_error().decode()


class Lattice:
    """Convenience owner of one handle: ``Lattice(L, k).run(seeds)``."""

    def __init__(self, L: int, k: int, seed: int = 1):
        self.L, self.k = L, k
        self.h = rsa_create(L, k, seed)

    def run(self, seeds, stream=None):
        seeds = np.asarray(seeds, dtype=np.uint64)
        rsa_run_seeds(self.h, seeds, stream)
        return rsa_results(self.h, seeds.size)

    def run_keys(self, keys, stream=None):
        rsa_run_keys(self.h, keys, stream)
        return rsa_results(self.h, 1)

    def stats(self, n):
        return rsa_sample_stats(self.h, n)

    def contacts(self, n):
        return rsa_contacts(self.h, n)

    def accepted(self, sample=0):
        return rsa_accepted(self.h, sample)

    def _m(self, sample, m):
        if m is None:   # the percolating state: m = n_c
            _, nc = rsa_results(self.h, sample + 1)
            m = int(nc[sample])
        return m

    def cluster_sizes(self, sample=0, m=None):
        """Cluster-size histogram of the first m k-mers (default m = n_c)."""
        return rsa_cluster_sizes(self.h, sample, self._m(sample, m))

    def wrap_dirs(self, sample=0, m=None):
        """Winding directions of the first m k-mers (default m = n_c)."""
        return rsa_wrap_dirs(self.h, sample, self._m(sample, m))

    def close(self):
        rsa_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            if self.h is not None:
                self.close()
        except Exception:
            pass
