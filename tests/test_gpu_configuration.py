"""The configuration of the first m accepted k-mers on the GPU against the
oracle, through the C ABI: the cluster-size histogram (Eq. CSD) and the
winding directions (Sec. II.D) must be identical for m = 0, 1, n_c - 1, n_c,
n_j and random m, on the tile, line and general round paths, with seeded and
caller-supplied priorities."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1810_06800_gb300 import rsa, workloads

pytestmark = pytest.mark.gpu


def _ms(nj, nc, rng):
    return sorted({0, 1, max(nc - 1, 0), nc, nj, int(rng.integers(1, nj + 1)),
                   int(rng.integers(1, nj + 1))})


def _compare(lat, i, L, k, acc, ms):
    for m in ms:
        want, wx, wy = oracle.configuration(L, k, acc, m)
        got = lat.cluster_sizes(i, m)
        assert got.size == m + 1
        assert np.array_equal(got.astype(np.int64), want), (L, k, i, m)
        assert lat.wrap_dirs(i, m) == (wx, wy), (L, k, i, m)


@pytest.mark.parametrize("L,k", [(1, 1), (2, 1), (2, 2), (3, 3), (5, 2), (8, 8), (16, 3),
                                 (33, 32), (64, 4), (96, 16), (100, 3), (128, 100),
                                 (256, 1), (320, 320), (1024, 32), (2048, 256)])
def test_configuration_matches_oracle(L, k):
    seeds = list(range(1, 5 if L <= 1024 else 3))
    rng = np.random.default_rng(L * 131 + k)
    lat = rsa.Lattice(L, k)
    nj, nc = lat.run(seeds)
    for i, s in enumerate(seeds):
        acc, _ = oracle.scan(L, k, oracle.keys(L, s))
        assert acc.size == nj[i]
        _compare(lat, i, L, k, acc, _ms(int(nj[i]), int(nc[i]), rng))
    lat.close()


@pytest.mark.parametrize("kind", ["perm", "monotone", "descending", "wide"])
def test_configuration_with_caller_keys(kind):
    # priorities packed into the lowest byte range (perm, monotone) or spread
    # over all 64 bits (wide) exercise every pass of the radix select
    L, k = 32, 4
    if kind == "perm":
        keys = workloads.permutation_keys(L, 7)
    elif kind == "wide":
        keys = workloads.wide_keys(L, 7)
    else:
        keys = workloads.monotone_keys(L, descending=(kind == "descending"))
    lat = rsa.Lattice(L, k)
    nj, nc = lat.run_keys(keys)
    _, _, _, acc = oracle.sample_keys(L, k, keys)
    _compare(lat, 0, L, k, acc, _ms(int(nj[0]), int(nc[0]), np.random.default_rng(3)))
    lat.close()


def test_percolating_and_jamming_states():
    # Sec. III: at m = n_c some cluster winds, one k-mer earlier none does;
    # at jamming every cluster wraps (Appendix A), so the lattice winds too
    L, k = 512, 16
    lat = rsa.Lattice(L, k)
    nj, nc = lat.run(range(1, 9))
    for i in range(8):
        assert lat.wrap_dirs(i, int(nc[i]) - 1) == (False, False)
        assert any(lat.wrap_dirs(i, int(nc[i])))
        assert any(lat.wrap_dirs(i, int(nj[i])))
        c = lat.cluster_sizes(i, int(nc[i]))
        assert int(np.sum(np.arange(c.size) * c.astype(np.int64))) == nc[i]
    lat.close()


def test_configuration_argument_errors():
    L, k = 64, 4
    lat = rsa.Lattice(L, k)
    nj, nc = lat.run([1, 2])
    lib = rsa.load()
    buf = np.zeros(4, dtype=np.uint32)
    assert lib.rsa_cluster_sizes(lat.h, 0, int(nj[0]) + 1, buf.ctypes.data, 4) == rsa.RSA_EINVAL
    assert lib.rsa_cluster_sizes(lat.h, 0, 10, buf.ctypes.data, 4) == rsa.RSA_EINVAL  # cap < m+1
    assert lib.rsa_cluster_sizes(lat.h, 2, 1, buf.ctypes.data, 4) == rsa.RSA_EINVAL   # sample
    assert lib.rsa_cluster_sizes(lat.h, 0, 1, None, 4) == rsa.RSA_EINVAL
    wx, wy = ctypes.c_uint32(7), ctypes.c_uint32(7)
    assert lib.rsa_wrap_dirs(lat.h, 0, 0, ctypes.byref(wx), ctypes.byref(wy)) == 0
    assert (wx.value, wy.value) == (0, 0)
    assert lib.rsa_cluster_sizes(lat.h, 1, 3, buf.ctypes.data, 4) == 0
    assert buf[0] == 0 and int(np.sum(np.arange(4) * buf)) == 3
    # the results of the run are untouched by the configuration passes
    nj2, nc2 = rsa.rsa_results(lat.h, 2)
    assert np.array_equal(nj, nj2) and np.array_equal(nc, nc2)
    lat.close()


def test_jammed_state_of_two_clusters():
    # Sec. III.C: a jammed state may hold several clusters.  Priorities that
    # put the hand-built two-band packing (k = 4, L = 40) first make it the
    # jammed state; its two clusters of 160 k-mers both wind along x and y.
    L, k = 40, 4
    packing = workloads.two_band_packing()
    keys = workloads.packing_first_keys(L, packing, 3)
    lat = rsa.Lattice(L, k)
    nj, nc = lat.run_keys(keys)
    wj, wc, _, acc = oracle.sample_keys(L, k, keys)
    assert (int(nj[0]), int(nc[0])) == (wj, wc) and wj == 320
    assert np.array_equal(lat.accepted(0), np.sort(packing))
    got = lat.cluster_sizes(0, 320)
    assert np.nonzero(got)[0].tolist() == [160] and got[160] == 2
    assert lat.wrap_dirs(0, 320) == (True, True)
    _compare(lat, 0, L, k, acc, _ms(320, int(nc[0]), np.random.default_rng(5)))
    lat.close()
