"""Workspace-free entry point rsa_run_static, for callers that cannot
allocate device memory: a process whose device memory belongs to another
allocator (a framework's caching allocator that has reserved the HBM), or a
latency-critical loop that must not call cudaMalloc/cudaFree, which can
synchronise the whole device.  All of its device state lives in one fixed
array inside the library.

Checked here, on two calls in a row that share that array: n_j and n_c equal
the oracle's (Sec. II.B-II.D) and the allocating path's (rsa_run_seeds +
rsa_results) exactly, and a call leaves the device's free memory unchanged.

This file is collected last so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

import oracle
from paper_1810_06800_gb300 import rsa

pytestmark = pytest.mark.gpu


def _allocating(L, k, seeds):
    h = rsa.rsa_create(L, k, 1)
    try:
        rsa.rsa_run_seeds(h, seeds)
        return rsa.rsa_results(h, len(seeds))
    finally:
        rsa.rsa_destroy(h)


@pytest.mark.parametrize("L,k", [(64, 4), (96, 16), (100, 3), (256, 64)])
def test_static_run_matches_oracle_and_allocating_run_twice(L, k):
    first = list(range(1, 25))
    second = list(range(500, 531))  # a different batch size and seeds
    for seeds in (first, second):
        nj, nc = rsa.rsa_run_static(L, k, seeds)
        oj, oc = oracle.samples(L, k, seeds)
        assert np.array_equal(nj, oj.astype(np.uint32)), (L, k, seeds[:3])
        assert np.array_equal(nc, oc.astype(np.uint32)), (L, k, seeds[:3])
        wj, wc = _allocating(L, k, seeds)
        assert np.array_equal(nj, wj) and np.array_equal(nc, wc)


def test_static_run_allocates_no_device_memory():
    import torch
    L, k = 96, 16
    rsa.rsa_run_static(L, k, list(range(1, 9)))       # warm-up: kernels loaded
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    nj, nc = rsa.rsa_run_static(L, k, list(range(40, 52)))
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    oj, oc = oracle.samples(L, k, list(range(40, 52)))
    assert np.array_equal(nj, oj.astype(np.uint32)) and np.array_equal(nc, oc.astype(np.uint32))


def test_static_run_rejects_sizes_beyond_the_array():
    with pytest.raises(rsa.RSAError) as e:
        rsa.rsa_run_static(1024, 32, list(range(1, 101)))
    assert e.value.code == rsa.RSA_EINVAL
    assert "static workspace" in str(e.value)
