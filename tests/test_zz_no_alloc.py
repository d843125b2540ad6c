"""Workspace-free entry point rsa_run_static: for callers that cannot
allocate device memory (another allocator owns the device pool, or a
latency-critical loop must not call cudaMalloc/cudaFree).  Its results must
equal the allocating path's (rsa_run_seeds + rsa_results) exactly, on two
calls in a row that share the library's fixed device array.

This file is collected last so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

from paper_1810_06800_gb300 import rsa

pytestmark = pytest.mark.gpu


def _reference(L, k, seeds):
    h = rsa.rsa_create(L, k, 1)
    try:
        rsa.rsa_run_seeds(h, seeds)
        return rsa.rsa_results(h, len(seeds))
    finally:
        rsa.rsa_destroy(h)


@pytest.mark.parametrize("L,k", [(64, 4), (96, 16), (100, 3)])
def test_static_run_matches_allocating_run_twice(L, k):
    first = list(range(1, 25))
    second = list(range(500, 531))  # a different batch size and seeds
    for seeds in (first, second):
        nj, nc = rsa.rsa_run_static(L, k, seeds)
        wj, wc = _reference(L, k, seeds)
        assert np.array_equal(nj, wj), (L, k, seeds[:3])
        assert np.array_equal(nc, wc), (L, k, seeds[:3])


def test_static_run_rejects_sizes_beyond_the_array():
    with pytest.raises(rsa.RSAError) as e:
        rsa.rsa_run_static(1024, 32, list(range(1, 101)))
    assert e.value.code == rsa.RSA_EINVAL
    assert "static workspace" in str(e.value)
