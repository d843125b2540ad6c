"""Failure detection without a GPU fault.

Every data-dependent device loop of the library has an iteration cap that
ends it with a status bit instead of spinning: the greedy round loop, each
union-find walk and link retry, the bisection for the first wrap, and the
contact-edge buffer.  rsa_test_caps lowers those caps on one handle so that
each runs out on purpose, small enough to run out at once.  Each test checks
that the run reports the right error code and that the next normal run, on
the same handle and the same GPU context, is still bit-exact to the oracle.
Nothing here traps, faults or waits without a limit.
"""
import numpy as np
import pytest

import oracle
from paper_1810_06800_gb300 import rsa

pytestmark = pytest.mark.gpu

# one shape per round path: 32 x 32 tiles, long-k lines, general kernels
SHAPES = [(128, 8), (256, 64), (100, 3)]
SEEDS = list(range(1, 7))


def _oracle(L, k, seeds):
    nj, nc = oracle.samples(L, k, seeds)
    return nj.astype(np.uint32), nc.astype(np.uint32)


def _run_expect(h, L, seeds, code):
    rsa.rsa_run_seeds(h, seeds)
    with pytest.raises(rsa.RSAError) as e:
        rsa.rsa_results(h, len(seeds))
    assert e.value.code == code, (e.value.code, str(e.value))
    st = rsa.rsa_sample_stats(h, len(seeds))
    assert np.all(st["status"] == code)
    return st


def _normal_run_is_exact(h, L, k, seeds):
    rsa.rsa_test_caps(h)           # defaults back
    rsa.rsa_run_seeds(h, seeds)
    nj, nc = rsa.rsa_results(h, len(seeds))
    wj, wc = _oracle(L, k, seeds)
    assert np.array_equal(nj, wj) and np.array_equal(nc, wc)


@pytest.mark.parametrize("L,k", SHAPES)
def test_round_cap_reports_timeout_then_recovers(L, k):
    h = rsa.rsa_create(L, k, 1)
    try:
        rsa.rsa_test_caps(h, round_cap=1)
        st = _run_expect(h, L, SEEDS, rsa.RSA_ETIMEOUT)
        assert np.all(st["rounds"] == 1)
        _normal_run_is_exact(h, L, k, SEEDS)
    finally:
        rsa.rsa_destroy(h)


@pytest.mark.parametrize("L,k", SHAPES)
def test_union_find_cap_reports_timeout_then_recovers(L, k):
    h = rsa.rsa_create(L, k, 1)
    try:
        # one step per walk: any node below a root runs the walk out
        rsa.rsa_test_caps(h, uf_steps=1)
        _run_expect(h, L, SEEDS, rsa.RSA_ETIMEOUT)
        _normal_run_is_exact(h, L, k, SEEDS)
    finally:
        rsa.rsa_destroy(h)


@pytest.mark.parametrize("L,k", SHAPES)
def test_probe_cap_reports_timeout_then_recovers(L, k):
    h = rsa.rsa_create(L, k, 1)
    try:
        # the first probe (the jammed lattice) wraps; the search would need
        # about log2 n_j more
        rsa.rsa_test_caps(h, probe_cap=1)
        st = _run_expect(h, L, SEEDS, rsa.RSA_ETIMEOUT)
        assert np.all(st["probes"] == 1)
        _normal_run_is_exact(h, L, k, SEEDS)
    finally:
        rsa.rsa_destroy(h)


@pytest.mark.parametrize("L,k", SHAPES)
def test_edge_buffer_cap_reports_enomem_then_recovers(L, k):
    h = rsa.rsa_create(L, k, 1)
    try:
        rsa.rsa_test_caps(h, edge_cap=4)
        _run_expect(h, L, SEEDS, rsa.RSA_ENOMEM)
        _normal_run_is_exact(h, L, k, SEEDS)
    finally:
        rsa.rsa_destroy(h)


def test_configuration_walk_cap_reports_timeout():
    # the on-demand configuration pass shares the union-find walk cap
    L, k = 128, 8
    h = rsa.rsa_create(L, k, 1)
    try:
        rsa.rsa_run_seeds(h, [3])
        nj, nc = rsa.rsa_results(h, 1)
        rsa.rsa_test_caps(h, uf_steps=1)
        with pytest.raises(rsa.RSAError) as e:
            rsa.rsa_cluster_sizes(h, 0, int(nj[0]))
        assert e.value.code == rsa.RSA_ETIMEOUT
        rsa.rsa_test_caps(h)
        acc, _ = oracle.scan(L, k, oracle.keys(L, 3))
        want, _, _ = oracle.configuration(L, k, acc, int(nc[0]))
        got = rsa.rsa_cluster_sizes(h, 0, int(nc[0]))
        assert np.array_equal(got.astype(np.int64), want)
    finally:
        rsa.rsa_destroy(h)


def test_other_handles_unaffected_while_one_is_capped():
    L, k = 128, 8
    bad = rsa.rsa_create(L, k, 1)
    good = rsa.rsa_create(L, k, 1)
    try:
        rsa.rsa_test_caps(bad, round_cap=1)
        _run_expect(bad, L, SEEDS, rsa.RSA_ETIMEOUT)
        rsa.rsa_run_seeds(good, SEEDS)
        nj, nc = rsa.rsa_results(good, len(SEEDS))
        wj, wc = _oracle(L, k, SEEDS)
        assert np.array_equal(nj, wj) and np.array_equal(nc, wc)
    finally:
        rsa.rsa_destroy(bad)
        rsa.rsa_destroy(good)
