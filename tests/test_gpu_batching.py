"""Batching of uneven shapes: the small-lattice one-CTA-per-sample mode
(samples of any mix of (L, k) in one persistent launch), mixed batches that
run every shape the way the autotuner picks, and the autotuner itself.
Every result is compared with the CPU oracle (Sec. II.B-II.D) or, for
L = 8192, with its stored results (tests/golden/fullsize.json); results must
not depend on the CTA size, the tuning or the batch mix."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1810_06800_gb300 import rsa

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 1
HERE = os.path.dirname(os.path.abspath(__file__))

SMALL_SHAPES = [(1, 1), (2, 1), (2, 2), (3, 2), (5, 2), (16, 3), (31, 7), (32, 1), (32, 2),
                (33, 32), (40, 4), (64, 1), (64, 4), (64, 64), (100, 3), (128, 4), (128, 8),
                (128, 128)]


def _oracle(L, k, seeds):
    nj, nc = oracle.samples(L, k, seeds, threads=THREADS)
    return nj.astype(np.uint32), nc.astype(np.uint32)


def _uneven_batch(shapes, seeds):
    L, k, sd = [], [], []
    for (a, b) in shapes:
        for s in seeds:
            L.append(a)
            k.append(b)
            sd.append(s)
    return np.array(L, np.uint32), np.array(k, np.uint32), np.array(sd, np.uint64)


def _expected(L, k, sd):
    want_j = np.zeros(sd.size, np.uint32)
    want_c = np.zeros(sd.size, np.uint32)
    for (a, b) in sorted(set(zip(L.tolist(), k.tolist()))):
        sel = (L == a) & (k == b)
        wj, wc = _oracle(a, b, [int(s) for s in sd[sel]])
        want_j[sel], want_c[sel] = wj, wc
    return want_j, want_c


def test_small_mode_uneven_shapes_in_one_launch():
    L, k, sd = _uneven_batch(SMALL_SHAPES, range(1, 9))
    rng = np.random.default_rng(5)
    perm = rng.permutation(sd.size)          # shapes interleaved in the job table
    L, k, sd = L[perm], k[perm], sd[perm]
    nj, nc = rsa.rsa_run_small(L, k, sd)
    wj, wc = _expected(L, k, sd)
    assert np.array_equal(nj, wj) and np.array_equal(nc, wc)


@pytest.mark.parametrize("threads", [256, 512, 1024])
def test_small_mode_results_do_not_depend_on_cta_size(threads):
    L, k, sd = _uneven_batch([(64, 4), (128, 8), (33, 32)], range(20, 26))
    nj, nc = rsa.rsa_run_small(L, k, sd, threads=threads)
    wj, wc = _expected(L, k, sd)
    assert np.array_equal(nj, wj) and np.array_equal(nc, wc)


def test_small_mode_plain_small_config_all_seeds():
    # L = 64, k = 4, seeds 1..100: the whole batch in one launch
    nj, nc = rsa.rsa_run_small(64, 4, list(range(1, 101)))
    wj, wc = _oracle(64, 4, list(range(1, 101)))
    assert np.array_equal(nj, wj) and np.array_equal(nc, wc)


@pytest.mark.parametrize("L,k", [(256, 4), (128, 2), (129, 64)])
def test_small_mode_rejects_shapes_that_do_not_fit(L, k):
    with pytest.raises(rsa.RSAError) as e:
        rsa.rsa_run_small(L, k, [1, 2])
    assert e.value.code == rsa.RSA_EINVAL


def _golden(L, k):
    with open(os.path.join(HERE, "golden", "fullsize.json")) as f:
        d = json.load(f)["samples"]
    return {r["seed"]: r for r in d.values() if r["L"] == L and r["k"] == k}


@pytest.mark.parametrize("autotune", ["0", "1"])
def test_mixed_batch_of_the_uneven_workload(monkeypatch, autotune):
    # the uneven workload's four shapes (k in {2, 8, 64, 512}, L = 16 k) in
    # one call, fewer samples; L = 8192 checked against the stored oracle
    monkeypatch.setenv("RSA_AUTOTUNE", autotune)
    shapes = [(32, 2), (128, 8), (1024, 64), (8192, 512)]
    per = {32: range(1, 33), 128: range(1, 17), 1024: range(1, 5), 8192: range(1, 3)}
    L, k, sd = [], [], []
    for (a, b) in shapes:
        for s in per[a]:
            L.append(a), k.append(b), sd.append(s)
    L, k, sd = np.array(L, np.uint32), np.array(k, np.uint32), np.array(sd, np.uint64)
    nj, nc = rsa.rsa_run_mix(L, k, sd)
    small = L < 8192
    wj, wc = _expected(L[small], k[small], sd[small])
    assert np.array_equal(nj[small], wj) and np.array_equal(nc[small], wc)
    gold = _golden(8192, 512)
    for i in np.nonzero(~small)[0]:
        rec = gold[int(sd[i])]
        assert (int(nj[i]), int(nc[i])) == (rec["n_j"], rec["n_c"])


def test_mixed_batch_equals_each_sample_alone():
    L = np.array([64, 1024, 64, 100, 1024, 32], np.uint32)
    k = np.array([4, 64, 4, 3, 32, 2], np.uint32)
    sd = np.array([7, 7, 8, 9, 10, 11], np.uint64)
    nj, nc = rsa.rsa_run_mix(L, k, sd)
    for i in range(sd.size):
        lat = rsa.Lattice(int(L[i]), int(k[i]))
        aj, ac = lat.run([int(sd[i])])
        lat.close()
        assert (int(nj[i]), int(nc[i])) == (int(aj[0]), int(ac[0]))


def test_autotuner_choice_is_cached(tmp_path, monkeypatch):
    monkeypatch.setenv("RSA_TUNE_CACHE", str(tmp_path / "tune.jsonl"))
    c = rsa.rsa_tune(64, 4, 100, measure=True)
    assert c["mode"] in ("small", "global") and c["ms_per_sample"] > 0
    again = rsa.rsa_tune(64, 4, 100, measure=False)
    assert again == c
    # a shape that does not fit a CTA never picks the small mode
    big = rsa.rsa_tune(1024, 64, 4, measure=True)
    assert big["mode"] == "global" and big["rounds_per_check"] in (2, 4, 8)


def test_rounds_per_check_does_not_change_results():
    L, k, seeds = 1024, 32, list(range(1, 9))
    wj, wc = _oracle(L, k, seeds)
    for r in (1, 3, 8):
        lat = rsa.Lattice(L, k)
        rsa.rsa_set_rounds_per_check(lat.h, r)
        nj, nc = lat.run(seeds)
        lat.close()
        assert np.array_equal(nj, wj) and np.array_equal(nc, wc)


@pytest.mark.parametrize("L,k", [(8192, 512), (2048, 256), (4096, 4096)])
def test_window_cta_size_does_not_change_results(L, k):
    seeds = [1, 2] if L == 8192 else [3, 4, 5]
    out = []
    for wt in (256, 128):
        lat = rsa.Lattice(L, k)
        rsa.rsa_set_window_threads(lat.h, wt)
        out.append(lat.run(seeds))
        acc = [lat.accepted(i) for i in range(len(seeds))]
        out.append(acc)
        lat.close()
    assert np.array_equal(out[0][0], out[2][0]) and np.array_equal(out[0][1], out[2][1])
    for a, b in zip(out[1], out[3]):
        assert np.array_equal(a, b)
    if L == 8192:
        gold = _golden(8192, 512)
        for i, s in enumerate(seeds):
            assert (int(out[2][0][i]), int(out[2][1][i])) == (gold[s]["n_j"], gold[s]["n_c"])
    else:
        wj, wc = _oracle(L, k, seeds)
        assert np.array_equal(out[2][0], wj) and np.array_equal(out[2][1], wc)


def test_window_cta_size_is_rejected_where_it_does_not_apply():
    lat = rsa.Lattice(1024, 32)       # tile path
    with pytest.raises(rsa.RSAError):
        rsa.rsa_set_window_threads(lat.h, 128)
    rsa.rsa_set_window_threads(lat.h, 256)
    lat.close()
