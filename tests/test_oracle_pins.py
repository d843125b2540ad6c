"""Pins of the CPU oracle against what the paper and the mathematics fix,
not against the oracle itself.

* splitmix64 against its published output vectors (tests/golden).
* The priority-order greedy scan equals RSA (Sec. II.A, II.B): the law of
  (n_j, n_c) over all (2L^2)! orders equals the exact RSA Markov chain
  (L = 2), and matches it by chi-square on seeded samples (L = 3, 4).
* n_c (Sec. II.C, II.D) against breadth-first search on the lifted lattice.
* The paper's |x1-x2|+|y1-y2| > 2k test agrees with the exact rule when
  L >= 3k + 2.
* Jamming: no candidate fits afterwards; k = 1 gives n_j = L^2 (Table I).
* Appendix A Proposition: every cluster of every jammed packing wraps
  (exhaustive on small tori), hence n_c <= n_j.
* Statistics against Table I and the known k = 1 and k = 2 values.
* The configuration of the first m k-mers (cluster-size histogram, winding
  directions) against breadth-first search on the lifted lattice, its
  transpose symmetry, and the Fisher exponent of Eq. CSD at k = 1.
"""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import brute
from paper_1810_06800_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
M64 = 2**64 - 1


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                rows.append(line.split())
    return rows


def test_splitmix64_published_vectors():
    for row in _golden("splitmix64.txt"):
        seed, outs = int(row[0]), [int(v) for v in row[1:]]
        state = seed
        for want in outs:
            state = (state + 0x9E3779B97F4A7C15) & M64
            assert oracle.mix64(state) == want
        # the per-sample base is the first output of the stream seeded by seed
        assert oracle.base(seed) == outs[0]


def _inv_xorshift_right(z, s):
    x = z
    for _ in range(64 // s + 1):
        x = z ^ (x >> s)
    return x & M64


def test_mix64_is_a_bijection():
    # invert each step: odd multipliers have inverses mod 2^64 and
    # z ^ (z >> s) is inverted by fixed-point iteration
    a_inv = pow(0xBF58476D1CE4E5B9, -1, 2**64)
    b_inv = pow(0x94D049BB133111EB, -1, 2**64)
    rng = np.random.default_rng(7)
    for z in rng.integers(0, 2**64 - 1, size=20000, dtype=np.uint64):
        z = int(z)
        y = oracle.mix64(z)
        x = _inv_xorshift_right(y, 31)
        x = (x * b_inv) & M64
        x = _inv_xorshift_right(x, 27)
        x = (x * a_inv) & M64
        x = _inv_xorshift_right(x, 30)
        assert x == z


def test_keys_are_distinct_and_balanced():
    L = 64
    for seed in (1, 2, 3):
        k = oracle.keys(L, seed)
        assert np.unique(k).size == 2 * L * L
        # which orientation comes first is a fair coin at every site
        h, v = k[: L * L], k[L * L:]
        frac = float(np.mean(h < v))
        assert abs(frac - 0.5) < 4 * 0.5 / math.sqrt(L * L)
    # different seeds give unrelated streams
    assert np.intersect1d(oracle.keys(L, 1), oracle.keys(L, 2)).size == 0


def _law_from_orders(L, k):
    n = 2 * L * L
    counts = {}
    for perm in itertools.permutations(range(n)):
        keys = np.empty(n, dtype=np.uint64)
        keys[list(perm)] = np.arange(n, dtype=np.uint64)
        nj, nc, _, _ = oracle.sample_keys(L, k, keys)
        counts[(nj, nc)] = counts.get((nj, nc), 0) + 1
    tot = math.factorial(n)
    return {key: Fraction(c, tot) for key, c in counts.items()}


@pytest.mark.parametrize("k", [1, 2])
def test_greedy_over_all_orders_is_exact_rsa_L2(k):
    assert _law_from_orders(2, k) == brute.rsa_exact_distribution(2, k)


@pytest.mark.parametrize("L,k,nsamp", [(3, 2, 6000), (3, 3, 3000), (4, 3, 4000)])
def test_greedy_matches_rsa_chain_chi2(L, k, nsamp):
    law = brute.rsa_exact_distribution(L, k)
    counts = {}
    for s in range(nsamp):
        nj, nc, _ = oracle.sample(L, k, 1000 + s)
        counts[(nj, nc)] = counts.get((nj, nc), 0) + 1
    assert set(counts) <= set(law)
    # pool cells with small expectation, then a chi-square test at p ~ 1e-4
    chi2, dof, rest_o, rest_e = 0.0, -1, 0, 0.0
    for key, p in law.items():
        e = float(p) * nsamp
        o = counts.get(key, 0)
        if e < 5:
            rest_o += o
            rest_e += e
            continue
        chi2 += (o - e) ** 2 / e
        dof += 1
    if rest_e > 0:
        chi2 += (rest_o - rest_e) ** 2 / max(rest_e, 1e-9)
        dof += 1
    from scipy.stats import chi2 as chi2d
    assert chi2d.sf(chi2, max(dof, 1)) > 1e-4, (chi2, dof)


@pytest.mark.parametrize("L,k", [(1, 1), (2, 1), (2, 2), (3, 1), (4, 2), (5, 2), (6, 3),
                                 (7, 1), (8, 4), (9, 2), (12, 3), (16, 4), (10, 10), (12, 5)])
def test_nc_matches_bfs_on_the_lift(L, k):
    for seed in range(1, 31 if L <= 9 else 11):
        keys = oracle.keys(L, seed)
        nj, nc, _, acc = oracle.sample_keys(L, k, keys)
        assert nc == brute.nc_bruteforce(L, k, acc)
        assert 1 <= nc <= nj


@pytest.mark.parametrize("L,k", [(5, 1), (8, 2), (16, 2), (16, 4), (32, 8), (64, 4), (64, 16),
                                 (100, 32)])
def test_paper_2k_test_agrees_when_L_ge_3k_plus_2(L, k):
    assert L >= 3 * k + 2
    for seed in range(1, 21):
        _, nc, ncp = oracle.sample(L, k, seed)
        assert ncp == nc


def test_paper_2k_test_can_disagree_when_lattice_is_short():
    # L = 4, k = 1: a wrapped neighbour pair can sit only 2 apart, so the
    # "> 2k" threshold misses wraps the exact rule sees (a reading to record)
    diffs = 0
    for seed in range(1, 200):
        _, nc, ncp = oracle.sample(4, 1, seed)
        diffs += nc != ncp
    assert diffs > 0


@pytest.mark.parametrize("L,k", [(3, 2), (4, 3), (8, 3), (16, 5), (20, 20), (33, 7)])
def test_scan_result_is_jammed(L, k):
    for seed in range(1, 6):
        acc, occ = oracle.scan(L, k, oracle.keys(L, seed))
        assert oracle.is_jammed(L, k, occ)
        assert int(occ.sum()) == k * acc.size
        cells = {tuple(c) for c in zip(*np.nonzero(occ))}
        if L <= 8:
            assert brute.viable(L, k, cells) == []
        assert acc.size == len(brute.greedy(L, k, np.argsort(oracle.keys(L, seed),
                                                            kind="stable").tolist()))


@pytest.mark.parametrize("L,k", [(5, 2), (8, 3), (16, 4), (21, 7), (12, 12)])
def test_free_run_jamming_check_agrees_with_brute_force(L, k):
    rng = np.random.default_rng(L * 100 + k)
    for trial in range(40):
        occ = (rng.random((L, L)) < rng.uniform(0.3, 0.95)).astype(np.uint8)
        h, v = oracle.max_free_runs(occ)
        assert (h < k and v < k) == oracle.is_jammed(L, k, occ)
    for seed in (1, 2):
        acc, occ = oracle.scan(L, k, oracle.keys(L, seed))
        h, v = oracle.max_free_runs(occ)
        assert h < k and v < k
        assert np.array_equal(oracle.occupancy_from_accepted(L, k, acc), occ)


def test_jamming_check_rejects_a_gap():
    occ = np.ones((6, 6), dtype=np.uint8)
    occ[2, 1:4] = 0
    assert oracle.is_jammed(6, 4, occ)
    assert not oracle.is_jammed(6, 3, occ)


@pytest.mark.parametrize("L", [1, 2, 7, 64])
def test_k1_fills_every_site(L):
    for seed in (1, 2):
        nj, nc, _ = oracle.sample(L, 1, seed)
        assert nj == L * L          # Table I: p_j(k = 1) = 1
        assert 1 <= nc <= nj


@pytest.mark.parametrize("L", [1, 2, 3, 9, 40])
def test_k_equal_L_is_a_ring_that_wraps_alone(L):
    nj, nc, _ = oracle.sample(L, L, 5)
    assert nc == 1
    assert nj == L  # parallel full rows (or columns): one orientation fills


@pytest.mark.parametrize("L,k", [(2, 1), (3, 1), (3, 2), (3, 3), (4, 2), (4, 3), (4, 4), (5, 3),
                                 (5, 4), (6, 4), (6, 5)])
def test_proposition_every_jammed_cluster_wraps(L, k):
    """Appendix A: every cluster of every jammed packing on the torus wraps."""
    packs = brute.maximal_packings(L, k)
    assert packs
    for occ in packs:
        for comp in brute.clusters(L, occ):
            assert brute.wraps(L, comp)


def test_proposition_on_oracle_samples():
    for L, k in [(12, 3), (20, 4), (24, 6)]:
        for seed in range(1, 11):
            acc, occ = oracle.scan(L, k, oracle.keys(L, seed))
            cells = [tuple(c) for c in zip(*np.nonzero(occ))]
            for comp in brute.clusters(L, cells):
                assert brute.wraps(L, comp)


def test_bfs_checker_basic_shapes():
    # a straight line around the torus wraps, a closed ring of 8 does not
    assert brute.wraps(5, [(2, x) for x in range(5)])
    assert not brute.wraps(5, [(2, x) for x in range(4)])
    ring = [(1, 1), (1, 2), (1, 3), (2, 3), (3, 3), (3, 2), (3, 1), (2, 1)]
    assert not brute.wraps(6, ring)
    # a diagonal staircase winding once in x and once in y
    stair = [(i, i) for i in range(4)] + [(i, i + 1) for i in range(3)] + [(3, 0)]
    assert brute.wraps(4, stair)
    # L = 1 and L = 2 multi-edges
    assert brute.wraps(1, [(0, 0)])
    assert brute.wraps(2, [(0, 0), (0, 1)])
    assert not brute.wraps(3, [(0, 0), (0, 1)])


def _table1():
    return {int(r[0]): (float(r[1]), float(r[2])) for r in _golden("table1.txt")}


def test_k2_jamming_coverage():
    # dimer RSA jamming coverage on the square lattice is 0.9068
    # (Table I: 0.9062 at L = 200)
    L, k = 128, 2
    nj, _ = oracle.samples(L, k, range(1, 41), threads=os.cpu_count() or 1)
    pj = k * nj / (L * L)
    assert abs(pj.mean() - 0.9068) < 0.003


def test_k1_first_wrap_coverage():
    # site percolation, first wrap in either direction: mean p_c near 0.5927
    # at finite L; Table I gives 0.5933
    L = 128
    _, nc = oracle.samples(L, 1, range(1, 81), threads=os.cpu_count() or 1)
    pc = nc / (L * L)
    assert abs(pc.mean() - _table1()[0][0]) < 0.02


@pytest.mark.parametrize("n", [2, 3, 5])
def test_table1_smoke(n):
    k = 2**n
    L = 32 * k if n <= 3 else 16 * k
    seeds = range(1, 25)
    nj, nc = oracle.samples(L, k, seeds, threads=os.cpu_count() or 1)
    pj, pc = k * nj / (L * L), k * nc / (L * L)
    want_pc, want_pj = _table1()[n]
    # finite-size offsets scale like (L/k)^-3/4 and L^-1 (Eqs. pcscaling,
    # pjscaling); these lattices are 3-6x shorter than the paper's L/k = 100
    assert abs(pj.mean() - want_pj) < 0.012
    assert abs(pc.mean() - want_pc) < 0.05
    assert np.all(nc <= nj)


@pytest.mark.parametrize("L,k", [(2, 1), (3, 2), (6, 2), (8, 3), (12, 4), (16, 16)])
def test_contacts_match_brute_force_and_edge_count(L, k):
    for seed in range(1, 9):
        acc, occ = oracle.scan(L, k, oracle.keys(L, seed))
        got = oracle.contacts(L, k, acc)
        assert got == brute.contacts(L, k, acc)
        # every occupied-occupied lattice edge is a contact or lies inside a
        # k-mer (k - 1 inner edges each, k for a k = L ring)
        edges = int(np.sum(occ & np.roll(occ, -1, axis=1)) + np.sum(occ & np.roll(occ, -1, axis=0)))
        inner = acc.size * (k if k == L else k - 1)
        if L > 2:
            assert sum(got) == edges - inner


def test_wrap_dirs_checker_basic_shapes():
    assert brute.wrap_dirs(5, [(2, x) for x in range(5)]) == (True, False)
    assert brute.wrap_dirs(5, [(y, 3) for y in range(5)]) == (False, True)
    assert brute.wrap_dirs(5, [(2, x) for x in range(4)]) == (False, False)
    ring = [(1, 1), (1, 2), (1, 3), (2, 3), (3, 3), (3, 2), (3, 1), (2, 1)]
    assert brute.wrap_dirs(6, ring) == (False, False)
    # winding (1, 1): one turn along x and one along y
    stair = [(i, i) for i in range(4)] + [(i, i + 1) for i in range(3)] + [(3, 0)]
    assert brute.wrap_dirs(4, stair) == (True, True)
    # a row plus a column: both directions, as two separate cycles
    cross = [(0, x) for x in range(6)] + [(y, 2) for y in range(1, 6)]
    assert brute.wrap_dirs(6, cross) == (True, True)
    # L = 1: the +x and +y edges of the only cell are both self-loops
    assert brute.wrap_dirs(1, [(0, 0)]) == (True, True)
    assert brute.wrap_dirs(2, [(0, 0), (0, 1)]) == (True, False)


def _transpose(L, acc):
    """Candidates mirrored in the diagonal: H(y, x) <-> V(x, y)."""
    LL = L * L
    a = np.asarray(acc, dtype=np.int64)
    o, r = np.divmod(a, LL)
    y, x = np.divmod(r, L)
    return (((1 - o) * L + x) * L + y).astype(np.uint32)


@pytest.mark.parametrize("L,k", [(1, 1), (2, 1), (2, 2), (3, 1), (4, 2), (5, 2), (6, 3),
                                 (7, 1), (8, 2), (8, 4), (9, 3), (10, 10), (12, 4)])
def test_configuration_matches_bfs_on_the_lift(L, k):
    for seed in range(1, 13 if L <= 8 else 6):
        nj, nc, _, acc = oracle.sample_keys(L, k, oracle.keys(L, seed))
        for m in range(nj + 1):
            counts, wx, wy = oracle.configuration(L, k, acc, m)
            cells = [c for idx in acc[:m] for c in brute.cells_of(L, k, int(idx))]
            want = np.zeros(m + 1, dtype=np.int64)
            for comp in brute.clusters(L, cells):
                assert len(comp) % k == 0
                want[len(comp) // k] += 1
            assert np.array_equal(counts, want), (seed, m)
            assert (wx, wy) == brute.wrap_dirs(L, cells), (seed, m)
            # Sec. II.D: a cluster wraps from the n_c-th k-mer on
            assert (wx or wy) == (m >= nc), (seed, m, nc)


@pytest.mark.parametrize("L,k", [(16, 2), (32, 4), (48, 8), (64, 1)])
def test_configuration_invariants(L, k):
    for seed in range(1, 6):
        nj, nc, _, acc = oracle.sample_keys(L, k, oracle.keys(L, seed))
        accT = _transpose(L, acc)
        for m in sorted({1, nc - 1, nc, nj, (nc + nj) // 2}):
            counts, wx, wy = oracle.configuration(L, k, acc, m)
            assert int(np.sum(np.arange(m + 1) * counts)) == m   # every k-mer once
            assert counts[0] == 0
            cT, wxT, wyT = oracle.configuration(L, k, accT, m)
            assert np.array_equal(cT, counts) and (wxT, wyT) == (wy, wx)
        # Appendix A Proposition: at jamming every cluster wraps, so the
        # lattice winds in some direction
        _, wx, wy = oracle.configuration(L, k, acc, nj)
        assert wx or wy


@pytest.mark.parametrize("L", [1, 3, 8])
def test_configuration_of_a_ring(L):
    # k = L: one k-mer closes on itself and winds along its own axis
    for o, want in ((0, (True, False)), (1, (False, True))):
        counts, wx, wy = oracle.configuration(L, L, np.array([o * L * L], dtype=np.uint32), 1)
        assert list(counts) == [0, 1]
        if L > 1:
            assert (wx, wy) == want
        else:
            assert (wx, wy) == (True, True)


def test_cluster_sizes_follow_the_fisher_exponent():
    # Eq. CSD: at the percolation threshold n_s ~ s^-tau, tau = 187/91, for
    # large s.  Site percolation (k = 1) at the first wrap, L = 256, 40
    # samples, log-binned s in [4, 1024]; corrections to scaling at these
    # sizes make the apparent slope somewhat shallower than -tau.
    L, k, N = 256, 1, 40
    tot = np.zeros(L * L + 1)
    for seed in range(1, N + 1):
        _, nc, _, acc = oracle.sample_keys(L, k, oracle.keys(L, seed))
        counts, _, _ = oracle.configuration(L, k, acc, nc)
        tot[:counts.size] += counts
    s = np.arange(tot.size) * k
    xs, ys = [], []
    for a in 2.0 ** np.arange(2, 10):
        sel = (s >= a) & (s < 2 * a)
        xs.append(a * math.sqrt(2))
        ys.append(tot[sel].sum() / N / (L * L) / a)
    slope = np.polyfit(np.log(xs), np.log(ys), 1)[0]
    assert abs(slope + 187 / 91) < 0.25, slope


def test_horizontal_wrapping_probability_at_pc():
    # Appendix A (proof of the Consequence): at p = p_c the probability that a
    # cluster wraps horizontally tends to R* = 0.521058290 (k = 1, site
    # percolation, p_c = 0.592746).  L = 128, 400 samples, both axes averaged
    # (standard error about 0.02).
    L, k, N = 128, 1, 400
    m = round(0.592746 * L * L)
    wx = wy = 0
    for seed in range(1, N + 1):
        _, _, _, acc = oracle.sample_keys(L, k, oracle.keys(L, seed))
        _, x, y = oracle.configuration(L, k, acc, m)
        wx += x
        wy += y
    assert abs((wx + wy) / (2 * N) - 0.521058290) < 0.06, (wx / N, wy / N)


@pytest.mark.parametrize("L,k", [(1, 1), (5, 2), (16, 3), (64, 4), (128, 64), (300, 17)])
def test_scan_from_seed_equals_scan_of_the_keys(L, k):
    # the seeded scan forms its (key, idx) pairs from the key function itself;
    # it must accept exactly what the scan of the materialised keys accepts,
    # however many key ranges it is split into (one bucket per range at
    # 65536; larger counts are clamped to that)
    for seed in (1, 7, 123456789):
        a1, o1 = oracle.scan(L, k, oracle.keys(L, seed))
        for parts in (1, 2, 7, 64) + ((65536, 10**6) if L <= 16 else ()):
            a2, o2 = oracle.scan_seed(L, k, seed, parts)
            assert np.array_equal(a1, a2) and np.array_equal(o1, o2), parts


def test_a_jammed_state_can_hold_two_clusters():
    """Sec. III.C: a jammed state may consist of several clusters (the
    paper's example is k = 4, L = 10k), though samples in practice end with
    one.  The two-band packing is built by hand (workloads.two_band_packing):
    jammed by brute force, two clusters of 160 k-mers by breadth-first
    search, each winding in both directions (the Proposition).  The oracle's
    configuration must see the same, and its scan, given priorities that put
    the packing first, must accept exactly the packing."""
    L, k = 40, 4
    acc = workloads.two_band_packing()
    occ = oracle.occupancy_from_accepted(L, k, acc)
    cells = [tuple(c) for c in zip(*np.nonzero(occ))]
    assert acc.size == 320 and len(cells) == 1280          # no overlap
    assert not brute.viable(L, k, set(cells))              # jammed
    comps = brute.clusters(L, cells)
    assert sorted(len(c) for c in comps) == [640, 640]
    assert all(brute.wrap_dirs(L, c) == (True, True) for c in comps)
    counts, wx, wy = oracle.configuration(L, k, acc, acc.size)
    assert np.nonzero(counts)[0].tolist() == [160] and counts[160] == 2
    assert wx and wy
    assert oracle.is_jammed(L, k, occ)
    keys = workloads.packing_first_keys(L, acc, 3)
    nj, nc, ncp, got = oracle.sample_keys(L, k, keys)
    assert nj == 320 and np.array_equal(np.sort(got), np.sort(acc))
    assert 1 <= nc <= nj and nc == ncp == oracle.percolation(L, k, got)[0]
    assert nc == brute.nc_bruteforce(L, k, got)


@pytest.mark.parametrize("L,k,n", [(40, 4, 30), (64, 4, 20), (128, 8, 10), (256, 32, 6)])
def test_seeded_samples_jam_as_a_single_cluster(L, k, n):
    # Sec. III.C: in practice the jammed state is one cluster
    for seed in range(1, n + 1):
        acc, _ = oracle.scan(L, k, oracle.keys(L, seed))
        counts, wx, wy = oracle.configuration(L, k, acc, acc.size)
        assert counts.sum() == 1 and counts[acc.size] == 1, (L, k, seed)
        assert wx or wy
