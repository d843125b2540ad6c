"""Host statistics of the study module (Sec. III): float64 means, standard
deviations and log binning, checked on inputs with known answers; then the
statistics the paper reports, computed through the GPU path."""
import math

import numpy as np
import pytest

import oracle
from paper_1810_06800_gb300 import study


def test_coverage_stats_definitions():
    L, k = 64, 4
    nj = np.array([800, 810, 820, 790], dtype=np.uint32)
    nc = np.array([500, 520, 480, 510], dtype=np.uint32)
    st = study.coverage_stats(L, k, nj, nc)
    pj = k * nj.astype(float) / L**2
    assert st["p_j"]["mean"] == pytest.approx(float(np.mean(pj)), rel=1e-15)
    # sample standard deviation (n - 1) and its standard error
    sd = math.sqrt(sum((x - np.mean(pj)) ** 2 for x in pj) / 3)
    assert st["p_j"]["sd"] == pytest.approx(sd, rel=1e-12)
    assert st["p_j"]["se"] == pytest.approx(sd / 2, rel=1e-12)
    assert st["p_c/p_j"]["mean"] == pytest.approx(float(np.mean(nc / nj)), rel=1e-14)


def test_log_binning_recovers_a_power_law():
    # averaging s^-tau over [a, 2a) gives a^-tau times a constant for a
    # continuous s; integer sizes leave a bias that shrinks as 1/a (about
    # 0.01 when the first bin starts at 32)
    s = np.arange(1, 1 << 14, dtype=float)
    for tau in (1.5, 187 / 91, 2.5):
        assert study.fisher_slope(s, s ** -tau, 32, 4096) == pytest.approx(-tau, abs=0.012)
        assert study.fisher_slope(s, s ** -tau, 4, 4096) == pytest.approx(-tau, abs=0.04)
    xs, ys = study.log_binned(s, s ** -2.0)
    # bin sums are preserved: sum of ys * width equals the total
    widths = np.array([2.0 ** (i + 1) - 2.0 ** i for i in range(xs.size)])
    assert float(np.sum(ys * widths)) == pytest.approx(float(np.sum(s ** -2.0)), rel=1e-12)


def test_cluster_size_distribution_counts_every_site():
    # sum over s of s n_s is the mean occupied fraction at the threshold
    L, k = 48, 3
    hists, ms = [], []
    for seed in range(1, 6):
        _, nc, _, acc = oracle.sample_keys(L, k, oracle.keys(L, seed))
        c, _, _ = oracle.configuration(L, k, acc, nc)
        hists.append(c)
        ms.append(nc)
    s, n_s = study.cluster_size_distribution(L, k, hists)
    assert np.all(s % k == 0) and np.all(n_s > 0)
    assert float(np.sum(s * n_s)) == pytest.approx(k * np.mean(ms) / L**2, rel=1e-12)


@pytest.mark.gpu
def test_std_decreases_with_lattice_size():
    # Sec. III.B: sigma(p_c) ~ L^-3/4 and sigma(p_j) ~ L^-1 (the paper fits
    # 0.74 +- 0.05 and 1.23 +- 0.17 at k = 256); k = 16, L/k = 8, 16, 32,
    # 128 runs each
    out = study.std_vs_size(16, [8, 16, 32], 128)
    sig = [r["sigma_p_c"] for r in out["rows"]]
    assert sig[0] > sig[1] > sig[2]
    assert 0.45 < out["exponent_p_c"] < 1.05, out
    assert 0.6 < out["exponent_p_j"] < 1.6, out


@pytest.mark.gpu
def test_wrapping_probability_at_pc_on_gpu():
    # Appendix A: R* = 0.521058290 for a horizontal wrap at p_c (k = 1);
    # the GPU and the oracle give the same flags sample by sample
    L, runs = 128, 400
    r = study.wrap_probabilities(L, 1, 0.592746, runs)
    assert r["samples"] == runs
    assert abs((r["R_x"] + r["R_y"]) / 2 - 0.521058290) < 0.06, r
    m = r["m"]
    wx = sum(oracle.configuration(L, 1, oracle.sample_keys(L, 1, oracle.keys(L, s))[3], m)[1]
             for s in range(1, runs + 1))
    assert wx == round(r["R_x"] * runs)


@pytest.mark.gpu
def test_cluster_sizes_at_pc_follow_fisher_exponent_on_gpu():
    # Sec. III.C, Eq. CSD, k = 1 at L = 256: same samples and bins as the
    # oracle pin, through the GPU path
    hists, nj, nc = study.percolation_cluster_sizes(256, 1, 40)
    s, n_s = study.cluster_size_distribution(256, 1, hists)
    assert abs(study.fisher_slope(s, n_s, 4, 1024) + 187 / 91) < 0.25
