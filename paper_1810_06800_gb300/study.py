"""Host-side statistics over batches of jammed samples (Sec. III).

Every number here is computed from per-sample integers the GPU path returns
(n_j, n_c, cluster-size histograms, winding bits); the host only averages, in
float64:

* :func:`coverage_stats`     p_j = k n_j / L^2, p_c = k n_c / L^2 and p_c / p_j
  (Sec. II.A), with mean, standard deviation and standard error.
* :func:`std_vs_size`        the accuracy study of Sec. III.B: the standard
  deviations of p_c and p_j against L / k at fixed k, and their power-law
  exponents (Eqs. pcscaling, pjscaling: sigma(p_c) ~ L^-3/4, sigma(p_j) ~ L^-1).
* :func:`cluster_size_distribution`, :func:`log_binned`, :func:`fisher_slope`
  n_s at the percolation threshold (Sec. III.C, Eq. CSD: n_s ~ s^-tau,
  tau = 187/91).
* :func:`wrap_probabilities` the probability that a cluster winds round the
  torus along x, along y, along either or both, with a fixed number of
  k-mers placed (Appendix A: R* = 0.521058290 for one direction at p_c).

Command line:
  python -m paper_1810_06800_gb300.study std  --k 256 --ratios 8 16 32 --runs 100
  python -m paper_1810_06800_gb300.study csd  --L 2048 --k 256 --runs 100
  python -m paper_1810_06800_gb300.study wrap --L 512 --k 1 --p 0.592746 --runs 400
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np

from . import rsa

# Device memory a batch may use; larger runs go in several batches.
BATCH_BYTES = 32 << 30


def _mean_sd_se(x: np.ndarray) -> dict:
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    sd = float(np.std(x, ddof=1)) if n > 1 else 0.0
    return {"mean": float(np.mean(x)), "sd": sd, "se": sd / math.sqrt(n) if n else 0.0}


def coverage_stats(L: int, k: int, n_j, n_c) -> dict:
    """Mean, SD and SE of p_j, p_c and p_c / p_j over the given samples."""
    nj = np.asarray(n_j, dtype=np.float64)
    nc = np.asarray(n_c, dtype=np.float64)
    pj = k * nj / (L * L)
    pc = k * nc / (L * L)
    return {"L": L, "k": k, "samples": int(nj.size), "p_j": _mean_sd_se(pj),
            "p_c": _mean_sd_se(pc), "p_c/p_j": _mean_sd_se(pc / pj)}


def batch_size(L: int, k: int, want: int) -> int:
    """Samples per batch that keep one batch's workspace under BATCH_BYTES."""
    per = rsa.rsa_workspace_bytes(L, k, 1)
    return max(1, min(want, BATCH_BYTES // max(per, 1)))


def run_samples(L: int, k: int, seeds, with_lattice=None):
    """n_j, n_c (uint32) of the given seeds, in batches; with_lattice(lat,
    seeds_of_batch, nj, nc) is called after each batch while its results
    (and configurations) are still on the device."""
    seeds = np.asarray(list(seeds), dtype=np.uint64)
    nj_all, nc_all = [], []
    b = batch_size(L, k, seeds.size)
    lat = rsa.Lattice(L, k)
    try:
        for i in range(0, seeds.size, b):
            part = seeds[i:i + b]
            nj, nc = lat.run(part)
            if with_lattice is not None:
                with_lattice(lat, part, nj, nc)
            nj_all.append(nj)
            nc_all.append(nc)
    finally:
        lat.close()
    return np.concatenate(nj_all), np.concatenate(nc_all)


def _power_exponent(xs, ys) -> float:
    """-d log y / d log x by least squares (positive for a decaying law)."""
    return float(-np.polyfit(np.log(np.asarray(xs, float)), np.log(np.asarray(ys, float)), 1)[0])


def std_vs_size(k: int, ratios, runs: int, seed0: int = 1) -> dict:
    """Sec. III.B: sigma(p_c), sigma(p_j) over `runs` samples for L = r k."""
    rows = []
    for r in ratios:
        L = int(r) * k
        nj, nc = run_samples(L, k, range(seed0, seed0 + runs))
        st = coverage_stats(L, k, nj, nc)
        rows.append({"L/k": int(r), "L": L, "sigma_p_c": st["p_c"]["sd"],
                     "sigma_p_j": st["p_j"]["sd"], "p_c": st["p_c"]["mean"],
                     "p_j": st["p_j"]["mean"], "sigma_p_c/p_j": st["p_c/p_j"]["sd"]})
    out = {"k": k, "runs": runs, "rows": rows}
    if len(rows) >= 2:
        Ls = [row["L"] for row in rows]
        out["exponent_p_c"] = _power_exponent(Ls, [row["sigma_p_c"] for row in rows])
        out["exponent_p_j"] = _power_exponent(Ls, [row["sigma_p_j"] for row in rows])
    return out


def cluster_size_distribution(L: int, k: int, hists) -> tuple[np.ndarray, np.ndarray]:
    """(s, n_s): cluster size s in sites (= k x k-mers) and the average number
    of clusters of size s per lattice site, over the given per-sample
    histograms (counts[m] = clusters of m k-mers).  Sizes that never occur are
    left out."""
    size = max(len(h) for h in hists)
    tot = np.zeros(size, dtype=np.float64)
    for h in hists:
        tot[:len(h)] += np.asarray(h, dtype=np.float64)
    m = np.nonzero(tot)[0]
    m = m[m > 0]
    return m * k, tot[m] / len(hists) / (L * L)


def log_binned(s, n_s, base: float = 2.0):
    """Logarithmic bins [base^i, base^(i+1)) of cluster size: (geometric bin
    centre, sum of n_s in the bin / bin width, i.e. the mean n_s per size)."""
    s = np.asarray(s, dtype=np.float64)
    n_s = np.asarray(n_s, dtype=np.float64)
    if s.size == 0:
        return np.zeros(0), np.zeros(0)
    top = int(math.floor(math.log(s.max(), base))) + 1
    xs, ys = [], []
    for i in range(top + 1):
        lo, hi = base ** i, base ** (i + 1)
        sel = (s >= lo) & (s < hi)
        if np.any(sel):
            xs.append(math.sqrt(lo * hi))
            ys.append(float(n_s[sel].sum()) / (hi - lo))
    return np.asarray(xs), np.asarray(ys)


def fisher_slope(s, n_s, lo: float, hi: float, base: float = 2.0) -> float:
    """Slope of log n_s against log s over log bins with centres in [lo, hi];
    Eq. CSD predicts -187/91."""
    xs, ys = log_binned(s, n_s, base)
    sel = (xs >= lo) & (xs <= hi) & (ys > 0)
    if np.count_nonzero(sel) < 2:
        raise ValueError("fewer than two populated bins in the range")
    return float(np.polyfit(np.log(xs[sel]), np.log(ys[sel]), 1)[0])


def percolation_cluster_sizes(L: int, k: int, runs: int, seed0: int = 1):
    """Per-sample cluster-size histograms at the percolation threshold
    (m = n_c), plus n_j and n_c."""
    hists = []

    def grab(lat, part, nj, nc):
        for i in range(part.size):
            hists.append(lat.cluster_sizes(i, int(nc[i])))

    nj, nc = run_samples(L, k, range(seed0, seed0 + runs), grab)
    return hists, nj, nc


def wrap_probabilities(L: int, k: int, p: float, runs: int, seed0: int = 1) -> dict:
    """With m = round(p L^2 / k) k-mers placed (samples that jam with fewer
    are skipped and counted): fraction of samples whose clusters wind along
    x, along y, along either and along both."""
    m = int(round(p * L * L / k))
    flags = []

    def grab(lat, part, nj, nc):
        for i in range(part.size):
            if int(nj[i]) >= m:
                flags.append(lat.wrap_dirs(i, m))

    run_samples(L, k, range(seed0, seed0 + runs), grab)
    f = np.asarray(flags, dtype=bool).reshape(-1, 2)
    n = f.shape[0]
    frac = (lambda a: float(np.mean(a)) if n else float("nan"))
    return {"L": L, "k": k, "p": p, "m": m, "samples": n, "skipped": runs - n,
            "R_x": frac(f[:, 0]), "R_y": frac(f[:, 1]),
            "R_either": frac(f[:, 0] | f[:, 1]), "R_both": frac(f[:, 0] & f[:, 1])}


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    sub = ap.add_subparsers(dest="cmd", required=True)
    a = sub.add_parser("std", help="sigma(p_c), sigma(p_j) against L/k (Sec. III.B)")
    a.add_argument("--k", type=int, default=256)
    a.add_argument("--ratios", type=int, nargs="+", default=[8, 16, 32])
    a.add_argument("--runs", type=int, default=100)
    b = sub.add_parser("csd", help="cluster sizes at p_c (Sec. III.C, Eq. CSD)")
    b.add_argument("--L", type=int, default=2048)
    b.add_argument("--k", type=int, default=256)
    b.add_argument("--runs", type=int, default=100)
    c = sub.add_parser("wrap", help="winding probabilities with m = p L^2 / k k-mers")
    c.add_argument("--L", type=int, default=512)
    c.add_argument("--k", type=int, default=1)
    c.add_argument("--p", type=float, default=0.592746)
    c.add_argument("--runs", type=int, default=400)
    args = ap.parse_args(argv)
    if args.cmd == "std":
        print(json.dumps(std_vs_size(args.k, args.ratios, args.runs)))
    elif args.cmd == "csd":
        hists, nj, nc = percolation_cluster_sizes(args.L, args.k, args.runs)
        s, n_s = cluster_size_distribution(args.L, args.k, hists)
        xs, ys = log_binned(s, n_s)
        print(json.dumps({"L": args.L, "k": args.k, "runs": args.runs,
                          "coverage": coverage_stats(args.L, args.k, nj, nc),
                          "log_bins": [[float(x), float(y)] for x, y in zip(xs, ys)]}))
    else:
        print(json.dumps(wrap_probabilities(args.L, args.k, args.p, args.runs)))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
