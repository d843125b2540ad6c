#!/usr/bin/env python3
"""Write tests/golden/fullsize.json: oracle results of full-size samples.

The oracle (a sequential priority-order scan plus union-find, Sec. II.B to
II.D of arXiv:1810.06800) needs minutes per sample at L = 8192 and over an
hour and 35 GB of host memory per sample at L = 32768, too long to rerun
inside a test.  This script runs it once, one sample at a time, and stores
per (L, k, seed):
  n_j       number of accepted k-mers at jamming,
  n_c       number placed when a cluster first wraps (exact rule),
  n_c_paper the same by the paper's |x1-x2|+|y1-y2| > 2k test (Sec. II.D),
  acc_sha256  SHA-256 of the accepted candidate indices, sorted ascending,
              as little-endian uint32 (idx = (o*L + y)*L + x),
  first_idx, nc_idx  the first accepted candidate and the n_c-th one in scan
              order (the k-mer whose placement makes the first wrap).
Only oracle/ is called; nothing here reads the CUDA library.

  python tests/golden/make_fullsize.py --case 8192,512 --seeds 1-8
  python tests/golden/make_fullsize.py --case 32768,4096 --seeds 1 --out part1.json
  python tests/golden/make_fullsize.py --merge part1.json part2.json
  python tests/golden/make_fullsize.py --case 32768,4096 --seeds 4 --parts 16 --out p4.json

Entries already in the file are kept, so runs can be split and resumed;
--out writes to another file (one process per sample, several at once, on a
host with room for them), and --merge adds such files' entries here.
--parts splits the oracle's sort into key ranges handled one at a time, so
that an L = 32768 sample holds about 2 GB of sort pairs instead of 34 GB.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "fullsize.json")


def parse_seeds(s: str):
    out = []
    for part in s.split(","):
        if "-" in part:
            a, b = part.split("-")
            out.extend(range(int(a), int(b) + 1))
        else:
            out.append(int(part))
    return out


def one(L: int, k: int, seed: int, parts: int = 1) -> dict:
    import numpy as np

    import oracle
    t0 = time.perf_counter()
    acc, occ = oracle.scan_seed(L, k, seed, parts)
    del occ
    nc, ncp = oracle.percolation(L, k, acc)
    srt = np.sort(acc).astype("<u4")
    return {
        "L": L, "k": k, "seed": seed,
        "n_j": int(acc.size), "n_c": int(nc), "n_c_paper": int(ncp),
        "acc_sha256": hashlib.sha256(srt.tobytes()).hexdigest(),
        "first_idx": int(acc[0]), "nc_idx": int(acc[nc - 1]) if nc > 0 else None,
        "oracle_s": round(time.perf_counter() - t0, 1),
    }


def load(path: str) -> dict:
    db = {"_note": ("Oracle results of full-size samples, written by "
                    "tests/golden/make_fullsize.py (oracle/ only): n_j, n_c "
                    "(Sec. II.B-II.D of arXiv:1810.06800) and a SHA-256 of the "
                    "sorted accepted candidate indices."),
          "samples": {}}
    if os.path.exists(path):
        with open(path) as f:
            db = json.load(f)
    return db


def save(db: dict, path: str) -> None:
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(db, f, indent=1, sort_keys=True)
        f.write("\n")
    os.replace(tmp, path)


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", help="L,k")
    ap.add_argument("--seeds", help="e.g. 1-8 or 1,2,5")
    ap.add_argument("--out", default=OUT, help="file to add the entries to")
    ap.add_argument("--merge", nargs="*", help="add the entries of these files")
    ap.add_argument("--parts", type=int, default=1,
                    help="split the oracle's sort into this many key ranges (less memory)")
    args = ap.parse_args()
    if args.merge:
        db = load(OUT)
        for path in args.merge:
            db["samples"].update(load(path)["samples"])
        save(db, OUT)
        return 0
    L, k = (int(v) for v in args.case.split(","))
    sys.path.insert(0, ROOT)
    out = args.out
    db = load(out)
    for seed in parse_seeds(args.seeds):
        key = f"{L},{k},{seed}"
        if key in db["samples"]:
            continue
        rec = one(L, k, seed, args.parts)
        rec["host"] = f"{platform.machine()}, {os.cpu_count()} cores"
        db["samples"][key] = rec
        save(db, out)
        print(json.dumps(rec), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
