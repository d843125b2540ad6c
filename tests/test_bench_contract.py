"""bench.py's host-side contract, checked without a GPU: the reference arm
(the CPU oracle) prints one JSON line with the keys the benchmark contract
requires, the seed sharding gives ranks disjoint seed ranges, and the
traffic-figure digest ignores comments but not code."""
import importlib.util
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "L64_k4_x100", "--steps", "2", "--warmup", "1"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == "L64_k4_x100"


def test_seed_shards_are_disjoint_and_cover_the_ranks():
    b = _bench()
    seen = set()
    for rank in range(4):
        s = [int(x) for x in b.shard_seeds(rank, 100)]
        assert len(s) == 100 and s == list(range(rank * 100 + 1, rank * 100 + 101))
        assert not seen & set(s)
        seen |= set(s)


def test_source_digest_ignores_comments_only(tmp_path, monkeypatch):
    b = _bench()
    csrc = tmp_path / "paper_1810_06800_gb300" / "csrc"
    csrc.mkdir(parents=True)
    f = csrc / "rsa_tile.cuh"
    f.write_text("int a = 1;  // one\n\nint b = 2;\n")
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    d0 = b.src_digest("k_tile_cmin")
    f.write_text("// a new header line\nint a = 1;  // the first\nint b = 2;\n")
    assert b.src_digest("k_tile_cmin") == d0
    f.write_text("int a = 1;\nint b = 3;\n")
    assert b.src_digest("k_tile_cmin") != d0


def test_roofline_arithmetic_and_traffic_freshness(tmp_path, monkeypatch):
    # achieved = byte model x cells processed / summed event time; frac
    # against the given peak; traffic = the stored bytes per cell x cells per
    # launch only while the kernel's source digest matches the stored one
    b = _bench()
    kst = {"k_lwin_h": (10.0, 2)}                     # 10 ms over 2 launches
    work = {"raw": [1_000_000_000, 0, 0, 0]}          # cells of the horizontal pass
    r = b.roofline("k_lwin_h", kst, work, 0, 0, 0, 5000.0, "measured", 152, 2070.0)
    assert r["alg_bytes_per_cell"] == 16.0 and r["steps"] == ["rowmin"]
    assert abs(r["achieved"] - 16.0 * 1e9 / 0.010 / 1e9) < 1e-6
    assert abs(r["frac"] - r["achieved"] / 5000.0) < 1e-12
    assert r["cells_per_launch"] == 5e8 and r["avg_launch_ms"] == 5.0
    csrc = tmp_path / "paper_1810_06800_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "rsa_lwin.cuh").write_text("int window_pass;\n")
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    entry = {"bytes_per_cell": 2.0, "src": b.src_digest("k_lwin_h")}
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(json.dumps({"k_lwin_h": entry}))
    r = b.roofline("k_lwin_h", kst, work, 0, 0, 0, 5000.0, "measured", 152, 2070.0)
    assert r["traffic"] == 2.0 * 5e8
    # a capture of one window-pass CTA size counts only for runs that ask for it
    entry["window_threads"] = 256
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(json.dumps({"k_lwin_h": entry}))
    r = b.roofline("k_lwin_h", kst, work, 0, 0, 0, 5000.0, "measured", 152, 2070.0, 256)
    assert r["traffic"] == 2.0 * 5e8
    for asked in (0, 128):
        r = b.roofline("k_lwin_h", kst, work, 0, 0, 0, 5000.0, "measured", 152, 2070.0, asked)
        assert r["traffic"] is None
    (csrc / "rsa_lwin.cuh").write_text("int window_pass_changed;\n")
    r = b.roofline("k_lwin_h", kst, work, 0, 0, 0, 5000.0, "measured", 152, 2070.0, 256)
    assert r["traffic"] is None
    # no byte model: no fraction
    r = b.roofline("k_edges", {"k_edges": (3.0, 1)}, work, 1, 64, 4096, 5000.0, "measured",
                   152, 2070.0)
    assert r["frac"] is None
