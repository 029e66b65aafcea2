"""Host-side logic of bench.py (CPU): the roofline's bound and figures, and
the committed per-launch ncu figures keyed to the kernels' sources."""
import os
import sys

import pytest

sys.path.insert(0, os.path.join(os.path.dirname(__file__), ".."))
import bench  # noqa: E402

SMS, MHZ, HBM = 152, 2070.0, 6803.8
PEAK = SMS * 128 * MHZ * 1e6 / 1e9


def test_l2_fed_family_is_issue_bound():
    alg, t = 10e9, 2.0e-3
    prof = {"bytes_per_launch": 2.2e9, "inst_per_launch": 40e9}
    r = bench.roofline_record(alg, 8e9, t, prof, HBM, "measured", SMS, MHZ)
    assert r["bound"] == "alu" and r["unit"] == "Ginst/s"
    assert r["achieved"] == pytest.approx(40e9 / t / 1e9, rel=1e-3)
    assert r["peak"] == pytest.approx(PEAK, rel=1e-3)
    assert r["frac"] == pytest.approx(40e9 / t / 1e9 / PEAK, abs=1e-4)
    assert r["traffic"] == 2.2e9
    assert r["hbm_view"]["frac"] == pytest.approx(alg / t / 1e9 / HBM, abs=1e-4)


def test_dram_bound_family_is_hbm_bound():
    alg, t = 10e9, 2.0e-3
    for prof in ({"bytes_per_launch": 6e9, "inst_per_launch": 40e9},  # traffic near the algorithmic bytes
                 {"bytes_per_launch": 1e9},                           # no instruction count
                 {}):                                                 # nothing committed for these sources
        r = bench.roofline_record(alg, 8e9, t, prof, HBM, "measured", SMS, MHZ)
        assert r["bound"] == "hbm" and r["unit"] == "GB/s"
        assert r["achieved"] == pytest.approx(alg / t / 1e9, rel=1e-3)
        assert r["frac"] == pytest.approx(alg / t / 1e9 / HBM, abs=1e-4)
        assert r["traffic"] == prof.get("bytes_per_launch")


def test_committed_profile_keyed_to_sources(tmp_path):
    cur = bench.source_hash()
    f = tmp_path / "traffic.txt"
    f.write_text("# comment\n"
                 f"kernel=k:w source={cur} bytes_per_launch=123 inst_per_launch=456 units_per_launch=7\n"
                 "kernel=k:old source=0000000000000000 bytes_per_launch=1 inst_per_launch=2\n")
    assert bench.committed_profile("k:w", str(f)) == {"bytes_per_launch": 123.0, "inst_per_launch": 456.0}
    assert bench.committed_profile("k:old", str(f)) == {}   # taken on other sources
    assert bench.committed_profile("k:none", str(f)) == {}


def test_committed_traffic_file_parses():
    """Every line of the committed file names a known kernel family and
    carries numeric per-launch figures and a 16-hex-digit source hash."""
    path = os.path.join(os.path.dirname(bench.__file__), "profiles", "traffic.txt")
    lines = [ln for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert lines
    for ln in lines:
        kv = dict(x.split("=", 1) for x in ln.split() if "=" in x)
        fam, _, workload = kv["kernel"].partition(":")
        assert fam in bench.KERNEL_NAMES and workload
        assert len(kv["source"]) == 16 and int(kv["source"], 16) >= 0
        assert float(kv["bytes_per_launch"]) > 0 and float(kv["inst_per_launch"]) > 0


def test_source_hash_ignores_comments_and_whitespace():
    src = 'int a = 1; // note\n/* block\n comment */ const char *s = "x // y";  int b;'
    assert bench._code_only(src) == bench._code_only('int a = 1;\nconst char *s = "x // y"; int b; // other')
    assert bench._code_only(src) != bench._code_only('int a = 2; const char *s = "x // y"; int b;')
    assert bench._code_only(src) != bench._code_only('int a = 1; const char *s = "x / y"; int b;')
