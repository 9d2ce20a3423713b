"""bench.py's host-side arithmetic without a GPU: the committed ncu records are used only
while they match the sources, the HBM roofline entry, and the e2e floor the host link
sets."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_ncu_records_are_complete():
    d = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
    assert {"k_step_soa_fused_gather", "k_step_soa", "k_adj_forward", "k_adj_reverse", "k_step_batched_fused",
            "k_step_aos"} <= set(d)
    for k, e in d.items():
        assert len(e["source_hash"]) == 16, k
        assert bench.source_hash(e["unit"]) == e["source_hash"], k
        assert e["inst_per_particle_step"] > 0 and e["dram_bytes_per_launch_full_size"] > 0, k
        assert os.path.exists(os.path.join(ROOT, e["summary"])), k


def test_records_ignored_when_the_sources_differ(monkeypatch):
    monkeypatch.setattr(bench, "source_hash", lambda unit: "0" * 16)
    assert bench.ncu_record("k_step_soa_fused_gather") is None
    assert bench.ncu_traffic("k_step_soa_fused_gather") is None
    assert bench.hbm_roofline(72, 1000, 1e-6, "k_step_soa")["traffic"] is None


def test_unit_sources_follow_includes():
    src = [os.path.basename(f) for f in bench.unit_sources("step_fused.cu")]
    for f in ("step_fused.cu", "step_fused.cuh", "rk2_turns.cuh", "rk2_fast.cuh", "trig_table.inc", "cell_key.cuh",
              "step_core.cuh", "soax_internal.h", "soax.h", "build.py"):
        assert f in src, f
    assert "sort.cu" not in src and "api.cu" not in src


def test_hbm_roofline(monkeypatch):
    monkeypatch.setattr(bench, "measured_peaks", lambda: (6500.0, "measured"))
    r = bench.hbm_roofline(72, 16777216, 0.5e-3)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == 6500.0
    assert r["achieved"] == pytest.approx(72 * 16777216 / 0.5e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6500.0)


def test_e2e_floor():
    link = {"h2d_GB/s": 50.0, "d2h_GB/s": 50.0, "both_GB/s": 100.0}
    # A full-duplex link (both directions at once at twice one direction's rate): the k
    # intervals' sort gaps, k - 1 round trips between them at the combined rate (one
    # direction's time each), and the first upload and the last download alone.
    b, t, k, u = 1e9, 2e-3, 5, 1e9
    per = b / 50e9
    want = u * k / (k * t + (k - 1) * per + 2 * per)
    assert bench.e2e_floor(u, k, t, b, link) == pytest.approx(want)
    # One interval: the upload, the gap and the download in sequence.
    assert bench.e2e_floor(u, 1, t, b, link) == pytest.approx(u / (t + 2 * per))
    # A faster combined link can only raise the floor; the floor never beats the gaps
    # alone.
    fast = dict(link, **{"both_GB/s": 200.0})
    assert bench.e2e_floor(u, k, t, b, fast) > bench.e2e_floor(u, k, t, b, link)
    assert bench.e2e_floor(u, k, t, b, link) < u / t


def test_source_hash_ignores_comments_only():
    a = "int f(int x) {  // the step\n  return x + 1; /* one */\n}\n# build flag\n"
    b = "/* header */\nint f(int x) {\n  return x + 1;\n}\n"
    c = "int f(int x) {\n  return x + 2;\n}\n"
    assert bench.code_only(a) == bench.code_only(b)
    assert bench.code_only(a) != bench.code_only(c)
    assert "#include <x>" in bench.code_only("#include <x>\n// note\n")


def test_sort_kernel_launches():
    assert bench.sort_kernel_launches(32) == 6 + 1   # 15 bits: counting sort + the conditional's kernel
    assert bench.sort_kernel_launches(64) == 6 + 1   # 18 bits
    assert bench.sort_kernel_launches(100) == 9      # 20 bits: the radix passes alone
