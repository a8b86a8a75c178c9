"""Host-side logic of bench.py on CPU: the defaults the timing rules need, the end-to-end leg's
thread and context layout, and the binning roofline's byte count."""
import os
import sys
from types import SimpleNamespace

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_defaults_meet_the_timing_rules():
    a = bench.parse_args([])
    assert a.gpus == 1 and a.warmup >= 3 and a.steps >= 1
    assert a.workload == "c4" and a.impl == "ours"
    assert a.e2e_threads == 0 and not a.bin_only
    assert bench.parse_args(["--bin-only", "--workload", "c4"]).bin_only


def test_e2e_layout():
    # small outputs: three threads with a context each; gigabytes: one thread alternating two contexts
    assert bench.e2e_layout(192_472_876, 0) == (3, 1)
    assert bench.e2e_layout(10_348_729_530, 0) == (1, 2)
    assert bench.e2e_layout(int(2e9) - 1, 0) == (3, 1)
    assert bench.e2e_layout(int(2e9), 0) == (1, 2)
    # an explicit thread count wins, one context each
    assert bench.e2e_layout(10_348_729_530, 4) == (4, 1)
    assert bench.e2e_layout(1, 1) == (1, 1)


def test_bin_roofline_bytes():
    # the method's bytes: coordinates read twice (2 x 36 B per face), 16 B per bin, and per incidence
    # the 4-byte id plus the face's 36 B of coordinates
    w = SimpleNamespace(dim=3, bins=4, n_faces=10)
    r = bench.bin_roofline(w, 15, 1e-3)
    assert r["bytes"] == 720 + 16 * 64 + 40 * 15
    assert abs(r["achieved"] - r["bytes"] / 1e-6 / 1e9) < 1e-9
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    # the implementation's bytes beside it: bin ranges written and read (2 x 12 B per face), 4 + 64 B per
    # incidence
    assert r["impl_bytes"] == 720 + 240 + 16 * 64 + 68 * 15
    assert r["impl_frac"] > r["frac"]
    # 2D: 16 B of coordinates per face and incidence (32-byte entries in the implementation)
    w2 = SimpleNamespace(dim=2, bins=8, n_faces=5)
    r2 = bench.bin_roofline(w2, 7, 1e-3)
    assert r2["bytes"] == 2 * 16 * 5 + 16 * 64 + 20 * 7
    assert r2["impl_bytes"] == 2 * 16 * 5 + 2 * 8 * 5 + 16 * 64 + 36 * 7


def test_links_roofline_counts_the_survey_ops():
    # 40 ops per (adjacent cell, face, lattice direction); the per-pair setup is reported beside it
    w = SimpleNamespace(dim=3, bins=4, n_faces=10)
    k = {"ms_per_step": 2.0, "launches_per_step": 1.0}
    r = bench.roofline("links", k, w, {}, 0, 0, 0, 1000, [], {})
    assert abs(r["achieved"] - 1000 * 18 * 40 / 2e-3 / 1e12) < 1e-12
    assert r["with_per_pair_setup_tops"] > r["achieved"]
    assert r["bound"] == "alu" and abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-15
