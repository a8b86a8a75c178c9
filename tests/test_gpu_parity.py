"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Small workloads are compared in full (every bin, every level's blocks and masks
in lockstep, every adjacency list and link).  Full-size workloads run on the GPU
in the configuration the bench times and are checked on seeded samples the
oracle evaluates one by one, plus exact integer properties at every size.
"""
import numpy as np
import pytest

from synth import small_workload, workload
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


def _oracle(w, B=None):
    from oracle.oracle import Domain, OracleGeometry

    geo = OracleGeometry(w.dim, w.verts, w.idx)
    off, ids = geo.bin(Domain.unit(w.dim, w.root), w.bins if B is None else B)
    return geo, off, ids


def _full_check(w, out, geo, sample=None, links=True, B=None):
    from oracle.oracle import root_blocks

    lv = out["levels"]
    assert np.array_equal(lv[0]["blocks"], root_blocks(w.dim, (w.root,) * w.dim))
    rng = np.random.default_rng(123)
    stats = []
    for L in range(len(lv)):
        n, nb = U.compare_level(geo, w.dim, L, lv[L]["blocks"], lv[L]["mask"], sample=sample, d_abs=w.d_abs,
                                d_rel=w.d_rel, rng=rng)
        assert np.array_equal(lv[L]["flag"].astype(bool), lv[L]["mask"] != 0)
        stats.append((n, nb))
        if L + 1 < len(lv):
            U.check_children(w.dim, lv[L]["blocks"], lv[L]["mask"], lv[L + 1]["blocks"], lv[L + 1]["parent"])
    fin = lv[-1]
    Lf = len(lv) - 1
    U.compare_adjacency(geo, w.dim, Lf, fin["blocks"], fin["mask"], out["adj_cell"], out["adj_off"], out["adj_ids"],
                        sample=sample, d_abs=w.d_abs, d_rel=w.d_rel, rng=rng)
    if links:
        U.compare_links(geo, w.dim, Lf, w.lattice, fin["blocks"], out["adj_cell"], out["link_cell"],
                        out["link_dir"], out["link_q"], out["link_face"], sample=sample, rng=rng, d_abs=w.d_abs,
                        d_rel=w.d_rel)
    return stats


@pytest.mark.parametrize("kind", ["circle", "sphere3", "bumpy3"])
def test_small_full_parity(kind):
    w = small_workload(kind)
    out = U.run_gpu(w)
    geo, off, ids = _oracle(w)
    U.compare_bins(out["offsets"], out["ids"], off, ids)
    _full_check(w, out, geo)


def test_c1_full_parity():
    import json
    import os

    w = workload("c1")
    out = U.run_gpu(w)
    geo, off, ids = _oracle(w)
    U.compare_bins(out["offsets"], out["ids"], off, ids)
    _full_check(w, out, geo)
    # and the stored oracle summary (level sizes are integer results)
    want = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "c1_levels.json")))
    for L, lv in enumerate(want["levels"]):
        assert out["levels"][L]["blocks"].shape[0] == lv["blocks"]
        assert int((out["levels"][L]["mask"] != 0).sum()) == lv["marked"]
    assert out["adj_cell"].shape[0] == want["levels"][-1]["adjacent_cells"]


def test_facelist_equals_indexed():
    w = small_workload("bumpy3")
    a = U.run_gpu(w)
    b = U.run_gpu(w, facelist=True)
    for L in range(len(a["levels"])):
        assert np.array_equal(a["levels"][L]["mask"], b["levels"][L]["mask"])
    assert np.array_equal(a["adj_ids"], b["adj_ids"])
    assert np.array_equal(a["link_q"], b["link_q"]) and np.array_equal(a["link_face"], b["link_face"])


@pytest.mark.parametrize("B", [1, 2, 5, 40])
def test_bin_density_independence(B):
    """Exact binning only prunes candidates: results for any B equal those of the paper's naive B = 1."""
    w = small_workload("sphere3")
    ref = U.run_gpu(w)
    out = U.run_gpu(w, B=B)
    geo, off, ids = _oracle(w, B)
    U.compare_bins(out["offsets"], out["ids"], off, ids)
    for L in range(len(ref["levels"])):
        assert np.array_equal(ref["levels"][L]["mask"], out["levels"][L]["mask"])
    assert np.array_equal(ref["adj_ids"], out["adj_ids"])
    assert np.array_equal(ref["link_q"], out["link_q"])


@pytest.mark.parametrize("B", [200, 256])
def test_fine_bin_grid(B):
    """Grids of 8.0 M and 16.8 M bins: thousands of scan tiles chained by the look-back (at B = 200
    the last tile is partial).  Bins exact against the oracle; every result equal to that of B = 1."""
    w = small_workload("sphere3")
    ref = U.run_gpu(w, B=1)
    out = U.run_gpu(w, B=B)
    geo, off, ids = _oracle(w, B)
    U.compare_bins(out["offsets"], out["ids"], off, ids)
    for L in range(len(ref["levels"])):
        assert np.array_equal(ref["levels"][L]["mask"], out["levels"][L]["mask"])
    assert np.array_equal(ref["adj_ids"], out["adj_ids"])
    assert np.array_equal(ref["link_q"], out["link_q"])


def test_deterministic_repeat():
    w = small_workload("bumpy3")
    a = U.run_gpu(w)
    b = U.run_gpu(w)
    assert np.array_equal(a["adj_ids"], b["adj_ids"])
    assert np.array_equal(a["link_q"], b["link_q"]) and np.array_equal(a["link_face"], b["link_face"])


@pytest.mark.parametrize("name", ["c2", "c3"])
def test_full_size_sampled(name):
    w = workload(name)
    out = U.run_gpu(w, use_graph=True)
    geo, off, ids = _oracle(w)
    U.compare_bins(out["offsets"], out["ids"], off, ids)
    _full_check(w, out, geo, sample=300)


@pytest.mark.slow
def test_c4_full_size_sampled():
    w = workload("c4")
    out = U.run_gpu(w, use_graph=True)
    geo, off, ids = _oracle(w)
    U.compare_bins(out["offsets"], out["ids"], off, ids)
    _full_check(w, out, geo, sample=200)
