"""GPU edge cases and error statuses through the C ABI."""
import numpy as np
import pytest

from synth import Workload, small_workload
from synth import geometry as G
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


def _oracle_check(w, out, B=None):
    from oracle.oracle import Domain, OracleGeometry

    geo = OracleGeometry(w.dim, w.verts, w.idx)
    off, ids = geo.bin(Domain.unit(w.dim, w.root), w.bins if B is None else B)
    U.compare_bins(out["offsets"], out["ids"], off, ids)
    lv = out["levels"]
    for L in range(len(lv)):
        U.compare_level(geo, w.dim, L, lv[L]["blocks"], lv[L]["mask"], d_abs=w.d_abs, d_rel=w.d_rel)
        if L + 1 < len(lv):
            U.check_children(w.dim, lv[L]["blocks"], lv[L]["mask"], lv[L + 1]["blocks"], lv[L + 1]["parent"])
    U.compare_adjacency(geo, w.dim, len(lv) - 1, lv[-1]["blocks"], lv[-1]["mask"], out["adj_cell"], out["adj_off"],
                        out["adj_ids"], d_abs=w.d_abs, d_rel=w.d_rel)
    if "link_q" in out:
        U.compare_links(geo, w.dim, len(lv) - 1, w.lattice, lv[-1]["blocks"], out["adj_cell"], out["link_cell"],
                        out["link_dir"], out["link_q"], out["link_face"], d_abs=w.d_abs, d_rel=w.d_rel)


def test_empty_geometry():
    w = Workload("empty", 3, np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32), root=3, n_levels=3, bins=4,
                 lattice=19)
    out = U.run_gpu(w)
    assert out["ids"].shape[0] == 0 and np.all(out["offsets"] == 0)
    assert out["levels"][0]["blocks"].shape[0] == 27
    assert np.all(out["levels"][0]["mask"] == 0)
    assert out["levels"][1]["blocks"].shape[0] == 0 and out["levels"][2]["blocks"].shape[0] == 0
    assert out["adj_cell"].shape[0] == 0 and out["link_q"].shape[0] == 0


def test_single_level_and_ragged_root():
    v, f = G.jittered_sphere(2, radius=0.3, centre=(0.45, 0.52, 0.5), sigma=1e-3, seed=3)
    w = Workload("ragged", 3, v, f, root=5, n_levels=1, bins=7, lattice=19)
    out = U.run_gpu(w)
    _oracle_check(w, out)


def test_faces_outside_domain_and_degenerate():
    rng = np.random.default_rng(4)
    v, f = G.jittered_sphere(1, radius=0.3, centre=(0.5, 0.5, 0.5), sigma=1e-3, seed=8)
    tri = v[f]
    extra = np.array([
        [[1.5, 0.5, 0.5], [1.6, 0.5, 0.5], [1.5, 0.6, 0.5]],     # outside the domain
        [[0.2, 0.2, 0.2], [0.2, 0.2, 0.2], [0.2, 0.2, 0.2]],     # a point
        [[0.1, 0.1, 0.1], [0.3, 0.3, 0.3], [0.2, 0.2, 0.2]],     # collinear
        [[0.125, 0.3, 0.3], [0.125, 0.35, 0.3], [0.125, 0.3, 0.4]],  # on a cell boundary plane
    ], np.float32)
    fv = np.concatenate([tri, extra, (rng.uniform(0.05, 0.95, (5, 1, 3)) + rng.normal(0, 0.01, (5, 3, 3)))
                         .astype(np.float32)])
    verts = fv.reshape(-1, 3)
    idx = np.arange(verts.shape[0], dtype=np.int32).reshape(-1, 3)
    w = Workload("odd", 3, verts, idx, root=4, n_levels=3, bins=6, lattice=19)
    out = U.run_gpu(w)
    _oracle_check(w, out)


def test_links_beyond_the_first_capacity_guess():
    """A flat square just off the cell centres: about 5 links per cell next to it and 3 per (cell, face)
    pair, so the first eager pass's link capacity (a quarter above the pair count) is too small and the
    level's links are run again at their exact count; eager and graph-replay outputs agree with each
    other and, on sampled rows, with the oracle."""
    h = 1.0 / 128.0
    z0 = 0.5 + 0.37 * h
    v = np.array([[0.1, 0.1, z0], [0.9, 0.1, z0], [0.9, 0.9, z0], [0.1, 0.9, z0]], np.float32)
    f = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    w = Workload("flat", 3, v, f, root=16, n_levels=2, bins=16, lattice=19)
    out = U.run_gpu(w)
    n_pairs, n_links = out["adj_ids"].shape[0], out["link_q"].shape[0]
    assert n_links > n_pairs + n_pairs // 4 + 1024, (n_links, n_pairs)  # the re-run path ran
    again = U.run_gpu(w, use_graph=True)
    for k in ("adj_cell", "adj_off", "adj_ids", "link_cell", "link_dir", "link_face"):
        assert np.array_equal(out[k], again[k]), k
    assert np.array_equal(out["link_q"].view(np.uint32), again["link_q"].view(np.uint32))
    from oracle.oracle import Domain, OracleGeometry

    geo = OracleGeometry(3, w.verts, w.idx)
    geo.bin(Domain.unit(3, w.root), w.bins)
    lv = out["levels"]
    rng = np.random.default_rng(5)
    U.compare_adjacency(geo, 3, 1, lv[1]["blocks"], lv[1]["mask"], out["adj_cell"], out["adj_off"], out["adj_ids"],
                        sample=300, rng=rng, d_abs=w.d_abs, d_rel=w.d_rel)
    U.compare_links(geo, 3, 1, 19, lv[1]["blocks"], out["adj_cell"], out["link_cell"], out["link_dir"],
                    out["link_q"], out["link_face"], sample=400, rng=rng, d_abs=w.d_abs, d_rel=w.d_rel)


def _wall_grid(lo, hi, h, n_walls, off):
    """Axis-aligned square walls, each two triangles spanning [lo, hi]^2 in the other two axes, at
    coordinates (i + off) h for the given wall indices, in all three axes."""
    tris = []
    for axis in range(3):
        u, v = [(axis + 1) % 3, (axis + 2) % 3]
        for i in n_walls:
            c = (i + off) * h
            corners = []
            for a, b in ((lo, lo), (hi, lo), (hi, hi), (lo, hi)):
                p = [0.0, 0.0, 0.0]
                p[axis], p[u], p[v] = c, a, b
                corners.append(p)
            tris += [[corners[0], corners[1], corners[2]], [corners[0], corners[2], corners[3]]]
    t = np.array(tris, np.float32)
    return t.reshape(-1, 3), np.arange(t.shape[0] * 3, dtype=np.int32).reshape(-1, 3)


def test_links_dense_tile():
    """Walls between every pair of neighbouring cell centres in all three axes: every inner cell has all
    18 links, so a tile of 128 cells holds more links than the link kernel gathers in shared memory
    (1,792) and stores them directly; the outputs agree with the oracle on sampled rows."""
    h = 1.0 / 64.0
    v, f = _wall_grid(0.36, 0.64, h, range(23, 40), 0.87)
    w = Workload("walls", 3, v, f, root=8, n_levels=2, bins=16, lattice=19)
    out = U.run_gpu(w)
    per_tile = np.bincount(out["link_cell"].astype(np.int64) // 128)
    assert per_tile.max() > 1792, per_tile.max()
    assert np.all(np.diff(out["link_cell"].astype(np.int64) * 32 + out["link_dir"]) > 0)
    from oracle.oracle import Domain, OracleGeometry

    geo = OracleGeometry(3, w.verts, w.idx)
    geo.bin(Domain.unit(3, w.root), w.bins)
    lv = out["levels"]
    rng = np.random.default_rng(6)
    U.compare_links(geo, 3, 1, 19, lv[1]["blocks"], out["adj_cell"], out["link_cell"], out["link_dir"],
                    out["link_q"], out["link_face"], sample=300, rng=rng, d_abs=w.d_abs, d_rel=w.d_rel)


def test_2d_naive_bins_and_half_cell_distance():
    w = small_workload("circle")
    w.d_rel = 0.5  # the smallest near-wall distance links allow
    out = U.run_gpu(w, B=1)
    _oracle_check(w, out, B=1)


def test_status_codes():
    import torch

    from paper_2502_16310_gb300 import AmrError, AmrGeom
    from paper_2502_16310_gb300 import binding as Bd

    g = AmrGeom(3, (4, 4, 4))
    with pytest.raises(AmrError) as e:
        g.bin(8)
    assert e.value.status == Bd.AMR_ESTATE
    v = torch.rand(10, 3, device="cuda")
    bad = torch.tensor([[0, 1, 10]], dtype=torch.int32, device="cuda")
    g.load(v, bad)
    with pytest.raises(AmrError) as e:
        g.bin(4)
    assert e.value.status == Bd.AMR_EDEVICE_CHECK
    nanv = v.clone()
    nanv[3, 1] = float("nan")
    g.load(nanv, torch.tensor([[0, 1, 3]], dtype=torch.int32, device="cuda"))
    with pytest.raises(AmrError) as e:
        g.bin(4)
    assert e.value.status == Bd.AMR_EDEVICE_CHECK
    # context stays usable after device-check errors
    g.load(v, torch.tensor([[0, 1, 2]], dtype=torch.int32, device="cuda"))
    g.bin(4)
    with pytest.raises(AmrError) as e:
        g.refine(2, 0.0, 0.25, 19, True, True)  # d < h/2 with links
    assert e.value.status == Bd.AMR_EINVAL
    with pytest.raises(AmrError) as e:
        g.bin(0)
    assert e.value.status == Bd.AMR_EINVAL
    g.close()
