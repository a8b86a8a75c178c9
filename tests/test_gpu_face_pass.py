"""Face-by-face marking of the mask-only levels (k_mark_faces) against the block walk: the two make the
same certified decisions (FP64 where not certified), so every output is identical bit for bit — block
lists, masks, flags, parents, adjacency lists and links — for both predicates, in 2D and 3D, on odd
geometry (faces outside the domain, degenerate faces, a non-cubic root grid) and when the finest level
is mask-only too (no adjacency).  Parity with the oracle under the face pass is covered by the other
parity tests, which run with the default (automatic) choice."""
import numpy as np
import pytest

from synth import Workload, small_workload
from synth import geometry as G
from tests import gpu_util as U

pytestmark = pytest.mark.gpu

ON, OFF = 2, 1


def _same(a, b):
    assert len(a["levels"]) == len(b["levels"])
    for L, (x, y) in enumerate(zip(a["levels"], b["levels"])):
        for k in ("blocks", "mask", "flag", "parent"):
            if x[k] is None:
                assert y[k] is None
                continue
            assert np.array_equal(x[k], y[k]), (L, k)
    # bin lists are sets (the scatter's order within a bin is not fixed)
    assert np.array_equal(a["offsets"], b["offsets"])
    seg = np.repeat(np.arange(a["offsets"].shape[0] - 1), np.diff(a["offsets"].astype(np.int64)))
    assert np.array_equal(a["ids"][np.lexsort((a["ids"], seg))], b["ids"][np.lexsort((b["ids"], seg))])
    for k in ("adj_cell", "adj_off", "adj_ids", "link_cell", "link_dir", "link_q", "link_face"):
        if k in a or k in b:
            assert np.array_equal(np.asarray(a[k]).view(np.uint8), np.asarray(b[k]).view(np.uint8)), k


@pytest.mark.parametrize("kind", ["circle", "sphere3", "bumpy3"])
@pytest.mark.parametrize("predicate", [0, 1])
def test_face_pass_equals_block_walk(kind, predicate):
    w = small_workload(kind)
    d = {} if predicate == 0 else {"d_abs": 0.0, "d_rel": 1.5}
    links = predicate == 0
    on = U.run_gpu(w, face_pass=ON, predicate=predicate, want_links=links, **d)
    off = U.run_gpu(w, face_pass=OFF, predicate=predicate, want_links=links, **d)
    _same(on, off)
    assert on["n_face_setups"] > 0 and on["n_face_tests"] > 0
    assert off["n_face_setups"] == 0 and off["n_face_tests"] == 0
    assert sum(int(lv["flag"].sum()) for lv in on["levels"][:-1]) > 0


def test_face_pass_mask_only_finest_level():
    w = small_workload("bumpy3")
    on = U.run_gpu(w, face_pass=ON, want_links=False, want_adjacency=False)
    off = U.run_gpu(w, face_pass=OFF, want_links=False, want_adjacency=False)
    _same(on, off)
    assert int((on["levels"][-1]["mask"] != 0).sum()) > 0


def test_face_pass_odd_geometry_and_non_cubic_root():
    rng = np.random.default_rng(21)
    v, f = G.jittered_sphere(2, radius=0.3, centre=(0.5, 0.5, 0.5), sigma=1e-3, seed=5)
    tri = v[f]
    extra = np.array([
        [[1.5, 0.5, 0.5], [1.6, 0.5, 0.5], [1.5, 0.6, 0.5]],        # outside the domain
        [[-0.4, -0.2, 0.3], [-0.3, -0.2, 0.3], [-0.4, -0.1, 0.3]],  # outside, negative side
        [[0.2, 0.2, 0.2], [0.2, 0.2, 0.2], [0.2, 0.2, 0.2]],        # a point
        [[0.1, 0.1, 0.1], [0.3, 0.3, 0.3], [0.2, 0.2, 0.2]],        # collinear
        [[0.125, 0.3, 0.3], [0.125, 0.35, 0.3], [0.125, 0.3, 0.4]],  # on a cell boundary plane
        [[-0.1, 0.4, 0.4], [1.1, 0.45, 0.4], [0.5, 0.5, 1.2]],       # larger than the domain
    ], np.float32)
    fv = np.concatenate([tri, extra, (rng.uniform(0.05, 0.95, (7, 1, 3)) + rng.normal(0, 0.02, (7, 3, 3)))
                         .astype(np.float32)])
    verts = fv.reshape(-1, 3)
    idx = np.arange(verts.shape[0], dtype=np.int32).reshape(-1, 3)
    w = Workload("odd", 3, verts, idx, root=5, n_levels=3, bins=6, lattice=19)
    for root in ((5, 5, 5), (6, 3, 4)):
        on = U.run_gpu(w, face_pass=ON, root=root)
        off = U.run_gpu(w, face_pass=OFF, root=root)
        _same(on, off)


def test_face_pass_2d_odd_segments():
    v, f = G.circle_polygon(61, 0.3, (0.5, 0.5))
    extra_v = np.array([[1.2, 0.5], [1.4, 0.6], [0.3, 0.3], [0.3, 0.3], [-0.2, 0.5], [1.3, 0.52]], np.float32)
    verts = np.concatenate([v, extra_v]).astype(np.float32)
    n = v.shape[0]
    idx = np.concatenate([f, np.array([[n, n + 1], [n + 2, n + 3], [n + 4, n + 5]], np.int32)]).astype(np.int32)
    w = Workload("odd2", 2, verts, idx, root=7, n_levels=4, bins=5, lattice=9)
    on = U.run_gpu(w, face_pass=ON)
    off = U.run_gpu(w, face_pass=OFF)
    _same(on, off)


def test_face_pass_graph_replay():
    import torch

    from paper_2502_16310_gb300 import AmrGeom

    w = small_workload("sphere3")
    g = AmrGeom(3, (w.root,) * 3)
    g.load(torch.from_numpy(w.verts).cuda(), torch.from_numpy(w.idx).cuda())
    g.bin(w.bins)
    outs = []
    for use_graph in (False, True, True):
        res = g.refine(w.n_levels, w.d_abs, w.d_rel, w.lattice, True, True, use_graph=use_graph, face_pass=ON)
        torch.cuda.synchronize()
        outs.append([U.to_np(lv["mask"]).copy() for lv in res["levels"]] +
                    [U.to_np(res[k]).view(np.uint8).copy() for k in ("adj_ids", "link_q", "link_face")])
    assert res["graph_replay"]
    for o in outs[1:]:
        for x, y in zip(outs[0], o):
            assert np.array_equal(x, y)
    g.close()


def test_face_pass_status():
    import torch

    from paper_2502_16310_gb300 import AmrError, AmrGeom
    from paper_2502_16310_gb300 import binding as Bd

    w = small_workload("sphere3")
    g = AmrGeom(3, (w.root,) * 3)
    g.load(torch.from_numpy(w.verts).cuda(), torch.from_numpy(w.idx).cuda())
    g.bin(w.bins)
    with pytest.raises(AmrError) as e:
        g.refine(w.n_levels, w.d_abs, w.d_rel, w.lattice, True, True, face_pass=3)
    assert e.value.status == Bd.AMR_EINVAL
    g.close()
