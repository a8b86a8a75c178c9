"""Re-adaptation maps between two successive hierarchies (moving geometry): per level, every new
block's index in the previous list (-1 = created by refinement) and every previous block's index
in the new list (-1 = removed by coarsening).  Integer work: compared exactly with maps built on
the host from the two block lists."""
import numpy as np
import pytest

from synth import small_workload
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


def _maps(a, b):
    """index of each row of b in a (-1 when absent)"""
    where = {tuple(r): i for i, r in enumerate(a.tolist())}
    return np.array([where.get(tuple(r), -1) for r in b.tolist()], np.int64)


def _refine(g, w, v, levels=None, keep=False, use_graph=False):
    import torch

    g.load(torch.from_numpy(v).cuda(), torch.from_numpy(w.idx).cuda())
    g.bin(w.bins)
    res = g.refine(levels or w.n_levels, w.d_abs, w.d_rel, w.lattice, True, True, use_graph=use_graph,
                   keep_previous=keep)
    torch.cuda.synchronize()
    return [U.to_np(lv["blocks"]).copy() for lv in res["levels"]]


@pytest.mark.parametrize("use_graph", [False, True])
def test_moving_sphere_maps(use_graph):
    from paper_2502_16310_gb300 import AmrGeom

    w = small_workload("sphere3")
    g = AmrGeom(3, (w.root,) * 3)
    shift = np.array([0.011, -0.004, 0.007], np.float32)
    old = _refine(g, w, w.verts, use_graph=use_graph)
    for step in range(3):  # several moves: graph replays keep the previous lists too
        new = _refine(g, w, w.verts + (step + 1) * shift, keep=True, use_graph=use_graph)
        d = g.adapt_diff()
        assert len(d) == len(new)
        for L in range(len(new)):
            n2o, o2n = _maps(old[L], new[L]), _maps(new[L], old[L])
            assert np.array_equal(U.to_np(d[L]["new_to_old"]).astype(np.int64), n2o), (step, L)
            assert np.array_equal(U.to_np(d[L]["old_to_new"]).astype(np.int64), o2n), (step, L)
            assert d[L]["created"] == int((n2o < 0).sum()) and d[L]["removed"] == int((o2n < 0).sum())
        assert d[-1]["created"] > 0 and d[-1]["removed"] > 0  # the finest level moved with the wall
        old = new
    g.close()


def test_identity_and_depth_change():
    from paper_2502_16310_gb300 import AmrGeom

    w = small_workload("bumpy3")
    g = AmrGeom(3, (w.root,) * 3)
    a = _refine(g, w, w.verts)
    b = _refine(g, w, w.verts, keep=True)
    d = g.adapt_diff()
    for L in range(len(b)):
        assert np.array_equal(U.to_np(d[L]["new_to_old"]), np.arange(b[L].shape[0]))
        assert d[L]["created"] == 0 and d[L]["removed"] == 0
    # one level shallower: the dropped level's previous blocks are all removed
    c = _refine(g, w, w.verts, levels=w.n_levels - 1, keep=True)
    d = g.adapt_diff()
    assert len(d) == len(c) == len(b) - 1
    for L in range(len(c)):
        assert d[L]["created"] == 0 and d[L]["removed"] == 0
    g.close()
    del a


def test_adapt_diff_state_error():
    from paper_2502_16310_gb300 import AmrError, AmrGeom
    from paper_2502_16310_gb300 import binding as Bd

    w = small_workload("sphere3")
    g = AmrGeom(3, (w.root,) * 3)
    _refine(g, w, w.verts)
    with pytest.raises(AmrError) as e:
        g.adapt_diff()  # no previous hierarchy was kept
    assert e.value.status == Bd.AMR_ESTATE
    g.close()


def _arrays(res):
    out = [U.to_np(lv["blocks"]).copy() for lv in res["levels"]]
    for k in ("adj_cell", "adj_off", "adj_ids", "link_cell", "link_dir", "link_q", "link_face"):
        out.append(U.to_np(res[k]).view(np.uint8).copy())
    return out


def test_graph_replays_follow_a_moving_wall():
    """A wall moving by a fraction of the finest cell per step keeps replaying the captured level loop
    (the capacities leave room for the sizes to drift), with results identical to eager calls."""
    import torch

    from paper_2502_16310_gb300 import AmrGeom

    w = small_workload("sphere3")
    g, e = AmrGeom(3, (w.root,) * 3), AmrGeom(3, (w.root,) * 3)
    h_fin = 1.0 / (4 * w.root * 2 ** (w.n_levels - 1))
    delta = np.array([0.25, 0.1, 0.05], np.float32) * np.float32(h_fin)
    idx = torch.from_numpy(w.idx).cuda()
    replays = []
    for k in range(6):
        v = torch.from_numpy(w.verts + np.float32(k) * delta).cuda()
        got = []
        for ctx, graph in ((g, True), (e, False)):
            ctx.load(v, idx)
            ctx.bin(w.bins)
            res = ctx.refine(w.n_levels, w.d_abs, w.d_rel, w.lattice, True, True, use_graph=graph,
                             keep_previous=graph and k > 0)
            torch.cuda.synchronize()
            got.append(_arrays(res))
            if graph:
                replays.append(res["graph_replay"])
        assert len(got[0]) == len(got[1])
        for a, b in zip(*got):
            assert np.array_equal(a, b), k
        if k > 0:
            g.adapt_diff()  # its buffers are outside the graph: the next step still replays
    assert replays[0] is False and all(replays[1:]), replays
    g.close()
    e.close()


def test_moved_steps_against_oracle():
    """Each moved step's hierarchy is the oracle's hierarchy of the moved vertices (re-adaptation rebuilds
    from the roots, so the marks depend only on the geometry), and the new <-> old maps equal the maps
    between the oracle's own block lists of the two steps.  The shifts put no decision in the margin band
    (checked), so the block lists must agree exactly."""
    import torch

    from oracle.oracle import run_pipeline
    from paper_2502_16310_gb300 import AmrGeom

    w = small_workload("sphere3")
    g = AmrGeom(3, (w.root,) * 3)
    shift = np.array([0.011, -0.004, 0.007], np.float32)
    prev = None
    for step in range(3):
        v = w.verts + step * shift
        g.load(torch.from_numpy(v).cuda(), torch.from_numpy(w.idx).cuda())
        g.bin(w.bins)
        res = g.refine(w.n_levels, w.d_abs, w.d_rel, w.lattice, True, True, keep_previous=step > 0,
                       use_graph=step > 1)
        torch.cuda.synchronize()
        blocks = [U.to_np(lv["blocks"]).copy() for lv in res["levels"]]
        masks = [U.to_np(lv["mask"], np.uint64).copy() for lv in res["levels"]]
        orc = run_pipeline(3, v, w.idx, root=w.root, n_levels=w.n_levels, B=w.bins, lattice=w.lattice, links=False)
        assert all(int(np.count_nonzero(lv["band"])) == 0 for lv in orc["levels"]), "shift puts cells in the band"
        for L, lv in enumerate(orc["levels"]):
            assert np.array_equal(blocks[L], lv["blocks"]), (step, L)
            assert np.array_equal(masks[L], lv["mask"]), (step, L)
        if prev is not None:
            d = g.adapt_diff()
            for L, lv in enumerate(orc["levels"]):
                n2o, o2n = _maps(prev[L], lv["blocks"]), _maps(lv["blocks"], prev[L])
                assert np.array_equal(U.to_np(d[L]["new_to_old"]).astype(np.int64), n2o), (step, L)
                assert np.array_equal(U.to_np(d[L]["old_to_new"]).astype(np.int64), o2n), (step, L)
            assert d[-1]["created"] > 0 and d[-1]["removed"] > 0
        prev = [lv["blocks"] for lv in orc["levels"]]
    g.close()


def test_moving_c2_step_sampled():
    """The bench's moving wall (the c2 sphere, a quarter of a finest cell per step, graph replays): after
    several moves, every level of the current hierarchy is checked against the oracle on sampled blocks
    (lockstep: the oracle takes the GPU's blocks of each level), children exactly."""
    import torch

    from oracle.oracle import Domain, OracleGeometry
    from paper_2502_16310_gb300 import AmrGeom
    from synth import workload

    w = workload("c2")
    g = AmrGeom(3, (w.root,) * 3)
    h_fin = 1.0 / (4 * w.root * 2 ** (w.n_levels - 1))
    delta = np.array([0.25 * h_fin, 0.1 * h_fin, 0.05 * h_fin], np.float32)
    idx = torch.from_numpy(w.idx).cuda()
    for k in range(4):
        v = (w.verts + np.float32(k) * delta).astype(np.float32)
        g.load(torch.from_numpy(v).cuda(), idx)
        g.bin(w.bins)
        res = g.refine(w.n_levels, w.d_abs, w.d_rel, w.lattice, True, True, use_graph=True, keep_previous=k > 0)
    torch.cuda.synchronize()
    geo = OracleGeometry(3, v, w.idx)
    geo.bin(Domain.unit(3, w.root), w.bins)
    rng = np.random.default_rng(12)
    lv = res["levels"]
    for L in range(len(lv)):
        b = U.to_np(lv[L]["blocks"]).copy()
        m = U.to_np(lv[L]["mask"], np.uint64).copy()
        U.compare_level(geo, 3, L, b, m, sample=200, rng=rng)
        if L + 1 < len(lv):
            U.check_children(3, b, m, U.to_np(lv[L + 1]["blocks"]).copy(), U.to_np(lv[L + 1]["parent"]).copy())
    g.close()
