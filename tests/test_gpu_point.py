"""GPU parity of the point predicate (Alg. 1: a cell centre within the near-wall distance d
of the closed face), with the paper's absolute distance (d_abs = d_spec, d_rel = 0).

Same criteria as the box predicate: bins as sorted sets, masks identical outside the
oracle's 1e-6*h band (here |distance - d| <= 1e-6 h), adjacency lists identical up to
band pairs, links within 1e-5 (the point predicate needs d >= sqrt(2) h for links).
"""
import numpy as np
import pytest

from synth import small_workload, workload
from tests import gpu_util as U

pytestmark = pytest.mark.gpu

PRED_POINT = 1


def _check(w, d_abs, sample=None, B=None):
    from oracle.oracle import Domain, OracleGeometry, root_blocks

    B = w.bins if B is None else B
    out = U.run_gpu(w, B=B, d_abs=d_abs, d_rel=0.0, predicate=PRED_POINT)
    geo = OracleGeometry(w.dim, w.verts, w.idx)
    off, ids = geo.bin(Domain.unit(w.dim, w.root), B)
    U.compare_bins(out["offsets"], out["ids"], off, ids)
    lv = out["levels"]
    assert np.array_equal(lv[0]["blocks"], root_blocks(w.dim, (w.root,) * w.dim))
    rng = np.random.default_rng(7)
    for L in range(len(lv)):
        U.compare_level(geo, w.dim, L, lv[L]["blocks"], lv[L]["mask"], sample=sample, d_abs=d_abs, d_rel=0.0,
                        rng=rng, pred=PRED_POINT)
        if L + 1 < len(lv):
            U.check_children(w.dim, lv[L]["blocks"], lv[L]["mask"], lv[L + 1]["blocks"], lv[L + 1]["parent"])
    fin = lv[-1]
    Lf = len(lv) - 1
    U.compare_adjacency(geo, w.dim, Lf, fin["blocks"], fin["mask"], out["adj_cell"], out["adj_off"], out["adj_ids"],
                        sample=sample, d_abs=d_abs, d_rel=0.0, rng=rng, pred=PRED_POINT)
    U.compare_links(geo, w.dim, Lf, w.lattice, fin["blocks"], out["adj_cell"], out["link_cell"], out["link_dir"],
                    out["link_q"], out["link_face"], sample=sample, rng=rng, d_abs=d_abs, d_rel=0.0, pred=PRED_POINT)
    return out


@pytest.mark.parametrize("kind,d", [("circle", 0.03), ("sphere3", 0.035), ("bumpy3", 0.03)])
def test_point_small_full_parity(kind, d):
    out = _check(small_workload(kind), d)
    assert out["adj_cell"].shape[0] > 0 and out["link_q"].shape[0] > 0


@pytest.mark.parametrize("B", [1, 5])
def test_point_bin_density_independence(B):
    w = small_workload("sphere3")
    ref = U.run_gpu(w, d_abs=0.035, d_rel=0.0, predicate=PRED_POINT)
    out = U.run_gpu(w, B=B, d_abs=0.035, d_rel=0.0, predicate=PRED_POINT)
    for L in range(len(ref["levels"])):
        assert np.array_equal(ref["levels"][L]["mask"], out["levels"][L]["mask"])
    assert np.array_equal(ref["adj_ids"], out["adj_ids"])
    assert np.array_equal(ref["link_q"], out["link_q"])


def test_point_inside_box():
    """The ball of radius d lies in the cell box inflated by d - h/2 ... by d (half-width h/2 + d):
    on the root level, a point-adjacent cell is box-adjacent at the same d (outside both bands)."""
    from oracle.oracle import Domain, OracleGeometry

    w = small_workload("bumpy3")
    d = 0.03
    pt = U.run_gpu(w, n_levels=1, want_links=False, d_abs=d, d_rel=0.0, predicate=PRED_POINT)
    bx = U.run_gpu(w, n_levels=1, want_links=False, d_abs=d, d_rel=0.0, predicate=0)
    geo = OracleGeometry(w.dim, w.verts, w.idx)
    geo.bin(Domain.unit(w.dim, w.root), w.bins)
    blocks = pt["levels"][0]["blocks"]
    _, band_p, _, _ = geo.refine_blocks(0, blocks, d, 0.0, pred=PRED_POINT)
    _, band_b, _, _ = geo.refine_blocks(0, blocks, d, 0.0, pred=0)
    extra = pt["levels"][0]["mask"] & ~bx["levels"][0]["mask"] & ~(band_p | band_b)
    assert not np.any(extra)
    assert int(np.count_nonzero(pt["levels"][0]["mask"])) > 0


def test_point_links_need_reach():
    import torch

    from paper_2502_16310_gb300 import AmrError, AmrGeom
    from paper_2502_16310_gb300 import binding as Bd

    w = small_workload("sphere3")
    g = AmrGeom(3, (w.root,) * 3)
    g.load(torch.from_numpy(w.verts).cuda(), torch.from_numpy(w.idx).cuda())
    g.bin(w.bins)
    h_fin = 1.0 / (4 * w.root * 2 ** (w.n_levels - 1))
    with pytest.raises(AmrError) as e:
        g.refine(w.n_levels, 1.2 * h_fin, 0.0, 19, True, True, predicate=PRED_POINT)  # d < sqrt(2) h
    assert e.value.status == Bd.AMR_EINVAL
    with pytest.raises(AmrError) as e:
        g.refine(w.n_levels, 0.03, 0.0, 19, True, True, predicate=7)
    assert e.value.status == Bd.AMR_EINVAL
    g.close()


def test_point_graph_equals_eager():
    import torch

    from paper_2502_16310_gb300 import AmrGeom

    w = small_workload("bumpy3")
    outs = []
    for use_graph in (False, True, True):
        g = AmrGeom(3, (w.root,) * 3)
        g.load(torch.from_numpy(w.verts).cuda(), torch.from_numpy(w.idx).cuda())
        g.bin(w.bins)
        for _ in range(2 if use_graph else 1):
            res = g.refine(w.n_levels, 0.03, 0.0, 19, True, True, use_graph=use_graph, predicate=PRED_POINT)
        torch.cuda.synchronize()
        outs.append({k: res[k].cpu().numpy().copy() for k in ("adj_cell", "adj_off", "adj_ids", "link_q",
                                                              "link_face")})
        g.close()
    for o in outs[1:]:
        for k in o:
            assert np.array_equal(o[k].view(np.uint8), outs[0][k].view(np.uint8)), k


def test_point_c2_sampled():
    """c2 with the paper's absolute distance: d = 2 h of the finest level."""
    w = workload("c2")
    h_fin = 1.0 / (4 * w.root * 2 ** (w.n_levels - 1))
    _check(w, 2.0 * h_fin, sample=300)


@pytest.mark.parametrize("name", ["p2", "p3"])
def test_paper_setups_sampled(name):
    """The paper's speed-up setups (absolute d_spec = 0.1 / 0.05, refined twice), marking only as in
    the paper: every level's masks on seeded samples of blocks, children exact, at B = 1 and B = 16."""
    import torch

    from oracle.oracle import Domain, OracleGeometry, root_blocks
    from paper_2502_16310_gb300 import AmrGeom

    w = workload(name)
    geo = OracleGeometry(w.dim, w.verts, w.idx)
    geo.bin(Domain.unit(w.dim, w.root), 16)
    rng = np.random.default_rng(11)
    masks = []
    for B in (1, 16):
        g = AmrGeom(w.dim, (w.root,) * w.dim)
        g.load(torch.from_numpy(w.verts).cuda(), torch.from_numpy(w.idx).cuda())
        g.bin(B)
        res = g.refine(w.n_levels, w.d_abs, w.d_rel, 0, False, False, predicate=PRED_POINT)
        torch.cuda.synchronize()
        lv = [{"blocks": x["blocks"].cpu().numpy(), "mask": x["mask"].cpu().numpy().view(np.uint64),
               "parent": None if x["parent"] is None else x["parent"].cpu().numpy()} for x in res["levels"]]
        g.close()
        assert np.array_equal(lv[0]["blocks"], root_blocks(w.dim, (w.root,) * w.dim))
        for L in range(len(lv)):
            U.compare_level(geo, w.dim, L, lv[L]["blocks"], lv[L]["mask"], sample=100, d_abs=w.d_abs,
                            d_rel=w.d_rel, rng=rng, pred=PRED_POINT)
            if L + 1 < len(lv):
                U.check_children(w.dim, lv[L]["blocks"], lv[L]["mask"], lv[L + 1]["blocks"], lv[L + 1]["parent"])
        masks.append([x["mask"] for x in lv])
    # exact binning: the marks do not depend on B (the paper needs its propagation step for that)
    for a, b in zip(*masks):
        assert np.array_equal(a, b)
