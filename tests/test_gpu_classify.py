"""GPU node classification (solid = the adjacent cell's centre lies inside the closed mesh) against
the oracle's generalized winding number, and the restriction of the links to fluid cells.

Criteria: classes identical outside the oracle's band (centres within 1e-6 h of the mesh); the
fluid links are exactly the links of cells classified fluid, in the original order."""
import numpy as np
import pytest

from synth import small_workload, workload
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


def _run(w, B=None):
    import torch

    from paper_2502_16310_gb300 import AmrGeom

    g = AmrGeom(w.dim, (w.root,) * w.dim)
    g.load(torch.from_numpy(w.verts).cuda(), torch.from_numpy(w.idx).cuda())
    g.bin(w.bins if B is None else B)
    res = g.refine(w.n_levels, w.d_abs, w.d_rel, w.lattice, True, True)
    cls, nfb = g.classify()
    torch.cuda.synchronize()
    return g, res, cls.cpu().numpy().astype(bool), nfb


def _oracle_classes(w, res, rows):
    from oracle.oracle import Domain, OracleGeometry

    nc = 64 if w.dim == 3 else 16
    fin = res["levels"][-1]["blocks"].cpu().numpy()
    adj = U.to_np(res["adj_cell"], np.uint32)[rows]
    cells = U.cells_of(w.dim, fin, (adj // nc).astype(np.int64), (adj % nc).astype(np.int64))
    geo = OracleGeometry(w.dim, w.verts, w.idx)
    return geo.classify(len(res["levels"]) - 1, cells, Domain.unit(w.dim, w.root))


@pytest.mark.parametrize("kind", ["circle", "sphere3", "bumpy3"])
def test_classify_small_full(kind):
    w = small_workload(kind)
    g, res, solid, nfb = _run(w)
    rows = np.arange(solid.shape[0])
    want, band = _oracle_classes(w, res, rows)
    bad = (solid != want) & ~band
    assert not bad.any(), f"{int(bad.sum())} of {rows.size} cells differ"
    assert 0.2 < solid.mean() < 0.8  # the near-wall band straddles the surface
    g.close()


def test_classify_c2_sampled():
    w = workload("c2")
    g, res, solid, nfb = _run(w)
    rows = np.sort(np.random.default_rng(9).choice(solid.shape[0], size=300, replace=False))
    want, band = _oracle_classes(w, res, rows)
    assert not np.any((solid[rows] != want) & ~band)
    g.close()


def test_fluid_links_compaction_and_adjoint():
    import torch

    w = small_workload("bumpy3")
    g, res, solid, _ = _run(w)
    before = {k: U.to_np(res[k]).copy() for k in ("link_cell", "link_dir", "link_q", "link_face")}
    keep = ~solid[before["link_cell"].view(np.uint32).astype(np.int64)]
    out = g.fluid_links()
    torch.cuda.synchronize()
    for k in before:
        got = U.to_np(out[k])
        assert np.array_equal(got.view(np.uint8), before[k][keep].view(np.uint8)), k
    assert 0 < keep.sum() < keep.size
    # the q adjoint runs on the kept links
    nk = int(keep.sum())
    grad = g.q_backward(torch.ones(nk, device="cuda"))
    assert torch.isfinite(grad).all()
    g.close()


def test_classify_state_errors():
    import torch

    from paper_2502_16310_gb300 import AmrError, AmrGeom
    from paper_2502_16310_gb300 import binding as Bd

    w = small_workload("sphere3")
    g = AmrGeom(3, (w.root,) * 3)
    g.load(torch.from_numpy(w.verts).cuda(), torch.from_numpy(w.idx).cuda())
    g.bin(w.bins)
    with pytest.raises(AmrError) as e:
        g.classify()
    assert e.value.status == Bd.AMR_ESTATE
    with pytest.raises(AmrError) as e:
        g.fluid_links()
    assert e.value.status == Bd.AMR_ESTATE
    g.bin(w.bins, sampled=True)
    g.refine(w.n_levels, 0.03, 0.0, 0, True, False, predicate=1, search=1)
    with pytest.raises(AmrError) as e:
        g.classify()
    assert e.value.status == Bd.AMR_EINVAL
    g.close()
