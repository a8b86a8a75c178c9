"""GPU parity of the paper's own binned search (Sec. "Spatial Binning Algorithm"): sampled-point
bin membership, face detection in the cell's own bin with the point predicate, and the
refinement-mark propagation.

Criteria: sampled bins bit-exact as sorted sets (the sample points are FP64 with a fixed order
of operations on both sides); every level's masks identical to the oracle outside the band (the
oracle evaluated on the GPU's block list); the propagated flags identical to the oracle's
propagation of the GPU's own masks (integer work); children exact from the flags.
"""
import numpy as np
import pytest

from synth import small_workload, workload
from tests import gpu_util as U

pytestmark = pytest.mark.gpu

PRED_POINT, OWN_BIN = 1, 1


def _gpu(w, B, d_abs, propagate, sampled=True, n_levels=None):
    import torch

    from paper_2502_16310_gb300 import AmrGeom

    g = AmrGeom(w.dim, (w.root,) * w.dim)
    g.load(torch.from_numpy(w.verts).cuda(), torch.from_numpy(w.idx).cuda())
    bins = g.bin(B, sampled=sampled)
    res = g.refine(n_levels or w.n_levels, d_abs, 0.0, 0, False, False, predicate=PRED_POINT, search=OWN_BIN,
                   propagate=propagate)
    torch.cuda.synchronize()
    out = {"offsets": U.to_np(bins["offsets"], np.uint32), "ids": U.to_np(bins["ids"], np.uint32),
           "levels": [{"blocks": U.to_np(lv["blocks"]), "mask": U.to_np(lv["mask"], np.uint64),
                       "flag": U.to_np(lv["flag"]),
                       "parent": None if lv["parent"] is None else U.to_np(lv["parent"])} for lv in res["levels"]]}
    g.close()
    return out


def _check(w, B, d_abs, propagate=-1, sample=None, sampled=True):
    from oracle.oracle import Domain, OracleGeometry, propagate as o_propagate, propagation_rounds, root_blocks

    out = _gpu(w, B, d_abs, propagate, sampled)
    dom = Domain.unit(w.dim, w.root)
    geo = OracleGeometry(w.dim, w.verts, w.idx)
    off, ids = geo.bin(dom, B, sampled=sampled)
    U.compare_bins(out["offsets"], out["ids"], off, ids)
    lv = out["levels"]
    assert np.array_equal(lv[0]["blocks"], root_blocks(w.dim, (w.root,) * w.dim))
    rng = np.random.default_rng(3)
    for L in range(len(lv)):
        blocks = lv[L]["blocks"]
        idx = np.arange(blocks.shape[0])
        if sample is not None and idx.size > sample:
            idx = np.sort(rng.choice(idx.size, size=sample, replace=False))
        if idx.size:
            m_o, band, _, _ = geo.refine_blocks(L, blocks[idx], d_abs, 0.0, pred=PRED_POINT, search=OWN_BIN)
            bad = (m_o ^ lv[L]["mask"][idx]) & ~band
            assert not np.any(bad), f"level {L}: {int(np.count_nonzero(bad))} blocks differ outside the band"
        if L + 1 < len(lv):
            rounds = 0
            if propagate:
                h = dom.h(L)
                rounds = propagate if propagate > 0 else propagation_rounds(d_abs, 4 * h)
            want = o_propagate(w.dim, blocks, (lv[L]["mask"] != 0).astype(np.uint8), rounds)
            assert np.array_equal(lv[L]["flag"].astype(np.uint8), want), f"level {L} propagation"
            U.check_children(w.dim, blocks, lv[L]["flag"].astype(np.uint64), lv[L + 1]["blocks"],
                             lv[L + 1]["parent"])
    return out


@pytest.mark.parametrize("kind,B,d", [("circle", 7, 0.03), ("sphere3", 6, 0.035), ("bumpy3", 9, 0.03)])
def test_paper_mode_small(kind, B, d):
    out = _check(small_workload(kind), B, d)
    assert sum(int(np.count_nonzero(x["mask"])) for x in out["levels"]) > 0


@pytest.mark.parametrize("B", [4, 16, 40])
def test_sampled_bins_match(B):
    """Sampled membership, bit-exact (as sorted sets), on a surface with faces of all sizes."""
    import torch

    from oracle.oracle import Domain, OracleGeometry
    from paper_2502_16310_gb300 import AmrGeom

    w = small_workload("bumpy3")
    g = AmrGeom(3, (w.root,) * 3)
    g.load(torch.from_numpy(w.verts).cuda(), torch.from_numpy(w.idx).cuda())
    bins = g.bin(B, sampled=True)
    off_g, ids_g = U.to_np(bins["offsets"], np.uint32), U.to_np(bins["ids"], np.uint32)
    g.close()
    off_o, ids_o = OracleGeometry(3, w.verts, w.idx).bin(Domain.unit(3, w.root), B, sampled=True)
    U.compare_bins(off_g, ids_g, off_o, ids_o)


def test_own_bin_single_bin_is_full_search():
    """With one bin every cell sees every face: the own-bin search equals the query-box search."""
    import torch

    from paper_2502_16310_gb300 import AmrGeom

    w = small_workload("sphere3")
    a = _gpu(w, 1, 0.035, 0, sampled=False)
    g = AmrGeom(3, (w.root,) * 3)
    g.load(torch.from_numpy(w.verts).cuda(), torch.from_numpy(w.idx).cuda())
    g.bin(8)
    res = g.refine(w.n_levels, 0.035, 0.0, 0, False, False, predicate=PRED_POINT)
    torch.cuda.synchronize()
    for L, lv in enumerate(res["levels"]):
        assert np.array_equal(U.to_np(lv["mask"], np.uint64), a["levels"][L]["mask"]), L
    g.close()


@pytest.mark.parametrize("name", ["p2", "p3"])
def test_paper_setups_paper_mode(name):
    w = workload(name)
    _check(w, 8, w.d_abs, sample=150)


def test_paper_mode_validation():
    import torch

    from paper_2502_16310_gb300 import AmrError, AmrGeom
    from paper_2502_16310_gb300 import binding as Bd

    w = small_workload("sphere3")
    g = AmrGeom(3, (w.root,) * 3)
    g.load(torch.from_numpy(w.verts).cuda(), torch.from_numpy(w.idx).cuda())
    g.bin(8, sampled=True)
    for kw in ({"predicate": PRED_POINT},                        # sampled bins need the own-bin search
               {"predicate": 0, "search": OWN_BIN},              # the own-bin search needs the point predicate
               {"predicate": PRED_POINT, "search": OWN_BIN, "propagate": -2}):
        with pytest.raises(AmrError) as e:
            g.refine(w.n_levels, 0.03, 0.0, 0, False, False, **kw)
        assert e.value.status == Bd.AMR_EINVAL, kw
    with pytest.raises(AmrError) as e:  # no links with the own-bin search
        g.refine(w.n_levels, 0.03, 0.0, 19, True, True, predicate=PRED_POINT, search=OWN_BIN)
    assert e.value.status == Bd.AMR_EINVAL
    g.close()
