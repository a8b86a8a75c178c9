"""The algorithmic cell-face test count (amr_candidate_count) equals the oracle's per level, exactly
(integer work): per cell of every level's blocks, the distinct faces in the bins its inflated box
overlaps."""
import numpy as np
import pytest

from synth import small_workload
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", ["circle", "sphere3", "bumpy3"])
def test_candidate_count_matches_oracle(kind):
    import torch

    from oracle.oracle import Domain, OracleGeometry
    from paper_2502_16310_gb300 import AmrGeom

    w = small_workload(kind)
    g = AmrGeom(w.dim, (w.root,) * w.dim)
    g.load(torch.from_numpy(w.verts).cuda(), torch.from_numpy(w.idx).cuda())
    g.bin(w.bins)
    res = g.refine(w.n_levels, w.d_abs, w.d_rel, w.lattice, True, True)
    per, tot = g.candidate_count()
    geo = OracleGeometry(w.dim, w.verts, w.idx)
    geo.bin(Domain.unit(w.dim, w.root), w.bins)
    want = []
    for L, lv in enumerate(res["levels"]):
        blocks = U.to_np(lv["blocks"]).copy()
        _, _, _, nc = geo.refine_blocks(L, blocks, w.d_abs, w.d_rel, count_candidates=True)
        want.append(nc)
    assert per == want
    assert tot == sum(want) > 0
    g.close()


def test_candidate_count_state_error():
    import torch

    from paper_2502_16310_gb300 import AmrError, AmrGeom
    from paper_2502_16310_gb300 import binding as Bd

    w = small_workload("sphere3")
    g = AmrGeom(3, (w.root,) * 3)
    g.load(torch.from_numpy(w.verts).cuda(), torch.from_numpy(w.idx).cuda())
    g.bin(w.bins)
    with pytest.raises(AmrError) as e:
        g.candidate_count()
    assert e.value.status == Bd.AMR_ESTATE
    g.close()
