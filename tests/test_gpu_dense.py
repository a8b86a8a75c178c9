"""Finest blocks that meet many faces (a fine mesh on a coarse grid): more survivor records than a
warp stages in shared memory.  The first call re-walks those blocks for their lists and sorts each
cell's list with the warp; later calls keep the records in a spill area (up to 1,024 per block) and
sort them by face id.  Every output of the two calls is identical, and equal to the oracle's."""
import numpy as np
import pytest

from synth import Workload
from synth import geometry as G
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


def _host(res):
    import torch

    torch.cuda.synchronize()
    out = [U.to_np(lv[k]).copy() for lv in res["levels"] for k in ("blocks", "mask")]
    out += [U.to_np(res[k]).view(np.uint8).copy() for k in ("adj_cell", "adj_off", "adj_ids", "link_cell",
                                                                 "link_dir", "link_q", "link_face")]
    return out


@pytest.mark.parametrize("subdiv,rows", [(5, 400), (6, 150)])
def test_dense_finest_blocks(subdiv, rows):
    import torch

    from oracle.oracle import Domain, OracleGeometry
    from paper_2502_16310_gb300 import AmrGeom

    v, f = G.jittered_sphere(subdiv, radius=0.3, centre=(0.5, 0.49, 0.51), sigma=1e-4, seed=40 + subdiv)
    w = Workload("dense", 3, v, f, root=4, n_levels=2, bins=16, lattice=19)
    g = AmrGeom(3, (w.root,) * 3)
    g.load(torch.from_numpy(w.verts).cuda(), torch.from_numpy(w.idx).cuda())
    g.bin(w.bins)
    outs = []
    for _ in range(3):  # re-walk, then the spill area (eager), then a graph capture and replay
        res = g.refine(w.n_levels, w.d_abs, w.d_rel, w.lattice, True, True, use_graph=len(outs) == 2)
        outs.append(_host(res))
    for o in outs[1:]:
        for x, y in zip(outs[0], o):
            assert np.array_equal(x, y)
    fin = res["levels"][-1]
    blocks, mask = U.to_np(fin["blocks"]).copy(), U.to_np(fin["mask"], np.uint64).copy()
    K = np.array([bin(int(m)).count("1") for m in mask])
    assert K.max() > 0
    geo = OracleGeometry(3, w.verts, w.idx)
    geo.bin(Domain.unit(3, w.root), w.bins)
    adj_cell = U.to_np(res["adj_cell"], np.uint32)
    adj_off = U.to_np(res["adj_off"], np.uint32)
    adj_ids = U.to_np(res["adj_ids"], np.uint32)
    # cells with long lists: the blocks hold far more faces than the 64 records staged per warp
    lens = np.diff(adj_off.astype(np.int64))
    assert lens.max() > 64
    U.compare_adjacency(geo, 3, w.n_levels - 1, blocks, mask, adj_cell, adj_off, adj_ids, sample=rows,
                        d_abs=w.d_abs, d_rel=w.d_rel)
    U.compare_links(geo, 3, w.n_levels - 1, w.lattice, blocks, adj_cell, U.to_np(res["link_cell"], np.uint32),
                    U.to_np(res["link_dir"]), U.to_np(res["link_q"]), U.to_np(res["link_face"], np.uint32),
                    sample=rows // 2, d_abs=w.d_abs, d_rel=w.d_rel)
    g.close()
