"""Graph mode, batched mode and the autotuner against the eager single-geometry path.

Graph replays and batched runs execute the same per-block arithmetic as the
eager single-geometry path, so every output must be bitwise identical (after
subtracting the batch bases from batch-global indices).
"""
import numpy as np
import pytest

from synth import Workload, small_workload
from synth import geometry as G
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


def _single(w, use_graph=False, repeats=1, B=None, warps=0, face_pass=0):
    import torch

    from paper_2502_16310_gb300 import AmrGeom

    g = AmrGeom(w.dim, (w.root,) * w.dim)
    v = torch.from_numpy(w.verts).cuda()
    ix = torch.from_numpy(w.idx).cuda()
    outs = []
    for _ in range(repeats):
        g.load(v, ix)
        g.bin(w.bins if B is None else B)
        res = g.refine(w.n_levels, w.d_abs, w.d_rel, w.lattice, True, True, use_graph=use_graph,
                       warps_per_cta=warps, face_pass=face_pass)
        outs.append(_host(res))
    launches = g.launch_count()
    g.close()
    return outs, launches


def _host(res):
    import torch

    torch.cuda.synchronize()
    out = {"levels": [{k: (None if lv[k] is None else lv[k].cpu().numpy().copy()) for k in ("blocks", "mask", "flag",
                                                                                             "parent")}
                      for lv in res["levels"]]}
    for k in ("adj_cell", "adj_off", "adj_ids", "link_cell", "link_dir", "link_q", "link_face"):
        if k in res:
            a = res[k].cpu().numpy().copy()
            out[k] = a.astype(np.int64) if a.dtype == np.int32 else a
    return out


def _same(a, b, what=""):
    assert len(a["levels"]) == len(b["levels"]), what
    for L, (x, y) in enumerate(zip(a["levels"], b["levels"])):
        for k in ("blocks", "mask", "flag", "parent"):
            if x[k] is None:
                assert y[k] is None or y[k].size == 0
                continue
            assert np.array_equal(x[k].astype(np.int64), y[k].astype(np.int64)), f"{what} level {L} {k}"
    for k in ("adj_cell", "adj_off", "adj_ids", "link_cell", "link_dir", "link_face"):
        assert np.array_equal(np.asarray(a[k]).astype(np.int64), np.asarray(b[k]).astype(np.int64)), f"{what} {k}"
    assert np.array_equal(a["link_q"].view(np.uint32), b["link_q"].view(np.uint32)), f"{what} link_q"


@pytest.mark.parametrize("kind", ["circle", "sphere3", "bumpy3"])
def test_graph_equals_eager(kind):
    w = small_workload(kind)
    (eager,), _ = _single(w)
    outs, _ = _single(w, use_graph=True, repeats=4)
    for i, o in enumerate(outs):
        _same(eager, o, f"graph call {i}")


def test_graph_overflow_falls_back():
    """A geometry that needs more blocks than the captured graph's capacities re-runs eagerly, correctly."""
    import torch

    from paper_2502_16310_gb300 import AmrGeom

    small = small_workload("sphere3")
    v2, f2 = G.jittered_sphere(3, radius=0.33, centre=(0.5, 0.5, 0.5), sigma=1e-4, seed=12)
    big = Workload("big", 3, v2, f2, root=small.root, n_levels=small.n_levels, bins=small.bins, lattice=19)
    (want,), _ = _single(big)
    g = AmrGeom(3, (small.root,) * 3)
    for w in (small, small, big, big):
        g.load(torch.from_numpy(w.verts).cuda(), torch.from_numpy(w.idx).cuda())
        g.bin(w.bins)
        res = g.refine(w.n_levels, w.d_abs, w.d_rel, 19, True, True, use_graph=True)
        got = _host(res)
    _same(want, got, "after fallback")
    g.close()


def _batch_set():
    ws = [small_workload("sphere3"), small_workload("bumpy3")]
    v, f = G.jittered_sphere(2, radius=0.3, centre=(0.48, 0.52, 0.5), sigma=1e-3, seed=21)
    ws.append(Workload("s2", 3, v, f, root=5, n_levels=2, bins=10, lattice=19))
    u, f = G.geodesic_sphere_unit(5)
    v, f = G.perturbed_surface(u, f, seed=22, lmax=4)
    ws.append(Workload("geo5", 3, v, f, root=7, n_levels=4, bins=20, lattice=19))
    ws.append(Workload("empty", 3, np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32), root=3, n_levels=2,
                       bins=4, lattice=19))
    return ws


@pytest.mark.parametrize("use_graph,face_pass", [(False, 1), (False, 2), (True, 0)])
def test_batch_matches_single(use_graph, face_pass):
    """Batched runs (block walk only, face by face wherever it applies, automatic) equal single-geometry
    runs by the block walk alone, bit for bit."""
    import torch

    from paper_2502_16310_gb300 import AmrBatch

    ws = _batch_set()
    singles = [_single(w, face_pass=1)[0][0] for w in ws]
    b = AmrBatch(3)
    for w in ws:
        b.add(torch.from_numpy(w.verts).cuda(), torch.from_numpy(w.idx).cuda(), w.root, w.n_levels, w.d_abs, w.d_rel,
              w.bins)
    for rep in range(3 if use_graph else 1):
        r = b.run(19, True, True, use_graph=use_graph, face_pass=face_pass)
        assert (r.n_face_setups > 0) == (face_pass != 1)
        for i, w in enumerate(ws):
            got = _host(b.view(i))
            _same(singles[i], got, f"geometry {i} rep {rep}")
    b.close()


def test_batch_adjoint_matches_single():
    import torch

    from paper_2502_16310_gb300 import AmrBatch, AmrGeom

    ws = _batch_set()[:4]
    b = AmrBatch(3)
    for w in ws:
        b.add(torch.from_numpy(w.verts).cuda(), torch.from_numpy(w.idx).cuda(), w.root, w.n_levels, w.d_abs, w.d_rel,
              w.bins)
    r = b.run(19, True, True)
    nl = int(r.n_links)
    wts = torch.randn(nl, device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    gb = b.q_backward(wts).cpu().numpy()
    vbase = 0
    for i, w in enumerate(ws):
        vw = b.view(i)
        lb = vw["bases"]["link"]
        n_i = vw["link_q"].shape[0]
        g = AmrGeom(3, (w.root,) * 3)
        g.load(torch.from_numpy(w.verts).cuda(), torch.from_numpy(w.idx).cuda())
        g.bin(w.bins)
        g.refine(w.n_levels, w.d_abs, w.d_rel, 19, True, True)
        gs = g.q_backward(wts[lb:lb + n_i]).cpu().numpy()
        g.close()
        assert np.array_equal(gs.view(np.uint32), gb[vbase:vbase + w.verts.shape[0]].view(np.uint32)), i
        vbase += w.verts.shape[0]
    b.close()


def test_autotune_picks_a_candidate():
    import torch

    from paper_2502_16310_gb300 import AmrGeom

    w = small_workload("sphere3")
    g = AmrGeom(3, (w.root,) * 3)
    g.load(torch.from_numpy(w.verts).cuda(), torch.from_numpy(w.idx).cuda())
    B, warps, ms = g.autotune(w.n_levels, w.d_abs, w.d_rel, 19, True, True, b_candidates=[8, 16, 32],
                              w_candidates=[2, 4, 8])
    assert B in (8, 16, 32) and warps in (2, 4, 8) and ms > 0
    g.bin(B)
    res = _host(g.refine(w.n_levels, w.d_abs, w.d_rel, 19, True, True, warps_per_cta=warps))
    g.close()
    (ref,), _ = _single(w)
    _same(ref, res, "tuned")


@pytest.mark.slow
def test_c5_batched_sampled():
    """The 48-geometry workload in one batch (bin densities from the autotuner, graph replay), checked
    against the oracle on seeded samples of six geometries: bins in full, blocks, adjacency and links
    sampled."""
    import torch

    from oracle.oracle import Domain, OracleGeometry
    from paper_2502_16310_gb300 import AmrBatch, AmrGeom
    from synth import batched_workloads

    ws = batched_workloads(48)
    data = [(torch.from_numpy(w.verts).cuda(), torch.from_numpy(w.idx).cuda()) for w in ws]
    for w, (v, ix) in zip(ws, data):
        g = AmrGeom(3, (w.root,) * 3)
        g.load(v, ix)
        w.bins, _, _ = g.autotune(w.n_levels, w.d_abs, w.d_rel, 19, True, True, b_candidates=[16, 32, 64, 128],
                                  w_candidates=[4])
        g.close()
    b = AmrBatch(3)
    for w, (v, ix) in zip(ws, data):
        b.add(v, ix, w.root, w.n_levels, w.d_abs, w.d_rel, w.bins)
    for _ in range(2):
        b.run(19, True, True, use_graph=True)
    rng = np.random.default_rng(55)
    big = int(np.argmax([w.n_faces for w in ws]))
    deep = int(np.argmax([w.n_levels * 1000 + w.root for w in ws]))
    pick = sorted({big, deep, *rng.choice(len(ws), size=4, replace=False).tolist()})
    for i in pick:
        w = ws[i]
        out = _host(b.view(i))
        geo = OracleGeometry(3, w.verts, w.idx)
        # bins of this geometry, in full, from the single-geometry path at the tuned density
        g = AmrGeom(3, (w.root,) * 3)
        g.load(*data[i])
        bins = g.bin(w.bins)
        off_g = bins["offsets"].cpu().numpy().view(np.uint32)
        ids_g = bins["ids"].cpu().numpy().view(np.uint32)
        g.close()
        off_o, ids_o = geo.bin(Domain.unit(3, w.root), w.bins)
        U.compare_bins(off_g, ids_g, off_o, ids_o)
        lv = out["levels"]
        for L in range(len(lv)):
            U.compare_level(geo, 3, L, lv[L]["blocks"], lv[L]["mask"].view(np.uint64), sample=40, rng=rng)
            if L + 1 < len(lv):
                U.check_children(3, lv[L]["blocks"], lv[L]["mask"].view(np.uint64), lv[L + 1]["blocks"],
                                 lv[L + 1]["parent"])
        fin = lv[-1]
        U.compare_adjacency(geo, 3, len(lv) - 1, fin["blocks"], fin["mask"].view(np.uint64),
                            out["adj_cell"].astype(np.uint32), out["adj_off"].astype(np.uint32),
                            out["adj_ids"].astype(np.uint32), sample=60, rng=rng)
        U.compare_links(geo, 3, len(lv) - 1, 19, fin["blocks"], out["adj_cell"].astype(np.uint32),
                        out["link_cell"].astype(np.uint32), out["link_dir"], out["link_q"],
                        out["link_face"].astype(np.uint32), sample=60, rng=rng)
    b.close()
