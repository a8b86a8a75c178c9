"""The q adjoint at full size: c4 (1,310,720 triangles, 6 levels, 256^3 bins, level loop replayed as a CUDA
graph, as the bench runs it) and the 48-geometry batch c5 (one amr_batch_q_backward over all geometries).

The oracle cannot differentiate hundreds of millions of links, so the upstream weights are seeded normal
numbers on the links of a seeded sample of faces and zero on every other link.  The adjoint is linear in
the weights, so the library's full-size launch must then return exactly the gradient of
L = sum over the sampled faces' links of w q.  The sampled faces share no vertex, so the gradient at each
of their vertices is that face's own, and FP64 central differences of L can be taken one face at a time.

Checks, with the tolerance of the other adjoint tests (per entry 1e-4 |ref| + 1e-4 rms(ref)):
  * every vertex of a sampled face against the oracle's FP64 analytic gradient;
  * a sub-sample of those faces against FP64 central differences of L;
  * every other vertex exactly zero.
"""
import numpy as np
import pytest

from synth import workload
from tests import gpu_util as U

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
REL = 1e-4


def independent_faces(idx, n, rng, allowed=None):
    """Up to n faces (seeded order) of which no two share a vertex."""
    order = rng.permutation(idx.shape[0]) if allowed is None else rng.permutation(allowed)
    used, out = set(), []
    for f in order:
        vs = idx[f].tolist()
        if any(v in used for v in vs):
            continue
        used.update(vs)
        out.append(int(f))
        if len(out) == n:
            break
    return np.array(sorted(out), np.int64)


def assert_close(g, ref, what):
    scale = np.sqrt(np.mean(ref ** 2)) + 1e-300
    err = np.abs(g - ref)
    bad = err > REL * np.abs(ref) + REL * scale
    assert not np.any(bad), (f"{what}: {int(bad.sum())}/{bad.size} entries off; worst rel "
                             f"{float(np.max(err / (np.abs(ref) + scale))):.3e}")


def oracle_vertex_grad(geo, w, level, cells, dirs, faces, wts):
    gf = geo.q_grad(level, 19, cells, dirs.astype(np.int32), faces.astype(np.int64), wts.astype(np.float64))
    gv = np.zeros((w.verts.shape[0], 3))
    for k in range(3):
        np.add.at(gv, w.idx[:, k], gf[:, k, :])
    return gv


def central_differences(geo, w, level, cells, dirs, faces, wts, fd_faces):
    """FP64 central differences of L = sum w q with respect to the vertices of each face in fd_faces
    (one face at a time; links whose hit disappears under the perturbation are skipped whole)."""
    h = 1.0 / (4 * w.root) * 2.0 ** (-level)
    delta = 1e-6 * h
    fv = w.verts[w.idx].astype(np.float64)
    out = {}
    for f in fd_faces:
        sel = np.nonzero(faces == f)[0]
        for k in range(3):
            for c in range(3):
                num, stable = 0.0, True
                for j in sel:
                    vp, vm = fv[f].copy(), fv[f].copy()
                    vp[k, c] += delta
                    vm[k, c] -= delta
                    qp = geo.link_q(level, 19, cells[j], int(dirs[j]), int(f), vp)
                    qm = geo.link_q(level, 19, cells[j], int(dirs[j]), int(f), vm)
                    if not (np.isfinite(qp) and np.isfinite(qm)):
                        stable = False
                        break
                    num += float(wts[j]) * (qp - qm) / (2 * delta)
                if stable:
                    out[(int(w.idx[f, k]), c)] = num
    return out


def test_adjoint_c4_sampled_faces():
    import torch

    from oracle.oracle import Domain, OracleGeometry
    from paper_2502_16310_gb300 import AmrGeom

    w = workload("c4")
    L = w.n_levels - 1
    g = AmrGeom(3, (w.root,) * 3)
    g.load(torch.from_numpy(w.verts).cuda(), torch.from_numpy(w.idx).cuda())
    g.bin(w.bins)
    for _ in range(2):  # the second call replays the captured level loop
        res = g.refine(w.n_levels, w.d_abs, w.d_rel, 19, True, True, use_graph=True)
    rng = np.random.default_rng(404)
    fs = independent_faces(w.idx, 1500, rng)
    sel_f = torch.zeros(w.n_faces, dtype=torch.bool, device="cuda")
    sel_f[torch.from_numpy(fs).cuda()] = True
    lf = res["link_face"].long()
    rows = torch.nonzero(sel_f[lf]).flatten()
    nl = lf.numel()
    wts = torch.zeros(nl, dtype=torch.float32, device="cuda")
    wsel = torch.randn(rows.numel(), device="cuda", generator=torch.Generator("cuda").manual_seed(5))
    wts[rows] = wsel
    # the sampled links on the host: cell coordinates, direction, face, weight
    lc = res["link_cell"].long()[rows]
    ids = res["adj_cell"].long()[lc]
    blocks = res["levels"][-1]["blocks"].long()[ids // 64].cpu().numpy()
    bits = (ids % 64).cpu().numpy()
    loc = np.stack([bits & 3, (bits >> 2) & 3, (bits >> 4) & 3], axis=1)
    cells = (4 * blocks + loc).astype(np.int32)
    dirs = res["link_dir"][rows].cpu().numpy()
    faces = lf[rows].cpu().numpy()
    wh = wsel.cpu().numpy()
    grad = g.q_backward(wts).cpu().numpy().astype(np.float64)
    g.close()
    assert rows.numel() > 100_000 and set(np.unique(faces).tolist()) <= set(fs.tolist())

    geo = OracleGeometry(3, w.verts, w.idx)
    geo.bin(Domain.unit(3, w.root), w.bins)  # sets the oracle's domain
    ref = oracle_vertex_grad(geo, w, L, cells, dirs, faces, wh)
    touched = np.zeros(w.verts.shape[0], bool)
    touched[w.idx[fs].ravel()] = True
    assert np.all(grad[~touched] == 0.0), "a vertex of no sampled face has a non-zero gradient"
    assert_close(grad[touched], ref[touched], "c4 vs the oracle's analytic gradient")
    fd = central_differences(geo, w, L, cells, dirs, faces, wh, fs[rng.choice(fs.size, 20, replace=False)])
    assert len(fd) > 100
    keys = list(fd)
    assert_close(np.array([grad[v, c] for v, c in keys]), np.array([fd[k] for k in keys]),
                 "c4 vs FP64 central differences")


@pytest.fixture(scope="module")
def c5_batch():
    """The 48-geometry workload in one batch: bin densities from the autotuner, level loop replayed as a
    CUDA graph."""
    import torch

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
    yield ws, data, b
    b.close()


def test_adjoint_c5_batched(c5_batch):
    """One amr_batch_q_backward over all 48 geometries, weights on sampled faces of six geometries (the
    largest, the deepest and four seeded others): each one's vertices against its oracle gradient, a few
    faces against central differences, every other vertex of the batch exactly zero."""
    import torch

    from oracle.oracle import Domain, OracleGeometry
    from paper_2502_16310_gb300.binding import _view

    ws, data, b = c5_batch
    r = b.result
    nl = int(r.n_links)
    lf_all = _view(r.link_face, (nl,), torch.int32).long()
    nf_tot = sum(w.n_faces for w in ws)
    rng = np.random.default_rng(77)
    big = int(np.argmax([w.n_faces for w in ws]))
    deep = int(np.argmax([w.n_levels * 1000 + w.root for w in ws]))
    pick = sorted({big, deep, *rng.choice(len(ws), size=4, replace=False).tolist()})
    views = {i: b.view(i) for i in pick}
    sel_f = torch.zeros(nf_tot, dtype=torch.bool, device="cuda")
    picked = {}
    for i in pick:
        fs = independent_faces(ws[i].idx, 300, rng)
        picked[i] = fs
        sel_f[torch.from_numpy(fs + views[i]["bases"]["face"]).cuda()] = True
    rows = torch.nonzero(sel_f[lf_all]).flatten()
    wts = torch.zeros(nl, dtype=torch.float32, device="cuda")
    wts[rows] = torch.randn(rows.numel(), device="cuda", generator=torch.Generator("cuda").manual_seed(8))
    grad = b.q_backward(wts).cpu().numpy().astype(np.float64)
    wh_all = wts.cpu().numpy()
    vbase, checked = 0, 0
    for i, w in enumerate(ws):
        nv = w.verts.shape[0]
        gi = grad[vbase:vbase + nv]
        vbase += nv
        if i not in picked:
            assert np.all(gi == 0.0), f"geometry {i}: non-zero gradient without weighted links"
            continue
        vw = views[i]
        lb = vw["bases"]["link"]
        faces = vw["link_face"].cpu().numpy()
        loc_rows = np.nonzero(np.isin(faces, picked[i]))[0]
        wloc = wh_all[lb + loc_rows]
        ids = vw["adj_cell"].cpu().numpy()[vw["link_cell"].cpu().numpy()[loc_rows]]
        fin = vw["levels"][-1]["blocks"].cpu().numpy()
        cells = U.cells_of(3, fin, (ids // 64).astype(np.int64), (ids % 64).astype(np.int64))
        dirs = vw["link_dir"].cpu().numpy()[loc_rows]
        fsel = faces[loc_rows]
        L = w.n_levels - 1
        geo = OracleGeometry(3, w.verts, w.idx)
        geo.bin(Domain.unit(3, w.root), w.bins)  # sets the oracle's domain
        ref = oracle_vertex_grad(geo, w, L, cells, dirs, fsel, wloc)
        touched = np.zeros(nv, bool)
        touched[w.idx[picked[i]].ravel()] = True
        assert np.all(gi[~touched] == 0.0), f"geometry {i}: a vertex of no sampled face has a gradient"
        assert_close(gi[touched], ref[touched], f"c5 geometry {i} vs the oracle")
        fd = central_differences(geo, w, L, cells, dirs, fsel, wloc,
                                 picked[i][rng.choice(picked[i].size, min(5, picked[i].size), replace=False)])
        keys = list(fd)
        if keys:
            assert_close(np.array([gi[v, c] for v, c in keys]), np.array([fd[k] for k in keys]),
                         f"c5 geometry {i} vs central differences")
        checked += len(keys)
    assert checked > 50
