"""GPU q adjoint against the oracle's FP64 analytic gradient and FP64 central differences.

Criterion: per gradient entry |g_gpu - g_ref| <= 1e-4 |g_ref| + 1e-4 * rms(g_ref) (relative 1e-4, with a
floor at 1e-4 of the gradient's RMS for entries that nearly cancel).  Determinism: bitwise identical results
over repeated calls.
"""
import numpy as np
import pytest

from synth import small_workload, workload
from tests import gpu_util as U

pytestmark = pytest.mark.gpu
REL = 1e-4


def _run(w, facelist=False, seed=0):
    import torch

    from paper_2502_16310_gb300 import AmrGeom

    g = AmrGeom(w.dim, (w.root,) * w.dim)
    if facelist:
        g.load(torch.from_numpy(w.verts[w.idx]).cuda())
    else:
        g.load(torch.from_numpy(w.verts).cuda(), torch.from_numpy(w.idx).cuda())
    g.bin(w.bins)
    res = g.refine(w.n_levels, w.d_abs, w.d_rel, w.lattice, True, True)
    nl = res["link_q"].shape[0]
    rng = np.random.default_rng(seed)
    wts = rng.normal(size=nl).astype(np.float32)
    grad = g.q_backward(torch.from_numpy(wts).cuda())
    torch.cuda.synchronize()
    out = {"wts": wts, "grad": grad.cpu().numpy().astype(np.float64),
           "link_cell": U.to_np(res["link_cell"], np.uint32).copy(), "link_dir": U.to_np(res["link_dir"]).copy(),
           "link_face": U.to_np(res["link_face"], np.uint32).copy(), "link_q": U.to_np(res["link_q"]).copy(),
           "adj_cell": U.to_np(res["adj_cell"], np.uint32).copy(),
           "blocks": U.to_np(res["levels"][-1]["blocks"]).copy(), "geom": g}
    return out


def _oracle_grad(w, out):
    from oracle.oracle import Domain, OracleGeometry

    geo = OracleGeometry(w.dim, w.verts, w.idx)
    geo.bin(Domain.unit(w.dim, w.root), w.bins)
    nc = 64 if w.dim == 3 else 16
    rows = out["link_cell"].astype(np.int64)
    ids = out["adj_cell"][rows]
    cells = U.cells_of(w.dim, out["blocks"], (ids // nc).astype(np.int64), (ids % nc).astype(np.int64))
    gf = geo.q_grad(w.n_levels - 1, w.lattice, cells, out["link_dir"].astype(np.int32),
                    out["link_face"].astype(np.int64), out["wts"].astype(np.float64))
    return geo, cells, gf


def _to_vertices(w, gf):
    gv = np.zeros((w.verts.shape[0], w.dim))
    for k in range(w.dim):
        np.add.at(gv, w.idx[:, k], gf[:, k, :])
    return gv


def _assert_close(g, ref, what):
    scale = np.sqrt(np.mean(ref ** 2)) + 1e-300
    err = np.abs(g - ref)
    tol = REL * np.abs(ref) + REL * scale
    bad = err > tol
    assert not np.any(bad), (f"{what}: {int(bad.sum())}/{bad.size} entries off; worst rel "
                             f"{float(np.max(err / (np.abs(ref) + scale))):.3e}")
    return float(np.max(err / (np.abs(ref) + scale)))


@pytest.mark.parametrize("kind", ["circle", "bumpy3", "sphere3"])
def test_adjoint_matches_oracle_indexed(kind):
    w = small_workload(kind)
    out = _run(w)
    _, _, gf = _oracle_grad(w, out)
    _assert_close(out["grad"], _to_vertices(w, gf), kind)
    out["geom"].close()


@pytest.mark.parametrize("kind", ["circle", "bumpy3"])
def test_adjoint_matches_oracle_facelist(kind):
    w = small_workload(kind)
    out = _run(w, facelist=True)
    _, _, gf = _oracle_grad(w, out)
    _assert_close(out["grad"], gf, kind)
    out["geom"].close()


def test_adjoint_matches_central_differences():
    """GPU dL/dv against FP64 central differences of L = sum w q (face-vertex layout, sampled faces)."""
    w = small_workload("bumpy3")
    out = _run(w, facelist=True, seed=3)
    geo, cells, _ = _oracle_grad(w, out)
    L = w.n_levels - 1
    h = 1.0 / (4 * w.root) * 2.0 ** (-L)
    fv = w.verts[w.idx].astype(np.float64)
    faces = out["link_face"].astype(np.int64)
    rng = np.random.default_rng(9)
    cand = np.unique(faces)
    pick = rng.choice(cand, size=min(40, cand.size), replace=False)
    delta = 1e-6 * h
    got, want = [], []
    for f in pick:
        sel = np.nonzero(faces == f)[0]
        for k in range(3):
            for c in range(3):
                num, stable = 0.0, True
                for j in sel:
                    vp, vm = fv[f].copy(), fv[f].copy()
                    vp[k, c] += delta
                    vm[k, c] -= delta
                    qp = geo.link_q(L, 19, cells[j], int(out["link_dir"][j]), f, vp)
                    qm = geo.link_q(L, 19, cells[j], int(out["link_dir"][j]), f, vm)
                    if not (np.isfinite(qp) and np.isfinite(qm)):
                        stable = False
                        break
                    num += float(out["wts"][j]) * (qp - qm) / (2 * delta)
                if not stable:
                    continue
                got.append(out["grad"][f, k, c])
                want.append(num)
    assert len(got) > 100
    _assert_close(np.array(got), np.array(want), "central differences")
    out["geom"].close()


def test_adjoint_deterministic():
    import torch

    w = small_workload("bumpy3")
    out = _run(w)
    g = out["geom"]
    wts = torch.from_numpy(out["wts"]).cuda()
    first = g.q_backward(wts).cpu().numpy()
    for _ in range(9):
        again = g.q_backward(wts).cpu().numpy()
        assert np.array_equal(first.view(np.uint32), again.view(np.uint32))
    g.close()


def test_autograd_function():
    import torch

    from paper_2502_16310_gb300 import AmrGeom, q_links

    w = small_workload("bumpy3")
    g = AmrGeom(3, (w.root,) * 3)
    v = torch.from_numpy(w.verts).cuda().requires_grad_(True)
    idx = torch.from_numpy(w.idx).cuda()
    q = q_links(g, v, idx, w.bins, w.n_levels, w.d_abs, w.d_rel, 19)
    wts = torch.randn(q.shape[0], device="cuda", generator=torch.Generator("cuda").manual_seed(1))
    (wts * q).sum().backward()
    direct = g.q_backward(wts)
    assert torch.equal(v.grad, direct)
    g.close()


def test_adjoint_c3_full():
    w = workload("c3")
    out = _run(w, seed=5)
    _, _, gf = _oracle_grad(w, out)
    _assert_close(out["grad"], _to_vertices(w, gf), "c3")
    out["geom"].close()
