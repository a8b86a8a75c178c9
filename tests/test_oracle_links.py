"""Pins of the oracle's wall links q and of their vertex gradient.

  * exact rational segment/face intersection (Cramer's rule in Fractions) over
    every face, for every link of sampled adjacent cells: hit/miss, min t and
    the smallest-id tie-break;
  * closed forms: the circle (polygon between the inscribed and circumscribed
    radii) and the sphere (polyhedron likewise) bound q by the analytic hit
    parameters of the two radii;
  * invariants: q in [0, 1]; opposite links of neighbouring cells through the
    same face give q + q' = 1;
  * the analytic dq/dv against FP64 central finite differences of q.
"""
import numpy as np
import pytest

from synth import geometry as G
from synth import small_workload
from tests.exact import segment_face_hit


def _pipeline(w, links=True):
    from oracle.oracle import run_pipeline

    return run_pipeline(w.dim, w.verts, w.idx, root=w.root, n_levels=w.n_levels, B=w.bins, lattice=w.lattice,
                        links=links)


@pytest.mark.parametrize("kind", ["circle", "bumpy3"])
def test_links_match_exact_rational(oracle_lib, kind):
    from oracle.oracle import lattice_dirs

    w = small_workload(kind)
    out = _pipeline(w)
    dom = out["dom"]
    L = w.n_levels - 1
    h = dom.h(L)
    dirs = lattice_dirs(w.lattice)
    fv = w.verts[w.idx]
    rng = np.random.default_rng(1)
    cells = out["adj_cells"]
    pick = rng.choice(cells.shape[0], size=min(25, cells.shape[0]), replace=False)
    n_hit = 0
    for i in pick:
        o = (cells[i].astype(np.float64) + 0.5) * h
        # faces that can possibly be hit: vertices within 3h of the cell (cheap exact prefilter)
        near = np.nonzero(np.abs(fv.astype(np.float64) - o).min(axis=1).max(axis=1) < 3 * h)[0]
        for k in range(1, dirs.shape[0]):
            d = dirs[k, :w.dim] * h
            best, bf = None, -1
            for f in near:
                t = segment_face_hit(o, d, fv[f].astype(np.float64))
                if t is not None and (best is None or t < best):
                    best, bf = t, f
            q, face, band = out["q"][i, k - 1], out["q_face"][i, k - 1], out["q_band"][i, k - 1]
            if band:
                continue
            if best is None:
                assert np.isnan(q) and face == -1
            else:
                n_hit += 1
                assert q == pytest.approx(float(best), abs=1e-12)
                # tie-break: the oracle's face hits at the same t
                tf = segment_face_hit(o, d, fv[face].astype(np.float64))
                assert tf is not None and abs(float(tf) - float(best)) < 1e-12
    assert n_hit > 20


def test_links_range_and_reciprocity(oracle_lib):
    from oracle.oracle import lattice_dirs

    w = small_workload("bumpy3")
    out = _pipeline(w)
    q = out["q"]
    ok = np.isfinite(q)
    assert np.all((q[ok] >= 0) & (q[ok] <= 1))
    dirs = lattice_dirs(19)
    opp = {k: int(np.nonzero(np.all(dirs == -dirs[k], axis=1))[0][0]) for k in range(1, 19)}
    index = {tuple(c): i for i, c in enumerate(out["adj_cells"].tolist())}
    pairs = 0
    for i, c in enumerate(out["adj_cells"]):
        for k in range(1, 19):
            if not ok[i, k - 1] or out["q_band"][i, k - 1]:
                continue
            nb = tuple((c + dirs[k]).tolist())
            j = index.get(nb)
            if j is None:
                continue
            ko = opp[k]
            if ok[j, ko - 1] and out["q_face"][j, ko - 1] == out["q_face"][i, k - 1] and not out["q_band"][j, ko - 1]:
                assert q[i, k - 1] + q[j, ko - 1] == pytest.approx(1.0, abs=1e-12)
                pairs += 1
    assert pairs > 1000


def _annulus_check(out, lattice, centre, r_in, r_out, h):
    """q of every adjacent cell against the inscribed / circumscribed circle (sphere).

    From a cell inside r_in the segment leaves the polygon (polyhedron) between
    the leaving roots of r_in and r_out; from a cell outside r_out it enters
    between the entering roots of r_out and r_in.  A segment that never reaches
    the shell cannot hit.  FP32 rounding of the vertices (< 1e-7) is allowed for
    through the radial rate of the segment at the crossings.
    """
    from oracle.oracle import lattice_dirs

    D = centre.shape[0]
    dirs = lattice_dirs(lattice)[:, :D]
    o = (out["adj_cells"].astype(np.float64) + 0.5) * h - centre
    rad0 = np.linalg.norm(o, axis=1)
    inside = rad0 < r_in - 1e-7
    outside = rad0 > r_out + 1e-7
    oo = np.einsum("ij,ij->i", o, o)
    n_firm = n_short = 0
    for k in range(1, dirs.shape[0]):
        d = dirs[k] * h
        a = d @ d
        b = 2 * o @ d

        def root(rho, leaving):
            disc = b * b - 4 * a * (oo - rho ** 2)
            sq = np.sqrt(np.maximum(disc, 0))
            t = (-b + sq) / (2 * a) if leaving else (-b - sq) / (2 * a)
            return np.where(disc > 0, t, np.nan)

        def rate(t):
            return np.abs(b + 2 * a * t) / (2 * np.sqrt(np.maximum(oo + b * t + a * t * t, 1e-30)))

        q = out["q"][:, k - 1]
        band = out["q_band"][:, k - 1]
        t_a = np.where(inside, root(r_in, True), root(r_out, False))
        t_b = np.where(inside, root(r_out, True), root(r_in, False))
        slack = 1e-7 / np.maximum(np.minimum(rate(np.nan_to_num(t_a)), rate(np.nan_to_num(t_b))), 1e-30)
        firm = ((inside | outside) & np.isfinite(t_a) & np.isfinite(t_b) & (t_a > slack) & (t_b < 1 - slack)
                & (slack < 1e-3) & ~band)
        assert np.all(np.isfinite(q[firm]))
        assert np.all((q[firm] >= t_a[firm] - slack[firm]) & (q[firm] <= t_b[firm] + slack[firm]))
        never = (inside & (t_a > 1 + slack)) | (outside & (np.isnan(t_a) | (t_a > 1 + slack) | (t_a < 0)))
        assert np.all(np.isnan(q[never & ~band]))
        n_firm += int(firm.sum())
        n_short += int((never & ~band).sum())
    return n_firm, n_short


def test_circle_closed_form_links(oracle_lib):
    from synth import workload

    w = workload("c1")
    out = _pipeline(w)
    h = out["dom"].h(w.n_levels - 1)
    n_firm, n_short = _annulus_check(out, 9, np.array([0.5, 0.5]), 0.2 * np.cos(np.pi / 512), 0.2, h)
    assert n_firm > 500 and n_short > 500


def test_sphere_closed_form_links(oracle_lib):
    from oracle.oracle import run_pipeline

    u, f = G.icosphere_unit(3)
    R, c = 0.29, np.array([0.5, 0.5, 0.5])
    v = (u * R + c).astype(np.float32)
    tri = v[f].astype(np.float64) - c
    nrm = np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0])
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    r_in = np.min(np.abs(np.einsum("ij,ij->i", nrm, tri[:, 0])))
    r_out = np.max(np.linalg.norm(v.astype(np.float64) - c, axis=1))
    out = run_pipeline(3, v, f, root=4, n_levels=2, B=16, lattice=19)
    h = out["dom"].h(1)
    n_firm, n_short = _annulus_check(out, 19, c, r_in, r_out, h)
    assert n_firm > 500 and n_short > 500


@pytest.mark.parametrize("kind", ["circle", "bumpy3"])
def test_q_grad_matches_finite_differences(oracle_lib, kind):
    w = small_workload(kind)
    out = _pipeline(w)
    geo, L, D = out["geo"], w.n_levels - 1, w.dim
    h = out["dom"].h(L)
    q = out["q"]
    ok = np.isfinite(q) & ~out["q_band"]
    ci, ki = np.nonzero(ok)
    rng = np.random.default_rng(5)
    sel = rng.choice(ci.shape[0], size=min(200, ci.shape[0]), replace=False)
    cells = out["adj_cells"][ci[sel]]
    dirs = (ki[sel] + 1).astype(np.int32)
    faces = out["q_face"][ci[sel], ki[sel]]
    wts = rng.normal(size=sel.shape[0])
    grad = geo.q_grad(L, w.lattice, cells, dirs, faces, wts)
    fv = w.verts[w.idx].astype(np.float64)
    delta = 1e-6 * h
    n_cmp = 0
    for f in np.unique(faces)[:40]:
        for k in range(D):
            for c in range(D):
                num = 0.0
                stable = True
                for j in np.nonzero(faces == f)[0]:
                    vp = fv[f].copy()
                    vm = fv[f].copy()
                    vp[k, c] += delta
                    vm[k, c] -= delta
                    qp = geo.link_q(L, w.lattice, cells[j], dirs[j], f, vp)
                    qm = geo.link_q(L, w.lattice, cells[j], dirs[j], f, vm)
                    if not (np.isfinite(qp) and np.isfinite(qm)):
                        stable = False
                        break
                    num += wts[j] * (qp - qm) / (2 * delta)
                if not stable:
                    continue
                an = grad[f, k, c]
                assert an == pytest.approx(num, rel=1e-5, abs=1e-6 * (abs(an) + 1.0)), (f, k, c, an, num)
                n_cmp += 1
    assert n_cmp > 50


@pytest.mark.parametrize("lattice", [9, 19])
def test_velocity_sets(oracle_lib, lattice):
    """The oracle's velocity sets are DdQq (rest vector first): the 2D set is the 8 neighbours of the
    square, the 3D set the 6 face and 12 edge neighbours of the cube; each closed under negation, with
    zero sum, and isotropic second moments (sum c_a c_b proportional to the identity)."""
    from oracle.oracle import lattice_dirs

    c = lattice_dirs(lattice).astype(np.int64)
    D = 2 if lattice == 9 else 3
    assert c.shape == (lattice, 3) and np.all(c[0] == 0)
    if D == 2:
        assert np.all(c[:, 2] == 0)
    m = c[1:, :D]
    assert len({tuple(r) for r in m.tolist()}) == lattice - 1
    n2 = (m * m).sum(axis=1)
    want = [(1, 4), (2, 4)] if D == 2 else [(1, 6), (2, 12)]
    assert sorted(np.unique(n2, return_counts=True)[0].tolist()) == [w[0] for w in want]
    assert [int((n2 == k).sum()) for k, _ in want] == [n for _, n in want]
    assert np.all(np.abs(m) <= 1)
    assert {tuple(r) for r in m.tolist()} == {tuple(r) for r in (-m).tolist()}
    assert np.all(m.sum(axis=0) == 0)
    second = m.T @ m
    assert np.array_equal(second, second[0, 0] * np.eye(D, dtype=np.int64))
