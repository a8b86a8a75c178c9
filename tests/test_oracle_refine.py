"""Pins of the oracle's near-wall refinement (Sec. "Cell-Face Identification Algorithms").

  * brute force: every cell against every face (the paper's naive scheme, B = 1
    in its notation) through the bare predicate, with no bins at all;
  * bin independence: exact binning only prunes candidates, so the masks are
    identical for every bin density;
  * closed forms: for an inscribed polygon / polyhedron of a circle / sphere, a
    cell's inflated box that holds a point strictly inside the inscribed
    radius and a point strictly outside the circumscribed radius must meet the
    surface, and a box entirely inside or outside the annulus cannot;
  * children: 2^D per marked block, inside the parent, canonical order.
"""
import numpy as np
import pytest

from synth import geometry as G


def _box_dist_range(lo, hi, c):
    """min and max distance from point c to the axis-aligned box [lo, hi]."""
    near = np.clip(c, lo, hi)
    dmin = np.linalg.norm(near - c, axis=-1)
    far = np.where(np.abs(lo - c) > np.abs(hi - c), lo, hi)
    dmax = np.linalg.norm(far - c, axis=-1)
    return dmin, dmax


def _cells(dim, blocks):
    n = 64 if dim == 3 else 16
    c = np.arange(n)
    loc = np.stack([c & 3, (c >> 2) & 3] + ([(c >> 4) & 3] if dim == 3 else []), 1)
    return 4 * blocks[:, None, :] + loc[None]


def test_brute_force_tiny(oracle_lib):
    from oracle.oracle import Domain, OracleGeometry, root_blocks, sat_margin

    v, f = G.jittered_sphere(1, radius=0.3, centre=(0.52, 0.47, 0.5), sigma=2e-3, seed=9)
    fv = v[f].astype(np.float64)
    root = 3
    dom = Domain.unit(3, root)
    g = OracleGeometry(3, v, f)
    g.bin(dom, 5)
    blocks = root_blocks(3, (root,) * 3)
    for level in (0, 1):
        if level == 1:
            blocks = g.children(blocks, mask)[0][:40]
        mask, band, _, _ = g.refine_blocks(level, blocks, 0.0, 1.0)
        h = dom.h(level)
        r = 1.5 * h
        cells = _cells(3, blocks)
        want = np.zeros(blocks.shape[0], np.uint64)
        for b in range(blocks.shape[0]):
            for c in range(64):
                x = (cells[b, c] + 0.5) * h
                if any(sat_margin(3, fv[k] - x, r) <= 0 for k in range(fv.shape[0])):
                    want[b] |= np.uint64(1) << np.uint64(c)
        assert np.array_equal(mask, want)
        assert np.any(mask != 0)


@pytest.mark.parametrize("dim", [2, 3])
def test_bin_density_independence(oracle_lib, dim):
    from oracle.oracle import Domain, OracleGeometry, root_blocks

    if dim == 2:
        v, f = G.circle_polygon(61, 0.33, (0.51, 0.5))
        root = 8
    else:
        v, f = G.jittered_sphere(2, radius=0.31, centre=(0.5, 0.5, 0.5), sigma=1e-3, seed=4)
        root = 4
    dom = Domain.unit(dim, root)
    blocks = root_blocks(dim, (root,) * dim)
    ref = None
    for B in (1, 2, 3, 8, 13, 32):
        g = OracleGeometry(dim, v, f)
        g.bin(dom, B)
        m0, _, _, _ = g.refine_blocks(0, blocks)
        ch, _ = g.children(blocks, m0)
        m1, _, _, _ = g.refine_blocks(1, ch)
        cur = (m0, m1)
        if ref is None:
            ref = cur
        assert np.array_equal(ref[0], cur[0]) and np.array_equal(ref[1], cur[1]), B


def test_children_canonical(oracle_lib):
    from oracle.oracle import OracleGeometry

    g = OracleGeometry(3, np.zeros((0, 3, 3), np.float32), None)
    blocks = np.array([[0, 0, 0], [1, 2, 3], [5, 0, 1]], np.int32)
    mask = np.array([1, 0, 2**63], np.uint64)
    cb, cp = g.children(blocks, mask)
    assert cb.shape == (16, 3) and cp.tolist() == [0] * 8 + [2] * 8
    for k in range(16):
        s = k % 8
        assert np.array_equal(cb[k], 2 * blocks[cp[k]] + np.array([s & 1, (s >> 1) & 1, (s >> 2) & 1]))


def test_circle_closed_form_c1(oracle_lib):
    """c1 (512-gon, r = 0.2) on all three levels against the analytic circle annulus."""
    from oracle.oracle import run_pipeline
    from synth import workload

    w = workload("c1")
    out = run_pipeline(2, w.verts, w.idx, root=w.root, n_levels=w.n_levels, B=w.bins, lattice=9, links=False)
    R = 0.2
    r_in = R * np.cos(np.pi / 512)
    slack = 1e-7  # FP32 rounding of the polygon vertices
    checked = 0
    for L, lv in enumerate(out["levels"]):
        h = out["dom"].h(L)
        rr = 1.5 * h
        cells = _cells(2, lv["blocks"])
        x = (cells + 0.5) * h
        dmin, dmax = _box_dist_range(x - rr, x + rr, np.array([0.5, 0.5]))
        bits = ((lv["mask"][:, None] >> np.arange(16, dtype=np.uint64)) & np.uint64(1)).astype(bool)
        must = (dmin < r_in - slack) & (dmax > R + slack)
        never = (dmin > R + slack) | (dmax < r_in - slack)
        assert not np.any(must & ~bits), L
        assert not np.any(never & bits), L
        checked += int(must.sum() + never.sum())
        # blocks: every one on level L>0 is a child of a marked block
    assert checked > 5000
    # level block counts follow from the masks
    for L in range(len(out["levels"]) - 1):
        assert out["levels"][L + 1]["blocks"].shape[0] == 4 * int((out["levels"][L]["mask"] != 0).sum())


def test_sphere_closed_form(oracle_lib):
    from oracle.oracle import run_pipeline

    u, f = G.icosphere_unit(3)
    R, c = 0.29, np.array([0.5, 0.5, 0.5])
    v = (u * R + c).astype(np.float32)
    tri = v[f].astype(np.float64) - c
    nrm = np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0])
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    r_in = np.min(np.abs(np.einsum("ij,ij->i", nrm, tri[:, 0])))  # inradius of the polyhedron
    r_out = np.max(np.linalg.norm(v.astype(np.float64) - c, axis=1))
    out = run_pipeline(3, v, f, root=4, n_levels=2, B=16, lattice=19, links=False)
    checked = 0
    for L, lv in enumerate(out["levels"]):
        h = out["dom"].h(L)
        rr = 1.5 * h
        cells = _cells(3, lv["blocks"])
        x = (cells + 0.5) * h
        dmin, dmax = _box_dist_range(x - rr, x + rr, c)
        bits = ((lv["mask"][:, None] >> np.arange(64, dtype=np.uint64)) & np.uint64(1)).astype(bool)
        must = (dmin < r_in - 1e-7) & (dmax > r_out + 1e-7)
        never = (dmin > r_out + 1e-7) | (dmax < r_in - 1e-7)
        assert not np.any(must & ~bits)
        assert not np.any(never & bits)
        checked += int(must.sum() + never.sum())
    assert checked > 10000
