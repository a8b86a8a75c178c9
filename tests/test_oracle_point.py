"""Pins of the oracle's point predicate (Alg. 1, Sec. "Face Detection"): a cell centre
is adjacent to a face when its Euclidean distance to the closed face is at most the
near-wall distance.  The oracle's distance is checked against things fixed without it:
closed forms for each region of the triangle, brute force over a dense sampling of
the face, the ball/box bracket with the separating-axis predicate, and the circle.
"""
import math

import numpy as np
import pytest

from oracle.oracle import Domain, OracleGeometry, point_face_dist, root_blocks, sat_margin


def _rotation(rng):
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    return q * np.sign(np.diag(r))


def test_point_face_dist_regions():
    """Right triangle (0,0,0), (1,0,0), (0,1,0) seen from points whose closest feature is
    known: the interior (plane distance), an edge (distance to the edge's line) and a
    vertex (distance to the vertex), under random rigid motions."""
    rng = np.random.default_rng(1)
    tri = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    cases = [
        (np.array([0.2, 0.3, 0.7]), 0.7),                             # above the interior
        (np.array([0.5, -0.4, 0.3]), math.hypot(0.4, 0.3)),           # beside edge v0-v1
        (np.array([0.6, 0.6, -0.2]), math.sqrt(2 * 0.1 ** 2 + 0.04)),  # beside the hypotenuse
        (np.array([-0.3, -0.4, 0.0]), 0.5),                           # beyond vertex v0, in the plane
        (np.array([1.3, -0.1, 0.2]), math.sqrt(0.09 + 0.01 + 0.04)),  # beyond vertex v1
        (np.array([0.25, 0.25, 0.0]), 0.0),                           # on the face
    ]
    for x, want in cases:
        for _ in range(5):
            R = _rotation(rng)
            t = rng.normal(size=3)
            v = (tri @ R.T + t) - (x @ R.T + t)
            assert point_face_dist(3, v) == pytest.approx(want, abs=1e-12)


def test_point_segment_dist_regions():
    seg = np.array([[0.0, 0.0], [2.0, 0.0]])
    for x, want in [((1.0, 0.5), 0.5), ((-0.3, 0.4), 0.5), ((2.6, -0.8), 1.0), ((0.7, 0.0), 0.0)]:
        assert point_face_dist(2, seg - np.array(x)) == pytest.approx(want, abs=1e-14)


def _brute_tri(v, n=300):
    """Minimum distance from the origin over a barycentric grid on the triangle, plus
    each edge sampled 20x finer; an upper bound within the grid spacing."""
    a, b, c = v
    i, j = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")
    keep = i + j <= n
    s, t = i[keep] / n, j[keep] / n
    pts = a + s[:, None] * (b - a) + t[:, None] * (c - a)
    best = np.sqrt((pts ** 2).sum(1)).min()
    u = np.linspace(0.0, 1.0, 20 * n + 1)[:, None]
    for p, q in ((a, b), (b, c), (c, a)):
        e = p + u * (q - p)
        best = min(best, np.sqrt((e ** 2).sum(1)).min())
    return best


def test_point_face_dist_brute_force():
    rng = np.random.default_rng(2)
    for _ in range(40):
        v = rng.normal(size=(3, 3))
        if rng.random() < 0.2:
            v[2] = v[0] + 1e-3 * rng.normal(size=3)  # near-degenerate slivers
        d = point_face_dist(3, v)
        brute = _brute_tri(v)
        diam = max(np.linalg.norm(v[0] - v[1]), np.linalg.norm(v[1] - v[2]), np.linalg.norm(v[2] - v[0]))
        assert d <= brute + 1e-12
        assert brute - d <= diam / 300 + 1e-12


def test_point_face_dist_degenerate_faces():
    # zero-area faces: a segment (collinear vertices) and a point
    v = np.array([[1.0, 0.0, 0.0], [2.0, 0.0, 0.0], [3.0, 0.0, 0.0]]) - np.array([2.0, 1.0, 0.0])
    assert point_face_dist(3, v) == pytest.approx(1.0, abs=1e-14)
    p = np.tile(np.array([[0.3, 0.4, 0.0]]), (3, 1))
    assert point_face_dist(3, p) == pytest.approx(0.5, abs=1e-14)


def test_point_predicate_box_bracket():
    """The ball of radius R lies in the box of half-width R and contains the box of
    half-width R / sqrt(D): point-adjacent => box-adjacent at R, and box-adjacent at
    R / sqrt(D) => point-adjacent."""
    rng = np.random.default_rng(3)
    for D in (2, 3):
        n_pos = 0
        for _ in range(600):
            v = rng.uniform(-1.0, 1.0, size=(D, D))
            R = rng.uniform(0.05, 1.0)
            d = point_face_dist(D, v)
            if d <= R:
                n_pos += 1
                assert sat_margin(D, v, R) <= 1e-12
            if sat_margin(D, v, R / math.sqrt(D)) <= -1e-12:
                assert d <= R + 1e-12
        assert 50 < n_pos < 550


def test_point_refine_circle_closed_form():
    """512-gon inscribed in the circle r = 0.2: the polygon lies within the sagitta
    s = r (1 - cos(pi/512)) of the circle, so a cell whose analytic distance to the circle
    is farther than s from d must be adjacent exactly when that distance is at most d."""
    from synth import workload

    w = workload("c1")
    geo = OracleGeometry(2, w.verts, w.idx)
    dom = Domain.unit(2, w.root)
    geo.bin(dom, w.bins)
    r0, c0 = 0.2, np.array([0.5, 0.5])
    sag = r0 * (1.0 - math.cos(math.pi / 512)) + 1e-7  # + FP32 rounding of the vertices
    d = 0.03
    blocks = root_blocks(2, (w.root, w.root))
    mask, band, _, _ = geo.refine_blocks(0, blocks, d_abs=d, d_rel=0.0, pred=1)
    h = dom.h(0)
    checked = 0
    for b in range(blocks.shape[0]):
        for bit in range(16):
            cell = 4 * blocks[b] + np.array([bit & 3, bit >> 2])
            x = dom.origin[:2] + (cell + 0.5) * h
            dist = abs(np.linalg.norm(x - c0) - r0)
            if abs(dist - d) > sag:
                assert bool((int(mask[b]) >> bit) & 1) == (dist <= d), (cell, dist)
                checked += 1
    assert checked > 3000


def test_point_refine_bin_density_independence():
    from synth import small_workload

    w = small_workload("sphere3")
    dom = Domain.unit(3, w.root)
    blocks = root_blocks(3, (w.root,) * 3)
    ref = None
    for B in (1, 3, 16):
        geo = OracleGeometry(3, w.verts, w.idx)
        geo.bin(dom, B)
        mask, _, _, _ = geo.refine_blocks(0, blocks, d_abs=0.06, d_rel=0.0, pred=1)
        if ref is None:
            ref = mask
        assert np.array_equal(mask, ref), B
