"""Pins of the oracle's node classification (solid = inside the closed boundary mesh, by the
generalized winding number): closed forms for a cube and a sphere, the circle in 2D, the
orientation flip, and the winding number's values away from the mesh."""
import math

import numpy as np

from oracle.oracle import Domain, OracleGeometry


def _cube():
    v = np.array([[x, y, z] for z in (0.3, 0.7) for y in (0.3, 0.7) for x in (0.3, 0.7)], np.float32)
    # outward-oriented triangles of the 6 faces (vertex id = x + 2y + 4z)
    quads = [(0, 2, 3, 1), (4, 5, 7, 6), (0, 1, 5, 4), (2, 6, 7, 3), (0, 4, 6, 2), (1, 3, 7, 5)]
    f = []
    for a, b, c, d in quads:
        f += [(a, b, c), (a, c, d)]
    return v, np.array(f, np.int32)


def test_cube_exact():
    v, f = _cube()
    geo = OracleGeometry(3, v, f)
    rng = np.random.default_rng(1)
    pts = rng.uniform(0.0, 1.0, size=(400, 3))
    inside = np.all((pts > 0.3) & (pts < 0.7), axis=1)
    dist = np.min(np.abs(pts[:, :, None] - np.array([0.3, 0.7])[None, None, :]), axis=(1, 2))
    for p, want, dd in zip(pts, inside, dist):
        w = geo.winding_number(p)
        if dd > 1e-3 or not want:
            assert abs(abs(w) - (1.0 if want else 0.0)) < 1e-9, (p, w)
    # reversed orientation: w changes sign, the class does not
    geo_r = OracleGeometry(3, v, f[:, ::-1].copy())
    p = np.array([0.5, 0.45, 0.55])
    assert geo.winding_number(p) == -geo_r.winding_number(p) and abs(geo.winding_number(p)) > 0.99


def test_sphere_closed_form():
    """Icosphere inscribed in the sphere r = 0.3: the mesh lies between the sphere and the sphere
    of radius r cos(theta), theta the largest angle a face subtends at the centre; cells outside
    that shell are solid exactly when their centre is inside the sphere."""
    from synth import geometry as G

    u, f = G.icosphere_unit(3)
    c0, r = np.array([0.5, 0.5, 0.5]), 0.3
    v = (c0 + r * u).astype(np.float32)
    geo = OracleGeometry(3, v, f)
    dom = Domain.unit(3, 8)
    uf = u[f]
    cosmin = np.min(np.einsum("fij,fkj->fik", uf, uf))
    shell_lo = r * cosmin - 1e-6
    rng = np.random.default_rng(2)
    cells = rng.integers(0, 32, size=(600, 3)).astype(np.int32)
    solid, band = geo.classify(0, cells, dom)
    x = (cells + 0.5) / 32.0
    rad = np.linalg.norm(x - c0, axis=1)
    firm = (rad < shell_lo) | (rad > r + 1e-6)
    assert np.array_equal(solid[firm], rad[firm] < r)
    assert firm.sum() > 500 and not band[firm].any()


def test_circle_2d():
    from synth import geometry as G

    v, f = G.circle_polygon(97, 0.2, (0.5, 0.5))
    geo = OracleGeometry(2, v, f)
    dom = Domain.unit(2, 16)
    sag = 0.2 * (1 - math.cos(math.pi / 97)) + 1e-6
    cells = np.array([(i, j) for i in range(64) for j in range(64)], np.int32)
    solid, _ = geo.classify(0, cells, dom)
    rad = np.linalg.norm((cells + 0.5) / 64.0 - 0.5, axis=1)
    firm = np.abs(rad - 0.2) > sag
    assert np.array_equal(solid[firm], rad[firm] < 0.2)
    assert solid.sum() > 300


def test_winding_values_away_from_mesh():
    from synth import small_workload

    w = small_workload("bumpy3")
    geo = OracleGeometry(3, w.verts, w.idx)
    rng = np.random.default_rng(3)
    for p in rng.uniform(0.0, 1.0, size=(100, 3)):
        wn = geo.winding_number(p)
        assert min(abs(wn), abs(abs(wn) - 1.0)) < 1e-9
