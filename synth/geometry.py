"""Seeded synthetic surface meshes: the input data of the near-wall refinement path.

This module only builds input geometry (vertex coordinates and face index lists).
It holds none of the method's arithmetic: no binning, no adjacency predicate, no
link intersection.  Both the FP64 oracle and the CUDA path read what it returns.

Every generator returns ``(verts, idx)``:
  * ``verts``: float32 array ``[n_verts, D]`` (D = 2 for polylines, 3 for surfaces),
  * ``idx``:   int32 array ``[n_faces, D]`` of vertex indices per face
    (edges in 2D, triangles in 3D), faces oriented outward (counter-clockwise
    polygon in 2D, outward normals in 3D).

The shapes follow the paper's test geometries (Sec. "Results and Discussion":
a circle polygonised into equal edges in 2D, a closed triangle surface of
non-uniform triangle sizes in 3D) at the sizes of the synthetic workloads.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "circle_polygon",
    "icosahedron",
    "icosphere_unit",
    "geodesic_sphere_unit",
    "real_sph_harm_basis",
    "perturbed_surface",
    "jittered_sphere",
    "face_vertex_list",
]


def circle_polygon(n_seg: int, radius: float, centre=(0.5, 0.5)):
    """Regular ``n_seg``-gon inscribed in a circle; vertices computed in FP64, stored FP32.

    Edge k joins vertex k to vertex k+1 (mod n), so the polygon is counter-clockwise.
    """
    k = np.arange(n_seg, dtype=np.float64)
    ang = 2.0 * math.pi * k / n_seg
    v = np.stack([centre[0] + radius * np.cos(ang), centre[1] + radius * np.sin(ang)], axis=1)
    idx = np.stack([np.arange(n_seg), (np.arange(n_seg) + 1) % n_seg], axis=1)
    return v.astype(np.float32), idx.astype(np.int32)


def icosahedron():
    """Unit icosahedron (12 vertices, 20 outward-oriented faces), FP64."""
    p = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array(
        [
            [-1, p, 0], [1, p, 0], [-1, -p, 0], [1, -p, 0],
            [0, -1, p], [0, 1, p], [0, -1, -p], [0, 1, -p],
            [p, 0, -1], [p, 0, 1], [-p, 0, -1], [-p, 0, 1],
        ],
        dtype=np.float64,
    )
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array(
        [
            [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
            [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
            [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
            [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1],
        ],
        dtype=np.int64,
    )
    return v, f


def icosphere_unit(subdiv: int):
    """Icosahedron subdivided ``subdiv`` times by edge-midpoint split, projected to the unit sphere.

    Returns FP64 vertices ``[n_v,3]`` and int64 faces ``[20*4**subdiv, 3]``.
    """
    v, f = icosahedron()
    for _ in range(subdiv):
        nv = v.shape[0]
        e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]], axis=0)
        key = np.sort(e, axis=1)
        uniq, inv = np.unique(key, axis=0, return_inverse=True)
        inv = inv.reshape(-1)
        mid = v[uniq[:, 0]] + v[uniq[:, 1]]
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        v = np.concatenate([v, mid], axis=0)
        nf = f.shape[0]
        m01 = nv + inv[0:nf]
        m12 = nv + inv[nf:2 * nf]
        m20 = nv + inv[2 * nf:3 * nf]
        a, b, c = f[:, 0], f[:, 1], f[:, 2]
        f = np.concatenate(
            [
                np.stack([a, m01, m20], 1),
                np.stack([b, m12, m01], 1),
                np.stack([c, m20, m12], 1),
                np.stack([m01, m12, m20], 1),
            ],
            axis=0,
        )
    return v, f


def geodesic_sphere_unit(freq: int):
    """Class-I geodesic sphere of frequency ``freq``: every icosahedron face split into freq^2 triangles.

    Frequency 2**k equals the icosphere subdivided k times (same vertex set).
    Shared edge/vertex points are merged so the surface is closed.
    """
    if freq < 1:
        raise ValueError("freq must be >= 1")
    v0, f0 = icosahedron()
    n = freq
    # barycentric lattice points (i, j) with i + j <= n on each face
    ii, jj = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")
    keep = (ii + jj) <= n
    ii, jj = ii[keep], jj[keep]
    kk = n - ii - jj
    lut = -np.ones((n + 1, n + 1), dtype=np.int64)
    lut[ii, jj] = np.arange(ii.size)
    # triangles of the lattice ("up" and "down")
    tris = []
    for i in range(n):
        for j in range(n - i):
            tris.append((lut[i, j], lut[i + 1, j], lut[i, j + 1]))
            if i + j + 1 < n:
                tris.append((lut[i + 1, j], lut[i + 1, j + 1], lut[i, j + 1]))
    tris = np.asarray(tris, dtype=np.int64)
    pts = []
    faces = []
    base = 0
    for a, b, c in f0:
        p = (np.outer(ii, v0[a]) + np.outer(jj, v0[b]) + np.outer(kk, v0[c])) / n
        pts.append(p)
        # lattice axis i points to vertex a, j to b: triangle (i,j),(i+1,j),(i,j+1) keeps the face orientation
        faces.append(base + tris[:, [0, 2, 1]])
        base += p.shape[0]
    pts = np.concatenate(pts, 0)
    faces = np.concatenate(faces, 0)
    pts /= np.linalg.norm(pts, axis=1, keepdims=True)
    q = np.round(pts * 1e9).astype(np.int64)
    _, first, inv = np.unique(q, axis=0, return_index=True, return_inverse=True)
    inv = inv.reshape(-1)
    verts = pts[first]
    faces = inv[faces]
    # make orientation outward (all faces share one orientation by construction; flip if inward)
    tri = verts[faces]
    nrm = np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0])
    if np.sum(np.einsum("ij,ij->i", nrm, tri.mean(1))) < 0:
        faces = faces[:, [0, 2, 1]]
    return verts, faces


def real_sph_harm_basis(lmax: int, theta: np.ndarray, phi: np.ndarray):
    """Real orthonormal spherical harmonics Y_lm for 1 <= l <= lmax, all m (FP64).

    ``theta`` is the polar angle, ``phi`` the azimuth.  Returns a list of
    ``(l, m, values)``.  Normalised associated Legendre functions come from the
    standard three-term recurrences; the Condon-Shortley sign is omitted (the
    coefficients are symmetric random numbers, so the sign is immaterial).
    """
    x = np.cos(theta)
    s = np.sin(theta)
    out = []
    # Q[m] holds the normalised P_l^m for the running l, per m
    pmm = np.full_like(x, 1.0 / math.sqrt(4.0 * math.pi))
    diag = [pmm]
    for m in range(1, lmax + 1):
        pmm = math.sqrt((2.0 * m + 1.0) / (2.0 * m)) * s * pmm
        diag.append(pmm)
    table = {}
    for m in range(0, lmax + 1):
        p_lm2 = diag[m]
        table[(m, m)] = p_lm2
        if m + 1 <= lmax:
            p_lm1 = math.sqrt(2.0 * m + 3.0) * x * p_lm2
            table[(m + 1, m)] = p_lm1
            for l in range(m + 2, lmax + 1):
                a = math.sqrt((4.0 * l * l - 1.0) / (l * l - m * m))
                b = math.sqrt(((l - 1.0) ** 2 - m * m) / (4.0 * (l - 1.0) ** 2 - 1.0))
                p_l = a * (x * p_lm1 - b * p_lm2)
                table[(l, m)] = p_l
                p_lm2, p_lm1 = p_lm1, p_l
    r2 = math.sqrt(2.0)
    for l in range(1, lmax + 1):
        for m in range(-l, l + 1):
            if m == 0:
                out.append((l, m, table[(l, 0)]))
            elif m > 0:
                out.append((l, m, r2 * table[(l, m)] * np.cos(m * phi)))
            else:
                out.append((l, m, r2 * table[(l, -m)] * np.sin(-m * phi)))
    return out


def perturbed_surface(unit_verts: np.ndarray, faces: np.ndarray, *, seed: int, lmax: int,
                      radius: float = 0.25, sigma0: float = 0.05,
                      scale=(1.0, 0.8, 0.9), centre=(0.5, 0.5, 0.5)):
    """Star-shaped surface r(u) = radius * (1 + sum_{1<=l<=lmax} sum_m a_lm Y_lm(u)).

    a_lm ~ N(0, sigma0 / l) (standard deviation), drawn from ``numpy.random.default_rng(seed)``
    in (l, m) order; then the surface is scaled anisotropically about the centre.
    Returns FP32 vertices and int32 faces.
    """
    rng = np.random.default_rng(seed)
    u = unit_verts
    theta = np.arccos(np.clip(u[:, 2], -1.0, 1.0))
    phi = np.arctan2(u[:, 1], u[:, 0])
    pert = np.zeros(u.shape[0])
    for l, m, y in real_sph_harm_basis(lmax, theta, phi):
        a = rng.normal(0.0, sigma0 / l)
        pert += a * y
    r = radius * (1.0 + pert)
    if np.any(r <= 0):
        raise ValueError("perturbation produced a non-positive radius")
    p = u * r[:, None] * np.asarray(scale, dtype=np.float64)[None, :] + np.asarray(centre)[None, :]
    return p.astype(np.float32), faces.astype(np.int32)


def jittered_sphere(subdiv: int, *, radius: float, centre, sigma: float, seed: int):
    """Icosphere of ``subdiv`` subdivisions, radius ``radius``, vertices jittered by N(0, sigma)."""
    u, f = icosphere_unit(subdiv)
    rng = np.random.default_rng(seed)
    p = u * radius + np.asarray(centre, dtype=np.float64)[None, :]
    p = p + rng.normal(0.0, sigma, size=p.shape)
    return p.astype(np.float32), f.astype(np.int32)


def face_vertex_list(verts: np.ndarray, idx: np.ndarray) -> np.ndarray:
    """Coordinate-list form ``[n_faces, D(vertex), D(coord)]`` of an indexed mesh (a pure gather)."""
    return np.ascontiguousarray(verts[idx])
