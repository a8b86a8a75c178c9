"""The five synthetic workloads of the near-wall refinement path (input recipes only).

Each workload fixes: the geometry (seeded generator call), the root grid
(R_0 root blocks of 4^D cells per axis on the unit domain [0,1]^D), the total
number of grid levels, the bin density B (bins per axis), the lattice of the
wall links (D2Q9 or D3Q19) and whether the vertex adjoint of q is requested.

  c1  2D circle, 512 equal edges, r = 0.2 at (0.5, 0.5); 16^2 roots; 3 levels; B = 32; D2Q9.
  c2  3D icosphere subdivided 5x (20,480 triangles), r = 0.25 at the centre,
      vertices jittered by N(0, 1e-4); 32^3 roots; 4 levels; B = 64; D3Q19.
  c3  icosphere 6x (81,920 triangles) with r = 0.25(1 + sum_{l<=8} a_lm Y_lm),
      a_lm ~ N(0, 0.05/l), scaled (1, 0.8, 0.9); 32^3 roots; 5 levels; B = 128; D3Q19; adjoint.
  c4  same generator at 8 subdivisions (1,310,720 triangles), l <= 16;
      64^3 roots; 6 levels; B = 256; D3Q19; adjoint.
  c5  48 perturbed geodesic spheres, triangle count log-uniform in [1e3, 5e5],
      R_0 ~ U{16..48}, levels ~ U{2..6}; batched.

"levels" counts every level of the hierarchy, so a workload with n levels runs
n - 1 refinement passes (the paper's circle test: refined twice, three levels).
The near-wall distance is one cell width of the level being refined
(d_L = h_L), so the inflated cell box has half-width 1.5 h_L.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import geometry as G

__all__ = ["Workload", "workload", "batched_workloads", "small_workload", "NAMES"]

NAMES = ("c1", "c2", "c3", "c4", "c5")


@dataclass
class Workload:
    name: str
    dim: int
    verts: np.ndarray          # float32 [n_v, D]
    idx: np.ndarray            # int32 [n_f, D]
    root: int                  # R_0 root blocks per axis
    n_levels: int
    bins: int                  # bin density B
    lattice: int               # 9 (D2Q9) or 19 (D3Q19)
    d_abs: float = 0.0
    d_rel: float = 1.0
    predicate: int = 0         # 0: box (inflated cell meets the face), 1: point (centre within d, Alg. 1)
    adjoint: bool = False
    description: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_faces(self) -> int:
        return int(self.idx.shape[0])

    @property
    def h0(self) -> float:
        """Root-level cell size on the unit domain."""
        return 1.0 / (4.0 * self.root)


def _c1():
    v, f = G.circle_polygon(512, 0.2, (0.5, 0.5))
    return Workload("c1", 2, v, f, root=16, n_levels=3, bins=32, lattice=9,
                    description="2D circle r=0.2, 512 segments, 16^2 roots of 4^2 cells, 3 levels, 32^2 bins, D2Q9")


def _c2():
    v, f = G.jittered_sphere(5, radius=0.25, centre=(0.5, 0.5, 0.5), sigma=1e-4, seed=2)
    return Workload("c2", 3, v, f, root=32, n_levels=4, bins=64, lattice=19,
                    description="icosphere-5 (20,480 tris) r=0.25 jittered N(0,1e-4), 32^3 roots of 4^3 cells, "
                                "4 levels, 64^3 bins, D3Q19")


def _perturbed(subdiv, lmax, seed):
    u, f = G.icosphere_unit(subdiv)
    return G.perturbed_surface(u, f, seed=seed, lmax=lmax)


def _c3():
    v, f = _perturbed(6, 8, 3)
    return Workload("c3", 3, v, f, root=32, n_levels=5, bins=128, lattice=19, adjoint=True,
                    description="SH-perturbed icosphere-6 (81,920 tris, l<=8), 32^3 roots, 5 levels, 128^3 bins, "
                                "D3Q19, q adjoint")


def _c4():
    v, f = _perturbed(8, 16, 4)
    return Workload("c4", 3, v, f, root=64, n_levels=6, bins=256, lattice=19, adjoint=True,
                    description="SH-perturbed icosphere-8 (1,310,720 tris, l<=16), 64^3 roots, 6 levels, "
                                "256^3 bins, D3Q19, q adjoint")


def _p2():
    # the paper's 2D speed-up setup: 12,800 edges in the middle of a 256^2 grid on [0,1]^2,
    # d_spec = 0.1, refined twice (radius not stated: 0.25)
    v, f = G.circle_polygon(12800, 0.25, (0.5, 0.5))
    return Workload("p2", 2, v, f, root=64, n_levels=3, bins=16, lattice=9, d_abs=0.1, d_rel=0.0, predicate=1,
                    description="paper 2D setup: circle r=0.25, 12,800 segments, 256^2 cells (64^2 roots), "
                                "3 levels, d_spec=0.1, point predicate")


def _p3():
    # the paper's 3D setup with a synthetic stand-in for the 112,402-face bunny: a geodesic
    # sphere of frequency 75 (112,500 triangles), SH-perturbed and anisotropic like c3;
    # 64^3 grid on [0,1]^3, d_spec = 0.05, refined twice
    u, f = G.geodesic_sphere_unit(75)
    v, f = G.perturbed_surface(u, f, seed=31, lmax=8)
    return Workload("p3", 3, v, f, root=16, n_levels=3, bins=16, lattice=19, d_abs=0.05, d_rel=0.0, predicate=1,
                    description="paper 3D setup: SH-perturbed geodesic sphere (112,500 tris, bunny-scale), "
                                "64^3 cells (16^3 roots), 3 levels, d_spec=0.05, point predicate")


def batched_workloads(n: int = 48, base_seed: int = 5000):
    """The batched workload: ``n`` perturbed geodesic spheres of uneven size and depth.

    Geometry i uses ``default_rng(base_seed + i)`` for T_i = exp(U(ln 1e3, ln 5e5)),
    R_0 ~ U{16..48}, levels ~ U{2..6} and the SH coefficients.  Its frequency is
    round(sqrt(T_i / 20)), giving 20 * freq^2 triangles.  Bin density 0 means "pick by tuning".
    """
    out = []
    for i in range(n):
        rng = np.random.default_rng(base_seed + i)
        t = math.exp(rng.uniform(math.log(1e3), math.log(5e5)))
        freq = max(1, int(round(math.sqrt(t / 20.0))))
        root = int(rng.integers(16, 49))
        levels = int(rng.integers(2, 7))
        sh_seed = int(rng.integers(0, 2**31 - 1))
        u, f = G.geodesic_sphere_unit(freq)
        v, f = G.perturbed_surface(u, f, seed=sh_seed, lmax=8)
        out.append(Workload(f"c5[{i}]", 3, v, f, root=root, n_levels=levels, bins=0, lattice=19, adjoint=True,
                            description=f"geodesic sphere freq {freq} ({f.shape[0]} tris), {root}^3 roots, "
                                        f"{levels} levels",
                            meta={"freq": freq, "target_tris": t}))
    return out


def workload(name: str) -> Workload:
    """Build one named workload (c1..c4, the paper's setups p2 / p3); c5 is ``batched_workloads()``."""
    return {"c1": _c1, "c2": _c2, "c3": _c3, "c4": _c4, "p2": _p2, "p3": _p3}[name]()


def small_workload(kind: str, *, seed: int = 11):
    """Reduced cases the oracle finishes in seconds (several tiles plus a ragged tail)."""
    if kind == "sphere3":
        v, f = G.jittered_sphere(3, radius=0.27, centre=(0.5, 0.49, 0.51), sigma=1e-4, seed=seed)
        return Workload("sphere3", 3, v, f, root=8, n_levels=3, bins=32, lattice=19,
                        description="icosphere-3 (1,280 tris), 8^3 roots, 3 levels, 32^3 bins")
    if kind == "bumpy3":
        u, f = G.icosphere_unit(3)
        v, f = G.perturbed_surface(u, f, seed=seed, lmax=6)
        return Workload("bumpy3", 3, v, f, root=6, n_levels=3, bins=24, lattice=19, adjoint=True,
                        description="SH-perturbed icosphere-3, 6^3 roots (non-dyadic h), 3 levels, 24^3 bins")
    if kind == "circle":
        v, f = G.circle_polygon(97, 0.31, (0.47, 0.52))
        return Workload("circle97", 2, v, f, root=10, n_levels=4, bins=7, lattice=9, adjoint=True,
                        description="2D 97-gon, 10^2 roots (non-dyadic h), 4 levels, 7^2 bins")
    raise KeyError(kind)
