"""ctypes wrapper around the FP64 oracle library (``liboracle.so``) — test infrastructure.

``run_pipeline`` strings the oracle's per-step functions together in the
paper's order (import -> binning -> level-by-level near-wall refinement ->
adjacent-face lists and wall links on the finest level).  The loop over levels
and the child enumeration follow Sec. "Adaptive Mesh Refinement on GPUs"
(blocks of 4^D cells, one ID set per level) and the refine half of
M_RefineAndCoarsenBlocks.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "amr_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with g++ (no FMA contraction, no fast-math)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "amr_oracle.h"))):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB)
            P = C.c_void_p
            i64 = C.c_int64
            lib.orc_geom_new.restype = P
            lib.orc_geom_new.argtypes = [C.c_int, P, i64, P, i64, C.c_char_p, C.c_int]
            lib.orc_geom_free.argtypes = [P]
            lib.orc_geom_nfaces.restype = i64
            lib.orc_geom_nfaces.argtypes = [P]
            lib.orc_bins_build.restype = C.c_int
            lib.orc_bins_build.argtypes = [P, P, C.c_int]
            lib.orc_bins_nnz.restype = i64
            lib.orc_bins_nnz.argtypes = [P]
            lib.orc_bins_copy.argtypes = [P, P, P]
            lib.orc_face_bin_range.argtypes = [P, i64, P, P]
            lib.orc_sat_margin.restype = C.c_double
            lib.orc_sat_margin.argtypes = [C.c_int, P, C.c_double]
            lib.orc_refine_blocks.restype = C.c_int
            lib.orc_refine_blocks.argtypes = [P, P, C.c_int, C.c_double, C.c_double, C.c_int, C.c_int, P, i64, P, P,
                                              P, P]
            lib.orc_bins_build_sampled.restype = C.c_int
            lib.orc_bins_build_sampled.argtypes = [P, P, C.c_int]
            lib.orc_face_samples.restype = i64
            lib.orc_face_samples.argtypes = [P, i64, C.c_double, P, i64]
            lib.orc_winding_number.restype = C.c_double
            lib.orc_winding_number.argtypes = [P, P]
            lib.orc_classify.restype = C.c_int
            lib.orc_classify.argtypes = [P, P, C.c_int, P, i64, P, P]
            lib.orc_propagate.restype = C.c_int
            lib.orc_propagate.argtypes = [C.c_int, P, i64, P, C.c_int]
            lib.orc_point_face_dist.restype = C.c_double
            lib.orc_point_face_dist.argtypes = [C.c_int, P]
            lib.orc_children.restype = i64
            lib.orc_children.argtypes = [C.c_int, P, i64, P, P, P]
            lib.orc_cell_faces.restype = i64
            lib.orc_cell_faces.argtypes = [P, P, C.c_int, C.c_double, C.c_double, C.c_int, C.c_int, P, i64, P, P, P,
                                           i64]
            lib.orc_cell_links.restype = C.c_int
            lib.orc_cell_links.argtypes = [P, P, C.c_int, C.c_int, P, i64, P, P, P]
            lib.orc_lattice_dir.restype = C.c_int
            lib.orc_lattice_dir.argtypes = [C.c_int, C.c_int, P]
            lib.orc_link_q.restype = C.c_double
            lib.orc_link_q.argtypes = [P, P, C.c_int, C.c_int, P, C.c_int, i64, P]
            lib.orc_q_grad.restype = C.c_int
            lib.orc_q_grad.argtypes = [P, P, C.c_int, C.c_int, P, P, P, P, i64, P]
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class _CDomain(C.Structure):
    _fields_ = [("dim", C.c_int), ("root", C.c_int * 3), ("origin", C.c_double * 3), ("h0", C.c_double)]


@dataclass
class Domain:
    """Root grid: ``root`` blocks of 4^D cells per axis from ``origin`` with level-0 cell size ``h0``."""
    dim: int
    root: tuple
    origin: tuple = (0.0, 0.0, 0.0)
    h0: float = 0.0

    @staticmethod
    def unit(dim: int, root: int) -> "Domain":
        return Domain(dim, (root,) * dim, (0.0, 0.0, 0.0), 1.0 / (4.0 * root))

    def c(self) -> _CDomain:
        d = _CDomain()
        d.dim = self.dim
        r = list(self.root) + [1] * (3 - len(self.root))
        for a in range(3):
            d.root[a] = int(r[a])
            d.origin[a] = float(self.origin[a]) if a < len(self.origin) else 0.0
        d.h0 = float(self.h0)
        return d

    def h(self, level: int) -> float:
        return self.h0 * 2.0 ** (-level)


def lattice_dirs(lattice: int) -> np.ndarray:
    lib = _load()
    q = 9 if lattice == 9 else 19
    out = np.zeros((q, 3), np.int32)
    for i in range(q):
        c = np.zeros(3, np.int32)
        if lib.orc_lattice_dir(lattice, i, _p(c)):
            raise ValueError("bad lattice")
        out[i] = c
    return out


class OracleGeometry:
    """One imported geometry plus its bins (Sec. "Representation of the Complex Boundary Geometry")."""

    def __init__(self, dim: int, verts: np.ndarray, idx: np.ndarray | None = None):
        lib = _load()
        self.dim = dim
        v = np.ascontiguousarray(verts, dtype=np.float32)
        err = C.create_string_buffer(256)
        if idx is None:
            nf = v.shape[0]
            self._h = lib.orc_geom_new(dim, _p(v), 0, None, nf, err, 256)
        else:
            ix = np.ascontiguousarray(idx, dtype=np.int32)
            self._h = lib.orc_geom_new(dim, _p(v), v.shape[0], _p(ix), ix.shape[0], err, 256)
        if not self._h:
            raise ValueError(err.value.decode())
        self.n_faces = int(lib.orc_geom_nfaces(self._h))
        self.dom = None
        self.B = 0

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_geom_free(h)
            self._h = None

    # -- step 2 ----------------------------------------------------------
    def bin(self, dom: Domain, B: int, sampled: bool = False):
        """Step 2: exact AABB binning, or (sampled=True) the paper's sampled-point binning."""
        lib = _load()
        self._cdom = dom.c()
        build = lib.orc_bins_build_sampled if sampled else lib.orc_bins_build
        if build(self._h, C.byref(self._cdom), int(B)):
            raise ValueError("binning failed")
        self.dom, self.B = dom, int(B)
        nb = B ** self.dim
        nnz = int(lib.orc_bins_nnz(self._h))
        off = np.zeros(nb + 1, np.uint32)
        ids = np.zeros(max(nnz, 1), np.uint32)
        lib.orc_bins_copy(self._h, _p(off), _p(ids))
        return off, ids[:nnz]

    def face_bin_range(self, f: int):
        lo = np.zeros(3, np.int32)
        hi = np.zeros(3, np.int32)
        _load().orc_face_bin_range(self._h, int(f), _p(lo), _p(hi))
        return lo[:self.dim], hi[:self.dim]

    # -- step 3 ----------------------------------------------------------
    def refine_blocks(self, level: int, blocks: np.ndarray, d_abs=0.0, d_rel=1.0, count_candidates=False, pred=0,
                      search=0):
        b = np.ascontiguousarray(blocks, dtype=np.int32).reshape(-1, self.dim)
        n = b.shape[0]
        mask = np.zeros(max(n, 1), np.uint64)
        band = np.zeros(max(n, 1), np.uint64)
        nbp = C.c_int64(0)
        ncand = C.c_int64(0)
        rc = _load().orc_refine_blocks(self._h, C.byref(self._cdom), level, d_abs, d_rel, int(pred), int(search),
                                       _p(b), n,
                                       _p(mask),
                                       _p(band), C.byref(nbp), C.byref(ncand) if count_candidates else None)
        if rc:
            raise ValueError("orc_refine_blocks failed")
        return mask[:n], band[:n], int(nbp.value), int(ncand.value)

    def winding_number(self, x) -> float:
        """Generalized winding number of the mesh at point x."""
        p = np.zeros(3, np.float64)
        xs = np.asarray(x, dtype=np.float64).reshape(-1)
        p[:xs.size] = xs
        return float(_load().orc_winding_number(self._h, _p(p)))

    def classify(self, level: int, cells: np.ndarray, dom: "Domain" = None):
        """Per cell centre: solid (inside the closed mesh) and band (within 1e-6 h of the mesh)."""
        lib = _load()
        cd = dom.c() if dom is not None else self._cdom
        c = np.ascontiguousarray(cells, dtype=np.int32).reshape(-1, self.dim)
        n = c.shape[0]
        solid = np.zeros(max(n, 1), np.uint8)
        band = np.zeros(max(n, 1), np.uint8)
        lib.orc_classify(self._h, C.byref(cd), level, _p(c), n, _p(solid), _p(band))
        return solid[:n].astype(bool), band[:n].astype(bool)

    def face_samples(self, f: int, spacing: float) -> np.ndarray:
        """The sample points of face f of the paper's sampled binning, [k][dim]."""
        lib = _load()
        k = int(lib.orc_face_samples(self._h, int(f), float(spacing), None, 0))
        pts = np.zeros((max(k, 1), self.dim), np.float64)
        lib.orc_face_samples(self._h, int(f), float(spacing), _p(pts), k)
        return pts[:k]

    def children(self, blocks: np.ndarray, mask: np.ndarray):
        lib = _load()
        b = np.ascontiguousarray(blocks, dtype=np.int32).reshape(-1, self.dim)
        m = np.ascontiguousarray(mask, dtype=np.uint64)
        k = int(lib.orc_children(self.dim, _p(b), b.shape[0], _p(m), None, None))
        cb = np.zeros((max(k, 1), self.dim), np.int32)
        cp = np.zeros(max(k, 1), np.int32)
        lib.orc_children(self.dim, _p(b), b.shape[0], _p(m), _p(cb), _p(cp))
        return cb[:k], cp[:k]

    def cell_faces(self, level: int, cells: np.ndarray, d_abs=0.0, d_rel=1.0, pred=0, search=0):
        """Per cell: ascending adjacent face ids; band flags mark pairs inside the margin band."""
        lib = _load()
        c = np.ascontiguousarray(cells, dtype=np.int32).reshape(-1, self.dim)
        n = c.shape[0]
        counts = np.zeros(max(n, 1), np.int64)
        tot = int(lib.orc_cell_faces(self._h, C.byref(self._cdom), level, d_abs, d_rel, int(pred), int(search),
                                     _p(c), n,
                                     _p(counts),
                                     None, None, 0))
        ids = np.zeros(max(tot, 1), np.uint32)
        band = np.zeros(max(tot, 1), np.uint8)
        lib.orc_cell_faces(self._h, C.byref(self._cdom), level, d_abs, d_rel, int(pred), int(search), _p(c), n,
                           _p(counts),
                           _p(ids),
                           _p(band), tot)
        off = np.zeros(n + 1, np.int64)
        off[1:] = np.cumsum(counts[:n])
        return off, ids[:tot], band[:tot].astype(bool)

    def cell_links(self, level: int, lattice: int, cells: np.ndarray):
        lib = _load()
        c = np.ascontiguousarray(cells, dtype=np.int32).reshape(-1, self.dim)
        n = c.shape[0]
        Q = 9 if lattice == 9 else 19
        q = np.zeros((max(n, 1), Q - 1), np.float64)
        face = np.zeros((max(n, 1), Q - 1), np.int64)
        band = np.zeros((max(n, 1), Q - 1), np.uint8)
        if lib.orc_cell_links(self._h, C.byref(self._cdom), level, lattice, _p(c), n, _p(q), _p(face), _p(band)):
            raise ValueError("orc_cell_links failed")
        return q[:n], face[:n], band[:n].astype(bool)

    def link_q(self, level, lattice, cell, direction, face, verts_override=None):
        c = np.ascontiguousarray(cell, dtype=np.int32)
        ov = None if verts_override is None else np.ascontiguousarray(verts_override, dtype=np.float64)
        return float(_load().orc_link_q(self._h, C.byref(self._cdom), level, lattice, _p(c), int(direction),
                                        int(face), _p(ov)))

    def q_grad(self, level, lattice, cells, dirs, faces, grad_q):
        """d(sum grad_q * q)/d(face vertices) as [n_faces, D, D] (FP64)."""
        c = np.ascontiguousarray(cells, dtype=np.int32).reshape(-1, self.dim)
        d = np.ascontiguousarray(dirs, dtype=np.int32)
        f = np.ascontiguousarray(faces, dtype=np.int64)
        g = np.ascontiguousarray(grad_q, dtype=np.float64)
        out = np.zeros((self.n_faces, self.dim, self.dim), np.float64)
        rc = _load().orc_q_grad(self._h, C.byref(self._cdom), level, 9 if self.dim == 2 else 19, _p(c), _p(d),
                                _p(f), _p(g), c.shape[0], _p(out))
        if rc:
            raise ValueError("orc_q_grad failed")
        return out


def propagate(dim: int, blocks: np.ndarray, flags: np.ndarray, rounds: int) -> np.ndarray:
    """The paper's refinement-mark propagation over one level's block list; returns new flags (0/1)."""
    b = np.ascontiguousarray(blocks, dtype=np.int32).reshape(-1, dim)
    f = np.ascontiguousarray((np.asarray(flags) != 0).astype(np.uint8))
    _load().orc_propagate(dim, _p(b), b.shape[0], _p(f), int(rounds))
    return f


def propagation_rounds(d_spec: float, block_len: float) -> int:
    """N_prop = 1 + floor(d_spec / block length)."""
    return 1 + int(np.floor(d_spec / block_len))


def point_face_dist(dim: int, verts_local: np.ndarray) -> float:
    """Distance from the origin to the closed face (vertices relative to the point), Alg. 1's predicate."""
    v = np.ascontiguousarray(verts_local, dtype=np.float64).reshape(dim, dim)
    return float(_load().orc_point_face_dist(dim, _p(v)))


def sat_margin(dim: int, verts_local: np.ndarray, r: float) -> float:
    v = np.ascontiguousarray(verts_local, dtype=np.float64)
    return float(_load().orc_sat_margin(dim, _p(v), float(r)))


def root_blocks(dim: int, root) -> np.ndarray:
    """Level-0 blocks in x-fastest lexicographic order."""
    r = list(root) if hasattr(root, "__len__") else [root] * dim
    g = np.meshgrid(*[np.arange(r[a]) for a in range(dim)][::-1], indexing="ij")
    cols = [x.reshape(-1) for x in g][::-1]
    return np.stack(cols, axis=1).astype(np.int32)


def cells_of_mask(dim: int, blocks: np.ndarray, mask: np.ndarray):
    """Adjacent cells as (block index, cell bit) in canonical order, plus their global cell coords."""
    ncell = 64 if dim == 3 else 16
    bits = ((mask[:, None] >> np.arange(ncell, dtype=np.uint64)[None, :]) & np.uint64(1)).astype(bool)
    bi, ci = np.nonzero(bits)
    local = np.stack([ci & 3, (ci >> 2) & 3] + ([(ci >> 4) & 3] if dim == 3 else []), axis=1)
    cells = 4 * blocks[bi] + local
    return bi.astype(np.int64), ci.astype(np.int64), cells.astype(np.int32)


def run_pipeline(dim, verts, idx, *, root, n_levels, B, lattice, d_abs=0.0, d_rel=1.0, links=True,
                 max_level_blocks=None, pred=0, sampled=False, search=0, propagate_rounds=0):
    """Whole oracle pass: bins, every level's blocks/masks/band masks, finest-level adjacency and links."""
    geo = OracleGeometry(dim, verts, idx)
    dom = Domain.unit(dim, root)
    off, ids = geo.bin(dom, B, sampled=sampled)
    blocks = root_blocks(dim, (root,) * dim)
    levels = []
    for L in range(n_levels):
        if max_level_blocks is not None and blocks.shape[0] > max_level_blocks:
            raise ValueError("level too large for the oracle")
        mask, band, nbp, _ = geo.refine_blocks(L, blocks, d_abs, d_rel, pred=pred, search=search)
        flag = (mask != 0).astype(np.uint8)
        if propagate_rounds and L + 1 < n_levels:
            flag = propagate(dim, blocks, flag, propagate_rounds)
        lv = {"blocks": blocks, "mask": mask, "band": band, "n_band_pairs": nbp, "flag": flag}
        levels.append(lv)
        if L + 1 < n_levels:
            cb, cp = geo.children(blocks, flag.astype(np.uint64))
            lv["child_parent"] = cp
            blocks = cb
    out = {"geo": geo, "dom": dom, "offsets": off, "ids": ids, "levels": levels}
    fin = levels[-1]
    bi, ci, cells = cells_of_mask(dim, fin["blocks"], fin["mask"])
    out["adj_block"], out["adj_bit"], out["adj_cells"] = bi, ci, cells
    L = n_levels - 1
    out["adj_off"], out["adj_ids"], out["adj_band"] = geo.cell_faces(L, cells, d_abs, d_rel, pred=pred, search=search)
    if links:
        out["q"], out["q_face"], out["q_band"] = geo.cell_links(L, lattice, cells)
    return out
