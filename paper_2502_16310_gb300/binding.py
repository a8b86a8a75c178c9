"""ctypes binding of ``libamrgeom.so`` (C ABI in ``include/amrgeom.h``).

Argument marshalling only: every step of the refinement runs in the library's
CUDA kernels.  The functions keep the C names (``amr_create``,
``amr_geom_load``, ``amr_bin_faces``, ``amr_refine_near_wall`` ...).
``AmrGeom`` wraps one context for PyTorch users: inputs may be torch tensors
(CPU or CUDA) or numpy arrays, and outputs come back as zero-copy CUDA tensors
that borrow the context's buffers (``.clone()`` them to keep them past the next
call).  There is no CPU fallback: without the built library and a CUDA device
the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libamrgeom.so")
MAX_LEVELS = 16

_lib = None
_lock = threading.Lock()

AMR_OK, AMR_EINVAL, AMR_ENOMEM, AMR_ECUDA, AMR_EOVERFLOW, AMR_ETIMEOUT, AMR_ESTATE, AMR_EDEVICE_CHECK = range(8)
STATUS_NAMES = {0: "AMR_OK", 1: "AMR_EINVAL", 2: "AMR_ENOMEM", 3: "AMR_ECUDA", 4: "AMR_EOVERFLOW",
                5: "AMR_ETIMEOUT", 6: "AMR_ESTATE", 7: "AMR_EDEVICE_CHECK"}

EXPORTED = ["amr_create", "amr_destroy", "amr_status_str", "amr_last_error", "amr_set_stream", "amr_geom_load",
            "amr_bin_faces", "amr_bin_faces_sampled", "amr_refine_near_wall", "amr_sync", "amr_timing_enable",
            "amr_timing_reset", "amr_timing_get", "amr_launch_count", "amr_bin_faces_static", "amr_q_backward",
            "amr_classify_nodes", "amr_fluid_links", "amr_adapt_diff_get", "amr_candidate_count", "amr_autotune",
            "amr_batch_create", "amr_batch_destroy", "amr_batch_add", "amr_batch_set_bins", "amr_batch_run",
            "amr_batch_get_view", "amr_batch_q_backward", "amr_batch_last_error", "amr_batch_launch_count"]


class AmrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


DEV_ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
DEV_FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class amr_domain(C.Structure):
    _fields_ = [("dim", C.c_int), ("root_blocks", C.c_int * 3), ("origin", C.c_double * 3), ("h0", C.c_double),
                ("stream", C.c_void_p), ("dev_alloc", DEV_ALLOC), ("dev_free", DEV_FREE), ("user", C.c_void_p)]


class amr_bins_view(C.Structure):
    _fields_ = [("B", C.c_int), ("n_bins", C.c_int64), ("nnz", C.c_int64), ("offsets", C.c_void_p),
                ("ids", C.c_void_p), ("payload", C.c_void_p), ("payload_bytes", C.c_int64)]


class amr_refine_params(C.Structure):
    _fields_ = [("n_levels", C.c_int), ("d_abs", C.c_double), ("d_rel", C.c_double), ("lattice", C.c_int),
                ("want_adjacency", C.c_int), ("want_links", C.c_int), ("use_graph", C.c_int),
                ("warps_per_cta", C.c_int), ("predicate", C.c_int), ("search", C.c_int), ("propagate", C.c_int),
                ("keep_previous", C.c_int), ("face_pass", C.c_int)]


class amr_adapt_diff(C.Structure):
    _fields_ = [("n_levels", C.c_int), ("n_new", C.c_int64 * MAX_LEVELS), ("n_old", C.c_int64 * MAX_LEVELS),
                ("n_created", C.c_int64 * MAX_LEVELS), ("n_removed", C.c_int64 * MAX_LEVELS),
                ("new_to_old", C.c_void_p * MAX_LEVELS), ("old_to_new", C.c_void_p * MAX_LEVELS)]


AMR_PRED_BOX, AMR_PRED_POINT = 0, 1
AMR_SEARCH_QUERY_BOX, AMR_SEARCH_OWN_BIN = 0, 1
AMR_FACE_PASS_AUTO, AMR_FACE_PASS_OFF, AMR_FACE_PASS_ON = 0, 1, 2


class amr_refine_result(C.Structure):
    _fields_ = [("n_levels", C.c_int), ("n_blocks", C.c_int64 * MAX_LEVELS),
                ("block_coords", C.c_void_p * MAX_LEVELS), ("block_parent", C.c_void_p * MAX_LEVELS),
                ("cell_mask", C.c_void_p * MAX_LEVELS), ("block_flag", C.c_void_p * MAX_LEVELS),
                ("n_adj_cells", C.c_int64), ("n_adj_pairs", C.c_int64), ("adj_cell", C.c_void_p),
                ("adj_off", C.c_void_p), ("adj_ids", C.c_void_p), ("n_links", C.c_int64),
                ("link_cell", C.c_void_p), ("link_dir", C.c_void_p), ("link_q", C.c_void_p),
                ("link_face", C.c_void_p), ("n_fallback", C.c_int64), ("n_band", C.c_int64),
                ("n_candidates", C.c_int64), ("n_survivors", C.c_int64), ("n_link_candidates", C.c_int64),
                ("n_face_setups", C.c_int64), ("n_face_tests", C.c_int64), ("graph_replay", C.c_int)]


class amr_batch_view(C.Structure):
    _fields_ = [("r", amr_refine_result), ("level_base", C.c_int64 * MAX_LEVELS), ("adj_base", C.c_int64),
                ("pair_base", C.c_int64), ("link_base", C.c_int64), ("face_base", C.c_int64),
                ("vert_base", C.c_int64)]


def lib(build_if_missing: bool = True):
    """Load (building first when missing or stale and nvcc is available) the CUDA library."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        from . import build as _build

        if build_if_missing:
            try:
                _build.build()
            except Exception as e:  # no nvcc or a compile error: only an existing library may be used
                if not os.path.exists(LIB_PATH):
                    raise ImportError(f"libamrgeom.so is not built and cannot be built here: {e}") from e
        if not os.path.exists(LIB_PATH):
            raise ImportError("libamrgeom.so is not built; run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        P, i64 = C.c_void_p, C.c_int64
        L.amr_create.restype = C.c_int
        L.amr_create.argtypes = [C.POINTER(amr_domain), C.POINTER(P)]
        L.amr_destroy.restype = C.c_int
        L.amr_destroy.argtypes = [P]
        L.amr_status_str.restype = C.c_char_p
        L.amr_status_str.argtypes = [C.c_int]
        L.amr_last_error.restype = C.c_char_p
        L.amr_last_error.argtypes = [P]
        L.amr_set_stream.restype = C.c_int
        L.amr_set_stream.argtypes = [P, P]
        L.amr_geom_load.restype = C.c_int
        L.amr_geom_load.argtypes = [P, P, i64, P, i64]
        L.amr_bin_faces.restype = C.c_int
        L.amr_bin_faces.argtypes = [P, C.c_int, C.POINTER(amr_bins_view)]
        L.amr_bin_faces_sampled.restype = C.c_int
        L.amr_bin_faces_sampled.argtypes = [P, C.c_int, C.POINTER(amr_bins_view)]
        L.amr_refine_near_wall.restype = C.c_int
        L.amr_refine_near_wall.argtypes = [P, C.POINTER(amr_refine_params), C.POINTER(amr_refine_result)]
        L.amr_sync.restype = C.c_int
        L.amr_sync.argtypes = [P]
        L.amr_timing_enable.restype = C.c_int
        L.amr_timing_enable.argtypes = [P, C.c_int]
        L.amr_timing_reset.restype = C.c_int
        L.amr_timing_reset.argtypes = [P]
        L.amr_timing_get.restype = C.c_int
        L.amr_timing_get.argtypes = [P, C.POINTER(C.c_char_p), C.POINTER(C.c_double), C.POINTER(i64), C.c_int]
        L.amr_launch_count.restype = C.c_int64
        L.amr_launch_count.argtypes = [P]
        L.amr_q_backward.restype = C.c_int
        L.amr_q_backward.argtypes = [P, P, P]
        L.amr_classify_nodes.restype = C.c_int
        L.amr_classify_nodes.argtypes = [P, C.POINTER(C.c_void_p), C.POINTER(C.c_int64)]
        L.amr_fluid_links.restype = C.c_int
        L.amr_fluid_links.argtypes = [P, C.POINTER(amr_refine_result)]
        L.amr_adapt_diff_get.restype = C.c_int
        L.amr_adapt_diff_get.argtypes = [P, C.POINTER(amr_adapt_diff)]
        L.amr_candidate_count.restype = C.c_int
        L.amr_candidate_count.argtypes = [P, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        L.amr_autotune.restype = C.c_int
        L.amr_autotune.argtypes = [P, C.POINTER(amr_refine_params), P, C.c_int, P, C.c_int, C.POINTER(C.c_int),
                                   C.POINTER(C.c_int), C.POINTER(C.c_double)]
        L.amr_batch_create.restype = C.c_int
        L.amr_batch_create.argtypes = [C.c_int, P, C.POINTER(P)]
        L.amr_batch_destroy.restype = C.c_int
        L.amr_batch_destroy.argtypes = [P]
        L.amr_batch_add.restype = C.c_int
        L.amr_batch_add.argtypes = [P, C.POINTER(amr_domain), P, i64, P, i64, C.c_int, C.c_double, C.c_double,
                                    C.c_int, C.POINTER(C.c_int)]
        L.amr_batch_set_bins.restype = C.c_int
        L.amr_batch_set_bins.argtypes = [P, C.c_int, C.c_int]
        L.amr_batch_run.restype = C.c_int
        L.amr_batch_run.argtypes = [P, C.POINTER(amr_refine_params), C.POINTER(amr_refine_result)]
        L.amr_batch_get_view.restype = C.c_int
        L.amr_batch_get_view.argtypes = [P, C.c_int, C.POINTER(amr_batch_view)]
        L.amr_batch_q_backward.restype = C.c_int
        L.amr_batch_q_backward.argtypes = [P, P, P]
        L.amr_batch_last_error.restype = C.c_char_p
        L.amr_batch_last_error.argtypes = [P]
        L.amr_batch_launch_count.restype = C.c_int64
        L.amr_batch_launch_count.argtypes = [P]
        L.amr_bin_faces_static.restype = C.c_int
        L.amr_bin_faces_static.argtypes = [C.POINTER(amr_domain), P, i64, C.c_int, P, P, i64, C.POINTER(i64)]
        _lib = L
        return L


def _check(ctx, st: int):
    if st != AMR_OK:
        L = lib()
        msg = L.amr_last_error(ctx).decode() if ctx else L.amr_status_str(st).decode()
        raise AmrError(st, msg)


# -- C-named entry points ------------------------------------------------------

def amr_create(dim: int, root_blocks, origin=(0.0, 0.0, 0.0), h0: float | None = None, stream: int | None = None,
               dev_alloc=None, dev_free=None, user=None):
    """dev_alloc / dev_free: optional DEV_ALLOC / DEV_FREE callbacks (both or neither) that every device buffer
    of the context is taken from and returned to; the caller keeps them alive until amr_destroy."""
    L = lib()
    d = amr_domain()
    if dev_alloc is not None:
        d.dev_alloc = dev_alloc
    if dev_free is not None:
        d.dev_free = dev_free
    d.user = user
    d.dim = dim
    rb = list(root_blocks) + [1] * (3 - len(root_blocks))
    for a in range(3):
        d.root_blocks[a] = int(rb[a])
        d.origin[a] = float(origin[a]) if a < len(origin) else 0.0
    d.h0 = float(h0 if h0 is not None else 1.0 / (4.0 * rb[0]))
    d.stream = stream
    h = C.c_void_p()
    st = L.amr_create(C.byref(d), C.byref(h))
    if st != AMR_OK:
        raise AmrError(st, L.amr_status_str(st).decode())
    return h


def amr_destroy(ctx):
    _check(None, lib().amr_destroy(ctx))


def amr_set_stream(ctx, stream: int | None):
    _check(ctx, lib().amr_set_stream(ctx, stream))


def amr_geom_load(ctx, coords_ptr: int, n_verts: int, idx_ptr: int | None, n_faces: int):
    _check(ctx, lib().amr_geom_load(ctx, coords_ptr, int(n_verts), idx_ptr, int(n_faces)))


def amr_bin_faces(ctx, bin_density: int) -> amr_bins_view:
    v = amr_bins_view()
    _check(ctx, lib().amr_bin_faces(ctx, int(bin_density), C.byref(v)))
    return v


def amr_bin_faces_sampled(ctx, bin_density: int) -> amr_bins_view:
    v = amr_bins_view()
    _check(ctx, lib().amr_bin_faces_sampled(ctx, int(bin_density), C.byref(v)))
    return v


def amr_refine_near_wall(ctx, n_levels: int, d_abs=0.0, d_rel=1.0, lattice=0, want_adjacency=True,
                         want_links=True, use_graph=False, warps_per_cta=0, predicate=AMR_PRED_BOX,
                         search=AMR_SEARCH_QUERY_BOX, propagate=0, keep_previous=False,
                         face_pass=AMR_FACE_PASS_AUTO) -> amr_refine_result:
    p = _params(n_levels, d_abs, d_rel, lattice, want_adjacency, want_links, use_graph, warps_per_cta, predicate,
                search, propagate, keep_previous, face_pass)
    r = amr_refine_result()
    _check(ctx, lib().amr_refine_near_wall(ctx, C.byref(p), C.byref(r)))
    return r


def amr_q_backward(ctx, grad_q_ptr: int, grad_out_ptr: int):
    _check(ctx, lib().amr_q_backward(ctx, grad_q_ptr, grad_out_ptr))


def amr_sync(ctx):
    _check(ctx, lib().amr_sync(ctx))


def _params(n_levels=1, d_abs=0.0, d_rel=1.0, lattice=0, want_adjacency=True, want_links=True, use_graph=False,
            warps_per_cta=0, predicate=AMR_PRED_BOX, search=AMR_SEARCH_QUERY_BOX, propagate=0, keep_previous=False,
            face_pass=0):
    p = amr_refine_params()
    p.n_levels, p.d_abs, p.d_rel, p.lattice = int(n_levels), float(d_abs), float(d_rel), int(lattice)
    p.want_adjacency, p.want_links = int(bool(want_adjacency)), int(bool(want_links))
    p.use_graph, p.warps_per_cta = int(bool(use_graph)), int(warps_per_cta)
    p.predicate, p.search, p.propagate = int(predicate), int(search), int(propagate)
    p.keep_previous = int(bool(keep_previous))
    p.face_pass = int(face_pass)
    return p


def amr_autotune(ctx, n_levels, d_abs=0.0, d_rel=1.0, lattice=0, want_adjacency=True, want_links=True,
                 b_candidates=None, w_candidates=None):
    """(best bin density, best warps per block, best ms) on the loaded geometry."""
    p = _params(n_levels, d_abs, d_rel, lattice, want_adjacency, want_links)
    bc = (C.c_int * len(b_candidates))(*b_candidates) if b_candidates else None
    wc = (C.c_int * len(w_candidates))(*w_candidates) if w_candidates else None
    bb, bw, bt = C.c_int(0), C.c_int(0), C.c_double(0)
    _check(ctx, lib().amr_autotune(ctx, C.byref(p), bc, len(b_candidates or []), wc, len(w_candidates or []),
                                   C.byref(bb), C.byref(bw), C.byref(bt)))
    return int(bb.value), int(bw.value), float(bt.value)


def _bcheck(b, st):
    if st != AMR_OK:
        raise AmrError(st, lib().amr_batch_last_error(b).decode())


def amr_timing_enable(ctx, on: bool):
    _check(ctx, lib().amr_timing_enable(ctx, int(bool(on))))


def amr_timing_reset(ctx):
    _check(ctx, lib().amr_timing_reset(ctx))


def amr_timing_get(ctx) -> dict:
    L = lib()
    n = L.amr_timing_get(ctx, None, None, None, 0)
    names = (C.c_char_p * max(n, 1))()
    ms = (C.c_double * max(n, 1))()
    cnt = (C.c_int64 * max(n, 1))()
    n = L.amr_timing_get(ctx, names, ms, cnt, n)
    return {names[i].decode(): (float(ms[i]), int(cnt[i])) for i in range(n)}


def amr_launch_count(ctx) -> int:
    return int(lib().amr_launch_count(ctx))


STATIC_MAX_BINS = 1 << 18
STATIC_MAX_FACES = 1 << 17


def amr_bin_faces_static(dim, root_blocks, faces_soa_ptr: int, n_faces: int, bin_density: int, offsets_ptr: int,
                         ids_ptr: int, ids_capacity: int, origin=(0.0, 0.0, 0.0), h0=None, stream=None):
    """Allocation-free binning (device SoA faces in, caller-owned device offsets/ids out); returns nnz.

    Raises AmrError with the C status (EINVAL beyond the static maxima, EOVERFLOW when nnz > ids_capacity).
    """
    d = amr_domain()
    d.dim = dim
    rb = list(root_blocks) + [1] * (3 - len(root_blocks))
    for a in range(3):
        d.root_blocks[a] = int(rb[a])
        d.origin[a] = float(origin[a]) if a < len(origin) else 0.0
    d.h0 = float(h0 if h0 is not None else 1.0 / (4.0 * rb[0]))
    d.stream = stream
    nnz = C.c_int64(0)
    st = lib().amr_bin_faces_static(C.byref(d), faces_soa_ptr, int(n_faces), int(bin_density), offsets_ptr, ids_ptr,
                                    int(ids_capacity), C.byref(nnz))
    if st != AMR_OK:
        raise AmrError(st, lib().amr_status_str(st).decode() + f" (nnz={nnz.value})")
    return int(nnz.value)


# -- torch convenience layer ----------------------------------------------------

class _DevArray:
    """Minimal __cuda_array_interface__ holder for a borrowed device pointer."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(int(s) for s in shape), "typestr": typestr,
                                         "data": (int(ptr or 0), False), "version": 3, "strides": None}


class _Deferred:
    """A value built on first access (see _LazyDict)."""

    __slots__ = ("make",)

    def __init__(self, make):
        self.make = make


class _LazyDict(dict):
    """dict whose _Deferred entries are built on first access: the result views of a refinement
    cost nothing until they are read (a step that only needs the device state skips them)."""

    def __getitem__(self, k):
        v = dict.__getitem__(self, k)
        if isinstance(v, _Deferred):
            v = v.make()
            dict.__setitem__(self, k, v)
        return v

    def get(self, k, default=None):
        return self[k] if k in self else default

    def values(self):
        return [self[k] for k in self]

    def items(self):
        return [(k, self[k]) for k in self]

    def __iter__(self):
        # defined here so that dict(d) and {**d} go through keys() and __getitem__ (CPython copies a
        # dict subclass's raw entries when it keeps dict's own iterator)
        return dict.__iter__(self)

    def copy(self):
        return {k: self[k] for k in self}


def _view(ptr, shape, dtype):
    import torch

    n = int(np.prod(shape)) if len(shape) else 1
    if n == 0 or not ptr:
        return torch.empty(tuple(shape), dtype=dtype, device="cuda")
    typestr = {torch.float32: "<f4", torch.int32: "<i4", torch.int64: "<i8", torch.uint8: "|u1"}[dtype]
    t = torch.as_tensor(_DevArray(ptr, shape, typestr), device="cuda")
    return t


def _u32(ptr, n):
    # torch has limited uint32 support: expose as int32 bits, then widen to int64 for convenience
    import torch

    return _view(ptr, (n,), torch.int32)


class AmrGeom:
    """One refinement context: ``load`` -> ``bin`` -> ``refine`` on the current CUDA device.

    The context's work is ordered on the current torch CUDA stream at creation.
    """

    def __init__(self, dim: int, root_blocks, origin=(0.0, 0.0, 0.0), h0: float | None = None, dev_alloc=None,
                 dev_free=None):
        """dev_alloc / dev_free: optional DEV_ALLOC / DEV_FREE callbacks (both or neither) from which the
        context takes every device buffer (kept alive with the context)."""
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("AmrGeom needs a CUDA device")
        self.dim = dim
        self.root = tuple(int(r) for r in (root_blocks if hasattr(root_blocks, "__len__") else [root_blocks] * dim))
        self.stream = torch.cuda.current_stream()
        # torch's default stream has handle 0; pass the legacy default stream (handle 1) so the
        # context's work stays ordered with torch's own kernels and copies
        handle = self.stream.cuda_stream or 1
        self._hooks = (dev_alloc, dev_free)
        self.ctx = amr_create(dim, self.root, origin, h0, handle, dev_alloc=dev_alloc, dev_free=dev_free)
        self._keep = []
        self.bins = None
        self.last_result = None
        self.result = None

    def close(self):
        if getattr(self, "ctx", None):
            amr_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, verts, idx=None):
        """Step 1: faces from vertices + index list (idx) or a face-vertex list (idx None)."""
        import torch

        v = torch.as_tensor(verts, dtype=torch.float32)
        if not v.is_contiguous():
            v = v.contiguous()
        self._keep = [v]
        self.load_shape = tuple(v.shape)
        if idx is None:
            nf = v.shape[0]
            amr_geom_load(self.ctx, v.data_ptr(), 0, None, nf)
        else:
            ix = torch.as_tensor(idx, dtype=torch.int32)
            if not ix.is_contiguous():
                ix = ix.contiguous()
            self._keep.append(ix)
            amr_geom_load(self.ctx, v.data_ptr(), v.shape[0], ix.data_ptr(), ix.shape[0])
        return self

    def bin(self, B: int, sampled: bool = False):
        """Step 2: CSR bins; returns dict(offsets, ids) as borrowed int32 CUDA tensors (uint32 bits).
        sampled: the paper's sampled-point membership instead of the exact AABB overlap."""
        import torch

        v = amr_bin_faces_sampled(self.ctx, B) if sampled else amr_bin_faces(self.ctx, B)
        off, ids, nb, nnz = v.offsets, v.ids, int(v.n_bins), int(v.nnz)
        pay, pw = v.payload, int(v.payload_bytes) // 4
        # payload: [nnz, 16] (3D) or [nnz, 8] (2D) 32-bit words per entry (coordinates and normal as
        # float bits, then id with flags, then bin coordinates)
        self.bins = _LazyDict(B=v.B, n_bins=nb, nnz=nnz,
                              offsets=_Deferred(lambda: _view(off, (nb + 1,), torch.int32)),
                              ids=_Deferred(lambda: _view(ids, (nnz,), torch.int32)),
                              payload=_Deferred(lambda: _view(pay, (nnz, pw), torch.int32)))
        return self.bins

    def refine(self, n_levels: int, d_abs=0.0, d_rel=1.0, lattice=0, want_adjacency=True, want_links=None,
               use_graph=False, warps_per_cta=0, predicate=AMR_PRED_BOX, search=AMR_SEARCH_QUERY_BOX, propagate=0,
               keep_previous=False, face_pass=0):
        """Step 3: near-wall refinement; returns per-level tensors, adjacency CSR and links (borrowed).
        predicate: AMR_PRED_BOX (inflated cell box meets the face) or AMR_PRED_POINT (cell centre within
        d of the face, the paper's Alg. 1); search / propagate: the paper's binned search (own bin only)
        and its mark propagation (-1: 1 + floor(d / block length) rounds); face_pass: AMR_FACE_PASS_AUTO /
        _OFF / _ON, how mask-only levels are marked (identical results)."""
        if want_links is None:
            want_links = lattice != 0
        r = amr_refine_near_wall(self.ctx, n_levels, d_abs, d_rel, lattice, want_adjacency, want_links, use_graph,
                                 warps_per_cta, predicate, search, propagate, keep_previous, face_pass)
        self.last_result = r
        return self._wrap(r, want_adjacency, want_links)

    def _wrap(self, r, want_adjacency, want_links):
        import torch

        D = self.dim

        def lazy(ptr, shape, dtype):
            return _Deferred(lambda: _view(ptr, shape, dtype))

        levels = []
        for L in range(r.n_levels):
            n = int(r.n_blocks[L])
            levels.append(_LazyDict(
                blocks=lazy(r.block_coords[L], (n, D), torch.int32),
                parent=lazy(r.block_parent[L], (n,), torch.int32) if L > 0 else None,
                mask=lazy(r.cell_mask[L], (n,), torch.int64),
                flag=lazy(r.block_flag[L], (n,), torch.uint8),
            ))
        out = _LazyDict(levels=levels, n_fallback=int(r.n_fallback), n_band=int(r.n_band),
                        n_candidates=int(r.n_candidates), n_survivors=int(r.n_survivors),
                        n_link_candidates=int(r.n_link_candidates), n_face_setups=int(r.n_face_setups),
                        n_face_tests=int(r.n_face_tests), graph_replay=bool(r.graph_replay))
        if want_adjacency or want_links:
            na, npairs = int(r.n_adj_cells), int(r.n_adj_pairs)
            out["adj_cell"] = lazy(r.adj_cell, (na,), torch.int32)
            out["adj_off"] = lazy(r.adj_off, (na + 1,), torch.int32)
            out["adj_ids"] = lazy(r.adj_ids, (npairs,), torch.int32)
        if want_links:
            nl = int(r.n_links)
            out["link_cell"] = lazy(r.link_cell, (nl,), torch.int32)
            out["link_dir"] = lazy(r.link_dir, (nl,), torch.uint8)
            out["link_q"] = lazy(r.link_q, (nl,), torch.float32)
            out["link_face"] = lazy(r.link_face, (nl,), torch.int32)
        self.result = out
        return out

    def classify(self):
        """Node classes of the last refine's adjacent cells (row order of adj_cell): a borrowed uint8
        CUDA tensor, 1 = solid (inside the closed mesh), 0 = fluid; and the number of cells decided by
        the winding-number fallback."""
        import torch

        ptr = C.c_void_p()
        nfb = C.c_int64()
        _check(self.ctx, lib().amr_classify_nodes(self.ctx, C.byref(ptr), C.byref(nfb)))
        n = int(self.last_result.n_adj_cells) if self.last_result is not None else 0
        return _view(ptr.value, (n,), torch.uint8), int(nfb.value)

    def candidate_count(self):
        """Algorithmic cell-face test count of the last refine: (per-level list, total); per cell, the
        distinct faces in the bins its inflated box overlaps (exact, fixed by geometry and bins)."""
        per = (C.c_int64 * MAX_LEVELS)()
        tot = C.c_int64()
        _check(self.ctx, lib().amr_candidate_count(self.ctx, per, C.byref(tot)))
        n = int(self.last_result.n_levels) if self.last_result is not None else 0
        return [int(per[L]) for L in range(n)], int(tot.value)

    def adapt_diff(self):
        """Per level (after a refine with keep_previous): new_to_old / old_to_new index maps (borrowed int32
        CUDA tensors, -1 = created / removed) and the counts."""
        import torch

        d = amr_adapt_diff()
        _check(self.ctx, lib().amr_adapt_diff_get(self.ctx, C.byref(d)))
        out = []
        for L in range(max(d.n_levels, 0)):
            nn, no = int(d.n_new[L]), int(d.n_old[L])
            out.append({"new_to_old": _view(d.new_to_old[L], (nn,), torch.int32),
                        "old_to_new": _view(d.old_to_new[L], (no,), torch.int32),
                        "created": int(d.n_created[L]), "removed": int(d.n_removed[L])})
        return out

    def fluid_links(self):
        """Keep only the links of fluid cells (after classify); returns the updated link tensors."""
        r = amr_refine_result()
        _check(self.ctx, lib().amr_fluid_links(self.ctx, C.byref(r)))
        self.last_result = r
        return self._wrap(r, True, True)

    def q_backward(self, grad_q):
        """d(loss)/d(load input) from d(loss)/d(link_q) of the last refine (shape of the load input)."""
        import torch

        g = torch.as_tensor(grad_q, dtype=torch.float32, device="cuda").contiguous()
        out = torch.empty(self.load_shape, dtype=torch.float32, device="cuda")
        amr_q_backward(self.ctx, g.data_ptr(), out.data_ptr())
        return out

    def sync(self):
        amr_sync(self.ctx)

    def timing(self, on: bool = True):
        amr_timing_enable(self.ctx, on)

    def timing_reset(self):
        amr_timing_reset(self.ctx)

    def timings(self) -> dict:
        return amr_timing_get(self.ctx)

    def launch_count(self) -> int:
        return amr_launch_count(self.ctx)

    def autotune(self, n_levels, d_abs=0.0, d_rel=1.0, lattice=0, want_adjacency=True, want_links=True,
                 b_candidates=None, w_candidates=None):
        """Pick the bin density and warps per block by timing bin + refine on the loaded geometry."""
        return amr_autotune(self.ctx, n_levels, d_abs, d_rel, lattice, want_adjacency, want_links, b_candidates,
                            w_candidates)


def _make_qlinks():
    import torch

    class QLinks(torch.autograd.Function):
        """q of the wall links as a differentiable function of the vertex coordinates.

        Forward runs load -> bin -> refine (with links) on ``geom``; backward runs the
        library's deterministic adjoint.  Only q is differentiated (flags, adjacency and
        the choice of hit face are piecewise constant).  Call backward before the next
        refine on the same ``geom``.
        """

        @staticmethod
        def forward(ctx, verts, geom, idx, B, n_levels, d_abs, d_rel, lattice):
            geom.load(verts.detach(), idx)
            geom.bin(B)
            res = geom.refine(n_levels, d_abs, d_rel, lattice, True, True)
            ctx.geom = geom
            q = res["link_q"].clone()
            return q

        @staticmethod
        def backward(ctx, grad_q):
            g = ctx.geom.q_backward(grad_q)
            return g, None, None, None, None, None, None, None

    return QLinks


_QLINKS = None


def q_links(geom, verts, idx, B, n_levels, d_abs=0.0, d_rel=1.0, lattice=19):
    """Differentiable wall-link fractions q (see QLinks); returns a CUDA tensor [n_links]."""
    global _QLINKS
    if _QLINKS is None:
        _QLINKS = _make_qlinks()
    return _QLINKS.apply(verts, geom, idx, B, n_levels, d_abs, d_rel, lattice)


class AmrBatch:
    """Many geometries refined together (one launch per level for all of them).

    ``add`` takes each geometry's vertices/faces (torch or numpy, host or CUDA), its
    root grid, levels, near-wall distance and bin density (0 = tune later).
    ``run`` returns concatenated results (batch-global indices); ``view(i)``
    returns geometry i's results with local indices, as fresh CUDA tensors.
    """

    def __init__(self, dim: int):
        import torch

        self.dim = dim
        self.stream = torch.cuda.current_stream()
        h = C.c_void_p()
        st = lib().amr_batch_create(dim, self.stream.cuda_stream or 1, C.byref(h))
        if st != AMR_OK:
            raise AmrError(st, "amr_batch_create failed")
        self.b = h
        self.geoms = []
        self.result = None

    def close(self):
        if getattr(self, "b", None):
            lib().amr_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add(self, verts, idx, root, n_levels, d_abs=0.0, d_rel=1.0, bin_density=0, origin=(0.0, 0.0, 0.0),
            h0=None):
        import torch

        v = torch.as_tensor(verts, dtype=torch.float32).contiguous()
        root = tuple(int(r) for r in (root if hasattr(root, "__len__") else [root] * self.dim))
        d = amr_domain()
        d.dim = self.dim
        rb = list(root) + [1] * (3 - len(root))
        for a in range(3):
            d.root_blocks[a] = rb[a]
            d.origin[a] = float(origin[a]) if a < len(origin) else 0.0
        d.h0 = float(h0 if h0 is not None else 1.0 / (4.0 * rb[0]))
        out = C.c_int(-1)
        if idx is None:
            st = lib().amr_batch_add(self.b, C.byref(d), v.data_ptr(), 0, None, v.shape[0], int(n_levels),
                                     float(d_abs), float(d_rel), int(bin_density), C.byref(out))
            nv = 0
        else:
            ix = torch.as_tensor(idx, dtype=torch.int32).contiguous()
            st = lib().amr_batch_add(self.b, C.byref(d), v.data_ptr(), v.shape[0], ix.data_ptr(), ix.shape[0],
                                     int(n_levels), float(d_abs), float(d_rel), int(bin_density), C.byref(out))
            nv = v.shape[0]
        _bcheck(self.b, st)
        self.geoms.append({"n_levels": int(n_levels), "nv": nv, "nf": int(v.shape[0] if idx is None else idx.shape[0]),
                           "shape": tuple(v.shape)})
        return int(out.value)

    def set_bins(self, i, B):
        _bcheck(self.b, lib().amr_batch_set_bins(self.b, int(i), int(B)))

    def run(self, lattice=0, want_adjacency=True, want_links=None, use_graph=False, warps_per_cta=0,
            predicate=AMR_PRED_BOX, face_pass=AMR_FACE_PASS_AUTO):
        if want_links is None:
            want_links = lattice != 0
        p = _params(1, 0.0, 1.0, lattice, want_adjacency, want_links, use_graph, warps_per_cta, predicate,
                    face_pass=face_pass)
        r = amr_refine_result()
        _bcheck(self.b, lib().amr_batch_run(self.b, C.byref(p), C.byref(r)))
        self.want = (want_adjacency or want_links, want_links)
        self.result = r
        return r

    def view(self, i):
        """Geometry i's results with local indices (fresh tensors)."""
        import torch

        v = amr_batch_view()
        _bcheck(self.b, lib().amr_batch_get_view(self.b, int(i), C.byref(v)))
        r, D = v.r, self.dim
        nc = 64 if D == 3 else 16
        levels = []
        for L in range(r.n_levels):
            n = int(r.n_blocks[L])
            par = None
            if L > 0:
                par = _view(r.block_parent[L], (n,), torch.int32).clone() - int(v.level_base[L - 1])
            levels.append({"blocks": _view(r.block_coords[L], (n, D), torch.int32).clone(), "parent": par,
                           "mask": _view(r.cell_mask[L], (n,), torch.int64).clone(),
                           "flag": _view(r.block_flag[L], (n,), torch.uint8).clone()})
        out = {"levels": levels}
        adj, links = self.want
        Lf = r.n_levels - 1
        if adj:
            na, npairs = int(r.n_adj_cells), int(r.n_adj_pairs)
            out["adj_cell"] = _u32(r.adj_cell, na).long() - int(v.level_base[Lf]) * nc
            out["adj_off"] = _u32(r.adj_off, na + 1).long() - int(v.pair_base)
            out["adj_ids"] = _u32(r.adj_ids, npairs).long() - int(v.face_base)
        if links:
            nl = int(r.n_links)
            out["link_cell"] = _u32(r.link_cell, nl).long() - int(v.adj_base)
            out["link_dir"] = _view(r.link_dir, (nl,), torch.uint8).clone()
            out["link_q"] = _view(r.link_q, (nl,), torch.float32).clone()
            out["link_face"] = _u32(r.link_face, nl).long() - int(v.face_base)
        out["bases"] = {"face": int(v.face_base), "vert": int(v.vert_base), "link": int(v.link_base)}
        return out

    def q_backward(self, grad_q):
        import torch

        g = torch.as_tensor(grad_q, dtype=torch.float32, device="cuda").contiguous()
        if self.geoms and self.geoms[0]["nv"]:
            shape = (sum(x["nv"] for x in self.geoms), self.dim)
        else:
            shape = (sum(x["nf"] for x in self.geoms), self.dim, self.dim)
        out = torch.empty(shape, dtype=torch.float32, device="cuda")
        _bcheck(self.b, lib().amr_batch_q_backward(self.b, g.data_ptr(), out.data_ptr()))
        return out

    def launch_count(self):
        return int(lib().amr_batch_launch_count(self.b))
