"""The allocation-free binning entry point against the regular one.

amr_bin_faces_static serves callers that cannot allocate device memory (a
solver that owns all device memory through its own arena, a plugin whose host
owns every allocation, a time-critical loop that must not synchronise on
cudaMalloc/cudaFree).  It must produce exactly the bins of amr_bin_faces:
identical offsets and identical face sets per bin, on two calls in a row (its
scratch array keeps the previous call's contents, so the second call checks
that everything that must start at zero is cleared).

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

from synth import small_workload, workload
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


def _canonical(off, ids):
    """Face ids sorted within each bin (both entry points leave the order within a bin unspecified)."""
    seg = np.repeat(np.arange(off.shape[0] - 1), np.diff(off.astype(np.int64)))
    return ids[np.lexsort((ids, seg))]


def _same_bins(a, b):
    assert np.array_equal(a[0], b[0]), "offsets differ"
    assert np.array_equal(_canonical(*a), _canonical(*b)), "bin contents differ"


def _regular(w, B):
    import torch

    from paper_2502_16310_gb300 import AmrGeom

    g = AmrGeom(w.dim, (w.root,) * w.dim)
    g.load(torch.from_numpy(w.verts).cuda(), torch.from_numpy(w.idx).cuda())
    bins = g.bin(B)
    torch.cuda.synchronize()
    off = U.to_np(bins["offsets"], np.uint32).copy()
    ids = U.to_np(bins["ids"], np.uint32).copy()
    g.close()
    return off, ids


def _static(w, B, cap=None):
    import torch

    from paper_2502_16310_gb300 import amr_bin_faces_static

    fv = torch.from_numpy(w.verts[w.idx]).cuda()               # [n_faces, D(vertex), D(coord)]
    soa = fv.permute(1, 2, 0).contiguous()                       # [D(vertex), D(coord), n_faces]
    nb = B ** w.dim
    offsets = torch.full((nb + 1,), -1, dtype=torch.int32, device="cuda")
    cap = 64 * w.n_faces + 16 if cap is None else cap
    ids = torch.full((max(cap, 1),), -1, dtype=torch.int32, device="cuda")
    nnz = amr_bin_faces_static(w.dim, (w.root,) * w.dim, soa.data_ptr(), w.n_faces, B, offsets.data_ptr(),
                               ids.data_ptr(), cap, stream=1)
    torch.cuda.synchronize()
    return U.to_np(offsets, np.uint32).copy(), U.to_np(ids, np.uint32)[:nnz].copy()


@pytest.mark.parametrize("name,B", [("c2", 64), ("sphere3", 32), ("circle", 7)])
def test_static_matches_regular_twice(name, B):
    w = workload(name) if name == "c2" else small_workload(name)
    ref = _regular(w, B)
    for _ in range(2):
        _same_bins(_static(w, B), ref)
    # a different density in between, then the first again: stale counts must not leak
    _static(w, max(1, B // 2))
    _same_bins(_static(w, B), ref)


def test_static_limits_and_capacity():
    import torch

    from paper_2502_16310_gb300 import AmrError, amr_bin_faces_static
    from paper_2502_16310_gb300 import binding as Bd

    w = small_workload("sphere3")
    # beyond the fixed maxima: rejected before any launch
    soa = torch.zeros(9, 8, device="cuda")
    off = torch.zeros(2, dtype=torch.int32, device="cuda")
    with pytest.raises(AmrError) as e:
        amr_bin_faces_static(3, (4, 4, 4), soa.data_ptr(), Bd.STATIC_MAX_FACES + 1, 4, off.data_ptr(),
                             off.data_ptr(), 1, stream=1)
    assert e.value.status == Bd.AMR_EINVAL
    with pytest.raises(AmrError) as e:
        amr_bin_faces_static(3, (4, 4, 4), soa.data_ptr(), 8, 65, off.data_ptr(), off.data_ptr(), 1, stream=1)
    assert e.value.status == Bd.AMR_EINVAL
    # host pointers are rejected
    host = np.zeros(8, np.uint32)
    with pytest.raises(AmrError) as e:
        amr_bin_faces_static(3, (4, 4, 4), soa.data_ptr(), 8, 4, host.ctypes.data, off.data_ptr(), 1, stream=1)
    assert e.value.status == Bd.AMR_EINVAL
    # too small an id buffer: EOVERFLOW, and a later call still matches
    with pytest.raises(AmrError) as e:
        _static(w, 32, cap=10)
    assert e.value.status == Bd.AMR_EOVERFLOW
    _same_bins(_static(w, 32), _regular(w, 32))


def test_static_rejects_non_finite_then_recovers():
    """A NaN or infinite coordinate is an error (EINVAL), as it is for amr_geom_load, and the next call on
    valid faces still matches the regular binning."""
    import torch

    from paper_2502_16310_gb300 import AmrError, amr_bin_faces_static
    from paper_2502_16310_gb300 import binding as Bd

    w = small_workload("sphere3")
    B = 16
    for bad in (float("nan"), float("inf")):
        fv = torch.from_numpy(w.verts[w.idx]).cuda()
        soa = fv.permute(1, 2, 0).contiguous()
        soa[1, 2, w.n_faces // 2] = bad
        off = torch.zeros(B ** 3 + 1, dtype=torch.int32, device="cuda")
        ids = torch.zeros(64 * w.n_faces, dtype=torch.int32, device="cuda")
        with pytest.raises(AmrError) as e:
            amr_bin_faces_static(3, (w.root,) * 3, soa.data_ptr(), w.n_faces, B, off.data_ptr(), ids.data_ptr(),
                                 ids.numel(), stream=1)
        assert e.value.status == Bd.AMR_EINVAL
    _same_bins(_static(w, B), _regular(w, B))
