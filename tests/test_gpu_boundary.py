"""Boundary details of the C ABI on the GPU: a caller-supplied device allocator (every device buffer of the
context comes from it and goes back to it) and the bin payload view (one entry per (face, bin) entry, in the
order of the ids, holding the face's coordinates)."""
import numpy as np
import pytest

from synth import small_workload
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


def _refine_all(g, w):
    import torch

    g.load(torch.from_numpy(w.verts).cuda(), torch.from_numpy(w.idx).cuda())
    bins = g.bin(w.bins)
    res = g.refine(w.n_levels, w.d_abs, w.d_rel, w.lattice, True, True)
    torch.cuda.synchronize()
    out = {"ids": U.to_np(bins["ids"], np.uint32).copy(), "offsets": U.to_np(bins["offsets"], np.uint32).copy()}
    for k in ("adj_ids", "link_q", "link_face"):
        out[k] = U.to_np(res[k]).copy()
    out["masks"] = [U.to_np(lv["mask"]).copy() for lv in res["levels"]]
    return out


def test_caller_allocator_serves_every_buffer():
    import torch

    from paper_2502_16310_gb300 import AmrGeom
    from paper_2502_16310_gb300 import binding as Bd

    live, calls = {}, {"alloc": 0, "free": 0, "bytes": 0}

    @Bd.DEV_ALLOC
    def alloc(n, user):
        t = torch.empty(int(n), dtype=torch.uint8, device="cuda")
        live[t.data_ptr()] = t
        calls["alloc"] += 1
        calls["bytes"] += int(n)
        return t.data_ptr()

    @Bd.DEV_FREE
    def free(p, user):
        assert p in live, "freed a buffer the allocator did not hand out"
        del live[p]
        calls["free"] += 1

    w = small_workload("bumpy3")
    ref_g = AmrGeom(3, (w.root,) * 3)
    ref = _refine_all(ref_g, w)
    ref_g.close()
    g = AmrGeom(3, (w.root,) * 3, dev_alloc=alloc, dev_free=free)
    for _ in range(2):
        got = _refine_all(g, w)
        assert np.array_equal(got["offsets"], ref["offsets"])
        for k in ("adj_ids", "link_q", "link_face"):
            assert np.array_equal(got[k], ref[k]), k
        for a, b in zip(got["masks"], ref["masks"]):
            assert np.array_equal(a, b)
    assert calls["alloc"] > 10 and calls["bytes"] > 0
    g.close()
    assert calls["free"] == calls["alloc"] and not live, "every buffer goes back to the caller's allocator"


def test_allocator_needs_both_hooks():
    from paper_2502_16310_gb300 import AmrError, amr_create
    from paper_2502_16310_gb300 import binding as Bd

    alloc = Bd.DEV_ALLOC(lambda n, u: 0)
    with pytest.raises(AmrError) as e:
        amr_create(3, (4, 4, 4), dev_alloc=alloc)
    assert e.value.status == Bd.AMR_EINVAL


@pytest.mark.parametrize("kind", ["sphere3", "circle"])
def test_bin_payload_matches_ids_and_faces(kind):
    import torch

    from paper_2502_16310_gb300 import AmrGeom

    w = small_workload(kind)
    D = w.dim
    g = AmrGeom(D, (w.root,) * D)
    g.load(torch.from_numpy(w.verts).cuda(), torch.from_numpy(w.idx).cuda())
    bins = g.bin(w.bins)
    torch.cuda.synchronize()
    off = U.to_np(bins["offsets"], np.uint32).astype(np.int64)
    ids = U.to_np(bins["ids"], np.uint32)
    pay = U.to_np(bins["payload"], np.uint32)
    g.close()
    nc = D * D
    assert pay.shape == (ids.shape[0], 16 if D == 3 else 8)
    ent_id = pay[:, nc + (3 if D == 3 else 0)]
    assert np.array_equal(ent_id & ((1 << 29) - 1), ids), "entry k belongs to ids[k]"
    coords = pay[:, :nc].view(np.float32).reshape(-1, D, D)
    assert np.array_equal(coords, w.verts[w.idx][ids]), "entry coordinates are the face's"
    if D == 3:
        fv = w.verts[w.idx][ids].astype(np.float64)
        n64 = np.cross(fv[:, 1] - fv[:, 0], fv[:, 2] - fv[:, 0])
        n32 = pay[:, 9:12].view(np.float32).astype(np.float64)
        scale = np.abs(n64).max(axis=1, keepdims=True)
        assert np.all(np.abs(n32 - n64) <= 1e-6 * scale), "entry normal is the face's (v1-v0)x(v2-v0)"
    # bin coordinates of entry k: its bin b = bx + B by (+ B^2 bz)
    b = np.repeat(np.arange(off.shape[0] - 1), np.diff(off))
    bc = pay[:, nc + (4 if D == 3 else 1):nc + (7 if D == 3 else 4)].astype(np.int64)
    B = w.bins
    want = np.stack([b % B, (b // B) % B, b // (B * B)], axis=1)
    assert np.array_equal(bc[:, :D], want[:, :D])
    # first-bin flags: set exactly when the entry's bin is the first of its face's range along the axis
    for a in range(D):
        flag = (ent_id >> (29 + a)) & 1
        first = np.full(w.n_faces, np.iinfo(np.int64).max)
        np.minimum.at(first, ids.astype(np.int64), bc[:, a])
        assert np.array_equal(flag.astype(bool), bc[:, a] == first[ids]), a


def test_caller_allocator_failure_is_enomem():
    """An allocator that runs out (returns NULL) makes the call fail with AMR_ENOMEM; the context still
    closes and hands back every buffer it got, and a later context works."""
    import torch

    from paper_2502_16310_gb300 import AmrError, AmrGeom
    from paper_2502_16310_gb300 import binding as Bd

    live, budget = {}, {"left": 6}

    @Bd.DEV_ALLOC
    def alloc(n, user):
        if budget["left"] <= 0:
            return None
        budget["left"] -= 1
        t = torch.empty(int(n), dtype=torch.uint8, device="cuda")
        live[t.data_ptr()] = t
        return t.data_ptr()

    @Bd.DEV_FREE
    def free(p, user):
        del live[p]

    w = small_workload("bumpy3")
    g, err = None, None
    try:  # the budget runs out in the context's set-up or in one of the steps
        g = AmrGeom(3, (w.root,) * 3, dev_alloc=alloc, dev_free=free)
        g.load(torch.from_numpy(w.verts).cuda(), torch.from_numpy(w.idx).cuda())
        g.bin(w.bins)
        g.refine(w.n_levels, w.d_abs, w.d_rel, w.lattice, True, True)
    except AmrError as ex:
        err = ex
    assert err is not None and err.status == Bd.AMR_ENOMEM
    if g is not None:
        g.close()
    assert not live, "every buffer the context got went back"
    ref = AmrGeom(3, (w.root,) * 3)
    assert _refine_all(ref, w)["link_q"].size > 0
    ref.close()
