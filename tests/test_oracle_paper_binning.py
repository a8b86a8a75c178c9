"""Pins of the oracle's version of the paper's own binned search (Sec. "Spatial Binning
Algorithm"): sampled-point bin membership, the search of the cell's own bin and the
refinement-mark propagation.  Checked against facts fixed without the oracle's code:
the samples lie on the face, sampled membership is a subset of the AABB membership and
equals it for faces inside one bin, propagation marks the Chebyshev ball of the rounds
on a full grid, and with a single bin the own-bin search is the full search.
"""
import numpy as np

from oracle.oracle import Domain, OracleGeometry, propagate, propagation_rounds, root_blocks


def _tri_geo(seed=4, n=60, scale=0.08):
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.2, 0.8, size=(n, 1, 3))
    v = (c + rng.normal(0.0, scale, size=(n, 3, 3))).astype(np.float32).reshape(-1, 3)
    idx = np.arange(v.shape[0], dtype=np.int32).reshape(-1, 3)
    return v, idx


def _csr_sets(off, ids):
    return [set(ids[off[b]:off[b + 1]].tolist()) for b in range(off.shape[0] - 1)]


def test_samples_lie_on_the_face():
    v, idx = _tri_geo()
    geo = OracleGeometry(3, v, idx)
    s = 0.5 / 16
    for f in range(0, idx.shape[0], 7):
        tri = v[idx[f]].astype(np.float64)
        pts = geo.face_samples(f, s)
        # barycentric coordinates by least squares on the two edge vectors
        A = np.stack([tri[1] - tri[0], tri[2] - tri[0]], axis=1)
        lam, *_ = np.linalg.lstsq(A, (pts - tri[0]).T, rcond=None)
        l0 = 1.0 - lam.sum(0)
        assert np.all(lam >= -1e-9) and np.all(l0 >= -1e-9)
        assert np.allclose(A @ lam + tri[0][:, None], pts.T, atol=1e-12)
        for k in range(3):  # the vertices are samples
            assert np.min(np.abs(pts - tri[k]).sum(1)) <= 1e-15
        # consecutive samples along the first edge are at most s apart
        e = np.linalg.norm(tri[1] - tri[0])
        n = max(1, int(np.ceil(e / s)))
        assert e / n <= s + 1e-15


def test_sampled_membership_subset_and_rederived():
    v, idx = _tri_geo()
    for B in (4, 16, 40):
        dom = Domain.unit(3, 4)
        ex = OracleGeometry(3, v, idx)
        off_e, ids_e = ex.bin(dom, B)
        sp = OracleGeometry(3, v, idx)
        off_s, ids_s = sp.bin(dom, B, sampled=True)
        E, S = _csr_sets(off_e, ids_e), _csr_sets(off_s, ids_s)
        assert all(s_ <= e_ for s_, e_ in zip(S, E))
        for b in range(len(S)):  # ascending, unique per bin
            seg = ids_s[off_s[b]:off_s[b + 1]]
            assert np.all(np.diff(seg.astype(np.int64)) > 0)
        # membership re-derived from the sample points: bin = floor(x * B) clamped (unit domain)
        spacing = 0.5 / B
        want = [set() for _ in range(B ** 3)]
        for f in range(idx.shape[0]):
            pts = sp.face_samples(f, spacing)
            c = np.clip(np.floor(pts * B), 0, B - 1).astype(np.int64)
            for b in set((c[:, 0] + B * (c[:, 1] + B * c[:, 2])).tolist()):
                want[b].add(f)
        assert want == S


def test_sampled_equals_exact_for_faces_inside_one_bin():
    rng = np.random.default_rng(5)
    B = 8
    # tiny triangles well inside bins
    c = (rng.integers(0, B, size=(50, 1, 3)) + 0.5) / B
    v = (c + rng.uniform(-0.2, 0.2, size=(50, 3, 3)) / B).astype(np.float32).reshape(-1, 3)
    idx = np.arange(v.shape[0], dtype=np.int32).reshape(-1, 3)
    dom = Domain.unit(3, 2)
    off_e, ids_e = OracleGeometry(3, v, idx).bin(dom, B)
    off_s, ids_s = OracleGeometry(3, v, idx).bin(dom, B, sampled=True)
    assert np.array_equal(off_e, off_s) and np.array_equal(ids_e, ids_s)


def test_propagation_chebyshev_ball():
    """On a full grid of blocks, k rounds from one marked block mark the blocks within
    Chebyshev distance k (clipped to the grid)."""
    n = 9
    blocks = root_blocks(3, (n, n, n))
    centre = np.array([4, 4, 4])
    src = np.all(blocks == centre, axis=1)
    for k in range(4):
        flags = propagate(3, blocks, src.astype(np.uint8), k)
        want = np.abs(blocks - centre).max(1) <= k
        assert np.array_equal(flags.astype(bool), want), k
    # 2D, corner source: clipped quarter square
    b2 = root_blocks(2, (5, 5))
    f2 = propagate(2, b2, np.all(b2 == 0, axis=1).astype(np.uint8), 2)
    assert np.array_equal(f2.astype(bool), np.abs(b2).max(1) <= 2)


def test_propagation_stops_at_missing_blocks():
    """Marks only travel through blocks that exist on the level."""
    blocks = np.array([[0, 0, 0], [1, 0, 0], [3, 0, 0], [4, 0, 0]], np.int32)
    flags = propagate(3, blocks, np.array([1, 0, 0, 0], np.uint8), 5)
    assert flags.tolist() == [1, 1, 0, 0]


def test_propagation_rounds_formula():
    assert propagation_rounds(0.05, 4 / 256) == 1 + 3
    assert propagation_rounds(0.1, 4 / 256) == 1 + 6
    assert propagation_rounds(0.01, 4 / 64) == 1


def test_own_bin_search():
    """The own-bin search only drops candidates: its marks are a subset of the full search's;
    with one bin (the paper's naive B = 1) they are equal."""
    from synth import small_workload

    w = small_workload("sphere3")
    dom = Domain.unit(3, w.root)
    blocks = root_blocks(3, (w.root,) * 3)
    full = OracleGeometry(3, w.verts, w.idx)
    full.bin(dom, 8)
    m_full, _, _, _ = full.refine_blocks(0, blocks, 0.06, 0.0, pred=1)
    for B, sampled in ((1, True), (1, False), (8, True), (8, False)):
        geo = OracleGeometry(3, w.verts, w.idx)
        geo.bin(dom, B, sampled=sampled)
        m, _, _, _ = geo.refine_blocks(0, blocks, 0.06, 0.0, pred=1, search=1)
        assert not np.any(m & ~m_full)
        if B == 1:
            assert np.array_equal(m, m_full)
    assert np.count_nonzero(m_full) > 0
