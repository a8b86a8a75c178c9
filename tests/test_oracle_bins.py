"""Pins of the oracle's binning step (Sec. "Spatial Binning Algorithm").

Checked against what the definition fixes independently of the oracle's code:
  * exact rational re-derivation: face f is in bin b iff the closed AABB of f
    overlaps the bin's half-open box (last bin closed, outer bins unbounded);
  * invariants: sum of bin counts == sum over faces of their bin-range volumes,
    ids unique and ascending per bin;
  * special cases: B = 1 (the paper's naive scheme) holds every face once;
    vertices exactly on bin boundaries; faces outside the domain clamp inward.
"""
from fractions import Fraction as F

import numpy as np
import pytest

from synth import geometry as G


def _bins_rational(tri, B):
    """Set of bins for one face by interval overlap in exact arithmetic on the unit domain."""
    dim = tri.shape[1]
    rng = []
    for a in range(dim):
        lo = min(F(float(x)) for x in tri[:, a])
        hi = max(F(float(x)) for x in tri[:, a])
        ids = []
        for i in range(B):
            blo = F(i, B) if i > 0 else F(-10**9)
            bhi = F(i + 1, B)
            last = i == B - 1
            # half-open [blo, bhi) except the last bin, which is unbounded above
            if last:
                ok = hi >= blo
            else:
                ok = hi >= blo and lo < bhi
            if ok:
                ids.append(i)
        rng.append(ids)
    out = set()
    if dim == 2:
        for j in rng[1]:
            for i in rng[0]:
                out.add(i + B * j)
    else:
        for k in rng[2]:
            for j in rng[1]:
                for i in rng[0]:
                    out.add(i + B * j + B * B * k)
    return out


def _random_faces(rng, n, dim, grid=None):
    v = rng.uniform(-0.1, 1.1, size=(n, dim, dim))
    if grid:
        v = np.round(v * grid) / grid  # vertices on bin boundaries
    return v.astype(np.float32)


@pytest.mark.parametrize("dim,B,grid", [(2, 5, None), (2, 8, 8), (3, 4, None), (3, 6, 6), (3, 7, 14)])
def test_bins_match_rational_overlap(oracle_lib, dim, B, grid):
    from oracle.oracle import Domain, OracleGeometry

    rng = np.random.default_rng(100 + dim * 10 + B)
    fv = _random_faces(rng, 40, dim, grid)
    # small faces too, so many faces sit in a single bin
    small = (rng.uniform(0, 1, size=(20, 1, dim)) + rng.uniform(-0.02, 0.02, size=(20, dim, dim))).astype(np.float32)
    fv = np.concatenate([fv, small])
    g = OracleGeometry(dim, fv, None)
    off, ids = g.bin(Domain.unit(dim, 4), B)  # root 4 -> h0 = 1/16, domain [0,1]^D exactly
    nb = B ** dim
    assert off.shape[0] == nb + 1 and off[0] == 0 and off[-1] == ids.shape[0]
    members = {b: set(ids[off[b]:off[b + 1]].tolist()) for b in range(nb)}
    for b in range(nb):
        seg = ids[off[b]:off[b + 1]]
        assert np.all(np.diff(seg.astype(np.int64)) > 0), "ids must be unique and ascending"
    for f in range(fv.shape[0]):
        want = _bins_rational(fv[f], B)
        got = {b for b in range(nb) if f in members[b]}
        assert got == want, (f, fv[f], sorted(got), sorted(want))


def test_bin_count_invariant(oracle_lib):
    from oracle.oracle import Domain, OracleGeometry

    v, f = G.jittered_sphere(2, radius=0.3, centre=(0.5, 0.5, 0.5), sigma=1e-3, seed=5)
    g = OracleGeometry(3, v, f)
    B = 9
    off, ids = g.bin(Domain.unit(3, 8), B)
    tot = 0
    for k in range(f.shape[0]):
        lo, hi = g.face_bin_range(k)
        tot += int(np.prod(hi - lo + 1))
        assert np.all(lo <= hi) and np.all(lo >= 0) and np.all(hi < B)
    assert tot == ids.shape[0] == off[-1]


def test_naive_single_bin(oracle_lib):
    from oracle.oracle import Domain, OracleGeometry

    v, f = G.circle_polygon(33, 0.3, (0.5, 0.5))
    g = OracleGeometry(2, v, f)
    off, ids = g.bin(Domain.unit(2, 4), 1)
    assert off.tolist() == [0, 33]
    assert ids.tolist() == list(range(33))


def test_outside_domain_clamps(oracle_lib):
    from oracle.oracle import Domain, OracleGeometry

    fv = np.array([[[-5.0, -5.0], [-4.0, -4.0]], [[2.0, 0.5], [3.0, 0.5]], [[0.49, 0.5], [0.51, 0.5]]], np.float32)
    g = OracleGeometry(2, fv, None)
    off, ids = g.bin(Domain.unit(2, 2), 4)
    where = {int(x): [] for x in range(3)}
    for b in range(16):
        for x in ids[off[b]:off[b + 1]]:
            where[int(x)].append(b)
    assert where[0] == [0]            # far below: bin (0,0)
    assert where[1] == [3 + 4 * 2]    # far right at y = 0.5: bin (3, 2)
    assert where[2] == [1 + 4 * 2, 2 + 4 * 2]  # straddles x = 0.5


def test_empty_geometry(oracle_lib):
    from oracle.oracle import Domain, OracleGeometry

    g = OracleGeometry(3, np.zeros((0, 3, 3), np.float32), None)
    off, ids = g.bin(Domain.unit(3, 2), 3)
    assert ids.shape[0] == 0 and np.all(off == 0)


def test_invalid_inputs_rejected(oracle_lib):
    from oracle.oracle import OracleGeometry

    with pytest.raises(ValueError):
        OracleGeometry(3, np.zeros((4, 3), np.float32), np.array([[0, 1, 4]], np.int32))
    bad = np.zeros((1, 3, 3), np.float32)
    bad[0, 1, 2] = np.nan
    with pytest.raises(ValueError):
        OracleGeometry(3, bad, None)
