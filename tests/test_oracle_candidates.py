"""Pin of the oracle's algorithmic cell-face test count C_alg (the metric's denominator): per cell,
the distinct faces stored in the bins that the cell's inflated box overlaps.  Checked against a
brute force that never looks at the bin lists: a face is a candidate of a cell exactly when the
face's bin range (from its AABB) and the cell's bin range (from its inflated box) intersect on
every axis."""
import numpy as np
import pytest

from synth import geometry as G


def _bin(x, origin, s, B):
    t = np.floor((x - origin) * s)
    return np.clip(t, 0, B - 1).astype(np.int64)


def _brute(dim, fv, root, B, level, blocks, d_rel):
    h0 = 1.0 / (4.0 * root)
    h = h0 * 2.0 ** (-level)
    s = B / (4.0 * root * h0)
    flo = _bin(fv.min(axis=1), 0.0, s, B)  # [nf, D]
    fhi = _bin(fv.max(axis=1), 0.0, s, B)
    r = 0.5 * h + d_rel * h
    nc = 64 if dim == 3 else 16
    c = np.arange(nc)
    loc = np.stack([c & 3, (c >> 2) & 3] + ([(c >> 4) & 3] if dim == 3 else []), 1)
    cells = (4 * blocks[:, None, :] + loc[None]).reshape(-1, dim)
    x = 0.0 + (cells + 0.5) * h
    qlo, qhi = _bin(x - r, 0.0, s, B), _bin(x + r, 0.0, s, B)
    hit = np.all((qlo[:, None, :] <= fhi[None]) & (qhi[:, None, :] >= flo[None]), axis=2)
    return int(hit.sum())


@pytest.mark.parametrize("dim,B,level", [(3, 1, 0), (3, 5, 0), (3, 7, 1), (2, 6, 1), (2, 11, 2)])
def test_candidate_count_brute_force(oracle_lib, dim, B, level):
    from oracle.oracle import Domain, OracleGeometry, root_blocks

    if dim == 3:
        v, f = G.jittered_sphere(1, radius=0.3, centre=(0.52, 0.47, 0.5), sigma=2e-3, seed=5)
    else:
        v, f = G.circle_polygon(23, 0.31, (0.47, 0.52))
    root = 3
    geo = OracleGeometry(dim, v, f)
    geo.bin(Domain.unit(dim, root), B)
    blocks = root_blocks(dim, (root,) * dim)
    if level > 0:  # a few blocks of the deeper level, anywhere in the domain
        rng = np.random.default_rng(level + B)
        blocks = rng.integers(0, root * 2 ** level, size=(7, dim)).astype(np.int32)
    _, _, _, ncand = geo.refine_blocks(level, blocks, 0.0, 1.0, count_candidates=True)
    want = _brute(dim, v[f].astype(np.float64), root, B, level, blocks.astype(np.int64), 1.0)
    assert ncand == want
    assert want > 0
