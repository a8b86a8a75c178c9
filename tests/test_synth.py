"""The seeded synthetic inputs (CPU): sizes as documented, reproducible, closed meshes inside the
unit domain.  Node classification and the links of both senses rely on the meshes being closed."""
import numpy as np
import pytest

from synth import small_workload, workload

SIZES = {  # name: (dim, faces, roots per axis, levels, bins per axis, lattice)
    "c1": (2, 512, 16, 3, 32, 9),
    "c2": (3, 20480, 32, 4, 64, 19),
    "c3": (3, 81920, 32, 5, 128, 19),
    "p2": (2, 12800, 64, 3, 16, 9),
    "p3": (3, 112500, 16, 3, 16, 19),
}


def _closed(dim, idx):
    if dim == 2:  # every vertex ends exactly two segments
        return np.all(np.bincount(idx.ravel()) == 2)
    e = np.sort(np.concatenate([idx[:, [0, 1]], idx[:, [1, 2]], idx[:, [2, 0]]]), axis=1)
    _, cnt = np.unique(e, axis=0, return_counts=True)
    return np.all(cnt == 2)


@pytest.mark.parametrize("name", sorted(SIZES))
def test_workload_recipe(name):
    w = workload(name)
    dim, nf, root, levels, bins, lattice = SIZES[name]
    assert (w.dim, w.n_faces, w.root, w.n_levels, w.bins, w.lattice) == (dim, nf, root, levels, bins, lattice)
    assert w.verts.dtype == np.float32 and w.idx.dtype == np.int32
    assert w.verts.shape[1] == dim and w.idx.shape[1] == dim
    assert np.all((w.verts > 0) & (w.verts < 1))
    assert w.idx.min() == 0 and w.idx.max() == w.verts.shape[0] - 1
    assert _closed(dim, w.idx)
    if dim == 3:  # a sphere-like surface: V - E + F = 2
        assert w.verts.shape[0] - 3 * nf // 2 + nf == 2
    v = workload(name)
    assert np.array_equal(v.verts, w.verts) and np.array_equal(v.idx, w.idx)  # seeded


@pytest.mark.parametrize("kind", ["circle", "sphere3", "bumpy3"])
def test_small_workloads_closed(kind):
    w = small_workload(kind)
    assert _closed(w.dim, w.idx)
    assert np.all((w.verts > 0) & (w.verts < 1))
