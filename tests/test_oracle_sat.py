"""Pins of the oracle's adjacency predicate (separating-axis margin of box vs closed face).

The sign of the margin is checked against an independent construction:
exact-rational clipping of the face by the box's closed half-spaces
(Sutherland-Hodgman in 3D, parameter clipping in 2D) — non-empty iff they meet.
Closed forms fix the magnitude in simple configurations.
"""
import numpy as np
import pytest

from tests.exact import clip_nonempty


def _margin(dim, v, r):
    from oracle.oracle import sat_margin

    return sat_margin(dim, np.asarray(v, np.float64), r)


@pytest.mark.parametrize("dim", [2, 3])
def test_sign_matches_rational_clipping(oracle_lib, dim):
    rng = np.random.default_rng(7 + dim)
    r = 0.5
    n_touch = n_in = n_out = 0
    for it in range(1500 if dim == 3 else 3000):
        # coarse dyadic grid -> many exact touching / edge-on configurations
        scale = rng.choice([1.0, 0.5, 0.25])
        v = np.round(rng.uniform(-1.6, 1.6, size=(dim, dim)) * 8) / 8 * scale
        if it % 3 == 0:
            v = v + np.round(rng.uniform(-1.0, 1.0, size=(1, dim)) * 8) / 8  # shift whole face
        m = _margin(dim, v, r)
        hit = clip_nonempty(v, [-r] * dim, [r] * dim)
        assert (m <= 0.0) == hit, (v, m, hit)
        if m == 0.0:
            n_touch += 1
        elif m < 0:
            n_in += 1
        else:
            n_out += 1
    assert n_touch > 10 and n_in > 100 and n_out > 100


@pytest.mark.parametrize("dim", [2, 3])
def test_sign_random_continuous(oracle_lib, dim):
    rng = np.random.default_rng(70 + dim)
    r = 0.3
    for _ in range(800):
        v = rng.normal(0, 0.6, size=(dim, dim))
        m = _margin(dim, v, r)
        assert (m <= 0.0) == clip_nonempty(v, [-r] * dim, [r] * dim)


def test_closed_forms_3d(oracle_lib):
    r = 0.5
    # triangle parallel to the +z face at height r + delta
    for delta in [0.25, 1e-3, 0.0, -0.1]:
        z = r + delta
        v = [[-0.2, -0.2, z], [0.3, -0.1, z], [0.0, 0.4, z]]
        assert _margin(3, v, r) == pytest.approx(delta, abs=1e-15)
    # degenerate (point) face on the diagonal: only box axes count
    a = 0.9
    v = [[a, a, a]] * 3
    assert _margin(3, v, r) == pytest.approx(a - r, abs=1e-15)
    # big triangle through the box: negative margin
    v = [[-3, -3, 0.1], [3, -3, 0.1], [0, 3, 0.1]]
    assert _margin(3, v, r) < 0
    # tilted plane x + y + z = s: separated by (s - 3r)/sqrt(3) along the normal
    s = 2.0
    v = [[s, 0, 0], [0, s, 0], [0, 0, s]]
    assert _margin(3, v, r) == pytest.approx((s - 3 * r) / np.sqrt(3.0), abs=1e-12)
    # margin scales linearly with the configuration
    rng = np.random.default_rng(3)
    v = rng.normal(0, 1, size=(3, 3))
    assert _margin(3, 4.0 * v, 4.0 * r) == pytest.approx(4.0 * _margin(3, v, r), rel=1e-12, abs=1e-14)


def test_closed_forms_2d(oracle_lib):
    r = 0.5
    # segment along the diagonal x + y = s
    s = 1.5
    v = [[s, 0.0], [0.0, s]]
    assert _margin(2, v, r) == pytest.approx((s - 2 * r) / np.sqrt(2.0), abs=1e-12)
    v = [[0.7, -0.2], [0.7, 0.2]]
    assert _margin(2, v, r) == pytest.approx(0.2, abs=1e-15)
    v = [[-2.0, 0.5], [2.0, 0.5]]
    assert _margin(2, v, r) == 0.0
