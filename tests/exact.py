"""Exact rational geometry used to pin the oracle (independent constructions, not its formulas).

* box/face intersection by Sutherland-Hodgman clipping of the face against the
  six (four) closed half-spaces of the box, in ``fractions.Fraction``;
* segment/face intersection by Cramer's rule on the 3x3 (2x2) linear system
  ``o + t d = v0 + u (v1 - v0) + v (v2 - v0)``, in ``Fraction``.
"""
from __future__ import annotations

from fractions import Fraction as F


def _fr(x):
    return x if isinstance(x, F) else F(float(x))


def clip_nonempty(poly, box_lo, box_hi) -> bool:
    """True when the closed convex polygon/segment ``poly`` meets the closed box [lo, hi]."""
    pts = [tuple(_fr(c) for c in p) for p in poly]
    dim = len(box_lo)
    if len(pts) == 2:  # a segment: Liang-Barsky-style parameter clipping
        t0, t1 = F(0), F(1)
        a, b = pts
        for ax in range(dim):
            d = b[ax] - a[ax]
            lo, hi = _fr(box_lo[ax]), _fr(box_hi[ax])
            if d == 0:
                if a[ax] < lo or a[ax] > hi:
                    return False
                continue
            ta, tb = (lo - a[ax]) / d, (hi - a[ax]) / d
            if ta > tb:
                ta, tb = tb, ta
            t0, t1 = max(t0, ta), min(t1, tb)
            if t0 > t1:
                return False
        return True
    for ax in range(dim):
        for sign, bound in ((1, _fr(box_hi[ax])), (-1, _fr(box_lo[ax]))):
            # keep points with sign * x[ax] <= sign * bound
            out = []
            n = len(pts)
            if n == 0:
                return False
            for i in range(n):
                p, q = pts[i], pts[(i + 1) % n]
                fp = sign * p[ax] - sign * bound
                fq = sign * q[ax] - sign * bound
                if fp <= 0:
                    out.append(p)
                if (fp < 0 < fq) or (fq < 0 < fp):
                    t = fp / (fp - fq)
                    out.append(tuple(p[c] + t * (q[c] - p[c]) for c in range(dim)))
            pts = out
    return len(pts) > 0


def _det3(m):
    return (m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1])
            - m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0])
            + m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]))


def segment_face_hit(o, d, verts):
    """Exact hit parameter t in [0, 1] of o + t d with the closed face, or None.

    Parallel / coplanar configurations (singular system) are misses.
    """
    o = [_fr(c) for c in o]
    d = [_fr(c) for c in d]
    v = [[_fr(c) for c in p] for p in verts]
    if len(verts) == 2:
        e = [v[1][0] - v[0][0], v[1][1] - v[0][1]]
        rhs = [v[0][0] - o[0], v[0][1] - o[1]]
        # t d - s e = rhs
        det = d[0] * (-e[1]) - (-e[0]) * d[1]
        if det == 0:
            return None
        t = (rhs[0] * (-e[1]) - (-e[0]) * rhs[1]) / det
        s = (d[0] * rhs[1] - rhs[0] * d[1]) / det
        if 0 <= t <= 1 and 0 <= s <= 1:
            return t
        return None
    e1 = [v[1][c] - v[0][c] for c in range(3)]
    e2 = [v[2][c] - v[0][c] for c in range(3)]
    rhs = [v[0][c] - o[c] for c in range(3)]
    # t d - u e1 - w e2 = rhs ; columns (d, -e1, -e2)
    M = [[d[r], -e1[r], -e2[r]] for r in range(3)]
    det = _det3(M)
    if det == 0:
        return None

    def col(k):
        return [[rhs[r] if c == k else M[r][c] for c in range(3)] for r in range(3)]

    t = _det3(col(0)) / det
    u = _det3(col(1)) / det
    w = _det3(col(2)) / det
    if 0 <= t <= 1 and u >= 0 and w >= 0 and u + w <= 1:
        return t
    return None
