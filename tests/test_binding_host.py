"""Host-side pieces of the Python binding on CPU: result views built on first access."""
from paper_2502_16310_gb300.binding import _Deferred, _LazyDict


def test_lazy_views_build_once_and_survive_copies():
    made = []

    def make(v):
        def f():
            made.append(v)
            return v * 10
        return _Deferred(f)

    d = _LazyDict(a=make(1), b=make(2), c=3)
    assert made == []  # nothing is built until read
    assert d["a"] == 10 and d["a"] == 10 and made == [1]  # built once, then cached
    assert d.get("b") == 20 and d.get("zz", 7) == 7 and made == [1, 2]
    e = _LazyDict(x=make(4), y=make(5))
    for copy in (dict(e), {**e}, e.copy()):
        assert copy == {"x": 40, "y": 50}
    assert made == [1, 2, 4, 5]
    assert sorted(e.values()) == [40, 50] and dict(e.items()) == {"x": 40, "y": 50}
    assert list(e) == ["x", "y"] and "x" in e and len(e) == 2
