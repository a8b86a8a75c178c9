"""The C-ABI library builds, loads and exports every entry point its header declares (CPU only)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    inc = os.path.join(ROOT, "include")
    for fn in sorted(os.listdir(inc)):
        if fn.endswith(".h"):
            text = open(os.path.join(inc, fn)).read()
            names += re.findall(r"^AMR_API\s+[\w\s\*]+?\b(amr_\w+)\s*\(", text, flags=re.M)
    return names


def test_library_exports_header_symbols():
    from paper_2502_16310_gb300 import binding

    lib = binding.lib()
    names = _declared()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"
    assert set(binding.EXPORTED) <= set(names)


def test_status_strings_without_gpu():
    from paper_2502_16310_gb300 import binding

    lib = binding.lib()
    for s in range(8):
        assert lib.amr_status_str(s)
    # bad arguments are rejected before any device work
    h = ctypes.c_void_p()
    assert lib.amr_create(None, ctypes.byref(h)) == binding.AMR_EINVAL
    d = binding.amr_domain()
    d.dim = 4
    assert lib.amr_create(ctypes.byref(d), ctypes.byref(h)) == binding.AMR_EINVAL
    assert lib.amr_destroy(None) == binding.AMR_OK


def test_oracle_does_not_link_cuda_library():
    """The oracle is independent of the CUDA path: no shared headers or sources."""
    src = open(os.path.join(ROOT, "oracle", "amr_oracle.cpp")).read()
    assert "amrgeom" not in src and "internal.cuh" not in src
    py = open(os.path.join(ROOT, "oracle", "oracle.py")).read()
    assert "paper_2502_16310_gb300" not in py
    for fn in os.listdir(os.path.join(ROOT, "paper_2502_16310_gb300")):
        if fn.endswith(".py"):
            assert "oracle" not in open(os.path.join(ROOT, "paper_2502_16310_gb300", fn)).read().replace(
                "no oracle", "")


def test_product_path_never_reaches_the_oracle():
    """The package, its kernels and the public header name nothing of oracle/ (the checker is test
    infrastructure only), and the package fails loudly instead of falling back when the CUDA library
    cannot be loaded."""
    pkg = os.path.join(ROOT, "paper_2502_16310_gb300")
    files = [os.path.join(pkg, f) for f in os.listdir(pkg) if f.endswith(".py")]
    files += [os.path.join(pkg, "csrc", f) for f in os.listdir(os.path.join(pkg, "csrc"))
              if f.endswith((".cu", ".cuh", ".h"))]
    files += [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))]
    for fn in files:
        text = open(fn).read()
        assert not re.search(r"\boracle\b|amr_oracle|orc_", text), fn
    binding = open(os.path.join(pkg, "binding.py")).read()
    assert "raise ImportError" in binding
