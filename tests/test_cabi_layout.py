"""The ctypes mirrors of the C structs have the header's sizes and field offsets (gcc, no GPU)."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = ["amr_domain", "amr_bins_view", "amr_refine_params", "amr_refine_result", "amr_adapt_diff",
           "amr_batch_view"]


def _c_layout(tmp_path, names):
    from paper_2502_16310_gb300 import binding as Bd

    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "amrgeom.h"', "int main(void) {"]
    for n in names:
        lines.append(f'  printf("{n} %zu\\n", sizeof({n}));')
        for f, _ in getattr(Bd, n)._fields_:
            lines.append(f'  printf("{n}.{f} %zu\\n", offsetof({n}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return dict((k, int(v)) for k, v in (ln.split() for ln in out.splitlines()))


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_struct_layouts_match_header(tmp_path):
    from paper_2502_16310_gb300 import binding as Bd

    c = _c_layout(tmp_path, STRUCTS)
    for n in STRUCTS:
        t = getattr(Bd, n)
        assert c[n] == C.sizeof(t), n
        for f, _ in t._fields_:
            assert c[f"{n}.{f}"] == getattr(t, f).offset, (n, f)
