"""Write the stored expected values under tests/golden/ — calls only the oracle.

c1_levels.json: the 2D circle workload (512-gon, r = 0.2, 16^2 roots, 3 levels,
B = 32, D2Q9) as computed by the FP64 oracle: per level the block count, the
marked-block count, the adjacent-cell count and the band cells; the finest
level's adjacent-face pairs and wall links.  A regression pin of the oracle and
the expected counts of the GPU parity test.

Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.oracle import run_pipeline  # noqa: E402
from synth import workload  # noqa: E402


def c1_summary():
    w = workload("c1")
    out = run_pipeline(2, w.verts, w.idx, root=w.root, n_levels=w.n_levels, B=w.bins, lattice=9)
    lv = []
    for L, x in enumerate(out["levels"]):
        bits = [bin(int(m)).count("1") for m in x["mask"]]
        lv.append({"level": L, "blocks": int(x["blocks"].shape[0]), "marked": int((x["mask"] != 0).sum()),
                   "adjacent_cells": int(sum(bits)), "band_cells": int(sum(bin(int(m)).count("1") for m in x["band"]))})
    return {
        "workload": w.description,
        "nnz_bins": int(out["ids"].shape[0]),
        "levels": lv,
        "adjacent_face_pairs": int(out["adj_ids"].shape[0]),
        "links": int(np.isfinite(out["q"]).sum()),
        "band_links": int(out["q_band"].sum()),
        "q_sum": float(np.nansum(out["q"])),
    }


if __name__ == "__main__":
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "c1_levels.json"), "w") as f:
        json.dump(c1_summary(), f, indent=1)
        f.write("\n")
