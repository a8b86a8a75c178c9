"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and
compare its outputs with the FP64 oracle under the stated criteria.

Criteria (per output):
  * bins: identical sets of face ids per bin (order within a bin is unspecified
    on the GPU);
  * masks / blocks: identical outside the cells whose oracle decision lies in the
    1e-6*h margin band (box predicate: SAT margin; point predicate: distance
    minus d); children lists identical to the canonical children of the GPU's
    own masks (pure integer work);
  * adjacency lists: identical except for (cell, face) pairs in the band;
  * links: identical hit/miss outside the oracle's 1e-6 band, q within 1e-5
    absolute; the face must be one the oracle hits at that q (ties).
"""
from __future__ import annotations

import numpy as np

Q_TOL = 1e-5


def to_np(t, dtype=None):
    a = t.detach().cpu().numpy()
    return a.view(dtype) if dtype is not None else a


def run_gpu(w, *, B=None, n_levels=None, want_links=True, facelist=False, d_abs=None, d_rel=None, predicate=0,
            face_pass=0, want_adjacency=True, root=None, use_graph=False):
    """Whole CUDA pass for a workload; returns host copies of every output.  use_graph: refine twice with
    the level loop captured as a CUDA graph, so the outputs are those of a graph replay (as the bench
    runs it)."""
    import torch

    from paper_2502_16310_gb300 import AmrGeom

    B = w.bins if B is None else B
    n_levels = w.n_levels if n_levels is None else n_levels
    g = AmrGeom(w.dim, tuple(root) if root is not None else (w.root,) * w.dim)
    v = torch.from_numpy(w.verts).cuda()
    if facelist:
        g.load(torch.from_numpy(w.verts[w.idx]).cuda())
    else:
        g.load(v, torch.from_numpy(w.idx).cuda())
    bins = g.bin(B)
    for _ in range(2 if use_graph else 1):
        res = g.refine(n_levels, w.d_abs if d_abs is None else d_abs, w.d_rel if d_rel is None else d_rel,
                       w.lattice if want_links else 0, want_adjacency or want_links, want_links,
                       predicate=predicate, face_pass=face_pass, use_graph=use_graph)
    torch.cuda.synchronize()
    out = {"offsets": to_np(bins["offsets"], np.uint32), "ids": to_np(bins["ids"], np.uint32), "levels": []}
    for lv in res["levels"]:
        out["levels"].append({"blocks": to_np(lv["blocks"]), "mask": to_np(lv["mask"], np.uint64),
                              "flag": to_np(lv["flag"]),
                              "parent": None if lv["parent"] is None else to_np(lv["parent"])})
    if want_adjacency or want_links:
        out["adj_cell"] = to_np(res["adj_cell"], np.uint32)
        out["adj_off"] = to_np(res["adj_off"], np.uint32)
        out["adj_ids"] = to_np(res["adj_ids"], np.uint32)
    if want_links:
        out["link_cell"] = to_np(res["link_cell"], np.uint32)
        out["link_dir"] = to_np(res["link_dir"])
        out["link_q"] = to_np(res["link_q"])
        out["link_face"] = to_np(res["link_face"], np.uint32)
    for k in ("n_fallback", "n_band", "n_candidates", "n_survivors", "n_face_setups", "n_face_tests"):
        out[k] = res[k]
    g.close()
    return out


def compare_bins(off_g, ids_g, off_o, ids_o):
    assert off_g.shape == off_o.shape
    assert np.array_equal(off_g, off_o), "bin counts differ"
    nb = off_o.shape[0] - 1
    # sort within each bin: segment ids via repeat
    seg = np.repeat(np.arange(nb), np.diff(off_o.astype(np.int64)))
    og = np.lexsort((ids_g, seg))
    assert np.array_equal(ids_g[og], ids_o), "bin contents differ"


def cells_of(dim, blocks, block_idx, bits):
    loc = np.stack([bits & 3, (bits >> 2) & 3] + ([(bits >> 4) & 3] if dim == 3 else []), axis=1)
    return (4 * blocks[block_idx] + loc).astype(np.int32)


def compare_level(geo, dim, level, blocks, mask_gpu, sample=None, d_abs=0.0, d_rel=1.0, rng=None, pred=0):
    """Oracle masks for (a sample of) the GPU's blocks; returns (n_checked, n_band_cells)."""
    idx = np.arange(blocks.shape[0])
    if sample is not None and blocks.shape[0] > sample:
        rng = rng or np.random.default_rng(0)
        idx = np.sort(rng.choice(blocks.shape[0], size=sample, replace=False))
    if idx.size == 0:
        return 0, 0
    m_o, band, _, _ = geo.refine_blocks(level, blocks[idx], d_abs, d_rel, pred=pred)
    diff = (m_o ^ mask_gpu[idx]) & ~band
    bad = np.nonzero(diff)[0]
    assert bad.size == 0, (f"level {level}: {bad.size} blocks differ outside the band, e.g. block "
                           f"{blocks[idx[bad[0]]]} gpu {mask_gpu[idx[bad[0]]]:#x} oracle {m_o[bad[0]]:#x} "
                           f"band {band[bad[0]]:#x}")
    nband = int(sum(bin(int(b)).count("1") for b in band))
    return int(idx.size), nband


def check_children(dim, blocks, mask, child_blocks, child_parent):
    """GPU children == canonical children of the GPU's own marked blocks (integer exact)."""
    nch = 8 if dim == 3 else 4
    marked = np.nonzero(mask != 0)[0]
    want_p = np.repeat(marked, nch)
    s = np.tile(np.arange(nch), marked.size)
    off = np.stack([s & 1, (s >> 1) & 1] + ([(s >> 2) & 1] if dim == 3 else []), axis=1)
    want_b = 2 * blocks[want_p] + off
    assert child_blocks.shape == want_b.shape
    assert np.array_equal(child_parent, want_p)
    assert np.array_equal(child_blocks, want_b)


def compare_adjacency(geo, dim, level, fin_blocks, fin_mask, adj_cell, adj_off, adj_ids, sample=None,
                      d_abs=0.0, d_rel=1.0, rng=None, pred=0):
    nc = 64 if dim == 3 else 16
    # the adjacent cell list is exactly the set bits of the finest masks, ascending
    bits = ((fin_mask[:, None] >> np.arange(nc, dtype=np.uint64)[None, :]) & np.uint64(1)).astype(bool)
    bi, ci = np.nonzero(bits)
    want = (bi * nc + ci).astype(np.uint32)
    assert np.array_equal(adj_cell, want), "adjacent cell list differs from the finest masks"
    assert adj_off.shape[0] == adj_cell.shape[0] + 1 and adj_off[0] == 0 and adj_off[-1] == adj_ids.shape[0]
    assert np.all(np.diff(adj_off.astype(np.int64)) > 0), "every adjacent cell has at least one face"
    rows = np.arange(adj_cell.shape[0])
    if sample is not None and rows.size > sample:
        rng = rng or np.random.default_rng(1)
        rows = np.sort(rng.choice(rows.size, size=sample, replace=False))
    cells = cells_of(dim, fin_blocks, (adj_cell[rows] // nc).astype(np.int64), (adj_cell[rows] % nc).astype(np.int64))
    o_off, o_ids, o_band = geo.cell_faces(level, cells, d_abs, d_rel, pred=pred)
    n_band = 0
    for k, r in enumerate(rows):
        g = adj_ids[adj_off[r]:adj_off[r + 1]]
        assert np.all(np.diff(g.astype(np.int64)) > 0), "adjacency list not ascending"
        o = o_ids[o_off[k]:o_off[k + 1]]
        ob = o_band[o_off[k]:o_off[k + 1]]
        firm = set(o[~ob].tolist())
        allowed = set(o.tolist())
        gs = set(g.tolist())
        assert firm <= gs, (cells[k], sorted(firm - gs))
        assert gs <= allowed, (cells[k], sorted(gs - allowed))
        n_band += int(ob.sum())
    return int(rows.size), n_band


def compare_links(geo, dim, level, lattice, fin_blocks, adj_cell, link_cell, link_dir, link_q, link_face,
                  sample=None, rng=None, d_abs=0.0, d_rel=1.0, pred=0):
    nc = 64 if dim == 3 else 16
    Q1 = 18 if lattice == 19 else 8
    n_adj = adj_cell.shape[0]
    # links are sorted by (cell, dir) and unique
    key = link_cell.astype(np.int64) * 32 + link_dir.astype(np.int64)
    assert np.all(np.diff(key) > 0), "links not strictly sorted by (cell, direction)"
    assert np.all((link_dir >= 1) & (link_dir <= Q1))
    assert np.all((link_q >= 0) & (link_q <= 1))
    rows = np.arange(n_adj)
    if sample is not None and n_adj > sample:
        rng = rng or np.random.default_rng(2)
        rows = np.sort(rng.choice(n_adj, size=sample, replace=False))
    # the GPU's links of the checked rows as [rows, Q1] tables (links are sorted by cell)
    lo = np.searchsorted(link_cell, rows, "left")
    cnt = np.searchsorted(link_cell, rows, "right") - lo
    row_of = np.repeat(np.arange(rows.size), cnt)
    pos = np.arange(int(cnt.sum())) - np.repeat(np.cumsum(cnt) - cnt, cnt) + np.repeat(lo, cnt)
    gq = np.full((rows.size, Q1), np.nan)
    gf = np.full((rows.size, Q1), -1, np.int64)
    gq[row_of, link_dir[pos].astype(np.int64) - 1] = link_q[pos]
    gf[row_of, link_dir[pos].astype(np.int64) - 1] = link_face[pos]
    cells = cells_of(dim, fin_blocks, (adj_cell[rows] // nc).astype(np.int64), (adj_cell[rows] % nc).astype(np.int64))
    q_o, f_o, b_o = geo.cell_links(level, lattice, cells)
    # a link inherits the band of its face's adjacency decision: links are formed against the
    # cell's adjacency list, and a face in the adjacency band may be listed or not
    a_off, a_ids, a_band = geo.cell_faces(level, cells, d_abs, d_rel, pred=pred)
    inherit = np.zeros_like(b_o)
    for i in range(cells.shape[0]):
        bset = set(a_ids[a_off[i]:a_off[i + 1]][a_band[a_off[i]:a_off[i + 1]]].tolist())
        if bset:
            inherit[i] = np.isin(f_o[i], list(bset)) | np.isin(gf[i], list(bset))
    firm = ~(b_o | inherit)
    hit_o = np.isfinite(q_o)
    hit_g = np.isfinite(gq)
    bad = firm & (hit_o != hit_g)
    assert not np.any(bad), f"{int(bad.sum())} links differ in hit/miss, e.g. {np.argwhere(bad)[:3].tolist()}"
    both = firm & hit_o & hit_g
    err = np.abs(gq[both] - q_o[both])
    assert err.size == 0 or err.max() <= Q_TOL, f"max |dq| = {err.max()}"
    # face: either the oracle's face, or another face the oracle hits at the same q
    diff_face = both & (gf != f_o)
    for i, k in np.argwhere(diff_face):
        qf = geo.link_q(level, lattice, cells[i], k + 1, gf[i, k])
        assert np.isfinite(qf) and abs(qf - q_o[i, k]) <= Q_TOL, (cells[i], k + 1, gf[i, k], f_o[i, k])
    return int(both.sum()), int((~firm).sum()), float(err.max()) if err.size else 0.0
