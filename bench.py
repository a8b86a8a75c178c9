#!/usr/bin/env python
"""Throughput of the near-wall refinement hot path on GB300.

One step = the whole path on one synthetic geometry: import (gather to SoA +
face normals), binning (AABB count, scan, scatter), near-wall refinement of
every level with child compaction, the finest level's adjacent-face lists and
its D3Q19 wall links.  Headline value: near-wall cells identified per second
(adjacent cells summed over all levels), whole job over all ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c4] [--impl reference]

The default workload is the largest single-geometry one (c4: 1,310,720 triangles,
64^3 roots, 6 levels, 256^3 bins); c1-c3 are timed beside it (`per_workload`).

Multi-GPU: the path has no exchange step, so N ranks run N independent
replicas of the workload (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "near-wall cells/s & faces binned/s; batched vs single; adjoint/forward"
UNIT = "cells/s"
FP32_LANES_PER_SM = 128
N_SM = 152
SM_MAX_MHZ = 2070.0
L2_FLUSH_BYTES = 512 << 20

# Algorithmic work per unit (FP32-pipe operations counted from the kernel source):
OPS_BLOCK_CANDIDATE = 120.0   # face setup up to the AABB cull (vertex offsets, edges, three box axes)
OPS_CELL_TEST = 80.0          # one cell against one (face, block) survivor: 13 axes x (projection + interval test)
OPS_FACE_SETUP = 400.0        # face-by-face marking, per (face, level): cell range, frame, 13 axis intervals
OPS_LINK_DIR = 40.0           # per (adjacent cell, face, lattice direction): one watertight segment-triangle test
OPS_LINK_FACE = 150.0         # per (adjacent cell, face), executed on top: double-float offsets, plane offset,
                              # cross products and the line filters (reported beside the roofline, not in it)
# DRAM bytes (read + write) per launch of the current kernels, from one ncu capture each
# (dram__bytes_read.sum + dram__bytes_write.sum, one pass) of the named workload; others report null
MEASURED_TRAFFIC = {("c4", "refine_level"): 393028096 + 2277046272,
                    # the link step: k_links, the scan of its tile counts, k_links_place
                    ("c4", "links"): 3768263936 + 4520397312 + 12329216 + 5083136000 + 6614900736}


def parse_args(argv=None):
    p = argparse.ArgumentParser(description=__doc__)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--workload", default="c4")
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle sample")
    p.add_argument("--no-all-cores", action="store_true", help="skip the oracle timing on all host cores")
    p.add_argument("--no-graph", action="store_true", help="time the eager path instead of graph replays")
    p.add_argument("--no-extras", action="store_true", help="skip the batched and adjoint measurements")
    p.add_argument("--bin-only", action="store_true",
                   help="time the binning alone (load once, then count, scan and scatter per step)")
    p.add_argument("--batch-geoms", type=int, default=48)
    p.add_argument("--e2e-threads", type=int, default=0,
                   help="host threads (one context each) of the e2e leg; 0 = three threads for steps that "
                        "copy back less than 2 GB, else one thread alternating two contexts")
    return p.parse_args(argv)


def max_over_ranks(x: float, world: int, device="cpu") -> float:
    """The largest x over the ranks (one all-reduce over the job's process group; x for one rank)."""
    if world <= 1:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(units_per_rank: float, world: int, ms_step: float) -> float:
    """Units all ranks processed per second: every rank runs the same workload (replicas, weak
    scaling), timed by the slowest rank's step."""
    return units_per_rank * world / (ms_step * 1e-3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append({"sm": float(parts[1]), "max": float(parts[2]), "power": float(parts[3]),
                             "hw": parts[5], "hwth": parts[6], "swth": parts[7], "swpc": parts[8]})
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sms = sorted(r["sm"] for r in rows)
        reasons = set()
        for r in rows:
            for k, name in (("hw", "hw_slowdown"), ("hwth", "hw_thermal_slowdown"), ("swth", "sw_thermal_slowdown"),
                            ("swpc", "sw_power_cap")):
                if r[k].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": sms[len(sms) // 2], "sm_max_mhz": max(r["max"] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows),
                "power_w_max": max(r["power"] for r in rows)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def near_wall_cells(res):
    """Adjacent cells summed over all levels (popcount of every level's cell masks)."""
    import torch

    lut = torch.tensor([bin(i).count("1") for i in range(256)], dtype=torch.int64, device="cuda")
    tot = 0
    for lv in res["levels"]:
        m = lv["mask"]
        if m.numel():
            tot += int(lut[m.view(torch.uint8).long()].sum().item())
    return tot


def run_ours(args, rank, world, local):
    import numpy as np
    import torch

    from paper_2502_16310_gb300 import AmrGeom
    from synth import workload

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = workload(args.workload)
    verts = torch.from_numpy(w.verts).to(dev)
    idx = torch.from_numpy(w.idx).to(dev)
    g = AmrGeom(w.dim, (w.root,) * w.dim)
    stream = g.stream

    use_graph = not args.no_graph

    def step():
        g.load(verts, idx)
        g.bin(w.bins)
        return g.refine(w.n_levels, w.d_abs, w.d_rel, w.lattice, True, True, use_graph=use_graph)

    for _ in range(max(args.warmup, 1)):
        res = step()
    torch.cuda.synchronize()
    cells = near_wall_cells(res)
    n_links = int(res["link_q"].shape[0])
    n_adj = int(res["adj_cell"].shape[0])
    n_pairs = int(res["adj_ids"].shape[0])
    n_cand, n_surv = res["n_candidates"], res["n_survivors"]
    n_fb, n_band = res["n_fallback"], res["n_band"]
    n_lcand = res.get("n_link_candidates", 0)
    n_fsetup, n_ftest = res.get("n_face_setups", 0), res.get("n_face_tests", 0)
    blocks = [int(lv["blocks"].shape[0]) for lv in res["levels"]]
    nnz = int(g.bin(w.bins)["ids"].shape[0])  # (face, bin) incidences
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    # timed region: K steps, L2 flushed between steps (outside the events)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(local if "CUDA_VISIBLE_DEVICES" not in os.environ else 0)
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    launches0 = g.launch_count()
    t0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    launches = g.launch_count() - launches0
    barrier()
    clocks = sampler.stop()
    ms = [a.elapsed_time(b) for a, b in ev]
    ms_step = sum(ms) / len(ms)
    ms_step = max_over_ranks(ms_step, world, dev)
    value = whole_job_value(cells, world, ms_step)

    # per-kernel timing pass (CUDA events around each launch, on the context stream)
    g.timing(True)
    g.timing_reset()
    n_t = max(3, min(10, args.steps))
    for k in range(n_t):
        flush.fill_(k & 0xff)
        g.load(verts, idx)
        g.bin(w.bins)
        g.refine(w.n_levels, w.d_abs, w.d_rel, w.lattice, True, True, use_graph=False)
    tk = g.timings()
    g.timing(False)
    # the algorithmic cell-face test count of the step (per cell, the distinct faces in the bins its
    # inflated box overlaps; fixed by the geometry and the bins), outside every timed region
    c_alg_levels, c_alg = g.candidate_count()
    kern = {name: {"ms_per_step": v[0] / n_t, "launches_per_step": v[1] / n_t} for name, v in tk.items()}
    t_bin = sum(kern[k]["ms_per_step"] for k in ("bin_count", "bin_scan", "bin_scatter") if k in kern)
    t_refine = kern.get("refine_level", {}).get("ms_per_step", 0.0)
    t_mark = kern.get("mark_faces", {}).get("ms_per_step", 0.0)
    dom = max(kern.items(), key=lambda kv: kv[1]["ms_per_step"])
    roof = roofline(dom[0], dom[1], w, kern, n_cand, n_surv, n_adj, n_pairs, blocks, clocks, n_fsetup, n_ftest)
    roof["traffic"] = MEASURED_TRAFFIC.get((args.workload, dom[0]))
    NCe = 64 if w.dim == 3 else 16
    n_tests = n_surv * NCe + n_ftest  # block-walk cell tests + face-by-face (face, cell) tests
    binning = bin_roofline(w, nnz, t_bin)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"{args.workload}: {w.description}", "faces": w.n_faces, "levels": w.n_levels,
                   "bins_per_axis": w.bins, "blocks_per_level": blocks, "near_wall_cells_per_step": cells,
                   "adjacent_finest_cells": n_adj, "adjacent_pairs": n_pairs, "links": n_links,
                   "parallelism": f"replicas x{world}", "l2": "flushed between steps (512 MB write)",
                   "level_loop": "CUDA graph replay" if use_graph else "eager",
                   "fp64_fallbacks_per_step": n_fb, "band_cases_per_step": n_band,
                   "block_face_candidates": n_cand, "block_survivors": n_surv, "link_candidates": n_lcand,
                   "face_pass_setups": n_fsetup, "face_pass_tests": n_ftest,
                   "c_alg_per_step": c_alg, "c_alg_per_level": c_alg_levels},
        "faces_binned_per_s": w.n_faces / (t_bin * 1e-3) if t_bin > 0 else None,
        # algorithmic cell-face tests (C_alg) over the time of all marking kernels of the step
        "cell_face_tests_per_s": c_alg / ((t_refine + t_mark) * 1e-3) if t_refine + t_mark > 0 else None,
        # the tests the kernels ran: block-walk survivors x cells, plus the face-by-face (face, cell) tests
        "executed_cell_face_tests_per_s": n_tests / ((t_refine + t_mark) * 1e-3) if t_refine + t_mark > 0 else None,
        "binning": binning,
        "kernels_ms_per_step": {k: round(v["ms_per_step"], 5) for k, v in kern.items()},
        "wall_s": wall,
        "gpu_launches": int(launches),
        "clocks": clocks,
        "roofline": roof,
    }
    if not args.no_e2e:
        line["e2e"] = run_e2e(w, args, dev)
        line["e2e"]["single_stream"] = run_e2e_single_stream(w, args, dev)
        line["e2e"]["host_link"] = host_link_rates(dev)
    g.close()
    if not args.no_extras and world == 1:
        line["classify"] = run_classify("c2", dev, flush)
    if not args.no_extras and world == 1:
        names = [n for n in ("c3", args.workload) if workload(n).adjoint]
        line["adjoint"] = {n: run_adjoint(n, dev, flush) for n in dict.fromkeys(names)}
        line["per_workload"] = {n: run_device_steps(n, dev, flush, use_graph)
                                for n in ("c1", "c2", "c3", "c4") if n != args.workload}
        line["batched"] = run_batched(args, dev, flush)
        line["paper_setups"] = run_paper_setups(args, dev, flush)
        line["moving"] = run_moving(args, dev, flush)
    return line


def run_device_steps(name, dev, flush, use_graph, steps=10, warmup=3):
    """Device time of the whole step (load, bin, refine with adjacency and links) on another workload:
    CUDA events on the context's stream, L2 flushed between steps (outside the events)."""
    import torch

    from paper_2502_16310_gb300 import AmrGeom
    from synth import workload

    w = workload(name)
    g = AmrGeom(w.dim, (w.root,) * w.dim)
    v = torch.from_numpy(w.verts).to(dev)
    ix = torch.from_numpy(w.idx).to(dev)

    def step():
        g.load(v, ix)
        g.bin(w.bins)
        return g.refine(w.n_levels, w.d_abs, w.d_rel, w.lattice, True, True, use_graph=use_graph)

    for _ in range(warmup):
        res = step()
    torch.cuda.synchronize()
    cells = near_wall_cells(res)
    ms = _timed_steps(step, steps, flush, g.stream)
    g.close()
    return {"workload": f"{name}: {w.description}", "ms_per_step": ms, "near_wall_cells_per_step": cells,
            "cells_per_s": cells / (ms * 1e-3), "steps": steps}


def run_classify(name, dev, flush, reps=5):
    """Node classification of the finest adjacent cells (fluid / solid) and the restriction of the
    links to fluid cells, on the 20,480-triangle sphere: CUDA-event times on the context stream."""
    import torch

    from paper_2502_16310_gb300 import AmrGeom
    from synth import workload

    w = workload(name)
    g = AmrGeom(w.dim, (w.root,) * w.dim)
    verts = torch.from_numpy(w.verts).to(dev)
    idx = torch.from_numpy(w.idx).to(dev)
    g.load(verts, idx)
    g.bin(w.bins)
    res = g.refine(w.n_levels, w.d_abs, w.d_rel, w.lattice, True, True)
    n_links = int(res["link_q"].shape[0])
    st = g.stream
    ms = []
    for k in range(reps):
        flush.fill_(k & 0xff)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        cls, nfb = g.classify()
        b.record(st)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    solid = float(cls.float().mean().item()) if cls.numel() else 0.0
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    out = g.fluid_links()
    b.record(st)
    torch.cuda.synchronize()
    n_fluid = int(out["link_q"].shape[0])
    g.close()
    return {"workload": f"{name}: {w.description}", "cells": int(cls.numel()), "classify_ms": sum(ms) / len(ms),
            "solid_fraction": solid,
            "winding_fallbacks": nfb, "links": n_links, "fluid_links": n_fluid,
            "fluid_links_ms": a.elapsed_time(b),
            "note": "classify/fluid_links times include their host round trip (one read-back each)"}


def run_moving(args, dev, flush, steps=10):
    """Re-adaptation of a moving wall: the c2 sphere translated by a quarter of the finest cell per step;
    each step is load (new vertices) + bin + refine (graph replay, the previous hierarchy kept) + the
    new/old block maps.  CUDA-event time per step and the blocks created / removed on the finest level."""
    import torch

    from paper_2502_16310_gb300 import AmrGeom
    from synth import workload

    w = workload("c2")
    g = AmrGeom(3, (w.root,) * 3)
    idx = torch.from_numpy(w.idx).to(dev)
    h_fin = 1.0 / (4 * w.root * 2 ** (w.n_levels - 1))
    base = torch.from_numpy(w.verts).to(dev)
    delta = torch.tensor([0.25 * h_fin, 0.1 * h_fin, 0.05 * h_fin], device=dev)
    st = g.stream

    def step(k):
        g.load(base + k * delta, idx)
        g.bin(w.bins)
        g.refine(w.n_levels, w.d_abs, w.d_rel, w.lattice, True, True, use_graph=True, keep_previous=True)
        return g.adapt_diff()

    for k in range(3):
        step(k)
    ms, created, removed = [], [], []
    for k in range(3, 3 + steps):
        flush.fill_(k & 0xff)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        d = step(k)
        b.record(st)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
        created.append(d[-1]["created"])
        removed.append(d[-1]["removed"])
    g.close()
    return {"workload": "c2 sphere moving 0.25 h_fin per step", "ms_per_step": sum(ms) / len(ms),
            "finest_created_per_step": sum(created) / len(created),
            "finest_removed_per_step": sum(removed) / len(removed),
            "note": "includes the host read-back of the refine sizes and of the map counts"}


def _timed_steps(fn, n, flush, stream):
    """CUDA-event time (ms) of n calls of fn, L2 flushed before each (outside the events)."""
    import torch

    total = 0.0
    for k in range(n):
        flush.fill_(k & 0xff)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        total += a.elapsed_time(b)
    return total / n


def run_adjoint(name, dev, flush):
    """Adjoint vs forward on a workload with the q adjoint (c3, c4): forward = load + bin + refine with
    links (graph replay); backward = amr_q_backward for seeded random upstream weights (it includes
    regrouping the links by face).  CUDA-event times on the context's stream."""
    import torch

    from paper_2502_16310_gb300 import AmrGeom
    from synth import workload

    w = workload(name)
    g = AmrGeom(3, (w.root,) * 3)
    v = torch.from_numpy(w.verts).to(dev)
    ix = torch.from_numpy(w.idx).to(dev)
    st = g.stream

    def fwd():
        g.load(v, ix)
        g.bin(w.bins)
        return g.refine(w.n_levels, w.d_abs, w.d_rel, 19, True, True, use_graph=True)

    for _ in range(3):
        res = fwd()
    nl = int(res["link_q"].shape[0])
    wts = torch.randn(nl, device=dev, generator=torch.Generator(dev).manual_seed(0))

    def both():
        fwd()
        g.q_backward(wts)

    n = 10 if w.n_faces < 500_000 else 6
    t_f = _timed_steps(fwd, n, flush, st)
    t_fb = _timed_steps(both, n, flush, st)
    g.close()
    t_b = t_fb - t_f
    return {"workload": f"{name}: " + w.description, "links": nl, "forward_ms": t_f, "backward_ms": t_b,
            "adjoint_over_forward": t_b / t_f, "steps": n}


def run_batched(args, dev, flush):
    """The 48-geometry workload: one batched launch per level (graph replay) vs one geometry at a time
    (each with its own context and graph), bin densities and warps per block from the autotuner; forward
    alone, and forward plus the q adjoint (seeded random upstream weights) in both legs."""
    import torch

    from paper_2502_16310_gb300 import AmrBatch, AmrGeom
    from synth import batched_workloads

    t0 = time.perf_counter()
    ws = batched_workloads(args.batch_geoms)
    gen_s = time.perf_counter() - t0
    st = torch.cuda.current_stream()
    data = [(torch.from_numpy(w.verts).to(dev), torch.from_numpy(w.idx).to(dev)) for w in ws]
    # autotune the bin density of every geometry (one-time setup, not timed)
    t0 = time.perf_counter()
    ctxs = []
    for w, (v, ix) in zip(ws, data):
        g = AmrGeom(3, (w.root,) * 3)
        g.load(v, ix)
        B, warps, _ = g.autotune(w.n_levels, w.d_abs, w.d_rel, 19, True, True,
                                 b_candidates=[8, 16, 24, 32, 48, 64, 96, 128], w_candidates=[4])
        w.bins = B
        ctxs.append(g)
    tune_s = time.perf_counter() - t0

    def single():
        out = []
        for w, (v, ix), g in zip(ws, data, ctxs):
            g.load(v, ix)
            g.bin(w.bins)
            out.append(g.refine(w.n_levels, w.d_abs, w.d_rel, 19, True, True, use_graph=True))
        return out

    # one geometry at a time first, then the batch: the two never hold their buffers together
    for _ in range(3):
        res = single()
    gen = torch.Generator(dev).manual_seed(1)
    wts = [torch.randn(int(r["link_q"].shape[0]), device=dev, generator=gen) for r in res]
    wts_all = torch.cat(wts)

    def single_adj():
        single()
        for g, wt in zip(ctxs, wts):
            g.q_backward(wt)

    t_single = _timed_steps(single, 5, flush, st)
    single_adj()  # warm-up: every context's adjoint buffers
    t_single_adj = _timed_steps(single_adj, 5, flush, st)
    for g in ctxs:
        g.close()
    del res
    torch.cuda.synchronize()

    b = AmrBatch(3)
    for w, (v, ix) in zip(ws, data):
        b.add(v, ix, w.root, w.n_levels, w.d_abs, w.d_rel, w.bins)

    def batched():
        b.run(19, True, True, use_graph=True)

    def batched_adj():
        batched()
        b.q_backward(wts_all)

    for _ in range(3):
        batched()
    assert wts_all.numel() == int(b.result.n_links), "batched and single runs differ in their link counts"
    # near-wall cells of the whole set (from the batch's masks)
    r = b.result
    cells = 0
    lut = torch.tensor([bin(i).count("1") for i in range(256)], dtype=torch.int64, device=dev)
    from paper_2502_16310_gb300.binding import _view
    for L in range(r.n_levels):
        n = int(r.n_blocks[L])
        if n:
            m = _view(r.cell_mask[L], (n,), torch.int64)
            cells += int(lut[m.view(torch.uint8).long()].sum().item())
    t_batch = _timed_steps(batched, 5, flush, st)
    batched_adj()  # warm-up: the batch's adjoint buffers
    l0 = b.launch_count()
    t_batch_adj = _timed_steps(batched_adj, 5, flush, st)
    launches_batch = (b.launch_count() - l0) / 5
    b.close()
    return {"workload": f"{len(ws)} SH-perturbed geodesic spheres, {sum(w.n_faces for w in ws)} triangles, "
                        f"roots 16^3..48^3, 2..6 levels, bin density tuned per geometry",
            "near_wall_cells": cells, "links": int(wts_all.numel()),
            "single_ms": t_single, "batched_ms": t_batch,
            "single_cells_per_s": cells / (t_single * 1e-3), "batched_cells_per_s": cells / (t_batch * 1e-3),
            "batched_over_single": t_single / t_batch,
            "single_fwd_adj_ms": t_single_adj, "batched_fwd_adj_ms": t_batch_adj,
            "batched_over_single_fwd_adj": t_single_adj / t_batch_adj,
            "batched_launches_per_fwd_adj": launches_batch, "generate_s": gen_s, "tune_s": tune_s}


def run_paper_setups(args, dev, flush, bins=(1, 2, 4, 6, 7, 8, 9, 10, 12, 14, 16), reps=3):
    """The paper's two speed-up setups (point predicate, absolute d_spec, refined twice) at its bin
    densities, each in two modes: `exact` (AABB bins, every bin the test region overlaps: the marks do
    not depend on B) and `paper` (the paper's sampled bins, face detection in the cell's own bin, then
    1 + floor(d / block length) propagation rounds: the inserted blocks vary with B).  Per B: bin-setup
    and face-detection (marking, with propagation) times and the blocks per level."""
    import torch

    from paper_2502_16310_gb300 import AmrGeom
    from synth import workload

    out = {}
    for name in ("p2", "p3"):
        w = workload(name)
        v = torch.from_numpy(w.verts).to(dev)
        ix = torch.from_numpy(w.idx).to(dev)
        rows = {"workload": w.description, "faces": w.n_faces, "B": list(bins)}
        for mode in ("exact", "paper"):
            g = AmrGeom(w.dim, (w.root,) * w.dim)
            r = {"bin_ms": [], "detect_ms": [], "blocks_per_level": [], "near_wall_cells": []}
            for B in bins:
                def step():
                    g.load(v, ix)
                    if mode == "exact":
                        g.bin(B)
                        return g.refine(w.n_levels, w.d_abs, w.d_rel, 0, False, False, predicate=w.predicate)
                    g.bin(B, sampled=True)
                    return g.refine(w.n_levels, w.d_abs, w.d_rel, 0, False, False, predicate=w.predicate,
                                    search=1, propagate=-1)

                res = step()
                torch.cuda.synchronize()
                g.timing(True)
                g.timing_reset()
                for k in range(reps):
                    flush.fill_(k & 0xff)
                    step()
                torch.cuda.synchronize()
                tk = g.timings()
                g.timing(False)
                t_bin = sum(tk[k][0] for k in ("bin_count", "bin_scan", "bin_scatter") if k in tk) / reps
                t_det = sum(tk[k][0] for k in ("refine_level", "propagate", "mark_faces")
                            if k in tk) / reps
                r["bin_ms"].append(round(t_bin, 4))
                r["detect_ms"].append(round(t_det, 4))
                r["blocks_per_level"].append([int(lv["blocks"].shape[0]) for lv in res["levels"]])
                r["near_wall_cells"].append(near_wall_cells(res))
            g.close()
            rows[mode] = r
        out[name] = rows
    return out


def roofline(name, k, w, kern, n_cand, n_surv, n_adj, n_pairs, blocks, clocks, n_fsetup=0, n_ftest=0):
    """Roofline entry for the dominant kernel: algorithmic work per launch / average launch time."""
    hbm, src = measured_peaks()
    launches = max(k["launches_per_step"], 1e-9)
    t = k["ms_per_step"] / launches * 1e-3
    NC = 64 if w.dim == 3 else 16
    alu_peak = N_SM * FP32_LANES_PER_SM * SM_MAX_MHZ * 1e6 / 1e12  # FP32-pipe Tops/s at the max SM clock
    if name == "refine_level":
        # deduplicated candidates set up against the walked box (a parent group's on the levels below the
        # roots) and the cell tests of every (face, block) pair that passed the culls; the rest of the
        # survivors' setups and the child culls are left out (a lower bound)
        ops = (n_cand * OPS_BLOCK_CANDIDATE + n_surv * NC * OPS_CELL_TEST) / launches
        a = ops / t / 1e12
        return {"kernel": name, "bound": "alu", "achieved": a, "peak": alu_peak, "unit": "Tops/s (FP32 pipe)",
                "frac": a / alu_peak, "traffic": None, "peak_source": "152 SM x 128 FP32 lanes x 2070 MHz"}
    if name == "mark_faces":
        ops = (n_fsetup * OPS_FACE_SETUP + n_ftest * OPS_CELL_TEST) / launches
        a = ops / t / 1e12
        return {"kernel": name, "bound": "alu", "achieved": a, "peak": alu_peak, "unit": "Tops/s (FP32 pipe)",
                "frac": a / alu_peak, "traffic": None, "peak_source": "152 SM x 128 FP32 lanes x 2070 MHz"}
    if name == "links":
        # algorithmic work: one ~40-op watertight test per (adjacent cell, adjacent face, lattice direction)
        Q1 = 18 if w.dim == 3 else 8
        ops = n_pairs * Q1 * OPS_LINK_DIR / launches
        a = ops / t / 1e12
        ex = n_pairs * (OPS_LINK_FACE + Q1 * OPS_LINK_DIR) / launches / t / 1e12
        return {"kernel": name, "bound": "alu", "achieved": a, "peak": alu_peak, "unit": "Tops/s (FP32 pipe)",
                "frac": a / alu_peak, "traffic": None, "peak_source": "152 SM x 128 FP32 lanes x 2070 MHz",
                "ops_per_launch": ops, "with_per_pair_setup_tops": ex}
    if name == "adjacency":
        ops = n_surv * NC * OPS_CELL_TEST / launches
        a = ops / t / 1e12
        return {"kernel": name, "bound": "alu", "achieved": a, "peak": alu_peak, "unit": "Tops/s (FP32 pipe)",
                "frac": a / alu_peak, "traffic": None, "peak_source": "152 SM x 128 FP32 lanes x 2070 MHz"}
    # HBM-bound kernels: algorithmic bytes
    nb = w.bins ** w.dim
    D = w.dim
    byts = {"bin_count": w.n_faces * (4 * D * D + 4 * D) + 8.0 * nb,
            "bin_scan": 8.0 * nb,
            "bin_scatter": w.n_faces * (4 * D * D + 4 * D)}.get(name, 0.0) / launches
    a = byts / t / 1e9
    return {"kernel": name, "bound": "hbm", "achieved": a, "peak": hbm, "unit": "GB/s", "frac": a / hbm,
            "traffic": None, "peak_source": src}


def bin_method_bytes(D, n_faces, n_bins, nnz):
    """Algorithmic bytes of the binning as the method defines them: the face coordinates read by the
    count and scatter passes (2 x 4 D^2 per face), the bin counters zeroed, counted, scanned and read as
    offsets (16 bytes per bin), and per (face, bin) incidence its 4-byte id and its coordinates (4 D^2)."""
    return 2 * 4 * D * D * n_faces + 16 * n_bins + (4 + 4 * D * D) * nnz


def bin_impl_bytes(D, n_faces, n_bins, nnz):
    """Bytes the implementation moves on purpose: the method's bytes with the per-face bin range written and
    read back (2 x 4 D) and the full payload entry (64 bytes in 3D, 32 in 2D: coordinates, FP32 normal, id
    with flags, bin coordinates) in place of the bare coordinates."""
    entry = 64 if D == 3 else 32
    return 2 * 4 * D * D * n_faces + 2 * 4 * D * n_faces + 16 * n_bins + (4 + entry) * nnz


def bin_roofline(w, nnz, t_bin_ms):
    """HBM roofline of the binning kernels (count, scan, scatter) together.  `frac` counts the method's
    algorithmic bytes (bin_method_bytes); the implementation's larger figure is reported beside it."""
    hbm, src = measured_peaks()
    D = w.dim
    nb = w.bins ** D
    byts = bin_method_bytes(D, w.n_faces, nb, nnz)
    impl = bin_impl_bytes(D, w.n_faces, nb, nnz)
    t = t_bin_ms * 1e-3
    a = byts / t / 1e9 if t > 0 else 0.0
    ai = impl / t / 1e9 if t > 0 else 0.0
    return {"kernels": ["bin_count", "bin_scan", "bin_scatter"], "bound": "hbm", "faces_per_s": w.n_faces / t,
            "incidences": nnz, "bytes": byts, "achieved": a, "peak": hbm, "unit": "GB/s", "frac": a / hbm,
            "peak_source": src, "ms": t_bin_ms,
            "impl_bytes": impl, "impl_achieved": ai, "impl_frac": ai / hbm}


def run_bin_only(args, local):
    """Binning alone on the workload's geometry: per step the three binning kernels (count, scan,
    scatter), each timed by the library with CUDA events on its stream, L2 flushed between steps.  The
    device holds only the geometry and the bins, so this is also the small case for kernel captures of
    the binning."""
    import torch

    from paper_2502_16310_gb300 import AmrGeom
    from paper_2502_16310_gb300 import binding as Bd
    from synth import workload

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = workload(args.workload)
    g = AmrGeom(w.dim, (w.root,) * w.dim)
    g.load(torch.from_numpy(w.verts).to(dev), torch.from_numpy(w.idx).to(dev))
    for _ in range(max(args.warmup, 1)):
        nnz = int(g.bin(w.bins)["nnz"])
    torch.cuda.synchronize()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    sampler = ClockSampler(local if "CUDA_VISIBLE_DEVICES" not in os.environ else 0)
    g.timing(True)
    g.timing_reset()
    sampler.start()
    l0 = Bd.amr_launch_count(g.ctx)
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        g.bin(w.bins)
    torch.cuda.synchronize()
    launches = Bd.amr_launch_count(g.ctx) - l0
    clocks = sampler.stop()
    tk = g.timings()
    g.timing(False)
    names = ("bin_count", "bin_scan", "bin_scatter")
    kern = {k: tk[k][0] / args.steps for k in names if k in tk}
    t_bin = sum(kern.values())
    g.close()
    binning = bin_roofline(w, nnz, t_bin)
    return {"metric": "faces binned/s", "value": w.n_faces / (t_bin * 1e-3), "unit": "faces/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_bin, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {w.description}",
                       "faces": w.n_faces, "bins_per_axis": w.bins, "incidences": nnz,
                       "l2": "flushed between steps (512 MB write)"},
            "kernels_ms_per_step": {k: round(v, 5) for k, v in kern.items()},
            "roofline": binning, "clocks": clocks, "gpu_launches": int(launches)}


def e2e_layout(d2h_bytes, threads_arg):
    """(host threads, contexts per thread) of the e2e leg: as asked, else three threads with one
    context each for steps that copy back less than 2 GB, one thread alternating two contexts for
    larger ones."""
    if threads_arg > 0:
        return threads_arg, 1
    return (1, 2) if d2h_bytes >= 2e9 else (3, 1)


def run_e2e(w, args, dev):
    """Same metric through the public API with host buffers: every step uploads its inputs from pinned
    host memory (inside amr_geom_load) and copies every output back to pinned host memory, as a user
    streaming results to the host would run it.  Steps that copy back less than 2 GB: a few host
    threads, each with its own context and stream, take the steps in turn; one thread's uploads,
    host-side calls and copies overlap the others' GPU work, and their kernels share the GPU.  Steps
    that copy back more are long and bound by the copies: one host thread alternates two contexts, so
    a step's copies overlap the next step's compute without a third step's kernels and pinned output
    competing for the GPU and the host link.  Host wall clock from the start of the timed steps to the
    end of the last step's copies."""
    import threading

    import torch

    from paper_2502_16310_gb300 import AmrGeom

    hv = torch.from_numpy(w.verts).pin_memory()
    hi = torch.from_numpy(w.idx).pin_memory()
    bi = hv.numel() * 4 + hi.numel() * 4
    use_graph = not args.no_graph
    out = {}

    def new_slot():
        with torch.cuda.stream(torch.cuda.Stream(device=dev)):
            return [AmrGeom(w.dim, (w.root,) * w.dim), {}]

    def step(slot, i):
        g, out_bufs = slot
        g.load(hv, hi)
        g.bin(w.bins)
        res = g.refine(w.n_levels, w.d_abs, w.d_rel, w.lattice, True, True, use_graph=use_graph)
        nbytes = 0
        tensors = []
        for L, lv in enumerate(res["levels"]):
            tensors += [lv["blocks"], lv["mask"]]
        tensors += [res["adj_cell"], res["adj_off"], res["adj_ids"], res["link_cell"], res["link_dir"],
                    res["link_q"], res["link_face"]]
        with torch.cuda.stream(g.stream):  # the outputs' stream: ordered after the refinement
            for j, t in enumerate(tensors):
                buf = out_bufs.get(j)
                if buf is None or buf.numel() < t.numel() or buf.dtype != t.dtype:
                    buf = torch.empty(t.numel() + t.numel() // 8 + 1024, dtype=t.dtype).pin_memory()
                    out_bufs[j] = buf
                buf[:t.numel()].copy_(t.reshape(-1), non_blocking=True)
                nbytes += t.numel() * t.element_size()
        out[i] = (res, nbytes)

    # one untimed step gives the bytes a step copies back
    first = new_slot()
    step(first, 0)
    torch.cuda.synchronize()
    NT, NC = e2e_layout(out[0][1], args.e2e_threads)
    slots = [[first if i == 0 and c == 0 else new_slot() for c in range(NC)] for i in range(NT)]
    errors = []

    def worker(i, n, go):
        try:
            torch.cuda.set_device(dev)
            go.wait()
            for k in range(n):
                step(slots[i][k % NC], i)
        except Exception as e:  # surfaced by the main thread
            errors.append(e)

    def run_threads(n_each):
        go = threading.Event()
        th = [threading.Thread(target=worker, args=(i, n_each, go)) for i in range(NT)]
        for t in th:
            t.start()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        go.set()
        for t in th:
            t.join()
        torch.cuda.synchronize()
        if errors:
            raise errors[0]
        return time.perf_counter() - t0

    run_threads(NC * max(2, args.warmup))  # warm-up: allocations, graph captures, pinned buffers
    K = NT * NC * max(2, args.steps // (NT * NC))
    dt = run_threads(K // NT) / K
    res, bo = out[0]
    cells = near_wall_cells(res)
    for per_thread in slots:
        for g, _ in per_thread:
            g.close()
    return {"value": cells / dt, "unit": UNIT, "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo,
            "ms_per_step": dt * 1e3, "level_loop": "CUDA graph replay" if use_graph else "eager",
            "threads": NT, "contexts_per_thread": NC, "steps": K,
            "note": f"host wall clock over K steps: load(pinned host) -> bin -> refine -> D2H of every output to "
                    f"pinned host; {NT} host thread(s), each taking its steps in turn on {NC} context(s) with "
                    f"a stream each, so steps overlap on the GPU (the device-side value times one stream)"}


def host_link_rates(dev, nbytes=1 << 30, reps=3):
    """Device-to-pinned-host and pinned-host-to-device copy rates of this machine (one stream, best of a few
    1 GiB copies): the host link the e2e copies run over, which varies between boxes."""
    import torch

    d = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    h = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    out = {}
    for name, dst, src in (("d2h_gbps", h, d), ("h2d_gbps", d, h)):
        best = float("inf")
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            dst.copy_(src, non_blocking=True)
            torch.cuda.synchronize()
            best = min(best, time.perf_counter() - t0)
        out[name] = nbytes / best / 1e9
    del d, h
    return out


def run_e2e_single_stream(w, args, dev):
    """End-to-end latency of one step at a time through the public API: one context, one stream, one host
    thread; each step uploads its inputs from pinned host memory (inside amr_geom_load), bins, refines and
    copies every output back to pinned host memory, and the host waits for the copies before the next step
    starts.  Host wall clock per step (median and mean)."""
    import torch

    from paper_2502_16310_gb300 import AmrGeom

    hv = torch.from_numpy(w.verts).pin_memory()
    hi = torch.from_numpy(w.idx).pin_memory()
    use_graph = not args.no_graph
    with torch.cuda.stream(torch.cuda.Stream(device=dev)):
        g = AmrGeom(w.dim, (w.root,) * w.dim)
    bufs = {}

    def step():
        g.load(hv, hi)
        g.bin(w.bins)
        res = g.refine(w.n_levels, w.d_abs, w.d_rel, w.lattice, True, True, use_graph=use_graph)
        tensors = []
        for lv in res["levels"]:
            tensors += [lv["blocks"], lv["mask"]]
        tensors += [res["adj_cell"], res["adj_off"], res["adj_ids"], res["link_cell"], res["link_dir"],
                    res["link_q"], res["link_face"]]
        nbytes = 0
        with torch.cuda.stream(g.stream):
            for j, t in enumerate(tensors):
                buf = bufs.get(j)
                if buf is None or buf.numel() < t.numel() or buf.dtype != t.dtype:
                    buf = torch.empty(t.numel() + t.numel() // 8 + 1024, dtype=t.dtype).pin_memory()
                    bufs[j] = buf
                buf[:t.numel()].copy_(t.reshape(-1), non_blocking=True)
                nbytes += t.numel() * t.element_size()
        g.stream.synchronize()
        return nbytes

    for _ in range(max(2, min(args.warmup, 3))):
        step()
    ts = []
    n = max(3, min(args.steps, 10))
    for _ in range(n):
        t0 = time.perf_counter()
        bo = step()
        ts.append(time.perf_counter() - t0)
    g.close()
    ts.sort()
    return {"ms_median": ts[len(ts) // 2] * 1e3, "ms_mean": sum(ts) / len(ts) * 1e3, "steps": n,
            "d2h_bytes_per_step": bo,
            "note": "one context, one stream, one host thread: each step's copies end before the next step starts"}


# ---------------------------------------------------------------------------
# the oracle on the host (CPU baseline and the reference arm)
# ---------------------------------------------------------------------------
def oracle_sampled_step(w, frac0, rng, max_blocks=400, max_cells=400):
    """One oracle pass over a seeded subtree sample of the workload.

    Level 0: a random fraction `frac0` of the roots.  Deeper levels: the
    children of the sampled marked blocks, subsampled to at most `max_blocks`.
    The finest level's adjacency and links run on at most `max_cells` sampled
    adjacent cells.  Every time and count is scaled by the inverse inclusion
    probability, giving an estimate for the whole workload.
    Returns (estimated seconds, estimated near-wall cells, cpu seconds spent).
    """
    import numpy as np

    from oracle.oracle import Domain, OracleGeometry, cells_of_mask, root_blocks

    t_start = time.process_time()
    geo = OracleGeometry(w.dim, w.verts, w.idx)
    t0 = time.perf_counter()
    geo.bin(Domain.unit(w.dim, w.root), w.bins)
    est_t = time.perf_counter() - t0
    blocks = root_blocks(w.dim, (w.root,) * w.dim)
    sel = rng.random(blocks.shape[0]) < frac0
    blocks = blocks[sel]
    weight = 1.0 / frac0
    est_cells = 0.0
    for L in range(w.n_levels):
        if blocks.shape[0] > max_blocks:
            keep = rng.choice(blocks.shape[0], size=max_blocks, replace=False)
            weight *= blocks.shape[0] / max_blocks
            blocks = blocks[np.sort(keep)]
        t0 = time.perf_counter()
        mask, _, _, _ = geo.refine_blocks(L, blocks, w.d_abs, w.d_rel)
        est_t += (time.perf_counter() - t0) * weight
        est_cells += sum(bin(int(m)).count("1") for m in mask) * weight
        if L + 1 < w.n_levels:
            blocks, _ = geo.children(blocks, mask)
    _, _, cells = cells_of_mask(w.dim, blocks, mask)
    if cells.shape[0]:
        cw = weight
        if cells.shape[0] > max_cells:
            cw *= cells.shape[0] / max_cells
            cells = cells[rng.choice(cells.shape[0], size=max_cells, replace=False)]
        t0 = time.perf_counter()
        geo.cell_faces(w.n_levels - 1, cells, w.d_abs, w.d_rel)
        geo.cell_links(w.n_levels - 1, w.lattice, cells)
        est_t += (time.perf_counter() - t0) * cw
    return est_t, est_cells, time.process_time() - t_start


def host_cpu():
    """(CPU model, logical cores) of this host."""
    model = None
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    if model is None:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.startswith("Model name:"):
                    model = line.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    return model or "unknown", os.cpu_count() or 1


def _oracle_worker(job):
    """One host process of the all-cores oracle run: seeded subtree samples until `seconds` of CPU time."""
    w, seed, seconds = job
    import numpy as np

    import oracle

    oracle.build()
    rng = np.random.default_rng(seed)
    frac, spent, ts, cs = 1.0 / 64, 0.0, [], []
    while spent < seconds:
        et, ec, cpu = oracle_sampled_step(w, frac, rng)
        spent += cpu
        ts.append(et)
        cs.append(ec)
    return ts, cs, spent


def run_cpu_baseline_all_cores(w, seconds):
    """The oracle as it stands on every host core at once: one process per core (spawned), each timing its
    own seeded subtree samples of the workload while all the others run.  The whole workload splits over
    blocks with no exchange, so the all-cores throughput is the sum of the per-process throughputs measured
    under that load."""
    import multiprocessing as mp

    model, ncpu = host_cpu()
    oracle_build()
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(ncpu) as pool:
        res = pool.map(_oracle_worker, [(w, 1000 + i, seconds) for i in range(ncpu)])
    wall = time.perf_counter() - t0
    value = sum((sum(cs) / len(cs)) / (sum(ts) / len(ts)) for ts, cs, _ in res)
    n = sum(len(ts) for ts, _, _ in res)
    return {"value": value, "unit": UNIT, "cores": ncpu, "cpu_model": model, "kind": "oracle",
            "sample": (f"{ncpu} spawned processes, {n} seeded subtree samples of {w.name} in all (1/64 of the "
                       f"roots, <=400 blocks per level, <=400 finest adjacent cells each), times and counts scaled "
                       f"to the full workload; value = sum of the per-process throughputs under full load; "
                       f"{wall:.1f} s wall")}


def oracle_build():
    import oracle

    oracle.build()


def run_cpu_baseline(w, seconds):
    import numpy as np

    import oracle

    oracle.build()
    rng = np.random.default_rng(7)
    # grow the sample until it costs a few seconds, then repeat to fill the budget
    frac, spent, est_ts, est_cs = 1.0 / 256, 0.0, [], []
    while spent < seconds:
        et, ec, cpu = oracle_sampled_step(w, frac, rng)
        spent += cpu
        est_ts.append(et)
        est_cs.append(ec)
        if cpu < 1.0 and frac < 1.0 / 8:
            frac *= 2
    et, ec = float(np.mean(est_ts)), float(np.mean(est_cs))
    model, ncpu = host_cpu()
    return {"value": ec / et, "unit": UNIT, "cores": 1, "kind": "oracle", "cpu_model": model, "nproc": ncpu,
            "sample": (f"{len(est_ts)} seeded subtree samples of {w.name} (roots sampled at up to 1/8, <=400 "
                       f"blocks per level, <=400 finest adjacent cells for faces+links), times and counts scaled "
                       f"by inverse inclusion probability; {spent:.1f} s CPU"),
            "est_full_seconds": et, "est_near_wall_cells": ec}


def run_reference(args, rank, world):
    import numpy as np

    from synth import workload

    if rank != 0:
        return None
    import oracle

    oracle.build()
    w = workload(args.workload)
    rng = np.random.default_rng(11)
    frac = 1.0 / 64
    for _ in range(args.warmup):
        oracle_sampled_step(w, frac, rng)
    ts, cs, cpu = [], [], 0.0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        et, ec, c = oracle_sampled_step(w, frac, rng)
        ts.append(et)
        cs.append(ec)
        cpu += c
    wall = time.perf_counter() - t0
    value = float(np.mean(cs)) / float(np.mean(ts))
    sample = (f"each step: seeded subtree sample of {w.name} (1/64 of roots, <=400 blocks per level, <=400 finest "
              f"adjacent cells), oracle times scaled to the full workload")
    return {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": float(np.mean(ts)) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {w.description}"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                             "cpu_model": host_cpu()[0], "nproc": host_cpu()[1]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": wall}


def main(argv=None):
    args = parse_args(argv)
    rank, world, local = dist_env()
    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line), flush=True)
        return 0
    import torch

    if world > 1:
        torch.cuda.set_device(local)
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    if args.bin_only:
        if rank == 0:
            print(json.dumps(run_bin_only(args, local)), flush=True)
        return 0
    line = run_ours(args, rank, world, local)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from synth import workload

        wl = workload(args.workload)
        line["cpu_baseline"] = run_cpu_baseline(wl, args.cpu_seconds)
        if not args.no_all_cores:
            line["cpu_baseline"]["all_cores"] = run_cpu_baseline_all_cores(wl, args.cpu_seconds)
    if world > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
