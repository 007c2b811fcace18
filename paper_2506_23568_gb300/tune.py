"""Autotuner of the plan parameters (leaf size, lattice density, interpolation taps).

The paper leaves the factorisation depth and the sampling free and couples them to cost
(Sec. IV-B): the operation count is
    N_ops = C1 N_A N_f log2 N_f + C2 sum_leaves N_SA N_s,leaf + 2 C3 sum_merged-nodes N_s
(Eqs. eq4_nopsbpa, eq4_nopsinterp, eq4_nopstotal), with N_s the samples of each compressed
subimage.  The tuner evaluates these terms exactly for every candidate from a host-only plan
(its lattices and leaf memberships; no device work), turns them into a predicted time with
per-term costs calibrated on the device, times the few cheapest candidates, and accepts a
candidate only when its image stays within the accuracy bar of direct BPA (NRMSE in dB over
every k-th z-slab of the grid).  The interpolation term counts one interpolation per parent
sample and child (F children per node), with a per-tap cost (taps^3 multiply-adds).
"""
from __future__ import annotations

import math
import statistics

import numpy as np

DEFAULT_CANDIDATES = [dict(leaf_size=l, eta=e, taps=6) for l in (64, 128, 256, 512) for e in (1.5, 1.6, 1.75, 2.0)]
# per-term device costs (ns): range compression per N_f log2 N_f unit, leaf update per (member,
# lattice sample), interpolation per (parent sample, child) and tap^3; calibrated by calibrate()
DEFAULT_COEFFS = {"c1": 0.004, "c2": 0.0007, "c3": 0.00008}


def op_counts(traj, freqs, grid, **cfg):
    """The operation-count terms of Eq. eq4_nopstotal for one plan configuration, from the host
    planner alone: rc = N_A N_f log2 N_f, leaf = sum over leaves of members x lattice samples,
    interp = sum over merged nodes of lattice samples (voxels for the root) x children."""
    from . import Plan

    ex = Plan(traj, freqs, grid, host_only=True, **cfg).export()
    ls = ex["level_start"]
    n_a, n_f = len(traj), len(freqs)
    sizes = np.prod(ex["N"].astype(np.float64), axis=1)
    leaf = slice(ls[0], ls[1])
    leaf_updates = float(((ex["end"][leaf] - ex["begin"][leaf]) * sizes[leaf]).sum())
    interp = 0.0
    for lv in range(1, len(ls) - 1):
        nodes = slice(ls[lv], ls[lv + 1])
        if lv == len(ls) - 2:  # the root: its children are interpolated at every voxel
            interp += float(grid.nx * grid.ny * grid.nz) * float(ex["nchild"][ls[lv]])
        else:
            interp += float((sizes[nodes] * ex["nchild"][nodes]).sum())
    return {"rc": n_a * n_f * math.log2(n_f), "leaf": leaf_updates, "interp": interp, "levels": len(ls) - 1}


def predicted_ms(counts, taps, coeffs=None):
    c = coeffs or DEFAULT_COEFFS
    return 1e-6 * (c["c1"] * counts["rc"] + c["c2"] * counts["leaf"] + c["c3"] * taps ** 3 * counts["interp"])


def calibrate(traj, freqs, grid, echo, cfg=None):
    """Per-term costs from the stage times of one profiled image (median of three)."""
    from . import Plan

    cfg = cfg or dict(leaf_size=256, eta=1.6, taps=6)
    counts = op_counts(traj, freqs, grid, **cfg)
    plan = Plan(traj, freqs, grid, **cfg)
    plan.profile(True)
    runs = []
    for _ in range(4):
        plan.form_image(echo)
        runs.append(plan.stage_times())
    runs = runs[1:]
    agg = {}
    for name in ("range_compression", "leaf_subimages", "merge", "final", "need_final", "need_level"):
        agg[name] = statistics.median(sum(ms for n, _, ms in r if n == name) for r in runs)
    plan.close()
    interp_ms = agg["merge"] + agg["final"] + agg["need_final"] + agg["need_level"]
    return {"c1": 1e6 * agg["range_compression"] / counts["rc"],
            "c2": 1e6 * agg["leaf_subimages"] / max(counts["leaf"], 1.0),
            "c3": 1e6 * interp_ms / max(counts["interp"] * cfg["taps"] ** 3, 1.0)}


def _timed_ms(fn, reps=3):
    import torch

    fn()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def bpa_slabs(traj, freqs, grid, echo, every=8):
    """GPU direct BPA on every `every`-th z-slab of the grid (host complex64 array)."""
    import torch

    from . import bpa_form_image

    g = grid
    sub = g.__class__(g.x0, g.y0, g.z0, g.dx, g.dy, g.dz * every, g.nx, g.ny, (g.nz + every - 1) // every)
    ref = bpa_form_image(traj, freqs, sub, echo)
    torch.cuda.synchronize()
    return ref.cpu().numpy()


def accuracy_db(traj, freqs, grid, echo, image, every=8, ref=None):
    """NRMSE (dB) of an image against GPU direct BPA over every `every`-th z-slab of the grid
    (ref: those slabs, when already imaged)."""
    from .metrics import nrmse_db

    if ref is None:
        ref = bpa_slabs(traj, freqs, grid, echo, every)
    return nrmse_db(image[::every].cpu().numpy(), ref)


def tune(traj, freqs, grid, echo, target_db=-30.0, candidates=None, top=4, coeffs=None, every=8):
    """Pick plan parameters for one scan: rank the candidates by the operation-count model,
    time the `top` cheapest (plan + image, CUDA events), and return the fastest whose image is
    within target_db of direct BPA (over every `every`-th z-slab), with the table of what was
    tried.  When none qualifies, the most accurate one is returned and flagged."""
    from . import Plan

    cands = candidates or DEFAULT_CANDIDATES
    ranked = sorted(({**c, "predicted_ms": predicted_ms(op_counts(traj, freqs, grid, **c), c.get("taps", 6), coeffs)}
                     for c in cands), key=lambda r: r["predicted_ms"])
    ref = bpa_slabs(traj, freqs, grid, echo, every)
    tried = []
    for r in ranked[:top]:
        cfg = {k: v for k, v in r.items() if k != "predicted_ms"}
        holder = {}

        def run():
            holder["plan"] = Plan(traj, freqs, grid, **cfg)
            holder["img"] = holder["plan"].form_image(echo)

        ms = _timed_ms(run)
        db = accuracy_db(traj, freqs, grid, echo, holder["img"], every, ref)
        holder["plan"].close()
        tried.append({**r, "measured_ms": ms, "nrmse_db": db, "accepted": db <= target_db})
    ok = [t for t in tried if t["accepted"]]
    best = min(ok, key=lambda t: t["measured_ms"]) if ok else min(tried, key=lambda t: t["nrmse_db"])
    cfg = {k: v for k, v in best.items() if k in ("leaf_size", "eta", "taps", "merge_factor")}
    return {"config": cfg, "accepted": bool(ok), "tried": tried}
