"""Benchmark: seconds per volume of GPU HHFFBPA vs GPU direct BPA (same GB300),
with NRMSE between them, roofline fractions and the FP64 oracle as CPU baseline.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload large] [--impl reference]

One step = one pass of the whole hot path over one synthetic scan already
resident in HBM: plan (tree + sampling grids, per scan), HHFFBPA image (range
compression, demand passes, level-1 subimages, merges, final level), the
direct-BPA image of the same scan, and the NRMSE between them.  `value` is the
HHFFBPA seconds per volume (plan included) for the whole job.  Under torchrun
each rank images its own scan (weak scaling, no collective on the data path);
`value` = the slowest rank's mean HHFFBPA time per step (plan included) / ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "s/volume HHFFBPA vs direct BPA on same GPU at ≤-30 dB NRMSE; % of roofline"
WORKLOADS = {
    "large": "large: 65,536 positions (random-walk raster 0.5x0.5 m, +/-5 mm z), 512 freqs 76-81 GHz, "
             "256 point scatterers, 512x512x128 grid (0.98 x 0.98 x 1.5625 mm), FP32 bulk / FP64 references",
    "mid": "mid: 16,384 positions (zig-zag 0.4x0.4 m, sigma 3 mm), 256 freqs, 64 points + 4 plates, "
           "256x256x64 grid, SNR 20 dB",
    "tiny": "tiny: 2,048 positions, 128 freqs, 8 points, 64x64x16 grid",
    "sim1": "sim1 (shaped as the paper's point-scatterer simulation): 101 x 101 positions of a linear array "
            "scanned with position/angle fluctuations (depth within 8 cm), 24 freqs 12-15 GHz, 3x3x3 points at "
            "0.175 m pitch centred 0.4 m deep, 101x101x51 grid over 0.5 m^3",
}
# Plan per workload: the autotuner's choice (paper_2506_23568_gb300.tune: the Sec. IV-B
# operation count ranks the candidates, every candidate of a 16-point grid is timed, acceptance
# at NRMSE <= -32 dB against direct BPA over every 8th z-slab).  Large: leaf 1024, eta 1.5,
# 6 taps (-34.1 dB, 51.1 ms plan + image in the sweep; leaf 256 eta 1.5: -33.1 dB, 52.0 ms;
# eta 1.4 misses the bar; no 4-tap plan reached -32 dB at a lower cost).  Mid: leaf 1024,
# eta 1.5 (-36.1 dB, 15.6 ms; leaf 512 eta 1.5: -34.9 dB, 16.1 ms).
PLAN_CFG = {"large": dict(leaf_size=1024, eta=1.5), "mid": dict(leaf_size=1024, eta=1.5),
            "tiny": dict(leaf_size=32), "sim1": dict(leaf_size=32)}
# the paper's Table II (Sim I, one CPU core; BPA / HHFFBPA), quoted as context only
PAPER_SIM1 = {"speedup_hhffbpa_vs_bpa": 62.09, "psnr_hhffbpa_vs_bpa_db": 45.98,
              "centre_psf": {"bpa": [9.68, -12.77, -9.91], "hhffbpa": [9.68, -13.04, -10.63]},
              "squint_psf": {"bpa": [11.55, -12.28, -9.90], "hhffbpa": [11.70, -12.15, -9.99]},
              "psf_fields": ["mainlobe width mm", "PSLR dB", "ISLR dB"],
              "hardware": "one core of a 4.5 GHz Ryzen 9 7950X, C++ without parallelisation"}

# DRAM bytes (read + write) per evaluated sample of a stage's kernel, from an ncu capture of
# one launch on the mid workload in its benchmark plan (leaf 1024, eta 1.5: the large
# workload's leaf size; dram__bytes_read.sum + dram__bytes_write.sum = 44.7 MB + 45.3 MB for
# 5,713,647 evaluated leaf samples; profiles/k_stage0_mid.md), scaled to a launch by the
# samples it evaluates; keyed by the kernel revision, null for other kernels.
TRAFFIC_PER_SAMPLE = {("leaf_subimages", "paired two-sample loop, tile table, floor(256/npair) member groups"):
                      (44679936 + 45312512) / 5713647}
STAGE0_REVISION = "paired two-sample loop, tile table, floor(256/npair) member groups"

# Algorithmic work per unit: a BPA-type update (one position at one point) takes one
# rsqrt and one sincos (3 MUFU results) and about 25 FP32 operations
BPA_FLOP, BPA_MUFU = 25.0, 3.0            # per (voxel, position) update
MUFU_PER_SM_CLK = 16.0                    # SFU results per SM per clock (sm_100-class)
FP32_PER_SM_CLK = 256.0                   # 128 FMA lanes x 2 FLOP
SMEM_B_PER_SM_CLK = 128.0                 # shared-memory bytes per SM per clock (one wavefront)


def _peaks():
    p = {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "source": "fallback"}
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        m = json.load(open(path))
        p.update(hbm_gbs=float(m.get("hbm_gbs", p["hbm_gbs"])), sm_max_mhz=float(m.get("sm_max_mhz", 2070.0)),
                 source="measured")
    return p


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _scene(name, rank):
    import synth

    s = synth.CONFIGS[name]()
    if rank:  # independent scans per rank: same recipe, shifted trajectory seed
        rng = np.random.default_rng(5000 + rank)
        s.traj = s.traj + np.column_stack([rng.normal(0, 1e-4, len(s.traj)), rng.normal(0, 1e-4, len(s.traj)),
                                           np.zeros(len(s.traj))])
    return s


def reduce_over_ranks(dist, values, device):
    """Max over ranks of each timing (the slowest rank sets the job's time); identity
    without a process group."""
    if dist is None:
        return list(values)
    import torch

    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def per_volume_s(job_ms, ranks):
    """Whole-job seconds per volume: every rank images one volume per step, so the job's
    time per step is shared by `ranks` volumes."""
    return job_ms / 1e3 / ranks


def sm_count():
    """Streaming multiprocessors of the current device (152 on a GB300)."""
    import torch

    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def roofline_of(kind, ms, units, peaks, clk_mhz):
    """(achieved, peak, unit, bound, frac) for a kernel from its algorithmic work."""
    f = clk_mhz * 1e6
    sms = sm_count()
    if kind == "mufu":  # units = MUFU operations; the measured rate where there is one
        peak = peaks.get("mufu_tps") or MUFU_PER_SM_CLK * sms * f
        ach = units / (ms * 1e-3)
        return ach / 1e12, peak / 1e12, "TMUFU/s", "alu", ach / peak
    if kind == "fp32":  # units = FLOP
        peak = FP32_PER_SM_CLK * sms * f
        ach = units / (ms * 1e-3)
        return ach / 1e12, peak / 1e12, "TFLOP/s", "alu", ach / peak
    if kind == "hbm":  # units = bytes
        peak = peaks["hbm_gbs"] * 1e9
        ach = units / (ms * 1e-3)
        return ach / 1e9, peak / 1e9, "GB/s", "hbm", ach / peak
    raise ValueError(kind)


def kernel_work(stages, plan, info, levels, cnt, grid, n_pos, n_f, taps):
    """Algorithmic work per stage: FP32 FLOP, MUFU ops, HBM bytes (paper's cost model terms)."""
    out = []
    n_fft = info["n_fft"]
    for name, lev, ms in stages:
        flop = mufu = byts = 0.0
        if name == "range_compression":
            flop = 5.0 * n_fft * math.log2(n_fft) * n_pos
            byts = 8.0 * n_pos * (n_f + info["gate_bins"])
        elif name == "leaf_subimages":
            upd = plan["leaf_members_avg"] * levels[0]
            flop, mufu = BPA_FLOP * upd, BPA_MUFU * upd
            byts = 8.0 * levels[0] + 8.0 * n_pos * info["gate_bins"]
        elif name in ("merge", "final"):
            nch = plan["nchild"][lev]
            interp = levels[lev] * nch
            flop = interp * (4.0 * taps ** 3 + 100.0)
            mufu = interp * 11.0
            byts = 8.0 * levels[lev] + 8.0 * levels[lev - 1]
        # shared-memory reads of the separable interpolation: taps^3 complex64 samples per
        # (sample, child); not part of the FP32 / MUFU / HBM roofline, reported beside it
        smem = 8.0 * taps ** 3 * levels[lev] * plan["nchild"][lev] if name in ("merge", "final") else 0.0
        out.append(dict(stage=name, level=lev, ms=ms, flop=flop, mufu=mufu, bytes=byts, smem=smem))
    return out


def run_gpu(args):
    import torch

    import paper_2506_23568_gb300 as hh
    import synth

    ws, rank, local = _dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    peaks = _peaks()
    wl = args.workload
    s = _scene(wl, rank)
    echo = synth.scene_echo(s, device="cuda")
    cfg = dict(PLAN_CFG[wl])
    for key, val in (("leaf_size", args.leaf), ("taps", args.taps), ("eta", args.eta)):
        if val is not None:
            cfg[key] = val
    grid = s.grid
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    img = torch.empty(grid.shape, dtype=torch.complex64, device="cuda")
    bimg = torch.empty_like(img)

    def step(timed):
        ev[0].record(stream)
        plan = hh.Plan(s.traj, s.freqs, grid, **cfg)
        ev[4].record(stream)  # the plan is built (its constructor synchronises the stream)
        plan.profile(True)  # CUDA events around each stage, on the launching stream
        plan.form_image(echo, out=img)
        ev[1].record(stream)
        hh.bpa_form_image(s.traj, s.freqs, grid, echo, out=bimg)
        ev[2].record(stream)
        err = torch.linalg.vector_norm(img.to(torch.complex128) - bimg.to(torch.complex128)) / \
            torch.linalg.vector_norm(bimg.to(torch.complex128))  # FP64 reduce
        ev[3].record(stream)
        return plan, err

    for _ in range(args.warmup):
        plan, _ = step(False)
        plan.close()
    # the MUFU rate of this device, measured (one rsqrt feeding one sine and one cosine per
    # step, as in an update), before the timed region: the denominator of the MUFU rooflines
    peaks["mufu_tps"] = hh.mufu_throughput("update_mix", 4096)[0]
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    t_hh, t_bpa, t_step, t_plan, errs, stage_runs = [], [], [], [], [], []
    barrier()
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    launches0 = hh.kernel_launches()
    for _ in range(args.steps):
        plan, err = step(True)
        torch.cuda.synchronize()
        t_hh.append(ev[0].elapsed_time(ev[1]))
        t_plan.append(ev[0].elapsed_time(ev[4]))
        t_bpa.append(ev[1].elapsed_time(ev[2]))
        t_step.append(ev[0].elapsed_time(ev[3]))
        errs.append(float(err))
        stage_runs.append(plan.stage_times())
        plan.close()
    launches = hh.kernel_launches() - launches0  # the library's own kernels in the timed steps
    g1.record(stream)
    barrier()
    clk = clocks.stop()
    total_ms = g0.elapsed_time(g1)
    total_ms, mean_hh, mean_bpa = reduce_over_ranks(
        dist, [total_ms, statistics.mean(t_hh), statistics.mean(t_bpa)], "cuda")

    # per-stage durations averaged over the timed steps
    stages = [(name, lev, statistics.mean(run[i][2] for run in stage_runs))
              for i, (name, lev, _) in enumerate(stage_runs[0])]
    # --- untimed diagnostics: counters, level sizes, plan geometry, e2e
    plan = hh.Plan(s.traj, s.freqs, grid, **cfg)
    plan.form_image(echo, out=img)
    cnt = plan.counters()
    levels = plan.level_counts()
    info = plan.info()
    ex = plan.export()
    ls = ex["level_start"]
    leaves = slice(ls[0], ls[1])
    plan_meta = dict(leaf_members_avg=float(np.mean(ex["end"][leaves] - ex["begin"][leaves])),
                     nchild={l: int(ex["nchild"][ls[l]]) for l in range(1, info["n_levels"])})
    clk_mhz = clk["sm_mhz"] or peaks["sm_max_mhz"]
    work = kernel_work(stages, plan_meta, info, levels, cnt, grid, len(s.traj), len(s.freqs), plan.config.taps)
    # roofline time per stage: max of FP32, MUFU and HBM bound at the sampled clock
    f = clk_mhz * 1e6
    roof_ms = 0.0
    for w in work:
        t_fp = w["flop"] / (FP32_PER_SM_CLK * sm_count() * f)
        t_mu = w["mufu"] / (peaks.get("mufu_tps") or MUFU_PER_SM_CLK * sm_count() * f)
        t_hb = w["bytes"] / (peaks["hbm_gbs"] * 1e9)
        w["roof_ms"] = 1e3 * max(t_fp, t_mu, t_hb)
        w["bound"] = ["fp32", "mufu", "hbm"][int(np.argmax([t_fp, t_mu, t_hb]))]
        roof_ms += w["roof_ms"]
    hh_kernel_ms = sum(w["ms"] for w in work)
    dom = max(work, key=lambda w: w["ms"])
    # BPA kernel roofline (MUFU bound): updates = voxels x positions
    bpa_upd = grid.n_vox * len(s.traj)
    b_ach, b_peak, b_unit, b_bound, b_frac = roofline_of("mufu", mean_bpa, bpa_upd * BPA_MUFU, peaks, clk_mhz)
    kind = dom["bound"]
    units = {"fp32": dom["flop"], "mufu": dom["mufu"], "hbm": dom["bytes"]}[kind]
    d_ach, d_peak, d_unit, d_bound, d_frac = roofline_of(kind, dom["ms"], units, peaks, clk_mhz)
    d_kind_mufu = kind == "mufu"

    # position gradient of direct BPA on the differentiation scene (8,192 positions, 128 freqs,
    # 128x128x32 grid, echoes from a track with smooth 1 mm offsets): CUDA events around the call
    ds = synth.diff()
    d_echo = synth.diff_echo(ds, synth.diff_offsets(len(ds.traj)), device="cuda")
    d_g = torch.randn(ds.grid.shape, dtype=torch.complex64, device="cuda",
                      generator=torch.Generator(device="cuda").manual_seed(17))
    d_out = torch.empty((len(ds.traj), 3), dtype=torch.float64, device="cuda")
    d_times = []
    for i in range(4):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        hh.bpa_traj_gradient(ds.traj, ds.freqs, ds.grid, d_echo, d_g, out=d_out)
        e1.record(stream)
        torch.cuda.synchronize()
        if i:
            d_times.append(e0.elapsed_time(e1))
    d_ms = statistics.median(d_times)
    d_upd = ds.grid.n_vox * len(ds.traj)
    g_ach, g_peak, g_unit, g_bound, g_frac = roofline_of("mufu", d_ms, d_upd * BPA_MUFU, peaks, clk_mhz)

    # the fast method's adjoint and plan-fixed position gradient on the same scene (leaf 64):
    # CUDA events around each call, median of three after one warm-up call
    dplan = hh.Plan(ds.traj, ds.freqs, ds.grid, leaf_size=64)
    d_echo_out = torch.empty((len(ds.traj), len(ds.freqs)), dtype=torch.complex64, device="cuda")

    def _timed(fn):
        ts = []
        for i in range(4):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            if i:
                ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    fast_adj_ms = _timed(lambda: dplan.adjoint(d_g, out=d_echo_out))
    fast_grad_ms = _timed(lambda: dplan.traj_gradient(d_echo, d_g, out=d_out))
    fast_fwd_ms = _timed(lambda: dplan.form_image(d_echo))
    dplan.close()

    # e2e through the C ABI with pinned host buffers (H2D echo, D2H image inside the timed region)
    h_echo = echo.cpu().pin_memory()
    h_img = torch.empty(grid.shape, dtype=torch.complex64).pin_memory()
    e2e = []
    for i in range(max(2, min(args.steps, 4)) + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        p2 = hh.Plan(s.traj, s.freqs, grid, **cfg)
        p2.form_image(h_echo, out=h_img)
        torch.cuda.synchronize()
        if i:
            e2e.append(time.perf_counter() - t0)
        p2.close()

    nr_db = 20 * math.log10(statistics.mean(errs))
    hh_s = per_volume_s(mean_hh, ws)
    line = {
        "metric": METRIC,
        "value": hh_s,
        "unit": "s/volume",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 (FP64 tile references)",
        "data": "synthetic (seeded scene, exact Born-model echoes)",
        "config": {"workload": WORKLOADS[wl], "plan": cfg, "taps": plan.config.taps, "eta": plan.config.eta,
                   "merge_factor": plan.config.merge_factor, "l2": "inputs larger than L2 (echo 268 MB, "
                   "image 268 MB, level pools > 1 GB)", "parallelism": f"replicas x{ws}",
                   "step": "plan + HHFFBPA + direct BPA + NRMSE"},
        "bpa_s_per_volume": mean_bpa / 1e3,
        "speedup_vs_bpa": mean_bpa / mean_hh,
        "nrmse_db": nr_db,
        "stages_ms": [[w["stage"], w["level"], round(w["ms"], 3), round(w["roof_ms"], 3), w["bound"]] for w in work],
        "roofline": {"kernel": f'{dom["stage"]}(level {dom["level"]})', "bound": d_bound, "achieved": d_ach,
                     "peak": d_peak, "unit": d_unit, "frac": d_frac,
                     "traffic": (TRAFFIC_PER_SAMPLE[(dom["stage"], STAGE0_REVISION)] * levels[0]
                                 if (dom["stage"], STAGE0_REVISION) in TRAFFIC_PER_SAMPLE else None),
                     "traffic_source": "ncu dram bytes of one launch on the mid workload, scaled by the "
                                       "evaluated samples",
                     "peak_source": (f'measured: MUFU probe hh_mufu_throughput (rsqrt feeding sin and cos, '
                                     f'2048 threads/SM), {peaks["mufu_tps"] / 1e12:.3f} T/s = '
                                     f'{peaks["mufu_tps"] / (sm_count() * clk_mhz * 1e6):.2f} results/clk/SM at '
                                     f'the sampled {clk_mhz:.0f} MHz (nominal {MUFU_PER_SM_CLK:g})'
                                     if d_kind_mufu else
                                     f'derived ({FP32_PER_SM_CLK:g} FLOP/clk/SM x {sm_count()} SMs at the '
                                     f'sampled {clk_mhz:.0f} MHz)')},
        "plan_ms": statistics.mean(t_plan),
        "roofline_pipeline": {"roofline_ms": roof_ms, "kernels_ms": hh_kernel_ms,
                              "frac": roof_ms / hh_kernel_ms if hh_kernel_ms else None,
                              "frac_incl_plan": roof_ms / mean_hh},
        "smem_merges": [{"stage": w["stage"], "level": w["level"], "achieved": w["smem"] / (w["ms"] * 1e-3) / 1e12,
                         "peak": SMEM_B_PER_SM_CLK * sm_count() * clk_mhz * 1e6 / 1e12, "unit": "TB/s",
                         "frac": w["smem"] / (w["ms"] * 1e-3) / (SMEM_B_PER_SM_CLK * sm_count() * clk_mhz * 1e6),
                         "peak_source": f"derived ({SMEM_B_PER_SM_CLK:g} B/clk/SM x {sm_count()} SMs at "
                                        f"{clk_mhz:.0f} MHz)"}
                        for w in work if w["smem"] > 0],
        "roofline_bpa": {"bound": b_bound, "achieved": b_ach, "peak": b_peak, "unit": b_unit, "frac": b_frac,
                         "traffic": None},
        "counters": cnt,
        "level_samples_evaluated": levels,
        "e2e": {"value": statistics.median(e2e), "unit": "s/volume",
                "h2d_bytes_per_step": int(h_echo.numel() * 8 + s.traj.size * 8 + s.freqs.size * 8),
                "d2h_bytes_per_step": int(h_img.numel() * 8)},
        "gpu_launches": launches,
        "position_gradient": {"workload": "diff: 8,192 positions, 128 freqs, 32 points, 128x128x32 grid, "
                                          "smooth 1 mm track offsets", "ms": d_ms,
                              "updates": d_upd, "achieved": g_ach, "peak": g_peak, "unit": g_unit,
                              "bound": g_bound, "frac": g_frac,
                              "note": "bpa_traj_gradient incl. range compression; outside the timed steps"},
        "fast_differentiation": {"workload": "diff: 8,192 positions, 128 freqs, 32 points, 128x128x32 grid, "
                                               "smooth 1 mm track offsets; plan leaf 64, 4-way, 6 taps, eta 2",
                                 "forward_ms": fast_fwd_ms, "adjoint_ms": fast_adj_ms,
                                 "traj_gradient_ms": fast_grad_ms,
                                 "note": "hhffbp_form_image, hhffbp_adjoint, hhffbp_traj_gradient (plan held "
                                         "fixed); demand passes included; outside the timed steps"},
        "clocks": clk,
    }
    if wl == "sim1":
        line["evaluation"] = sim1_evaluation(hh, s, echo, img, bimg, cfg)
    if rank == 0 and not args.no_cpu_baseline:
        run = _oracle_run(wl, True)
        line["cpu_baseline"] = cpu_baseline(wl, run)
        line["cpu_baseline_bpa"], b_idx, b_ref = cpu_bpa_baseline(wl)
        line["precision"] = precision_study(hh, s, echo, cfg, img, bimg, run[2], np.asarray(run[3]), b_idx,
                                            np.asarray(b_ref))
        # the oracle's image against the GPU image of the same scan
        idx, ref = run[2], np.asarray(run[3])
        got = img.reshape(-1) if idx is None else img.reshape(-1)[torch.as_tensor(idx, device=img.device)]
        got = got.cpu().numpy().astype(np.complex128)
        line["parity_vs_oracle"] = {
            "rel_l2": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
            "max_abs_err_over_max_abs": float(np.abs(got - ref).max() / np.abs(ref).max()),
            "voxels": int(ref.size), "tolerance": 1e-4,
            "sample": "every voxel, same scan, same plan parameters (the oracle builds its own plan)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def sim1_evaluation(hh, s, echo, img, bimg, cfg):
    """The paper's Sim-I metrics for this scan: point-spread metrics along x through the centre
    (0, 0, 0.4) and squint (-0.175, 0, 0.4) scatterers on 0.5 mm line grids (both methods
    imaged there directly), PSNR of HHFFBPA against direct BPA over the volume, and the time of
    the maximum-intensity projection along z."""
    import torch

    import synth
    from paper_2506_23568_gb300 import metrics

    out = {"paper_table2_context": PAPER_SIM1}
    for name, (x0, y0, z0) in (("centre", (0.0, 0.0, 0.4)), ("squint", (-0.175, 0.0, 0.4))):
        lg = synth.Grid(x0 - 0.05, y0, z0, 5e-4, 1.0, 1.0, 201, 1, 1)
        h_line = hh.Plan(s.traj, s.freqs, lg, **cfg).form_image(echo).reshape(-1).cpu().numpy()
        b_line = hh.bpa_form_image(s.traj, s.freqs, lg, echo).reshape(-1).cpu().numpy()
        out[f"{name}_psf"] = {"hhffbpa": [1e3 * metrics.psf_metrics(h_line, 5e-4)[0], *metrics.psf_metrics(h_line, 5e-4)[1:]],
                              "bpa": [1e3 * metrics.psf_metrics(b_line, 5e-4)[0], *metrics.psf_metrics(b_line, 5e-4)[1:]],
                              "fields": ["mainlobe width mm", "PSLR dB", "ISLR dB"]}
    h, b = img.cpu().numpy(), bimg.cpu().numpy()
    out["psnr_hhffbpa_vs_bpa_db"] = metrics.psnr_db(h, b)
    out["psnr_magnitude_db"] = metrics.psnr_db(h, b, magnitude=True)
    mip = hh.mip(img)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(10):
        hh.mip(img, out=mip)
    e1.record()
    torch.cuda.synchronize()
    out["mip_ms"] = e0.elapsed_time(e1) / 10
    out["note"] = ("PSF metrics on 201-sample line grids at 0.5 mm through the scatterer (the method imaged "
                   "directly there, each with its own plan); readings of the metrics in metrics.py")
    return out


def run_batch(args):
    """Batching workload: 32 seeded scans of uneven length and grid (4k-32k positions,
    128-256 freqs, 128^2 x 32 to 384^2 x 64 voxels), plan parameters from the autotuner,
    imaged by one CUDA-graph launch per step.  value = graph time per step / 32 (s/volume);
    the plans are built once, before the timed steps (their time is reported per volume)."""
    import torch

    import paper_2506_23568_gb300 as hh
    import synth
    from paper_2506_23568_gb300 import tune

    ws, rank, local = _dist_env()
    torch.cuda.set_device(local)
    n_scans = 32
    scenes = [synth.batch_scene(i + 1000 * rank) for i in range(n_scans)]
    echos = [synth.scene_echo(sc, device="cuda") for sc in scenes]
    stream = torch.cuda.current_stream()
    # autotuner: calibrate the model's costs on the middle scan, tune three representatives
    order = sorted(range(n_scans), key=lambda i: len(scenes[i].traj))
    reps = [order[0], order[n_scans // 2], order[-1]]
    t0 = time.perf_counter()
    mid = scenes[reps[1]]
    coeffs = tune.calibrate(mid.traj, mid.freqs, mid.grid, echos[reps[1]])
    tuned = {}
    for r in reps:
        sc = scenes[r]
        tuned[r] = tune.tune(sc.traj, sc.freqs, sc.grid, echos[r], target_db=-30.0, top=3, coeffs=coeffs)
    tune_s = time.perf_counter() - t0
    cfg_of = {i: tuned[min(reps, key=lambda r: abs(len(scenes[r].traj) - len(scenes[i].traj)))]["config"]
              for i in range(n_scans)}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plans = [hh.Plan(sc.traj, sc.freqs, sc.grid, **cfg_of[i]) for i, sc in enumerate(scenes)]
    plan_s = time.perf_counter() - t0
    images = [torch.empty(sc.grid.shape, dtype=torch.complex64, device="cuda") for sc in scenes]
    batch = hh.Batch(plans, n_streams=8)
    for _ in range(max(args.warmup, 1)):
        batch.form_images(echos, images)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        batch.form_images(echos, images)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = e0.elapsed_time(e1)
    # the same scans one after another on one stream, for comparison
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    single = [torch.empty_like(im) for im in images]
    s0.record(stream)
    for p, e, im in zip(plans, echos, single):
        p.form_image(e, out=im)
    s1.record(stream)
    torch.cuda.synchronize()
    seq_ms = s0.elapsed_time(s1)
    equal = all(torch.equal(a, b) for a, b in zip(images, single))
    nr = [tune.accuracy_db(sc.traj, sc.freqs, sc.grid, e, im) for sc, e, im in zip(scenes, echos, images)]
    cnt_ok = all(p.counters()["errors"] == 0 for p in plans)
    value = total_ms / args.steps / 1e3 / n_scans
    line = {"metric": METRIC, "value": value, "unit": "s/volume", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 (FP64 tile references)",
            "data": "synthetic (seeded scenes, exact Born-model echoes)",
            "config": {"workload": "batch: 32 scans, 4k-32k positions, 128-256 freqs 76-81 GHz, grids 128^2x32 to "
                                   "384^2x64, one CUDA-graph launch per step (8 concurrent branches)",
                       "l2": "inputs larger than L2 (echoes and images of 32 scans, several GB)"},
            "sequential_s_per_volume": seq_ms / 1e3 / n_scans, "graph_speedup_vs_sequential": seq_ms / (total_ms / args.steps),
            "batch_images_equal_single_scan_images": equal, "counters_clean": cnt_ok,
            "nrmse_db_vs_bpa_every_8th_slab": {"min": min(nr), "max": max(nr)},
            "plans_s_per_volume": plan_s / n_scans, "tuning_s": tune_s,
            "tuner": {"coeffs_ns": coeffs, "chosen": {str(r): tuned[r]["config"] for r in reps},
                      "tried": {str(r): tuned[r]["tried"] for r in reps}},
            "roofline": None, "gpu_launches": None,
            "e2e": None, "clocks": clk,
            "note": "roofline, e2e and the CPU baseline are reported on the single-scan workloads"}
    batch.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


def _oracle_points(wl, g, full):
    """Voxels the oracle images: the whole volume, or (the reference arm's per-step sample)
    the central half x half of the middle z-slab -- the whole slab for tiny."""
    if full:
        return None, "the full volume"
    c = g.nz // 2
    if wl == "tiny":
        xs, ys = np.arange(g.nx), np.arange(g.ny)
    else:
        xs, ys = np.arange(g.nx // 4, g.nx // 4 + g.nx // 2), np.arange(g.ny // 4, g.ny // 4 + g.ny // 2)
    idx = ((c * g.ny + ys[:, None]) * g.nx + xs[None, :]).ravel()
    return idx, f"the central {len(xs)}x{len(ys)} voxels of z-slab {c} (1/{g.n_vox // idx.size} of D)"


def _oracle_run(wl, full, scene=None):
    """Time the FP64 oracle (its own plan + HHFFBPA, demand-driven, OpenMP on the host cores)
    over the full volume or the per-step sample: (seconds, what, voxel indices, values)."""
    import oracle
    import synth

    s, e = scene if scene is not None else (None, None)
    if s is None:
        s = synth.CONFIGS[wl]()
        e = synth.scene_echo(s, device="cpu").numpy()
    g = s.grid
    idx, what = _oracle_points(wl, g, full)
    pts = g.points() if idx is None else g.points(idx)
    t0 = time.perf_counter()
    pl = oracle.Plan(s.traj, s.freqs, g, **PLAN_CFG[wl])
    vals, _ = pl.hhffbpa(e, pts)
    return time.perf_counter() - t0, what, idx, vals


def cpu_bpa_baseline(wl):
    """The oracle's direct BPA-RC (FP64, OpenMP): the whole volume for tiny, else one z-slab
    extrapolated to the volume (exact: its cost is the same for every voxel)."""
    import oracle
    import synth

    s = synth.CONFIGS[wl]()
    e = synth.scene_echo(s, device="cpu").numpy()
    g = s.grid
    if wl == "tiny":
        idx, what, scale = np.arange(g.n_vox), "the full volume, timed in full", 1.0
    else:
        c = g.nz // 2
        idx = np.arange(g.nx * g.ny) + c * g.nx * g.ny
        what, scale = f"z-slab {c} ({g.nx * g.ny} voxels), x{g.nz} to the volume (linear in voxels)", float(g.nz)
    t0 = time.perf_counter()
    vals = oracle.bpa_rc(s.traj, s.freqs, e, g.points(idx))
    t = time.perf_counter() - t0
    return {"value": t * scale, "unit": "s/volume", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"oracle direct BPA-RC (FP64, OpenMP) over {what}: {t:.2f} s",
            "ns_per_update_core": t * oracle.num_threads() / (idx.size * len(s.traj)) * 1e9}, idx, vals


def precision_study(hh, s, echo, cfg, img, bimg, h_idx, h_ref, b_idx, b_ref):
    """Error against the FP64 oracle of the FP32 path as built (FP64 per-tile and per-node
    references, FP32 differences) and of the same path with those references in FP32, for
    HHFFBPA (the oracle's voxels) and direct BPA (the oracle's BPA voxels)."""
    import torch

    def rel(gpu, idx, ref):
        g = gpu.reshape(-1) if idx is None else gpu.reshape(-1)[torch.as_tensor(idx, device=gpu.device)]
        g = g.cpu().numpy().astype(np.complex128)
        return float(np.linalg.norm(g - ref) / np.linalg.norm(ref))

    f32 = hh.HH_FLAG_FP32_REFS
    img32 = hh.Plan(s.traj, s.freqs, s.grid, flags=f32, **cfg).form_image(echo)
    bimg32 = hh.bpa_form_image(s.traj, s.freqs, s.grid, echo, flags=f32)
    return {"hhffbpa_rel_l2": {"fp64_references": rel(img, h_idx, h_ref), "fp32_references": rel(img32, h_idx, h_ref)},
            "bpa_rel_l2": {"fp64_references": rel(bimg, b_idx, b_ref), "fp32_references": rel(bimg32, b_idx, b_ref)},
            "note": "relative L2 against the FP64 oracle; fp32_references = HH_FLAG_FP32_REFS (per-tile reference "
                    "ranges and phases of direct BPA and the merges' tile references in FP32)"}


def cpu_baseline(wl, run=None):
    """The oracle over the full volume, timed in full (run = a finished _oracle_run)."""
    import oracle

    t, what, _, _ = run if run is not None else _oracle_run(wl, True)
    return {"value": t, "unit": "s/volume", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"oracle plan + HHFFBPA (FP64, OpenMP) over {what} of the {wl} workload, timed in full"}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle on the host cores, bounded samples of the same workload."""
    ws, rank, _ = _dist_env()
    if rank != 0:
        return
    import oracle
    import synth

    wl = args.workload
    if wl == "batch":  # the oracle's baselines are reported on the single-scan workloads
        print(json.dumps({"impl": "reference", "workload": "batch", "note": "the CPU oracle is timed on the "
                          "single-scan workloads (tiny, mid, large, sim1), not on the 32-scan batch"}), flush=True)
        return
    sc = synth.CONFIGS[wl]()
    scene = (sc, synth.scene_echo(sc, device="cpu").numpy())
    # calibration (untimed): the full volume once, and the per-step sample once
    t_full = _oracle_run(wl, True, scene)[0]
    t_cal, what, _, _ = _oracle_run(wl, False, scene)
    ratio = t_full / t_cal
    for _ in range(args.warmup):
        _oracle_run(wl, False, scene)
    vals = []
    t_start = time.perf_counter()
    for _ in range(args.steps):
        vals.append(_oracle_run(wl, False, scene)[0] * ratio)
    wall = time.perf_counter() - t_start
    val = statistics.mean(vals)
    sample = (f"oracle plan + HHFFBPA (FP64, OpenMP) over {what} of the {wl} workload per step, scaled by the "
              f"measured full-volume / sample time ratio {ratio:.2f} (full volume {t_full:.1f} s, timed once "
              f"before the warm-up)")
    line = {"metric": METRIC, "value": val, "unit": "s/volume", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": wall * 1e3 / args.steps, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[wl], "plan": PLAN_CFG[wl]}, "impl": "reference",
            "cpu_baseline": {"value": val, "unit": "s/volume", "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": "s/volume", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="large", choices=sorted(WORKLOADS) + ["batch"])
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--leaf", type=int, default=None, help="override the plan's leaf size")
    ap.add_argument("--taps", type=int, default=None, help="override the interpolation taps")
    ap.add_argument("--eta", type=float, default=None, help="override the base lattice density")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
