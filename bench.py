#!/usr/bin/env python
"""Throughput of the two-phase shallow-flow step on one GB300 (cell-steps/s).

Headline workload: the large-scale release event -- 4096 x 4096 cells at 10 m
over a seeded 1/f^2.2 spectral DEM (1500 m relief) with one carved valley, a
2.5e7 m^3 parabolic-cap release (bed-normal volume) on a 30-40 degree slope,
solid fraction U(0.55, 0.65), transmissive boundaries, CFL 0.1, 10000 steps
(synthetic stand-in for the Hsiaolin event of Sect. 4.1; the real DEM is not
available).

A step is one full time step: CFL time step from the exact max-reduction, two
stages of the central scheme with all sources, Heun average, boundary fill.
Each stage is two launches: the wet/dry classification, which writes the
stage result of every tile without mass in reach (the zero state), and the
stage kernel on the listed tiles.  The event is first run through all its
10000 steps (timed as a whole, with the wet-tile fraction at the start of
each quarter); the headline then times K steps (after W warm-up steps) from
the checkpoint at the start of each quarter, so that the K-step figure
samples the whole event and not only its start.  Every cell of the grid
counts in cell-steps/s, as in the paper's speed-up figures (Sect. 3.2); the
kernel's own roofline comes from the same kernels on an all-wet state
(`dense`: every tile computes), against the measured FP64 FMA rate and
against HBM with 13 words per computed cell-step.  The headline is the FP64
form; the FP32 form (FP64 budgets and friction test) is measured the same
way in the same run.  The state (0.8 GB in FP64) is larger than L2, so no
flush is needed between steps.

The other configurations have lines of their own at their stated sizes and
lengths: the arc-plane release (128^2, 2000 steps, FP64), the inflow
hydrograph (2048 x 1024 to t = 600 s, FP32 with FP64 budgets), the 256-member
ensemble (3000 steps, FP32) and the adjoint calibration (1024^2, 5000 steps,
checkpoint every 71).

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

With N > 1 (torchrun, one rank per GPU) every rank advances its own replica of
the workload (independent problems, weak scaling, no data-path collective);
the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "cell-steps/s FP64 vs FP32 (% HBM roofline); ensemble cells/s; adjoint/fwd cost"
UNIT = "cell-steps/s"
N_SIDE = 4096
DX = 10.0

# Algorithmic work of one stage launch per cell (both counted from the
# formulas of stage.cuh; see the design notes): floating-point operations
# (add, sub, mul, div, sqrt = 1; fma = 2; comparisons, min/max, abs = 0) and
# bytes that must cross HBM for one cell-step: read U^n (6 words), write
# U^{n+1} (6), read the bed elevation (1).
FLOPS_PER_CELL_STAGE = 488
WORDS_PER_CELL_STEP = 13
EVENT_STEPS = 10000  # the large release event's length
N_WINDOWS = 4        # timed windows, at the start of each quarter of the event

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of the stage
# kernel on the all-wet state, per cell and stage launch, from an ncu capture of
# stage_kernel_list on a 2048^2 all-wet case (the per-cell traffic of a
# fully wet grid does not depend on its size once it exceeds L2); valid only
# for the stage kernel source it was taken on (sha256 of csrc/stage.cuh,
# first 12).
TRAFFIC_PER_CELL_STAGE = {
    # profiles/stage_kernel_list_all_wet_2048.md
    ("f64", "135442891e6c"): 330.74,
    ("f32", "135442891e6c"): 77.01,
}


def cell_step_gbs(cells, esz, step_s):
    """HBM rate [GB/s] of a step over `cells` computed cells that takes step_s
    seconds, at 13 words of esz bytes per cell-step (FP64 104 B, FP32 52 B)."""
    return WORDS_PER_CELL_STEP * esz * cells / step_s / 1e9


def _traffic(form, h, cells):
    b = TRAFFIC_PER_CELL_STAGE.get((form, h))
    return None if b is None else b * cells


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# FP64 vector peak of GB300 from its unit counts and clock: 152 SMs x 2 FP64
# FMA/clk x 2 flops x 2.07 GHz = 1.26 TFLOP/s (the 1.25 TFLOP/s nominal
# figure).  The roofline takes the measured FMA rate (moses_debug_fp64_rate)
# and keeps this one beside it.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# FP32 vector peak: 152 SMs x 128 FMA/clk x 2 flops x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def stage_hash():
    with open(os.path.join(ROOT, "paper_2104_06784_gb300", "csrc", "stage.cuh"), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:12]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region.

    The sampler runs every 20 ms from before the measurement (it waits for
    its first sample, so it is live) to after it; the timed window is marked
    with begin() / end().  The samples that arrive within the window (plus
    one interval) are summarised; a window shorter than the interval that
    caught none is reported with the two samples bracketing it."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    INTERVAL_MS = 20

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.p = None
        self.lines = []  # (arrival time, line)
        self.windows = []

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", str(self.INTERVAL_MS)],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.time()
            while not self.lines and time.time() - t0 < 5.0:
                time.sleep(0.01)
        except Exception:
            self.p = None
        return self

    def _read(self):
        for line in self.p.stdout:
            self.lines.append((time.time(), line.strip()))

    def begin(self):
        self.windows.append([time.time(), None])

    def end(self):
        if self.windows:
            self.windows[-1][1] = time.time()

    def __exit__(self, *a):
        if self.p:
            time.sleep(2.5 * self.INTERVAL_MS / 1e3)  # the samples of the window's end
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()

    @staticmethod
    def _parse(ln):
        f = [x.strip() for x in ln.split(",")]
        if len(f) < 9:
            return None
        try:
            return float(f[1]), float(f[2]), f[5:9]
        except ValueError:
            return None

    def summary(self):
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lag = 1.5 * self.INTERVAL_MS / 1e3
        parsed = [(t, self._parse(ln)) for t, ln in self.lines]
        parsed = [(t, v) for t, v in parsed if v is not None]
        inside = [v for t, v in parsed if any(w0 <= t <= (w1 or w0) + lag for w0, w1 in self.windows)]
        how = "in the timed window"
        if not inside and self.windows and parsed:
            w0, w1 = self.windows[0][0], self.windows[-1][1] or self.windows[-1][0]
            before = [v for t, v in parsed if t < w0][-1:]
            after = [v for t, v in parsed if t > w1][:1]
            inside = before + after
            how = "bracketing the timed window (shorter than the sampling interval)"
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        reasons = set()
        for _, _, act in inside:
            for n, v in zip(names, act):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(v[0] for v in inside), "sm_max_mhz": inside[-1][1],
                "reasons": sorted(reasons), "samples": len(inside), "window": how,
                "interval_ms": self.INTERVAL_MS}


def _oracle_window(cfg, window, library=None):
    """The oracle on a window x window crop of the workload centred on the release."""
    from oracle.oracle import OracleSim
    ic, jc = cfg["release_cell"]
    n = cfg["dem"].shape[0]
    i0 = int(min(max(ic - window // 2, 0), n - window))
    j0 = int(min(max(jc - window // 2, 0), n - window))
    sl = (slice(j0, j0 + window), slice(i0, i0 + window))
    o = OracleSim(cfg["dem"][sl], cfg["dx"], cfg["dy"], cfg["params"], library=library)
    o.set_release(cfg["h"][sl], cfg["phi_s"][sl])
    return o


def _omp_threads():
    return int(os.environ.get("OMP_NUM_THREADS", "0")) or os.cpu_count() or 1


def cpu_baseline(cfg, window=1024):
    """The FP64 oracle as it stands on the host, on a bounded sample: steps on
    a window x window crop of the workload centred on the release (throughput
    per cell-step does not depend on the size).  Two legs: the plain build on
    one core (the paper's single-core baseline, Sect. 3.2) and the OpenMP
    build over every host core; the line's value is the multi-core leg."""
    from oracle import oracle as O
    n = cfg["dem"].shape[0]
    o = _oracle_window(cfg, window)
    o.step(1)
    t0 = time.perf_counter()
    s1 = 20
    o.step(s1)
    el1 = time.perf_counter() - t0
    cores = _omp_threads()
    om = _oracle_window(cfg, window, library=O.lib_openmp())
    om.step(1)
    sm = 20 * max(1, min(cores, 16))
    t0 = time.perf_counter()
    om.step(sm)
    elm = time.perf_counter() - t0
    return dict(value=window * window * sm / elm, unit=UNIT, cores=cores, kind="oracle",
                sample=f"{sm} FP64 steps of the oracle (OpenMP build, {cores} threads) on the {window}x{window} "
                       f"window of the {n}x{n} workload around the release",
                single_core={"value": window * window * s1 / el1, "cores": 1,
                             "sample": f"{s1} steps of the plain build on the same window, 1 thread"},
                seconds=el1 + elm)


def run_reference(args, cfg, rank):
    """The reference arm: the CPU oracle (OpenMP build, every host core) timed
    on the host, K steps after W warm-up steps, each step one oracle step on a
    1024 x 1024 window of the workload around the release."""
    if rank != 0:
        return None
    from oracle import oracle as O
    window = 1024
    n = cfg["dem"].shape[0]
    o = _oracle_window(cfg, window, library=O.lib_openmp())
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    el = time.perf_counter() - t0
    v = window * window * args.steps / el
    cores = _omp_threads()
    sample = (f"each step: one FP64 oracle step (OpenMP build, {cores} threads) on the {window}x{window} window "
              f"of the {n}x{n} workload")
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(cfg, args),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def config_dict(cfg, args):
    n = cfg["dem"].shape[0]
    return {"workload": f"large-scale release event, {n}x{n} cells at {DX:g} m, spectral DEM "
                        f"(beta 2.2, 1500 m relief, carved valley), 2.5e7 m^3 release (bed-normal), CFL 0.1, "
                        f"{EVENT_STEPS} steps; K steps timed from each of {N_WINDOWS} checkpoints (the start of each "
                        f"quarter of the event)",
            "cells": n * n, "dx_m": DX, "l2": "state larger than L2 (0.8 GB FP64, 0.4 GB FP32); no flush",
            "parallelism": f"replicas x{args.gpus}" if args.gpus > 1 else "single GPU"}


def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def measure(sim, cells, K, W, torch, sampler=None):
    """Device time of K steps (after W warm-up steps) with CUDA events on the
    simulation's stream; per-stage launch times from moses_step_timed."""
    sim.step(W)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0, e1 = _events(torch)
    if sampler is not None:
        sampler.begin()
    e0.record(stream)
    sim.step(K)
    e1.record(stream)
    torch.cuda.synchronize()
    if sampler is not None:
        sampler.end()
    ms = e0.elapsed_time(e1)
    # per-launch timing of the stage kernel over K more steps
    _, stage_ms = sim.step_timed(K)
    return ms, stage_ms


def run_event(sim, torch, nsteps=EVENT_STEPS, nwin=N_WINDOWS, tile=(32, 8)):
    """The whole event: nsteps steps in nwin segments, each timed with CUDA
    events on the simulation's stream; before each segment the state is kept
    (a device checkpoint for the windows) and its wet-tile fraction taken."""
    seg = nsteps // nwin
    stream = torch.cuda.current_stream()
    ckpts, segs = [], []
    for w in range(nwin):
        ck = torch.empty((6, sim.ny, sim.nx), dtype=torch.float64, device="cuda")
        sim.get_conserved_device(ck.data_ptr())
        torch.cuda.synchronize()
        wet = wet_tile_fraction(ck.cpu().numpy(), *tile)
        t0 = sim.budget()["t"]
        e0, e1 = _events(torch)
        e0.record(stream)
        sim.step(seg)
        e1.record(stream)
        torch.cuda.synchronize()
        ckpts.append(ck)
        segs.append({"from_step": w * seg, "t_s": t0, "wet_tiles": wet, "ms": e0.elapsed_time(e1)})
    b = sim.budget()
    U = sim.get_conserved()
    total = sum(x["ms"] for x in segs)
    return ckpts, {"steps": nwin * seg, "ms": total, "value": sim.nx * sim.ny * nwin * seg / (total / 1e3),
                   "t_end_s": b["t"], "wet_tiles_end": wet_tile_fraction(U, *tile), "segments": segs}


def measure_windows(sim, ckpts, K, W, torch, sampler=None, nvtx=None):
    """K steps timed (after W warm-up steps) from each checkpoint: CUDA events
    on the simulation's stream around the K steps of each window.  With
    `nvtx` the timed steps sit in an NVTX range of that name (a profiler can
    then take exactly those launches)."""
    stream = torch.cuda.current_stream()
    out = []
    for ck in ckpts:
        sim.set_conserved_device(ck.data_ptr())
        sim.step(W)
        torch.cuda.synchronize()
        e0, e1 = _events(torch)
        if sampler is not None:
            sampler.begin()
        if nvtx:
            torch.cuda.nvtx.range_push(nvtx)
        e0.record(stream)
        sim.step(K)
        e1.record(stream)
        if nvtx:
            torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        if sampler is not None:
            sampler.end()
        out.append(e0.elapsed_time(e1))
    return out


def wet_tile_fraction(U, tx=32, ty=8):
    """Fraction of tx x ty tiles that compute (the stage kernel's wet/dry
    masking): tiles with mass (U1 or U4 non-zero) in the tile or within the
    2-cell halo of its stencil."""
    m = (U[0] != 0) | (U[3] != 0)
    d = m.copy()
    for s in (1, 2):  # dilate by 2 cells in x, then in y
        d[:, s:] |= m[:, :-s]
        d[:, :-s] |= m[:, s:]
    m = d.copy()
    for s in (1, 2):
        d[s:, :] |= m[:-s, :]
        d[:-s, :] |= m[s:, :]
    ny, nx = d.shape
    py, px = -ny % ty, -nx % tx
    d = np.pad(d, ((0, py), (0, px)))
    t = d.reshape(d.shape[0] // ty, ty, d.shape[1] // tx, tx).any(axis=(1, 3))
    return float(t.mean())


def measure_dense(cfg, K, Wm, torch, fp64_tflops, hbm_gbs, h):
    """The same 4096^2 terrain and release with a 5 cm mixture layer over every
    cell, so that every tile computes (no dry tile to skip): the stage's own
    rate.  Per form its roofline: FP64 against the measured FP64 FMA rate
    (the binding roof: 488 flops per cell and stage) and against HBM with the
    13 words per computed cell-step (104 B); FP32 against HBM (52 B) and
    against the FP32 FMA peak from unit counts and clock.  The launch time is
    the summed device time of the stage launches (the classification and the
    listed-tile stage kernel) from moses_step_timed, per launch pair."""
    from paper_2104_06784_gb300 import moses
    c = dict(cfg, h=cfg["h"] + 0.05)
    out = {"config": "the 4096^2 workload plus a 5 cm layer (phi_s as the release) on every cell: all tiles wet"}
    for form, prec, esz in (("f64", moses.FP64, 8), ("f32", moses.FP32, 4)):
        with moses.from_config(c, precision=prec) as sim:
            ms, stage_ms = measure(sim, sim.nx * sim.ny, K, Wm, torch)
            cells = sim.nx * sim.ny
        launch_ms = (stage_ms[0] + stage_ms[1]) / (2 * K)
        step_s = 2 * launch_ms / 1e3
        gbs = cell_step_gbs(cells, esz, step_s)
        tfl = FLOPS_PER_CELL_STAGE * cells / (launch_ms / 1e3) / 1e12
        out[form] = {"ms_per_step": ms / K, "value": cells * K / (ms / 1e3), "launch_ms": launch_ms,
                     "hbm": {"achieved": gbs, "peak": hbm_gbs, "unit": "GB/s", "frac": gbs / hbm_gbs,
                             "bytes_per_cell_step": WORDS_PER_CELL_STEP * esz}}
        if form == "f64":
            out[form]["alu"] = {"achieved": tfl, "peak": fp64_tflops, "unit": "TFLOP/s", "frac": tfl / fp64_tflops,
                                "peak_source": "measured FP64 FMA rate (moses_debug_fp64_rate)",
                                "peak_units_clock": FP64_PEAK_TFLOPS, "frac_units_clock": tfl / FP64_PEAK_TFLOPS}
            tr = _traffic("f64", h, cells)
            out[form]["traffic_per_launch"] = tr
        else:
            out[form]["alu"] = {"achieved": tfl, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                                "frac": tfl / FP32_PEAK_TFLOPS, "peak_source": "unit counts x 2.07 GHz"}
            out[form]["traffic_per_launch"] = _traffic("f32", h, cells)
    return out


def measure_variants(cfg, K, Wm, torch):
    """Step time of the model options the configurations leave off, on the
    all-wet form of the 4096^2 workload (`measure_dense`: every tile computes,
    so the options' arithmetic shows; 32 x 8 tiles, CUDA events): the
    central-upwind flux (scheme 1), the viscous term (nu_f = 1 m^2/s), the
    third-order WENO face values (recon 1), the three-stage SSP Runge-Kutta
    (rk 3) and WENO with the three-stage Runge-Kutta together."""
    from paper_2104_06784_gb300 import moses
    out = {}
    for name, over in (("central_upwind", dict(scheme=1)), ("viscous", dict(nu_f=1.0)), ("weno3", dict(recon=1)),
                       ("rk3", dict(rk=3)), ("weno3_rk3", dict(recon=1, rk=3))):
        out[name] = {}
        for form, prec in (("f64", moses.FP64), ("f32", moses.FP32)):
            c = dict(cfg, h=cfg["h"] + 0.05, params=dict(cfg["params"], **over))
            with moses.from_config(c, precision=prec) as sim:
                ms, _ = measure(sim, sim.nx * sim.ny, K, Wm, torch)
            out[name][form] = {"ms_per_step": ms / K, "value": sim.nx * sim.ny * K / (ms / 1e3)}
    return out


def reduce_over_ranks(x, op="max", dist=None, device="cpu"):
    """max (or sum) of a scalar over the ranks; x itself without a process group."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def shard(items, rank, world):
    """The members of an ensemble that one rank advances: every world-th one
    from `rank` (independent problems, no data-path exchange)."""
    return list(items)[rank::world]


def measure_ensemble(K, Wm, seed=0, n=256, rank=0, world=1, dist=None, device="cpu", steps=3000):
    """Batched ensemble, FP32: 256 members on square grids of lognormal side
    (64..1024 cells, 5 m), each its own spectral DEM, basal friction, drag and
    release volume; all the steps of a call in one cooperative launch (per
    stage the classification of every member's tiles and the stage on the wet
    ones, the CTAs meeting on a bounded grid barrier in between), with the
    tile shape the batch's tuner chose.  The members' 3000 steps are timed
    whole (after Wm warm-up steps), device time from CUDA events on the
    batch's stream.  With several ranks the members are sharded across them;
    the time is the max over ranks."""
    from paper_2104_06784_gb300 import moses, workloads as W
    cfgs = shard(W.ensemble_config(n, seed=seed), rank, world)
    cells_rank = int(sum(c["dem"].size for c in cfgs))
    sims = [moses.from_config(c, precision=moses.FP32) for c in cfgs]
    with moses.Batch(sims) as b:
        b.step(Wm)
        if dist is not None:
            dist.barrier()
        ms = b.step_timed(steps)
        tiles = b.tiles
        rows, tune_ms = b.tile_rows()
    wet = float(np.mean([wet_tile_fraction(s_.get_conserved()) for s_ in sims]))
    for s_ in sims:
        s_.close()
    ms = reduce_over_ranks(ms, "max", dist, device)
    cells = int(reduce_over_ranks(cells_rank, "sum", dist, device))
    return {"value": cells * steps / (ms / 1e3), "unit": "cell-steps/s", "members": n, "cells": cells,
            "members_per_rank": len(cfgs), "scaling": "strong" if world > 1 else None,
            "ms_per_step": ms / steps, "steps": steps, "warmup": Wm, "dtype": "f32", "gpu_launches": 1,
            "tiles": tiles, "tile": f"32x{rows}",
            "tile_tuning_ms": {"32x4": tune_ms[0], "32x8": tune_ms[1], "32x16": tune_ms[2]},
            "wet_tiles_end_mean": wet,
            "config": "256 scenarios, sides clip(round16(lognormal(ln 256, ln4/2)), 64, 1024), dx 5 m, "
                      "spectral DEMs, delta_b U(15,30) deg, c_D U(1e-4,1e-2) 1/s, release U(1e4,1e6) m^3, FP32, "
                      f"{steps} steps timed whole"}


def measure_arc_plane(torch):
    """The arc-plane release at its stated size and length: 128 x 128 cells at
    5 m, closed boundaries, CFL 0.5, 2000 steps, FP64 (CUDA events); the tile
    shape from the autotuner on the release state (its probes change no
    state)."""
    from paper_2104_06784_gb300 import moses, workloads as W
    cfg = W.release_config()
    with moses.from_config(cfg, precision=moses.FP64) as sim:
        sim.step(3)
        sim.set_release(cfg["h"], cfg["phi_s"])
        sim.autotune()
        tile = sim.tile_name()
        stream = torch.cuda.current_stream()
        torch.cuda.synchronize()
        e0, e1 = _events(torch)
        e0.record(stream)
        sim.step(cfg["steps"])
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        b = sim.budget()
    v0 = W.release_volume(cfg["h"], cfg["dem"], cfg["dx"])
    return {"config": "arc-plane release, 128x128 cells at 5 m, closed, CFL 0.5, 2000 steps, FP64",
            "steps": cfg["steps"], "ms": ms, "value": 128 * 128 * cfg["steps"] / (ms / 1e3), "dtype": "f64",
            "tile": tile,
            "t_end_s": b["t"], "clamp_cells": b["clamp_cells"],
            "volume_m3": b["vol_s"] + b["vol_f"], "release_volume_m3": v0}


def measure_inflow(torch, precision=None):
    """The inflow hydrograph at its stated size and length: 2048 x 1024 cells
    at 5 m, channel-and-fan DEM, triangular hydrograph (800 m^3/s at 60 s, 0 by
    300 s) at a 20-cell inlet, run to t = 600 s, FP32 state with FP64 budgets.
    Device time from CUDA events around the whole run; the mass budget closes
    on the boundary fluxes (volume - boundary inflow - clamp volume).  The
    run starts dry, so the tile shape comes from the autotuner on a second
    simulation of the same workload advanced to t = 120 s (untimed)."""
    from paper_2104_06784_gb300 import moses, workloads as W
    cfg = W.inflow_config()
    prec = moses.FP32 if precision is None else precision
    with moses.from_config(cfg, precision=prec) as probe:
        probe.run_until(120.0)
        tile_id, _ = probe.autotune()
    with moses.from_config(cfg, precision=prec) as sim:
        sim.set_tile(tile_id)
        tile = sim.tile_name()
        stream = torch.cuda.current_stream()
        torch.cuda.synchronize()
        e0, e1 = _events(torch)
        e0.record(stream)
        n = sim.run_until(cfg["t_end"])
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        b = sim.budget()
        U = sim.get_conserved()
    vol = b["vol_s"] + b["vol_f"]
    bnd = b["bnd_in_s"] + b["bnd_in_f"]
    clamp = b["clamp_s"] + b["clamp_f"]
    tq, Q = np.asarray(cfg["inflow"]["t"]), np.asarray(cfg["inflow"]["Q"])
    cells = U.shape[1] * U.shape[2]
    return {"config": "inflow hydrograph, 2048x1024 cells at 5 m, channel-and-fan DEM, triangular Q (800 m^3/s "
                      "peak at 60 s, 0 by 300 s), 20-cell inlet, to t = 600 s, FP32 state + FP64 budgets",
            "steps": n, "t_end_s": b["t"], "ms": ms, "value": cells * n / (ms / 1e3),
            "dtype": "f32" if prec == moses.FP32 else "f64", "tile": tile,
            "volume_m3": vol, "boundary_inflow_m3": bnd, "clamp_volume_m3": clamp,
            "mass_drift_rel": abs(vol - bnd - clamp) / max(bnd, 1e-300),
            "hydrograph_volume_m3": float(np.trapezoid(Q, tq)) if hasattr(np, "trapezoid") else float(np.trapz(Q, tq)),
            "wet_tiles_end": wet_tile_fraction(U), "gpu_launches": 4 * n}


def measure_adjoint(torch, n=1024, steps=None, ckpt=None):
    """Adjoint calibration workload, FP32 forward: 1024 x 1024 cells at 5 m,
    spectral DEM, internal friction 35 deg (Savage-Hutter earth pressure),
    5000 steps with a checkpoint every 71.  The target deposit
    comes from a forward run with the hidden basal friction 22 deg and drag
    3e-3 1/s; the gradient of the deposit misfit at 25 deg, 1e-3 1/s is taken
    with respect to delta_b, phi_int, c_D and the release thickness.  Times:
    the forward run alone (CUDA events), then the forward run with
    checkpoints and the backward pass (recompute + reverse sweep) of
    moses_adjoint_misfit (CUDA events inside the library)."""
    from paper_2104_06784_gb300 import moses, workloads as W
    cfg = W.adjoint_config(n=n)
    N, C = steps or cfg["steps"], ckpt or cfg["ckpt_every"]
    ct = dict(cfg)
    ct["params"] = dict(cfg["params"], **cfg["hidden"])
    with moses.from_config(ct, precision=moses.FP32) as gt:
        gt.step(N)
        st = gt.get_state()
    hs_t = st["h"] * st["phi_s"]
    with moses.from_config(cfg, precision=moses.FP32) as f:
        f.step(3)
        stream = torch.cuda.current_stream()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        f.step(N)
        e1.record(stream)
        torch.cuda.synchronize()
        fwd_ms = e0.elapsed_time(e1)
    with moses.from_config(cfg, precision=moses.FP32) as g:
        r = g.adjoint_misfit(N, hs_t, ckpt_every=C, release_phi=cfg["phi_s"])
    tf, tb = (float(x) for x in r["timing_ms"])
    gh = r["g_release_h"]
    return {"config": f"adjoint calibration, {n}x{n} cells at 5 m, spectral DEM, 1e6 m^3 release, phi_int 35 deg "
                      f"(k_mode 1), FP32 forward, {N} steps, checkpoint every {C}; target from delta_b 22 deg, c_D 3e-3",
            "steps": N, "ckpt_every": C, "dtype": "f32", "forward_ms": fwd_ms,
            "adjoint_forward_ms": tf, "adjoint_backward_ms": tb,
            "backward_over_forward": tb / fwd_ms, "total_over_forward": (tf + tb) / fwd_ms,
            "loss": r["loss"],
            "grad": {"delta_b_per_deg": float(r["g_params"][0]), "phi_int_per_deg": float(r["g_params"][1]),
                     "c_d": float(r["g_params"][2]), "release_h_l2": float(np.sqrt((gh * gh).sum()))},
            # forward: 2 stages of 2 launches per step (the first stage logs the clock), misfit;
            # backward: per step 2 recording stages of 2 launches and 2 x (cell, face; the face
            # kernel folds the ghosts on this grid); release gradient
            "gpu_launches": 4 * N + 1 + 8 * N + 1,
            "fp64_check": "gradients against FP64 central differences of the oracle: tests/test_gpu_adjoint.py"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-configs", action="store_true", help="skip the arc-plane and inflow lines")
    ap.add_argument("--side", type=int, default=N_SIDE, help="grid side (the workload is defined at 4096)")
    ap.add_argument("--event-steps", type=int, default=EVENT_STEPS, help="length of the event (10000)")
    ap.add_argument("--only", choices=["f64", "f32", "adjoint"], default=None,
                    help="measure one precision form (K steps from the start), or only the adjoint")
    ap.add_argument("--wet-layer", type=float, default=0.0,
                    help="add a mixture layer of this depth [m] on every cell (all tiles wet; for profiling)")
    ap.add_argument("--tile", choices=["auto", "32x8", "32x4", "32x16", "32x4-2t"], default="auto",
                    help="stage tile shape: autotuned (default) or pinned")
    ap.add_argument("--from-step", type=int, default=0,
                    help="--only f64 / f32: advance this many steps of the event first (untimed)")
    ap.add_argument("--adj-steps", type=int, default=None, help="adjoint: steps (default: the workload's 5000)")
    ap.add_argument("--adj-ckpt", type=int, default=None, help="adjoint: checkpoint interval (default 71)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.wet_layer > 0 and args.only not in ("f64", "f32"):
        ap.error("--wet-layer is for --only f64 / f32 profiling runs")

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    from paper_2104_06784_gb300 import workloads as W
    cfg = W.large_release_config(n=args.side, dx=DX, seed=0)
    if args.wet_layer > 0:
        cfg = dict(cfg, h=cfg["h"] + args.wet_layer)

    if args.impl == "reference":
        line = run_reference(args, cfg, rank)
        if line is not None:
            print(json.dumps(line), flush=True)
        return

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2104_06784_gb300 import moses
    if args.only == "adjoint":
        adj = measure_adjoint(torch, steps=args.adj_steps, ckpt=args.adj_ckpt)
        if rank == 0:
            print(json.dumps(adj), flush=True)
        return
    side = args.side
    cells = side * side
    K, Wm = args.steps, args.warmup

    def max_over_ranks(x):
        return reduce_over_ranks(x, "max", dist, "cuda")

    forms = [("f64", moses.FP64), ("f32", moses.FP32)]
    if args.only:
        # profiling runs: K steps from the start of the event (or of the wet layer)
        name, prec = [f for f in forms if f[0] == args.only][0]
        sim = moses.from_config(cfg, precision=prec)
        if args.tile != "auto":
            sim.set_tile({v: k for k, v in moses.Sim.TILES.items()}[args.tile])
        else:
            sim.autotune()
        if args.from_step > 0:
            sim.step(args.from_step)
        # the timed steps in an NVTX range `only_<form>` (for a profiler's filter)
        torch.cuda.nvtx.range_push(f"only_{name}")
        ms, stage_ms = measure(sim, cells, K, Wm, torch)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        if rank == 0:
            print(json.dumps({"form": name, "side": side, "from_step": args.from_step, "tile": sim.tile_name(),
                              "ms_per_step": ms / K, "launch_ms": (stage_ms[0] + stage_ms[1]) / (2 * K),
                              "value": world * cells * K / (ms / 1e3)}), flush=True)
        sim.close()
        return

    pk, pk_src = peaks()
    fp64_tflops = moses.fp64_rate()
    h = stage_hash()
    results, tiles = {}, {}
    sampler = ClockSampler(local)
    nwin = N_WINDOWS
    for name, prec in forms:
        sim = moses.from_config(cfg, precision=prec)
        if args.tile == "auto":
            tile, tile_ms = sim.autotune()  # the project's tile autotuner
            tiles[name] = {"tile": moses.Sim.TILES[tile],
                           "ms_per_launch": {moses.Sim.TILES[t]: tile_ms[t] for t in range(len(tile_ms))}}
        else:
            tile = {v: k for k, v in moses.Sim.TILES.items()}[args.tile]
            sim.set_tile(tile)
            tiles[name] = {"tile": args.tile, "pinned": True}
        ts = moses.Sim.TILE_SHAPES[tile]
        ckpts, event = run_event(sim, torch, nsteps=args.event_steps, nwin=nwin, tile=ts)
        if dist is not None:
            dist.barrier()
        with (sampler if name == "f64" else _Null()):
            win_ms = measure_windows(sim, ckpts, K, Wm, torch, sampler if name == "f64" else None,
                                     nvtx=f"headline_windows_{name}")
        del ckpts
        ms = max_over_ranks(sum(win_ms))
        results[name] = dict(ms=ms, win_ms=win_ms, event=event, sim=sim)
        if name == "f32":
            sim.close()

    f64, f32 = results["f64"], results["f32"]
    value = world * cells * K * nwin / (f64["ms"] / 1e3)

    # the kernels' own rate: every tile wet
    dense = measure_dense(cfg, K, Wm, torch, fp64_tflops, pk["hbm_gbs"], h)
    # the flux phase in double-float arithmetic (pairs of FP32 numbers, not
    # IEEE FP64) against FP64, on 4M synthetic faces: an evaluation, not a
    # stepping form
    dfe = moses.flux_eval(1 << 22, 10)
    dfe["speedup"] = dfe["df_gfaces_per_s"] / dfe["f64_gfaces_per_s"] if dfe["f64_gfaces_per_s"] > 0 else None
    dfe["note"] = "central face flux (face_flux2) only; double-float is not IEEE FP64"
    d64, d32 = dense["f64"], dense["f32"]
    roof64 = {"bound": "alu", "achieved": d64["alu"]["achieved"], "peak": fp64_tflops, "unit": "TFLOP/s",
              "frac": d64["alu"]["achieved"] / fp64_tflops, "traffic": d64["traffic_per_launch"],
              "kernel": "moses::stage_kernel_list<double,32,8> with its classification launch, one stage, "
                        "on the all-wet 4096^2 state (488 flops per cell and stage)",
              "peak_source": "measured FP64 FMA rate (moses_debug_fp64_rate); "
                             f"{FP64_PEAK_TFLOPS:.3f} TFLOP/s from unit counts and clock",
              "hbm": {"achieved": d64["hbm"]["achieved"], "peak": pk["hbm_gbs"], "unit": "GB/s",
                      "frac": d64["hbm"]["frac"], "bytes_per_cell_step": 104, "peak_source": pk_src}}
    roof32 = {"bound": "hbm", "achieved": d32["hbm"]["achieved"], "peak": pk["hbm_gbs"], "unit": "GB/s",
              "frac": d32["hbm"]["frac"], "traffic": d32["traffic_per_launch"],
              "kernel": "moses::stage_kernel_list<float,32,8> with its classification launch, one stage, "
                        "on the all-wet 4096^2 state (52 B per cell-step)",
              "peak_source": pk_src, "alu": d32["alu"]}

    # end to end through the C-ABI with pinned host buffers: per step, upload
    # the state, one step, download the state
    e2e = None
    if not args.no_e2e:
        sim = f64["sim"]
        Uh = torch.empty((6, side, side), dtype=torch.float64, pin_memory=True).numpy()
        sim.get_conserved(out=Uh)
        for _ in range(2):
            sim.set_conserved(Uh)
            sim.step(1)
            sim.get_conserved(out=Uh)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        t0 = time.perf_counter()
        Ke = max(3, K // 2)
        for _ in range(Ke):
            sim.set_conserved(Uh)
            sim.step(1)
            sim.get_conserved(out=Uh)
        torch.cuda.synchronize()
        el = max_over_ranks(time.perf_counter() - t0)
        e2e = {"value": world * cells * Ke / el, "unit": UNIT, "h2d_bytes_per_step": int(Uh.nbytes),
               "d2h_bytes_per_step": int(Uh.nbytes),
               "calls": "moses_set_conserved + moses_step(1) + moses_get_conserved, pinned host buffers, "
                        "on the state at the start of the last quarter of the event"}
    f64["sim"].close()

    ens = None if args.no_ensemble else measure_ensemble(K, Wm, rank=rank, world=world, dist=dist, device="cuda")
    adj = None if args.no_adjoint else measure_adjoint(torch)
    variants = None if args.no_variants else measure_variants(cfg, K, Wm, torch)
    arc = None if args.no_configs else measure_arc_plane(torch)
    infl = None if args.no_configs else measure_inflow(torch)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(cfg)
        cpu.pop("seconds", None)

    def windows(r):
        return [{"from_step": sg["from_step"], "wet_tiles": sg["wet_tiles"], "ms_per_step": m / K}
                for sg, m in zip(r["event"]["segments"], r["win_ms"])]

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": Wm,
        "ms_per_step": f64["ms"] / (K * nwin), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (seeded spectral DEM and release; see workloads.py)",
        "config": config_dict(cfg, args), "roofline": roof64, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": 4 * K * nwin, "clocks": sampler.summary(),
        "windows": windows(f64), "event": f64["event"],
        "f32": {"value": world * cells * K * nwin / (f32["ms"] / 1e3), "ms_per_step": f32["ms"] / (K * nwin),
                "dtype": "f32", "roofline": roof32, "gpu_launches": 4 * K * nwin, "windows": windows(f32),
                "event": f32["event"]},
        "dense": dense,
        "fp64_fma_tflops": fp64_tflops,
        "double_float_flux": dfe,
        "arc_plane": arc,
        "inflow": infl,
        "ensemble": ens,
        "adjoint": adj,
        "variants": variants,
        "tiles": tiles,
        "stage_source": h,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


class _Null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        pass


if __name__ == "__main__":
    main()
