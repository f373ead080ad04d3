#!/usr/bin/env python
"""Throughput of the two-phase shallow-flow step on one GB300 (cell-steps/s).

Workload: the large-scale release event -- 4096 x 4096 cells at 10 m over a
seeded 1/f^2.2 spectral DEM (1500 m relief) with one carved valley, a
2.5e7 m^3 parabolic-cap release on a 30-40 degree slope, solid fraction
U(0.55, 0.65), transmissive boundaries, CFL 0.1 (synthetic stand-in for the
Hsiaolin event of Sect. 4.1; the real DEM is not available).

A step is one full time step: CFL time step from the exact max-reduction, two
stages of the central scheme with all sources, Heun average, boundary fill.
Each stage is two launches: the wet/dry classification, which writes the
stage result of every tile without mass in reach (the zero state), and the
stage kernel on the listed tiles.  The release covers a small part of the
terrain, so most tiles are dry: the step streams the state through HBM and
the line reports the HBM roofline, the wet-tile fraction, and (`dense`) the
same kernels on an all-wet state, where the stage is bound by its FP64
arithmetic.  The headline is the FP64 form; the FP32 form (FP64 budgets and
friction test) is measured in the same run.  The state (0.8 GB in FP64) is
larger than L2, so no flush is needed between steps.

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
# With wet/dry masking a step need not touch a dry cell's state: it must read
# the two mass planes of every cell once (the wet test; FP32: 2 x 4 B masses
# and 2 x 4 B remainders, FP64: 2 x 8 B), and move the whole cell-step traffic
# above only for the cells of the tiles that compute.
MASS_TEST_BYTES = 16


def step_bytes(cells, wet_frac, esz):
    """Algorithmic HBM bytes of one masked step: the wet test over every cell
    plus the cell-step traffic of the cells in tiles with work."""
    return MASS_TEST_BYTES * cells + WORDS_PER_CELL_STEP * esz * wet_frac * cells

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one step --
# the wet/dry classification launch plus the listed-tile stage launch, both
# stages -- per cell of the 4096^2 workload, from an ncu capture of bench.py
# itself at full size (one-pass metrics) over the timed steps; valid only for
# the stage kernel source it was taken on (sha256 of csrc/stage.cuh, first
# 12) and for this workload (the wet fraction sets it).
TRAFFIC = {
    # profiles/stage_kernel_launch_list_4096_release.md (tile 32 x 8; the
    # classification's read of the mass planes is 95 % of it at any tile shape)
    ("f64", "beb8a8d2e738"): 16.87,
    # before the known-zero tile flags
    ("f64", "f1a1dc700d9f"): 108.86,
    ("f32", "f1a1dc700d9f"): 77.80,
}


def _traffic(form, h, side):
    b = TRAFFIC.get((form, h))
    return None if b is None or side != N_SIDE else b * side * side


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# FP64 vector peak of GB300: 152 SMs x 2 FP64 FMA/clk x 2 flops x 2.07 GHz
# = 1.26 TFLOP/s, matching the 1.25 TFLOP/s nominal figure.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


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


def cpu_baseline(cfg, steps=None, window=1024):
    """The FP64 oracle as it stands, single-threaded on the host, on a bounded
    sample: `steps` steps on a window x window crop of the workload centred on
    the release (throughput per cell-step does not depend on the size)."""
    from oracle.oracle import OracleSim
    ic, jc = cfg["release_cell"]
    n = cfg["dem"].shape[0]
    i0 = int(min(max(ic - window // 2, 0), n - window))
    j0 = int(min(max(jc - window // 2, 0), n - window))
    sl = (slice(j0, j0 + window), slice(i0, i0 + window))
    o = OracleSim(cfg["dem"][sl], cfg["dx"], cfg["dy"], cfg["params"])
    o.set_release(cfg["h"][sl], cfg["phi_s"][sl])
    o.step(1)
    steps = steps or 20
    t0 = time.perf_counter()
    o.step(steps)
    el = time.perf_counter() - t0
    return dict(value=window * window * steps / el, unit=UNIT, cores=1, kind="oracle",
                sample=f"{steps} FP64 steps of the oracle on the {window}x{window} window of the "
                       f"{n}x{n} workload around the release, 1 thread",
                seconds=el)


def run_reference(args, cfg, rank):
    """The reference arm: the CPU oracle timed on the host, K steps after W
    warm-up steps, each step one oracle step on a 1024 x 1024 window."""
    if rank != 0:
        return None
    from oracle.oracle import OracleSim
    window = 1024
    ic, jc = cfg["release_cell"]
    n = cfg["dem"].shape[0]
    i0 = int(min(max(ic - window // 2, 0), n - window))
    j0 = int(min(max(jc - window // 2, 0), n - window))
    sl = (slice(j0, j0 + window), slice(i0, i0 + window))
    o = OracleSim(cfg["dem"][sl], cfg["dx"], cfg["dy"], cfg["params"])
    o.set_release(cfg["h"][sl], cfg["phi_s"][sl])
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    el = time.perf_counter() - t0
    v = window * window * args.steps / el
    sample = f"each step: one FP64 oracle step on the {window}x{window} window of the {n}x{n} workload, 1 thread"
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(cfg, args),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def config_dict(cfg, args):
    n = cfg["dem"].shape[0]
    return {"workload": f"large-scale release event, {n}x{n} cells at {DX:g} m, spectral DEM "
                        f"(beta 2.2, 1500 m relief, carved valley), 2.5e7 m^3 release, CFL 0.1",
            "cells": n * n, "dx_m": DX, "l2": "state larger than L2 (0.8 GB FP64, 0.4 GB FP32); no flush",
            "parallelism": f"replicas x{args.gpus}" if args.gpus > 1 else "single GPU"}


def measure(sim, cells, K, W, torch, sampler=None):
    """Device time of K steps (after W warm-up steps) with CUDA events on the
    simulation's stream; per-stage launch times from moses_step_timed."""
    sim.step(W)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
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


def measure_dense(cfg, K, Wm, torch):
    """The same 4096^2 terrain and release with a 5 cm mixture layer over every
    cell, so that every tile computes (no dry tile to skip): the stage's
    arithmetic-bound rate, for comparison with the masked workload."""
    from paper_2104_06784_gb300 import moses
    c = dict(cfg, h=cfg["h"] + 0.05)
    out = {"config": "the 4096^2 workload plus a 5 cm layer (phi_s as the release) on every cell: all tiles wet"}
    for form, prec in (("f64", moses.FP64), ("f32", moses.FP32)):
        with moses.from_config(c, precision=prec) as sim:
            ms, stage_ms = measure(sim, sim.nx * sim.ny, K, Wm, torch)
            cells = sim.nx * sim.ny
        launch_ms = (stage_ms[0] + stage_ms[1]) / (2 * K)
        out[form] = {"ms_per_step": ms / K, "value": cells * K / (ms / 1e3), "launch_ms": launch_ms}
        if form == "f64":
            ach = FLOPS_PER_CELL_STAGE * cells / (launch_ms / 1e3) / 1e12
            out[form]["alu"] = {"achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                                "frac": ach / FP64_PEAK_TFLOPS}
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


def measure_ensemble(K, Wm, seed=0, n=256, rank=0, world=1, dist=None, device="cpu"):
    """Batched ensemble, FP32: 256 members on square grids of lognormal side
    (64..1024 cells, 5 m), each its own spectral DEM, basal friction, drag and
    release volume; per stage one batched classification launch and one
    batched launch over the wet tiles of all members, replayed from a CUDA graph.
    Device time from CUDA events on the batch's stream.  With several ranks
    the members are sharded across them; the time is the max over ranks."""
    from paper_2104_06784_gb300 import moses, workloads as W
    cfgs = shard(W.ensemble_config(n, seed=seed), rank, world)
    cells_rank = int(sum(c["dem"].size for c in cfgs))
    sims = [moses.from_config(c, precision=moses.FP32) for c in cfgs]
    with moses.Batch(sims) as b:
        b.step(Wm)
        if dist is not None:
            dist.barrier()
        ms = b.step_timed(K)
        tiles = b.tiles
    for s_ in sims:
        s_.close()
    ms = reduce_over_ranks(ms, "max", dist, device)
    cells = int(reduce_over_ranks(cells_rank, "sum", dist, device))
    return {"value": cells * K / (ms / 1e3), "unit": "cell-steps/s", "members": n, "cells": cells,
            "members_per_rank": len(cfgs), "scaling": "strong" if world > 1 else None,
            "ms_per_step": ms / K, "steps": K, "warmup": Wm, "dtype": "f32", "gpu_launches": 4 * K,
            "tiles_per_launch": tiles,
            "config": "256 scenarios, sides clip(round16(lognormal(ln 256, ln4/2)), 64, 1024), dx 5 m, "
                      "spectral DEMs, delta_b U(15,30) deg, c_D U(1e-4,1e-2) 1/s, release U(1e4,1e6) m^3, FP32"}


def measure_adjoint(torch, n=1024, steps=None, ckpt=None):
    """Adjoint calibration workload, FP32 forward: 1024 x 1024 cells at 5 m,
    spectral DEM, 5000 steps with a checkpoint every 71.  The target deposit
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
    return {"config": f"adjoint calibration, {n}x{n} cells at 5 m, spectral DEM, 1e6 m^3 release, FP32 forward, "
                      f"{N} steps, checkpoint every {C}; target from delta_b 22 deg, c_D 3e-3",
            "steps": N, "ckpt_every": C, "dtype": "f32", "forward_ms": fwd_ms,
            "adjoint_forward_ms": tf, "adjoint_backward_ms": tb,
            "backward_over_forward": tb / fwd_ms, "total_over_forward": (tf + tb) / fwd_ms,
            "loss": r["loss"],
            "grad": {"delta_b_per_deg": float(r["g_params"][0]), "phi_int_per_deg": float(r["g_params"][1]),
                     "c_d": float(r["g_params"][2]), "release_h_l2": float(np.sqrt((gh * gh).sum()))},
            # forward: 2 stages + 2 records per step, misfit; backward: per step 1 time reset,
            # 2 recording stages, 2 x (cell, face, fold); release gradient
            "gpu_launches": 4 * N + 1 + 9 * N + 1,
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
    ap.add_argument("--side", type=int, default=N_SIDE, help="grid side (the workload is defined at 4096)")
    ap.add_argument("--only", choices=["f64", "f32", "adjoint"], default=None,
                    help="measure one precision form, or only the adjoint")
    ap.add_argument("--wet-layer", type=float, default=0.0,
                    help="add a mixture layer of this depth [m] on every cell (all tiles wet; for profiling)")
    ap.add_argument("--tile", choices=["auto", "32x8", "32x4", "32x16"], default="auto",
                    help="stage tile shape: autotuned (default) or pinned")
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

    results = {}
    sampler = ClockSampler(local)
    forms = [("f64", moses.FP64), ("f32", moses.FP32)]
    if args.only:
        forms = [f for f in forms if f[0] == args.only]
    tiles = {}
    for name, prec in forms:
        sim = moses.from_config(cfg, precision=prec)
        if args.tile == "auto":
            tile, tile_ms = sim.autotune()  # the project's tile autotuner
            tiles[name] = {"tile": moses.Sim.TILES[tile],
                           "ms_per_launch": {moses.Sim.TILES[t]: tile_ms[t] for t in range(3)}}
        else:
            tile = {v: k for k, v in moses.Sim.TILES.items()}[args.tile]
            sim.set_tile(tile)
            tiles[name] = {"tile": args.tile, "pinned": True}
        if dist is not None:
            dist.barrier()
        with (sampler if name == "f64" else _Null()):
            ms, stage_ms = measure(sim, cells, K, Wm, torch, sampler if name == "f64" else None)
        ms = max_over_ranks(ms)
        launch_ms = (stage_ms[0] + stage_ms[1]) / (2 * K)
        results[name] = dict(ms=ms, launch_ms=launch_ms, stage_ms=[stage_ms[0] / K, stage_ms[1] / K], sim=sim)
        if not args.only:
            t = tiles[name]["tile"].split("x")
            results[name]["wet_tiles"] = wet_tile_fraction(sim.get_conserved(), int(t[0]), int(t[1]))
        if name == "f32":
            sim.close()

    if args.only:
        r = results[args.only]
        if rank == 0:
            print(json.dumps({"form": args.only, "side": side, "ms_per_step": r["ms"] / K,
                              "launch_ms": r["launch_ms"], "value": world * cells * K / (r["ms"] / 1e3)}), flush=True)
        r["sim"].close()
        return
    pk, pk_src = peaks()
    f64 = results["f64"]
    value = world * cells * K / (f64["ms"] / 1e3)
    h = stage_hash()
    t64, t32 = tiles["f64"]["tile"], tiles["f32"]["tile"]
    # The release covers a small part of the terrain: most tiles are dry, skip
    # their arithmetic and, once their output holds the zero state, their
    # writes too (wet/dry masking with known-zero tile flags).  A step then
    # reads the mass planes once (HBM) and runs the stage arithmetic on the
    # few wet tiles (FP64 pipe); the roofline counts the bytes such a step
    # must move (step_bytes).  The all-wet measurement (`dense`) gives the
    # arithmetic-bound rate of the same kernel.
    b64 = step_bytes(cells, f64["wet_tiles"], 8)
    gbs64 = b64 / (2 * f64["launch_ms"] / 1e3) / 1e9
    roof64 = {"bound": "hbm", "achieved": gbs64, "peak": pk["hbm_gbs"], "unit": "GB/s",
              "frac": gbs64 / pk["hbm_gbs"], "traffic": _traffic("f64", h, side),
              "kernel": f"one step: moses::classify_kernel<double,{t64.split('x')[1]}> + "
                        f"moses::stage_kernel_list<double,{t64.replace('x', ',')}>, two stages",
              "peak_source": pk_src, "wet_tiles": f64["wet_tiles"], "bytes_per_step": b64}
    f32 = results["f32"]
    b32 = step_bytes(cells, f32["wet_tiles"], 4)
    gbs32 = b32 / (2 * f32["launch_ms"] / 1e3) / 1e9
    roof32 = {"bound": "hbm", "achieved": gbs32, "peak": pk["hbm_gbs"], "unit": "GB/s",
              "frac": gbs32 / pk["hbm_gbs"], "traffic": _traffic("f32", h, side),
              "kernel": f"one step: moses::classify_kernel<float,{t32.split('x')[1]}> + "
                        f"moses::stage_kernel_list<float,{t32.replace('x', ',')}>, two stages",
              "peak_source": pk_src, "wet_tiles": f32["wet_tiles"], "bytes_per_step": b32}

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
               "calls": "moses_set_conserved + moses_step(1) + moses_get_conserved, pinned host buffers"}
    f64["sim"].close()

    ens = None if args.no_ensemble else measure_ensemble(K, Wm, rank=rank, world=world, dist=dist, device="cuda")

    adj = None if args.no_adjoint else measure_adjoint(torch)
    variants = None if args.no_variants else measure_variants(cfg, K, Wm, torch)
    dense = None if args.no_variants else measure_dense(cfg, K, Wm, torch)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(cfg)
        cpu.pop("seconds", None)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": Wm,
        "ms_per_step": f64["ms"] / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (seeded spectral DEM and release; see workloads.py)",
        "config": config_dict(cfg, args), "roofline": roof64, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": 4 * K, "clocks": sampler.summary(),
        "f32": {"value": world * cells * K / (f32["ms"] / 1e3), "ms_per_step": f32["ms"] / K, "dtype": "f32",
                "roofline": roof32, "gpu_launches": 4 * K},
        "ensemble": ens,
        "adjoint": adj,
        "variants": variants,
        "dense": dense,
        "stage_ms": {"f64": f64["stage_ms"], "f32": f32["stage_ms"]},
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
