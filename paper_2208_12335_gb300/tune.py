"""Autotuner for the batching settings of the tensor-core path.

The contractions run on fixed 128 x 128 tcgen05 tiles; what changes the
speed of a workload is how its batches are grouped: how many points an H
or density super-batch may gather (larger super-batches make the MMAs
deeper and cut the tiles and scatter atomics, but pad the union of active
functions) and how much operand-image workspace one wave may use.  `tune` plans the problem once per candidate
setting, times the H + density step with CUDA events on the device, and
writes the fastest setting to a text file that `fgi_plan` reads
(`Context.load(problem, precision, tune_path=...)`).

Only timing is done here; every candidate computes the same integrals.
"""
from __future__ import annotations

import os
import tempfile

import numpy as np
import torch

from .fgi import Context

DEFAULT_CANDIDATES = [
    {"density_sb_points": 0},
    {"h_sb_points": 0},
    {"h_sb_points": 256, "h_sb_growth": 1.25},
    {"h_sb_points": 400, "h_sb_growth": 1.25},
    {"h_sb_points": 512, "h_sb_growth": 1.25},
    # deeper H super-batches are faster but add FP32 truncation in the
    # remainder products: 576 points and more gave 1.2e-7 Ha on the Si64
    # cluster (over the 1e-7 bound), so they are not offered here
    {"density_sb_points": 512, "density_sb_growth": 1.35},
    {"density_sb_points": 768, "density_sb_growth": 1.35},
    {"density_sb_points": 1024, "density_sb_growth": 1.2},
    {"density_sb_points": 1024, "density_sb_growth": 1.35},
    {"density_sb_points": 1024, "density_sb_growth": 1.6},
    # operand images per wave (default 8192 MiB): the persistent contraction
    # kernels take a wave's tiles with a fixed stride, so shorter waves keep
    # their CTAs closer together in the tile list (less L2 thrash) at the
    # price of more launches
    {"wave_mb": 3072},
    {"wave_mb": 24576},
]


def write_settings(path: str, settings: dict) -> None:
    with open(path, "w") as f:
        for k, v in settings.items():
            f.write("%s %s\n" % (k, v))


def read_settings(path: str) -> dict:
    out = {}
    with open(path) as f:
        for line in f:
            parts = line.split()
            if len(parts) == 2:
                out[parts[0]] = float(parts[1])
    return out


def time_step(ctx: Context, v, d, steps: int = 3, warmup: int = 2) -> float:
    """Mean device time (ms) of integrate_h + density on the current stream."""
    ws = ctx.workspace()
    n_fn, nnz, n_pts, _ = ctx.sizes()
    h = torch.empty(nnz, dtype=torch.float64, device=v.device)
    n = torch.empty(n_pts, dtype=torch.float64, device=v.device)
    for _ in range(warmup):
        ctx.integrate_h(v, h, ws=ws)
        ctx.density(d, n, ws=ws)
    ctx.sync()
    stream = torch.cuda.current_stream(v.device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        ctx.integrate_h(v, h, ws=ws)
        ctx.density(d, n, ws=ws)
    e1.record(stream)
    e1.synchronize()
    ctx.sync()
    return e0.elapsed_time(e1) / steps


def tune(problem, path: str, precision: str = "split_bf16", device: int = 0, candidates=None,
         steps: int = 3, seed: int = 0, verbose: bool = False) -> dict:
    """Time every candidate setting on `problem` and write the fastest to
    `path`.  Returns {"best": settings, "ms": {label: ms}}.  The density
    matrix used for timing is seeded random (timing does not depend on it)."""
    candidates = DEFAULT_CANDIDATES if candidates is None else candidates
    dev = torch.device("cuda:%d" % device)
    v = torch.from_numpy(np.ascontiguousarray(problem.v)).to(dev)
    times = {}
    best, best_ms = None, float("inf")
    with tempfile.TemporaryDirectory() as tmp:
        for i, cand in enumerate(candidates):
            cpath = os.path.join(tmp, "cand%d.txt" % i)
            write_settings(cpath, cand)
            ctx = Context(device).load(problem, precision, tune_path=cpath)
            nnz = ctx.sizes()[1]
            rng = np.random.default_rng(seed)
            d = torch.from_numpy(rng.standard_normal(nnz) * 0.05).to(dev)
            ms = time_step(ctx, v, d, steps=steps)
            label = " ".join("%s=%s" % kv for kv in cand.items())
            times[label] = ms
            if verbose:
                print("tune: %-50s %.3f ms" % (label, ms), flush=True)
            if ms < best_ms:
                best, best_ms = cand, ms
            ctx.close()
    write_settings(path, best)
    return {"best": best, "ms": times}
