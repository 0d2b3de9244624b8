"""Benchmark: grid points/s and TFLOP/s of H integration + density on one GB300.

One step = one pass of the whole hot path over the workload: basis
evaluation, H contraction with sparse FP64 scatter, density contraction and
the FP64 electron-count traces, for every batch of the grid.  The plan
(active functions, pattern, work lists) is built once, off the timed path.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload si64]
                    [--precision split_bf16|bf16|fp64] [--impl reference]

Prints one JSON line (rank 0).  Under torchrun (N > 1) every rank runs an
independent replica of the workload (weak scaling, no collective on the data
path); the time is the max over ranks.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "grid pts/s and TFLOP/s for H-integ+density on 1 GB300, split-BF16 vs FP64 at stated err"
UNIT = "grid_pts/s"


def make_workload(name, accel=None):
    """The synthetic workloads; accel='cuda' builds partition weights and
    potentials with torch on the GPU (same definitions, faster)."""
    if name == "tiny":
        return W.tiny_water(), "tiny water: 3 atoms, 7 fns, 40x110 pts/atom"
    if name == "si64":
        return (W.si64(accel=accel),
                "Si64 cluster: 64 atoms, 1600 fns (6s3p2d), 60x302 pts/atom, batches <=300 pts")
    if name == "chno1000":
        return (W.chno_cluster(accel=accel),
                "1000-atom CHNO cluster, 19 fns/heavy atom, 5/H, 70x590 pts/atom, uneven batches 50-400 pts")
    if name.startswith("chno"):
        n = int(name[4:])
        return W.chno_cluster(n_atoms=n, accel=accel), "%d-atom CHNO cluster, 70x590 pts/atom" % n
    if name.startswith("many"):
        n = int(name[4:] or 512)
        return (W.many_molecules(n_mol=n, accel=accel),
                "%d independent CHNO molecules of 5-40 atoms, 30-60 x 110-302 pts/atom" % n)
    raise SystemExit("unknown workload " + name)


def gen_backend():
    """'cuda' when a CUDA device is present (input generation only), else None."""
    try:
        import torch
        return "cuda" if torch.cuda.is_available() else None
    except Exception:
        return None


def density_matrix(prob, rng):
    n = prob.n_fn_sys(0)
    if n <= 4000:
        D, _ = W.density_matrix_occ(n, max(1, int(round(0.28 * n))), rng)
        return D
    return None


def stored_values(ctx, M, s=0):
    rowptr, col = ctx.pattern(s)
    rows = np.repeat(np.arange(len(rowptr) - 1), np.diff(rowptr))
    return M[rows, col], rows, col


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.lines = []              # (host monotonic time, csv line)
        self.window = None           # (start, end) of the timed region
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200",
                                          "-i", str(self.index)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # wait (3 s at most) for the first sample, so that sampling is
            # running through the whole timed region that follows
            t0 = time.monotonic()
            while not self.lines and self.proc.poll() is None and time.monotonic() - t0 < 3.0:
                time.sleep(0.01)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def mark(self, start, end):
        """Keep only the samples taken while [start, end] ran (host clock)."""
        self.window = (start, end)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = self.lines
        if self.window is not None:
            # a sample line arrives up to one interval after it was taken
            inside = [r for r in rows if self.window[0] <= r[0] <= self.window[1] + 0.25]
            rows = inside if inside else rows
        for _, ln in rows:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, x in zip(names, f[5:9]):
                if x.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def fp64_gemm_peak(torch):
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    for _ in range(2):
        a @ b
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = 1e30
    for _ in range(5):
        e0.record()
        a @ b
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return 2.0 * n ** 3 / (best * 1e-3) / 1e12


def fp32_alu_peak(torch, mhz):
    """FP32 FMA issue rate of the device: SMs x 128 lanes x 2 FLOP per clock."""
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    return sms * 128 * 2 * mhz * 1e6 / 1e12


def traffic_for(kind, workload="chno1000"):
    """DRAM bytes per algorithmic flop of a kernel class from the committed
    ncu summary, if it was taken on the current kernel source and for this
    workload; else None.  Times a launch's algorithmic flops it gives the
    launch's DRAM traffic (launches change with the wave budget)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            tab = json.load(f)
    except Exception:
        return None
    ent = tab.get(kind)
    if not ent:
        return None
    src = os.path.join(ROOT, "paper_2208_12335_gb300", "csrc", ent["source"])
    try:
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except Exception:
        return None
    if h != ent.get("source_sha256_16"):
        return None
    if ent.get("workload", "chno1000") != workload:
        return None
    return ent.get("dram_bytes_per_algorithmic_flop")


def oracle_sample(prob, D, n_batches, seed=7, keep=False):
    """The FP64 oracle (H over the active functions + density) on a seeded
    sample of batches; returns (points, seconds, threads, batches) and, with
    keep, also (sub-problem, active functions, H, D, n) of the sample."""
    import oracle as O
    rng = np.random.default_rng(seed)
    cand = np.nonzero(prob.batch_sys == 0)[0]          # system 0 (D and the basis are its)
    ids = np.sort(rng.choice(cand, size=min(n_batches, len(cand)), replace=False))
    sub = prob.subgrid(ids)
    B = O.system_basis(sub)
    act = O.active_functions(B, sub.pts)
    t0 = time.perf_counter()
    Hs = O.h_matrix(B, sub.pts, sub.w, sub.v, sub=act)
    Ds = D[np.ix_(act, act)] if D is not None else np.eye(len(act))
    ns = O.density(B, sub.pts, Ds, sub=act)
    dt = time.perf_counter() - t0
    out = (sub.n_pts, dt, O.num_threads(), len(ids))
    return out + ((sub, act, Hs, Ds, ns) if keep else ())


def oracle_single_core(prob, D, n_batches=2, seed=3):
    """The oracle on one thread over a small seeded sample: points/s."""
    import oracle as O
    n = O.num_threads()
    O.set_num_threads(1)
    try:
        p, dt, _, _ = oracle_sample(prob, D, n_batches, seed=seed)
    finally:
        O.set_num_threads(n)
    return p / dt


def compare_on_sample(sample, precision, device, dev, torch, Context):
    """The library on the oracle's sample (the same sub-grid, planned on its
    own): max |dH| over the stored entries of system 0 and the density's
    relative L2 error, against the oracle results of the CPU-baseline leg."""
    sub, act, Hs, Ds, ns = sample
    cx = Context(device).load(sub, precision)
    rp, col = cx.pattern(0)
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    pos = -np.ones(len(rp) - 1, dtype=np.int64)
    pos[act] = np.arange(len(act))
    inside = (pos[rows] >= 0) & (pos[col] >= 0)
    nnz0 = len(col)
    h = cx.integrate_h(torch.from_numpy(sub.v).to(dev)).cpu().numpy()
    ref = np.zeros(nnz0)
    ref[inside] = Hs[pos[rows[inside]], pos[col[inside]]]
    dvals = np.zeros(cx.sizes()[1])        # functions outside act vanish on the sample
    dvals[:nnz0][inside] = Ds[pos[rows[inside]], pos[col[inside]]]
    n, _ = cx.density(torch.from_numpy(dvals).to(dev))
    cx.sync()
    n = n.cpu().numpy()
    res = {"max_abs_dH_sample": float(np.max(np.abs(h[:nnz0] - ref))),
           "max_abs_H_sample": float(np.max(np.abs(Hs))),
           "density_rel_l2_sample": float(np.linalg.norm(n - ns) / np.linalg.norm(ns)),
           "sample_points": int(sub.n_pts)}
    cx.close()
    return res


def executed_tensor_flops(ctx, products):
    """BF16 tensor-core FLOPs one step (H + density) executes, from the
    plan's schedules: 128 x 128 output tiles, contraction depth in chunks
    of 64, padding included; H over the upper tile triangle, the density
    over the upper block triangle of D."""
    tot = 0.0
    sh = ctx.schedule("h")
    for P_, n_, rank in zip(sh["sb_points"], sh["sb_fns"], sh["sb_rank"]):
        if rank < 0:
            continue
        nrb, nc = -(-int(n_) // 128), -(-int(P_) // 64)
        tot += nrb * (nrb + 1) / 2 * 2.0 * 128 * 128 * nc * 64
    sd = ctx.schedule("density")
    for P_, n_, rank in zip(sd["sb_points"], sd["sb_fns"], sd["sb_rank"]):
        if rank < 0:
            continue
        nrb, nkc, nc = -(-int(n_) // 128), -(-int(n_) // 64), -(-int(P_) // 64)
        tiles = (nc + 1) // 2
        for J in range(nrb):
            tot += tiles * 2.0 * 128 * 128 * (nkc - 2 * J) * 64
    return tot * products


def run_reference(args, rank):
    """Reference arm: the FP64 CPU oracle on bounded samples of the workload."""
    if rank != 0:
        return
    # the same generator backend as the library's arm (partition weights and
    # potential with torch on the device when one is present), so that both
    # arms integrate bit-identical inputs
    prob, desc = make_workload(args.workload, accel=gen_backend())
    D = density_matrix(prob, W.rng_for(1, W.PURPOSE_D))
    nb = args.ref_batches
    for _ in range(args.warmup):
        oracle_sample(prob, D, max(1, nb // 4), seed=1)
    pts_tot, t_tot = 0, 0.0
    threads = 1
    for k in range(args.steps):
        p, dt, threads, _ = oracle_sample(prob, D, nb, seed=100 + k)
        pts_tot += p
        t_tot += dt
    value = pts_tot / t_tot
    single = oracle_single_core(prob, D)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_tot / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": desc, "n_pts": prob.n_pts},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                            "sample": "%d seeded batches of %d per step (H + density)" % (nb, prob.n_batch),
                            "single_core_value": single, "single_core_sample": "2 seeded batches, 1 thread"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="chno1000")
    ap.add_argument("--precision", default="split_bf16", choices=["split_bf16", "bf16", "fp64"])
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--bf16-steps", type=int, default=2,
                    help="also time the plain BF16 variant and state its error (0: skip)")
    ap.add_argument("--many", type=int, default=512,
                    help="also run the many-instance workload of this many molecules (split BF16 in one "
                         "captured graph against a per-molecule FP64 loop); 0: skip")
    ap.add_argument("--adjoint-steps", type=int, default=2,
                    help="also time the adjoint (dL/dv, dL/dR) on the same plan (0: skip)")
    ap.add_argument("--hartree-steps", type=int, default=2,
                    help="also time the Hartree potential of the step's density (0: skip)")
    ap.add_argument("--no-check", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-batches", type=int, default=12)
    ap.add_argument("--graph", action=argparse.BooleanOptionalAction, default=True,
                    help="replay the step as a captured CUDA graph (default)")
    ap.add_argument("--fp64-per-system", action="store_true",
                    help="many-instance workloads: also time the FP64 path called molecule by molecule")
    ap.add_argument("--batches", type=int, default=0,
                    help="use a seeded subset of this many batches (small cases for profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda:%d" % local)
    from paper_2208_12335_gb300 import Context

    t0 = time.perf_counter()
    prob, desc = make_workload(args.workload, accel="cuda")
    gen_s = time.perf_counter() - t0
    torch.cuda.empty_cache()             # the generator's cached device blocks go back
    if args.batches:
        ids = np.sort(np.random.default_rng(99).choice(prob.n_batch, size=min(args.batches, prob.n_batch),
                                                        replace=False))
        prob = prob.subgrid(ids)
        desc += " (subset: %d seeded batches)" % len(ids)
    D = density_matrix(prob, W.rng_for(1, W.PURPOSE_D))
    t0 = time.perf_counter()
    ctx = Context(local).load(prob, args.precision)
    plan_s = time.perf_counter() - t0
    n_fn, nnz, n_pts, n_at = ctx.sizes()
    if prob.n_sys > 1:
        # one occupied-orbital density matrix per system; system 0 is checked
        rng = W.rng_for(1, W.PURPOSE_D)
        dvals = np.zeros(nnz)
        for s_ in range(prob.n_sys):
            _, nf, val0, nn = ctx.system(s_)
            Ds, _ = W.density_matrix_occ(nf, max(1, int(round(0.28 * nf))), rng)
            vals, r_, c_ = stored_values(ctx, Ds, s_)
            dvals[val0:val0 + nn] = vals
            if s_ == 0:
                D, rows, cols = Ds, r_, c_
    elif D is not None:
        dvals, rows, cols = stored_values(ctx, D)
    else:
        # large system: the stored values of the same occupied-orbital D,
        # computed on the pattern only (no dense n x n matrix); no oracle check
        rp, cl = ctx.pattern(0)
        r_ = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
        dvals = W.density_values_occ(n_fn, max(1, int(round(0.28 * n_fn))), r_, cl,
                                     W.rng_for(1, W.PURPOSE_D), accel="cuda:%d" % local)
        rows = cols = None
    v = torch.from_numpy(prob.v).to(dev)
    d = torch.from_numpy(dvals).to(dev)
    h = torch.empty(nnz, dtype=torch.float64, device=dev)
    n = torch.empty(n_pts, dtype=torch.float64, device=dev)
    tr = torch.empty(1, dtype=torch.float64, device=dev)
    ws = ctx.workspace()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        ctx.integrate_h(v, h, ws=ws)
        ctx.density(d, n, tr, ws=ws)

    def timed(nsteps, fn):
        times = []
        e = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
             for _ in range(nsteps)]
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        for k in range(nsteps):
            flush.fill_(k & 255)                  # evict L2 between steps (not timed)
            e[k][0].record(stream)
            fn()
            e[k][1].record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        times = [a.elapsed_time(b) for a, b in e]
        return times

    graph = None
    if args.graph:
        s2 = torch.cuda.Stream()
        with torch.cuda.stream(s2):
            step()
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            step()

    run = graph.replay if graph is not None else step
    for _ in range(args.warmup):
        run()
    ctx.sync()

    ctx.profile(True) if graph is None else None
    with ClockSampler(local) as clk:
        t_start = time.monotonic()
        times = timed(args.steps, run)
        clk.mark(t_start, time.monotonic())
    ms = statistics.mean(times)
    prof = {}
    if graph is None:
        for kind in ("basis", "h", "density", "other"):
            prof[kind] = ctx.profile_read(kind)
        ctx.profile(False)
    else:
        # the graph replays carry no per-kind events: the same steps run
        # eagerly once more, outside the timed region, for the per-kind
        # times, launch counts and the roofline line
        ctx.profile(True)
        for k in range(args.steps):
            flush.fill_(k & 255)
            step()
        ctx.sync()
        for kind in ("basis", "h", "density", "other"):
            prof[kind] = ctx.profile_read(kind)
        ctx.profile(False)
    ctx.sync()
    ms_t = torch.tensor([ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(ms_t, op=dist.ReduceOp.MAX)
    ms_max = float(ms_t.item())

    # end to end through the public API with host buffers
    v_h = torch.from_numpy(prob.v).pin_memory()
    d_h = torch.from_numpy(dvals).pin_memory()
    h_h = torch.empty(nnz, dtype=torch.float64).pin_memory()
    n_h = torch.empty(n_pts, dtype=torch.float64).pin_memory()
    v2 = torch.empty_like(v)
    d2 = torch.empty_like(d)

    def e2e_step():
        v2.copy_(v_h, non_blocking=True)
        d2.copy_(d_h, non_blocking=True)
        ctx.integrate_h(v2, h, ws=ws)
        ctx.density(d2, n, tr, ws=ws)
        h_h.copy_(h, non_blocking=True)
        n_h.copy_(n, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    e2e_times = timed(max(3, args.steps // 2), e2e_step)
    e2e_ms = statistics.mean(e2e_times)

    # FP64 GPU path on the same inputs (the comparator); its first step is
    # timed too (at tens of seconds per step, a warm-up step would double
    # the bench's run time for nothing: nothing is compiled at run time)
    fp64 = None
    h64 = n64 = None
    if args.precision != "fp64" and args.fp64_steps > 0:
        ctx.set_precision("fp64")
        t64 = timed(args.fp64_steps, step)
        ctx.sync()
        h64 = h.clone()
        n64 = n.clone()
        ctx.set_precision(args.precision)
        step()
        ctx.sync()
        fp64 = {"ms_per_step": statistics.mean(t64),
                "value": n_pts / (statistics.mean(t64) * 1e-3),
                "max_abs_dH_vs_fp64_gpu": float((h - h64).abs().max().item()),
                "density_rel_l2_vs_fp64_gpu": float(((n - n64).norm() / n64.norm()).item())}

    # the cheaper plain BF16 variant (one product per algorithmic FLOP) on
    # the same inputs: its time and its error against the FP64 GPU path
    # (every entry) and, below, the oracle sample
    variants = {}
    if args.precision == "split_bf16" and args.bf16_steps > 0:
        for prec in ("bf16",):
            ctx.set_precision(prec)
            step()
            ctx.sync()
            tb = timed(args.bf16_steps, step)
            ctx.sync()
            r = {"ms_per_step": statistics.mean(tb), "value": n_pts / (statistics.mean(tb) * 1e-3)}
            if h64 is not None:
                r["max_abs_dH_vs_fp64_gpu"] = float((h - h64).abs().max().item())
                r["density_rel_l2_vs_fp64_gpu"] = float(((n - n64).norm() / n64.norm()).item())
            variants[prec] = r
        ctx.set_precision(args.precision)
        step()
        ctx.sync()

    # the adjoint of L = sum_k g_k h_k (dL/dv, dL/dR) on the same plan, in
    # the context's precision (tensor cores for the split paths)
    adj = None
    if args.adjoint_steps > 0:
        g = torch.from_numpy(W.rng_for(3, W.PURPOSE_G).standard_normal(nnz)).to(dev)
        dv = torch.empty(n_pts, dtype=torch.float64, device=dev)
        dR = torch.empty((n_at, 3), dtype=torch.float64, device=dev)

        def adj_step():
            ctx.adjoint(g, v, dv, dR, ws=ws)

        adj_step()
        ctx.sync()
        ta = timed(args.adjoint_steps, adj_step)
        adj = {"ms_per_step": statistics.mean(ta), "value": n_pts / (statistics.mean(ta) * 1e-3),
               "unit": UNIT, "path": args.precision, "steps": args.adjoint_steps,
               "what": "dL/dv and dL/dR of L = sum_k g_k h_k, seeded random g on the H pattern"}

    # the step upstream: the Hartree potential of the step's density on the
    # same grid (multipole method, l_max 4; FP64 l = 0, FP32 l >= 1 terms)
    hart = None
    if args.hartree_steps > 0 and getattr(prob, "owner", None) is not None:
        step()
        ctx.sync()
        n_cur = n.clone()
        vh = ctx.hartree(n_cur, l_max=4)
        ctx.sync()
        th = timed(args.hartree_steps, lambda: ctx.hartree(n_cur, l_max=4, vh=vh))
        hms = statistics.mean(th)
        pairs = sum(int(np.sum(np.diff(prob.batch_off)[prob.batch_sys == s_])) *
                    int(prob.atom_off[s_ + 1] - prob.atom_off[s_]) for s_ in range(prob.n_sys))
        hart = {"ms_per_call": hms, "value": n_pts / (hms * 1e-3), "unit": UNIT, "l_max": 4,
                "point_atom_pairs_per_s": pairs / (hms * 1e-3), "steps": args.hartree_steps,
                "what": "v_H of the step's density n on the grid (multipoles on each atom's shells, "
                        "radial Poisson equation, evaluation at every point over every atom)"}
        if not args.no_check and n_pts <= 2_000_000 and rank == 0:
            import oracle.hartree as OH
            idx = np.sort(np.random.default_rng(11).choice(n_pts, min(n_pts, 400), replace=False))
            ref, bound = OH.hartree(prob, n_cur.cpu().numpy(), l_max=4, pts_idx=idx, l1_bound=True)
            err = np.abs(vh.cpu().numpy()[idx] - ref)
            hart["vs_oracle_sample"] = {"points": len(idx), "max_abs": float(err.max()),
                                        "max_rel_to_max_v": float(err.max() / np.abs(ref).max()),
                                        "max_err_over_l1_scale": float(np.max(err / np.maximum(bound, 1e-300)))}

    def many_leg(n_mol):
        """The many-instance workload: n_mol independent molecules in one plan,
        the split-BF16 step (H + density of every molecule) replayed as one
        captured CUDA graph, against the FP64 path called molecule by
        molecule on the same GPU (one context per molecule, one shared
        workspace); errors per molecule against that loop, and of molecule
        0 against the oracle on a sample of its batches."""
        t0 = time.perf_counter()
        mp, mdesc = make_workload("many%d" % n_mol, accel="cuda")
        mgen = time.perf_counter() - t0
        t0 = time.perf_counter()
        mc = Context(local).load(mp, "split_bf16")
        mplan = time.perf_counter() - t0
        _, m_nnz, m_pts, _ = mc.sizes()
        rng = W.rng_for(4, W.PURPOSE_D)
        mdv = np.zeros(m_nnz)
        D0 = None
        for s_ in range(mp.n_sys):
            _, nf, val0, nn = mc.system(s_)
            Ds, _ = W.density_matrix_occ(nf, max(1, int(round(0.28 * nf))), rng)
            mdv[val0:val0 + nn] = stored_values(mc, Ds, s_)[0]
            if s_ == 0:
                D0 = Ds
        mv = torch.from_numpy(mp.v).to(dev)
        md = torch.from_numpy(mdv).to(dev)
        mh = torch.empty(m_nnz, dtype=torch.float64, device=dev)
        mn = torch.empty(m_pts, dtype=torch.float64, device=dev)
        mtr = torch.empty(mp.n_sys, dtype=torch.float64, device=dev)
        mws = mc.workspace()

        def mstep():
            mc.integrate_h(mv, mh, ws=mws)
            mc.density(md, mn, mtr, ws=mws)

        s2 = torch.cuda.Stream()
        with torch.cuda.stream(s2):
            mstep()
        torch.cuda.synchronize()
        mg = torch.cuda.CUDAGraph()
        with torch.cuda.graph(mg):
            mstep()
        for _ in range(args.warmup):
            mg.replay()
        mc.sync()
        tm = timed(max(3, args.steps // 2), mg.replay)
        mc.sync()
        ms_many = statistics.mean(tm)
        # the per-molecule FP64 loop
        subs = [mp.system_problem(s_) for s_ in range(mp.n_sys)]
        ctxs = [Context(local).load(sp, "fp64") for sp in subs]
        ws64 = torch.empty(max(256, max(cx.workspace_size() for cx in ctxs)), dtype=torch.uint8, device=dev)
        ins = []
        for s_, (sp, cx) in enumerate(zip(subs, ctxs)):
            _, _, val0, nn = mc.system(s_)
            ins.append((torch.from_numpy(sp.v).to(dev), md[val0:val0 + nn].contiguous(),
                        torch.empty(nn, dtype=torch.float64, device=dev),
                        torch.empty(sp.n_pts, dtype=torch.float64, device=dev)))

        def loop_step():
            for cx, (vs, ds, hs, ns) in zip(ctxs, ins):
                cx.integrate_h(vs, hs, ws=ws64)
                cx.density(ds, ns, ws=ws64, with_traces=False)

        tl = timed(1, loop_step)
        for cx in ctxs:
            cx.sync()
        dh_max, dn_max, dn_tot, n_tot = 0.0, 0.0, 0.0, 0.0
        for s_, (_, _, hs, ns) in enumerate(ins):
            _, _, val0, nn = mc.system(s_)
            pts_s = torch.from_numpy(mp.system_points(s_)).to(dev)
            dh_max = max(dh_max, float((mh[val0:val0 + nn] - hs).abs().max().item()))
            dn = float((mn[pts_s] - ns).norm().item())
            nr = float(ns.norm().item())
            dn_max = max(dn_max, dn / nr)
            dn_tot += dn * dn
            n_tot += nr * nr
        for cx in ctxs:
            cx.close()
        out = {"workload": mdesc, "n_systems": mp.n_sys, "n_pts": int(m_pts), "gen_s": round(mgen, 1),
               "plan_s": round(mplan, 3), "graph": True,
               "ms_per_step": ms_many, "value": m_pts / (ms_many * 1e-3), "unit": UNIT,
               "fp64_per_molecule_loop": {"ms_per_step": statistics.mean(tl),
                                          "value": m_pts / (statistics.mean(tl) * 1e-3),
                                          "n_contexts": len(ctxs)},
               "speedup_vs_fp64_per_molecule_loop": statistics.mean(tl) / ms_many,
               "max_abs_dH_vs_fp64_loop": dh_max,
               "density_rel_l2_vs_fp64_loop": (dn_tot / n_tot) ** 0.5,
               "density_rel_l2_vs_fp64_loop_worst_molecule": dn_max}
        mc.close()
        return out, (mp, D0)

    many, many_inputs = (many_leg(args.many) if args.many > 0 and args.workload != "many%d" % args.many
                         else (None, None))

    # many-instance: the FP64 path called molecule by molecule (one context
    # and plan per molecule, one shared workspace), on the same inputs
    fp64_loop = None
    if args.fp64_per_system and prob.n_sys > 1:
        subs = [prob.system_problem(s_) for s_ in range(prob.n_sys)]
        ctxs = [Context(local).load(sp, "fp64") for sp in subs]
        wsb = max(cx.workspace_size() for cx in ctxs)
        ws64 = torch.empty(max(wsb, 256), dtype=torch.uint8, device=dev)
        ins = []
        for s_, (sp, cx) in enumerate(zip(subs, ctxs)):
            _, _, val0, nn = ctx.system(s_)
            ins.append((torch.from_numpy(sp.v).to(dev), d[val0:val0 + nn].contiguous(),
                        torch.empty(nn, dtype=torch.float64, device=dev),
                        torch.empty(sp.n_pts, dtype=torch.float64, device=dev)))

        def loop_step():
            for cx, (vs, ds, hs, ns) in zip(ctxs, ins):
                cx.integrate_h(vs, hs, ws=ws64)
                cx.density(ds, ns, ws=ws64, with_traces=False)

        loop_step()
        torch.cuda.synchronize()
        tl = timed(max(1, args.fp64_steps), loop_step)
        fp64_loop = {"ms_per_step": statistics.mean(tl), "value": n_pts / (statistics.mean(tl) * 1e-3),
                     "n_contexts": len(ctxs)}
        for cx in ctxs:
            cx.close()

    out = None
    if rank == 0:
        flops_step = sum(prof[k]["flops"] for k in ("h", "density")) / args.steps if prof else None
        value = n_pts * world / (ms_max * 1e-3)
        peaks, peak_src = measured_peaks()
        # dominant kernel class by measured time
        roof = None
        roof_all = None
        if prof:
            fp64_peak = fp64_gemm_peak(torch) if args.precision == "fp64" else None

            def roofline(kind):
                pk = prof[kind]
                avg_ms = pk["ms"] / max(1, pk["launches"])
                per_launch_flops = pk["flops"] / max(1, pk["launches"])
                ach = per_launch_flops / (avg_ms * 1e-3) / 1e12
                if kind == "basis":
                    # FP32 pipe: SMs x 128 lanes x 2 FLOP (FMA) per clock at the
                    # sampled maximum SM clock; the algorithmic count is ~30 FLOP
                    # per (point, function)
                    mhz = clk.summary().get("sm_max_mhz") or 2070.0
                    r = {"kernel": kind, "bound": "alu", "achieved": ach, "peak": fp32_alu_peak(torch, mhz),
                         "unit": "TFLOP/s",
                         "peak_note": "FP32 FMA issue rate: SMs x 128 lanes x 2 FLOP x %.0f MHz" % mhz}
                elif args.precision == "fp64":
                    r = {"kernel": kind, "bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                         "peak_note": "measured FP64 GEMM (cuBLAS) on this GPU"}
                else:
                    # BF16 products per algorithmic FLOP: 8 for the split H and density
                    products = 8 if args.precision == "split_bf16" else 1
                    r = {"kernel": kind, "bound": "tensor", "achieved": ach,
                         "peak": peaks["bf16_tflops_sustained"] / products, "unit": "TFLOP/s",
                         "peak_note": "%s sustained BF16 / %d BF16 products per algorithmic FLOP"
                                      % (peak_src, products)}
                r["frac"] = r["achieved"] / r["peak"]
                # the committed DRAM figures were taken on the split-BF16 kernels
                bpf = traffic_for(kind, args.workload) if args.precision == "split_bf16" else None
                r["traffic"] = bpf * per_launch_flops if bpf is not None else None
                # the DRAM traffic against the algorithmic bytes of the class
                # (operand images written and read, scatter, D blocks, points)
                alg_bytes = pk["bytes"] / max(1, pk["launches"])
                r["algorithmic_bytes"] = alg_bytes
                r["traffic_over_algorithmic"] = (r["traffic"] / alg_bytes
                                                 if r["traffic"] is not None and alg_bytes > 0 else None)
                r["launch_ms"] = avg_ms
                r["launches_per_step"] = pk["launches"] / args.steps
                return r

            dom = max(("basis", "h", "density"), key=lambda k: prof[k]["ms"])
            roof = roofline(dom)
            # the other kernel classes, for context (the line above is the dominant one)
            roof_all = {k: {q: roofline(k)[q] for q in ("bound", "achieved", "peak", "unit", "frac", "traffic",
                                                         "algorithmic_bytes", "traffic_over_algorithmic")}
                        for k in ("basis", "h", "density")}
        cpu = None
        errors = None
        if not args.no_cpu_baseline:
            # the CPU-baseline leg: the oracle timed on a sample of the
            # workload; its results also give the library's error on that sample
            res = oracle_sample(prob, D, args.ref_batches, keep=True)
            p, dt, thr, nbs = res[:4]
            cpu = {"value": p / dt, "unit": UNIT, "cores": thr, "kind": "oracle",
                   "sample": "%d seeded batches (%d points) of %d, H + density" % (nbs, p, prob.n_batch),
                   "single_core_value": oracle_single_core(prob, D),
                   "single_core_sample": "2 seeded batches, 1 thread"}
            if not args.no_check:
                errors = compare_on_sample(res[4:], args.precision, local, dev, torch, Context)
                for prec, r in variants.items():
                    # the cheaper variants on the same oracle sample
                    eb = compare_on_sample(res[4:], prec, local, dev, torch, Context)
                    r["max_abs_dH_vs_oracle_sample"] = eb["max_abs_dH_sample"]
                    r["density_rel_l2_vs_oracle_sample"] = eb["density_rel_l2_sample"]
                if many_inputs is not None:
                    # molecule 0 of the many-instance workload against the oracle
                    mp, D0 = many_inputs
                    rm = oracle_sample(mp, D0, args.ref_batches, keep=True)
                    many["molecule0_vs_oracle"] = compare_on_sample(rm[4:], "split_bf16", local, dev, torch,
                                                                    Context)
        launches = int(sum(prof[k]["launches"] for k in prof) / args.steps) if prof else None
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None,
               "dtype": {"split_bf16": "split-bf16x3 (f32 acc, f64 cross-batch)",
                         "bf16": "bf16 (f32 acc)",
                         "fp64": "f64"}[args.precision],
               "data": "synthetic",
               "config": {"workload": desc, "n_pts": n_pts, "n_fn": n_fn, "nnz": nnz, "n_atoms": n_at,
                          "n_batches": prob.n_batch, "precision": args.precision,
                          "l2": "flushed between steps (256 MiB write)",
                          "graph": bool(args.graph), "plan_s": round(plan_s, 3), "gen_s": round(gen_s, 1)},
               "tflops": flops_step / (ms_max * 1e-3) / 1e12 if flops_step else None,
               "roofline": roof,
               "roofline_by_kernel": roof_all,
               "cpu_baseline": cpu,
               "e2e": {"value": n_pts * world / (e2e_ms * 1e-3), "unit": UNIT,
                       "h2d_bytes_per_step": 8 * (n_pts + nnz), "d2h_bytes_per_step": 8 * (nnz + n_pts)},
               "gpu_launches": launches * args.steps if launches is not None else None,
               "fp64_path": fp64,
               "bf16_path": variants.get("bf16"),
               "many_instance": many,
               "adjoint": adj,
               "hartree": hart,
               "fp64_per_molecule_loop": fp64_loop,
               "errors_vs_oracle": errors,
               "clocks": clk.summary(),
               "profile_ms_per_step": {k: prof[k]["ms"] / args.steps for k in prof} if prof else None,
               # per step and kernel class: launches and algorithmic FLOPs (the units
               # the roofline and the DRAM-traffic scaling use)
               "profile_per_step": ({k: {"launches": prof[k]["launches"] / args.steps,
                                         "algorithmic_flops": prof[k]["flops"] / args.steps}
                                     for k in prof} if prof else None)}
        if fp64:
            out["speedup_vs_fp64_gpu"] = fp64["ms_per_step"] / ms_max
        if args.precision != "fp64":
            # executed tensor-core work of the whole step against the measured
            # sustained BF16 rate (padding of the 128 x 128 tiles included)
            ex = executed_tensor_flops(ctx, 8 if args.precision == "split_bf16" else 1)
            out["tensor_pipe"] = {"executed_bf16_tflop_per_step": ex / 1e12,
                                  "achieved_tflops": ex / (ms_max * 1e-3) / 1e12,
                                  "peak_tflops": peaks["bf16_tflops_sustained"],
                                  "frac_of_sustained": ex / (ms_max * 1e-3) / 1e12 / peaks["bf16_tflops_sustained"],
                                  "note": "%s sustained BF16; whole step (basis, scatter and gathers included)"
                                          % peak_src}
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
