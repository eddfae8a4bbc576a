#!/usr/bin/env python
"""Benchmark of the line-opacity + ODF hot path on the full ODF-table workload.

Workload: 5e6 seeded synthetic lines (30 species) over 9-10000 nm on an R = 2e6
log-lambda grid (14,026,236 points), the 57 x 25 DFSYNTHE T-P grid, 328 equal
log-lambda intervals x 12 ODF steps.  One step = one batch of (T, P) points of
that table through the whole hot path: populations are resident, then
synth_opacity (line prep, cut, profile synthesis) and build_odf (sort + step
means).  Metric: Voigt line-evaluations per second (the number of (line, grid
point) profile evaluations inside the cut windows, counted by the library),
plus ODF (T, P) points per second.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
Under torchrun each rank takes its own batch of points (independent units, no
data-path collective; weak scaling); timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# the serving legs run 16 CUDA streams (8 slots, two priorities each); with the default of 8
# hardware queues, streams share queues and a small request can wait behind another's kernels
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

import numpy as np  # noqa: E402

import workloads as wl  # noqa: E402

METRIC = "Voigt line-evals/s (line-by-line opacity synthesis + ODF binning)"
UNIT = "line-evals/s"
# FP32 operations of one far-wing profile evaluation in the form that takes 97-99.6 % of the
# evaluations of the table rows (plain rational form in units of sk, two points per
# reciprocal, packed FP32): per pair of points {v0, v1} = fma(G, B', E'), {D0, D1} =
# fma(v, v, c') and {s1, s0} += r {D0, D1} are three packed FFMAs (12 flop) and
# r = rcp(D0 D1) one FMUL (1 flop): 13 flop per pair, 6.5 per evaluation, plus half a
# reciprocal on the special-function unit (not counted).
FLOP_PER_EVAL = 6.5
FP32_LANES_PER_SM = 128
# kernels of the library per timed step: synth_opacity (k_place, k_consts, k_kappa0, k_med_init,
# three k_med_hist + k_med_pick levels, k_prep, k_windows, k_scan_class, k_scan_fin, k_scatter,
# k_ranges, k_tiles) and build_odf (k_odf_gather, then k_odf for the intervals it leaves)
LAUNCHES_PER_STEP = 19


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["native", "reference"], default="native")
    p.add_argument("--batch", type=int, default=8, help="(T, P) points per step and rank (table workload)")
    p.add_argument("--rows", type=str, default="",
                   help="comma-separated table rows (T index * 25 + P index) instead of the default batch")
    p.add_argument("--workload", choices=["table", "small"], default="table",
                   help="table: 5e6 lines, 9-10000 nm, 57x25 T-P grid; small: 20,000 lines, 300-400 nm, 4 points")
    p.add_argument("--mode", choices=["step", "serve", "batch", "precision", "bins", "table", "spectrum"],
                   default="step",
                   help="step: the throughput benchmark; serve: Poisson request stream through the server; "
                        "batch: persistent graph-captured batch against the plain per-point path; "
                        "spectrum: one spectrum request (80 depths) on windows of several lengths")
    p.add_argument("--spectrum-windows", type=str, default="1,10,100",
                   help="window lengths [nm] of the spectrum mode, from 500 nm at R = 5e5")
    p.add_argument("--batch-rows", type=int, default=4, help="ODF rows (composition, T, P) in the batch sample")
    p.add_argument("--batch-windows", type=int, default=200, help="spectrum windows in the batch sample")
    p.add_argument("--serve-seconds", type=float, default=60.0, help="arrival window of the latency stream")
    p.add_argument("--no-serve", action="store_true", help="skip the serving sub-measurement of the step mode")
    p.add_argument("--no-batch-leg", action="store_true", help="skip the batch sub-measurement of the step mode")
    p.add_argument("--bin-rays", type=int, default=8192, help="rays per step of the bin-intensity form")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    return p.parse_args()


# Rows (T index * 25 + P index) of the 57 x 25 table taken by one step, in increasing
# cost.  They sit at the 6, 19, 31, 44, 56, 69, 81 and 94 % quantiles of the per-row
# evaluation count W over all 1425 rows (W estimated once from a 20,000-line
# subsample of the same list): W per row from 1.6e10 to 1.4e13, about 2.2e13 per
# step, i.e. a cross-section of the table's cost distribution.
TABLE_ROWS = [277, 879, 232, 964, 1354, 1044, 1321, 297]


def batch_points(rank: int, B: int, world: int = 1):
    """Rows of `rank` among `world` ranks, B per rank, through the row-sharding helper: the
    first B rows of TABLE_ROWS, each with its temperature neighbours T index +- k (k < world)
    as rows of the same cost class, interleaved so that round-robin sharding gives rank k
    every class's k-th neighbour (the same cost mix on every rank; rank 0 takes TABLE_ROWS)."""
    from paper_2105_13611_gb300.sharding import rows_for_rank
    if not 1 <= B <= len(TABLE_ROWS):
        raise ValueError(f"--batch must be 1..{len(TABLE_ROWS)}")
    base = np.array(TABLE_ROWS[:B], dtype=np.int64)
    ti, pi = base // 25, base % 25
    # order[j * world + k] = k-th temperature neighbour of row j (downwards near the hot end)
    step = lambda t: 1 if t + world - 1 <= 56 else -1
    order = np.array([(t + step(t) * k) * 25 + p for t, p in zip(ti, pi) for k in range(world)], dtype=np.int64)
    return rows_for_rank(len(order), rank, world, order=order)


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm), "reasons": sorted(reasons)}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return d.get("hbm_gbs", 6800.0), d.get("sm_max_mhz", 2070.0), "measured"
    except (OSError, ValueError):
        return 6800.0, 2070.0, "fallback"


# ---------------------------------------------------------------------------
# CPU oracle sample (cpu_baseline and the reference arm)
def oracle_sample(seconds: float, w, lines, row_T, row_P, seed: int = 99):
    """Time the FP64 oracle (as it stands) on contiguous 0.2 nm slices of the same line list:
    each slice's lines, synthesised densely on the slice's grid at one (T, P) point, then the
    slice's ODF.  Returns (evals/s, evals, wall s, description)."""
    from oracle import odf as od
    from oracle import synthesis as sy
    el = wl.elements(w.n_metals)
    se, ss = wl.species_table(w.n_metals)
    rng = np.random.default_rng(seed)
    evals, t_total, n_slices = 0, 0.0, 0
    t_start = time.perf_counter()
    while time.perf_counter() - t_start < seconds:
        lo, hi = max(200.0, w.grid.lam0_nm), min(2000.0, w.grid.lam1_nm - 0.2)
        lam0 = float(np.exp(rng.uniform(math.log(lo), math.log(hi))))
        lam1 = lam0 + 0.2
        i0, i1 = np.searchsorted(lines.lam_nm, [lam0, lam1])
        if i1 - i0 < 2:
            continue
        sub = lines.subset(slice(i0, i1))
        g = wl.Grid(lam0, lam1, w.grid.R)
        t0 = time.perf_counter()
        pl = sy.prepare(sub, se, ss, el, row_T, row_P, g, w.cut, w.kc_factor)
        k, _, W = sy.kappa_dense(pl)
        od.odf(k, wl.equal_intervals(pl.N, 2), w.widths)
        t_total += time.perf_counter() - t0
        evals += W
        n_slices += 1
    desc = (f"{n_slices} slices of 0.2 nm (lines of the {len(lines)}-line list inside each slice, dense FP64 synthesis "
            f"on the slice grid at R=2e6 and T={row_T:.0f} K, P={row_P:.3g}, plus the slice ODF)")
    return evals / t_total, evals, t_total, desc


_WORKER_STATE = None


def _oracle_worker_init(workload: str):
    # each process builds its own copy of the seeded workload once
    global _WORKER_STATE
    w = wl.config_table() if workload == "table" else wl.config_small()
    _WORKER_STATE = (w, w.lines())


def _oracle_worker(job):
    seconds, seed, row_T, row_P = job
    w, lines = _WORKER_STATE
    return oracle_sample(seconds, w, lines, row_T, row_P, seed=seed)[1:3]


def oracle_pool(workload: str = "table"):
    """One process per host core (spawned, so that no child inherits the parent's CUDA state),
    each holding the seeded line list."""
    import multiprocessing as mp
    n = os.cpu_count() or 1
    return mp.get_context("spawn").Pool(n, initializer=_oracle_worker_init, initargs=(workload,)), n


def oracle_all_cores(seconds: float, row_T: float, row_P: float, pool=None, n=None, seed0: int = 1000):
    """The oracle slice sample on every host core at once, each process on its own slices.
    Returns (aggregate evals/s, processes, evals)."""
    own = pool is None
    if own:
        pool, n = oracle_pool()
    try:
        res = pool.map(_oracle_worker, [(seconds, seed0 + i, row_T, row_P) for i in range(n)])
    finally:
        if own:
            pool.close()
            pool.join()
    return sum(e / t for e, t in res if t > 0), n, int(sum(e for e, _ in res))


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = wl.config_table() if args.workload == "table" else wl.config_small()
    pts = batch_points(0, args.batch, 1) if args.workload == "table" else np.arange(len(w.T))
    T, P = float(w.T[pts[0]]), float(w.P[pts[0]])
    per_step = max(5.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    pool, n = oracle_pool(args.workload)
    try:
        for i in range(args.warmup):
            oracle_all_cores(per_step / 4, T, P, pool, n, seed0=100 * i)
        vals, evs = [], 0
        for i in range(args.steps):
            v, _, e = oracle_all_cores(per_step, T, P, pool, n, seed0=10000 + 100 * i)
            vals.append(v)
            evs += e
    finally:
        pool.close()
        pool.join()
    value = statistics.mean(vals)
    desc = (f"{n} processes (one per host core), each timing the FP64 oracle for {per_step:.0f} s per step on its own "
            f"0.2 nm slices of the {w.name} line list (dense synthesis at T={T:.0f} K, P={P:.3g}, plus the slice ODF)")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": w.name, "sample": "bounded oracle sample per step on every host core"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": n, "kind": "oracle", "sample": desc,
                            "evals": evs},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
def native_arm(args):
    import torch
    import torch.distributed as dist

    from paper_2105_13611_gb300 import binding

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    from paper_2105_13611_gb300.sharding import reduce_scalar

    def max_over_ranks(x):
        return reduce_scalar(x, "max")

    def sum_over_ranks(x):
        return reduce_scalar(x, "sum")

    w = wl.config_table() if args.workload == "table" else wl.config_small()
    lines = w.lines()
    el = wl.elements(w.n_metals)
    se, ss = wl.species_table(w.n_metals)
    ctx = binding.Context(local)
    ctx.load_linelist(lines, se, ss)
    ctx.set_atmosphere_grid(el, w.T, w.P)
    N = binding.grid_size(w.grid.lam0_nm, w.grid.lam1_nm, w.grid.R)
    K = w.n_intervals
    bounds = wl.equal_intervals(N, K)
    if args.rows:
        sel = np.array([int(x) for x in args.rows.split(",")], dtype=np.int32)
    else:
        sel = batch_points(rank, args.batch, world) if args.workload == "table" else np.arange(len(w.T), dtype=np.int32)
    B = len(sel)
    stream = torch.cuda.current_stream()
    kap = torch.empty((B, N), dtype=torch.float32, device=dev)
    kc = torch.empty(B, dtype=torch.float32, device=dev)
    ev = torch.empty(B, dtype=torch.int64, device=dev)
    ev_tot = torch.zeros(B, dtype=torch.int64, device=dev)
    odf = torch.empty((B, K, len(w.widths)), dtype=torch.float64, device=dev)
    opts = binding.make_opts(w.cut, w.kc_factor)

    def step():
        ctx.synth_opacity(w.grid, sel, kap, kc, ev, opts=opts, stream=stream)
        ctx.build_odf(kap, bounds, w.widths, odf, stream=stream)

    for _ in range(args.warmup):
        step()
    barrier()
    ctx.profile_enable(True)
    ctx.profile_read(binding.KERNEL_PROFILE)
    ctx.profile_read(binding.KERNEL_ODF)
    clocks = Clocks(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        step()
        ev_tot.add_(ev)
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    tiles_ms, tiles_n = ctx.profile_read(binding.KERNEL_PROFILE)
    odf_ms, odf_n = ctx.profile_read(binding.KERNEL_ODF)
    ctx.profile_enable(False)
    evals_rank = float(ev_tot.sum().item())
    evals = sum_over_ranks(evals_rank)
    ms_max = max_over_ranks(ms)
    value = evals / (ms_max / 1e3)
    odf_pts = B * args.steps * world / (ms_max / 1e3)

    # ---- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        Tb = np.ascontiguousarray(w.T[sel])
        Pb = np.ascontiguousarray(w.P[sel])
        odf_h = torch.empty((B, K, len(w.widths)), dtype=torch.float64, pin_memory=True)
        kc_h = torch.empty(B, dtype=torch.float32, pin_memory=True)
        ev_h = torch.empty(B, dtype=torch.int64, pin_memory=True)
        rows = np.arange(B, dtype=np.int32)
        ctx2 = binding.Context(local)
        ctx2.load_linelist(lines, se, ss)

        def e2e_step():
            ctx2.set_atmosphere_grid(el, Tb, Pb)
            ctx2.synth_opacity(w.grid, rows, kap, kc, ev, opts=opts, stream=stream)
            ctx2.build_odf(kap, bounds, w.widths, odf, stream=stream)
            odf_h.copy_(odf, non_blocking=True)
            kc_h.copy_(kc, non_blocking=True)
            ev_h.copy_(ev, non_blocking=True)
            stream.synchronize()
            return int(ev_h.sum())

        e2e_step()
        barrier()
        n_e2e = args.steps
        t0 = time.perf_counter()
        ev_e2e = 0
        for _ in range(n_e2e):
            ev_e2e += e2e_step()
        barrier()
        dt = max_over_ranks(time.perf_counter() - t0)
        ev_e2e = sum_over_ranks(ev_e2e)
        n_el = el.n
        h2d = (Tb.nbytes + Pb.nbytes + 5 * n_el * 8 + n_el * 8          # set_atmosphere_grid
               + rows.nbytes                                           # synth_opacity rows
               + bounds.nbytes + 8 * (2 * len(w.widths) + 1))          # build_odf bounds and widths
        d2h = odf_h.numel() * 8 + kc_h.numel() * 4 + ev_h.numel() * 8
        e2e = {"value": ev_e2e / dt, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "steps": n_e2e,
               "note": "line list resident (loaded once); per step: populations from host T, P, synthesis, ODF, "
                       "ODF table + kappa_c + evaluation counts copied to pinned host memory"}
        ctx2.close()

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    hbm, sm_max, peak_kind = peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    tiles_avg = tiles_ms / max(tiles_n, 1)
    evals_per_launch = evals_rank / max(tiles_n, 1)
    fp32_peak = sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12        # TFLOP/s at the maximum SM clock
    achieved = evals_per_launch * FLOP_PER_EVAL / (tiles_avg / 1e3) / 1e12
    traffic = measured_traffic("k_tiles", ["synth.cu", "voigt.cuh", "common.cuh"], sel)
    counted = profile_value("k_tiles_fp32_ops_row1044.md", "flop_per_eval_counted", "k_tiles",
                            ["synth.cu", "voigt.cuh", "common.cuh"])
    roofline = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak, "traffic": traffic, "kernel": "k_tiles (profile synthesis)",
                "fp32_counted": None if counted is None else {
                    "flop_per_eval": counted, "achieved": achieved * counted / FLOP_PER_EVAL,
                    "frac": achieved * counted / FLOP_PER_EVAL / fp32_peak,
                    "source": "ncu FP32 thread-instruction counters (FFMA2 x4, FFMA x2, FMUL, FADD) on row 1044, "
                              "profiles/k_tiles_fp32_ops_row1044.md"},
                "peak_kind": f"FP32 FMA peak {sms} SMs x {FP32_LANES_PER_SM} lanes x 2 flop x {sm_max:.0f} MHz",
                "sms": sms, "flop_per_eval": FLOP_PER_EVAL, "avg_launch_ms": tiles_avg, "launches": tiles_n}
    odf_avg = odf_ms / max(odf_n, 1)
    odf_bytes = B * N * 4 + B * K * 12 * 8
    roofline_odf = {"bound": "hbm", "achieved": odf_bytes / (odf_avg / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                    "frac": odf_bytes / (odf_avg / 1e3) / 1e9 / hbm,
                    "traffic": measured_traffic("build_odf", ["odf.cu", "common.cuh"], sel),
                    "kernel": "build_odf: k_odf_gather, then k_odf on the intervals it leaves",
                    "peak_kind": f"{peak_kind} HBM copy bandwidth", "avg_launch_ms": odf_avg, "launches": odf_n}
    ctx.close()
    # the other parts of the headline metric: the batched form against the plain per-point path,
    # and continuous batching against one request at a time (throughput, p50 / p99 latency)
    batch = serving = None
    if world == 1 and args.workload == "table" and not args.no_batch_leg:
        batch = batch_measure(w, lines, el, se, ss, n_rows=2, n_windows=200, steps=2)
    if world == 1 and args.workload == "table" and not args.no_serve:
        serving = serve_measure(w, lines, el, se, ss, n_burst=20, stream_s=args.serve_seconds)
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        T0, P0 = float(w.T[sel[0]]), float(w.P[sel[0]])
        v, e, s, desc = oracle_sample(15.0, w, lines, T0, P0)
        va, na, ea = oracle_all_cores(10.0, T0, P0)
        cpu = {"value": va, "unit": UNIT, "cores": na, "kind": "oracle",
               "sample": f"{na} processes x 10 s of the slice sample below, each on its own slices ({ea} evaluations)",
               "one_core": {"value": v, "cores": 1, "sample": desc, "evals": int(e), "seconds": s}}
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": w.name, "lines": len(lines), "species": w.n_species, "grid_points": N,
                      "R": w.grid.R, "lambda_nm": [w.grid.lam0_nm, w.grid.lam1_nm],
                      "tp_grid": "57 T x 25 P" if args.workload == "table" else "4 points, log P = 4",
                      "points_per_step_per_rank": B, "rows": [int(x) for x in sel], "intervals": K, "odf_steps": 12,
                      "l2": "inputs larger than L2 (no flush needed)", "parallelism": f"independent points x{world}"},
           "odf_points_per_s": odf_pts, "evals_per_step": evals / args.steps,
           "roofline": roofline, "roofline_odf": roofline_odf, "cpu_baseline": cpu, "e2e": e2e,
           "batch": batch, "serving": serving,
           "gpu_launches": LAUNCHES_PER_STEP * args.steps, "clocks": clk}
    print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
def make_request_stream(rate, seconds, seed, spectrum_fraction=0.9, n_max=None):
    """Poisson arrivals of mixed requests (the serving workload).

    Spectrum: grey atmosphere with D ~ U{40..120} depths, Teff ~ U(3500, 12000) K, log g ~ U(1, 5);
    window length ~ logU(1, 500) nm placed uniformly in 9-10000 nm at R = 5e5; 5 mu angles.
    ODF: one composition x the 57 x 25 T-P grid over 1-10 contiguous intervals of the 328-interval grid."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while n_max is None or len(out) < n_max:
        t += rng.exponential(1.0 / rate)
        if t > seconds:
            break
        if rng.random() < spectrum_fraction:
            D = int(rng.integers(40, 121))
            Teff, logg = rng.uniform(3500, 12000), rng.uniform(1, 5)
            L = float(np.exp(rng.uniform(math.log(1.0), math.log(500.0))))
            lam0 = float(rng.uniform(9.0, 10000.0 - L))
            m, T, P = wl.grey_atmosphere(D, Teff, logg)
            out.append((t, "spectrum", (m, T, P, wl.Grid(lam0, lam0 + L, 5e5))))
        else:
            nint = int(rng.integers(1, 11))
            k0 = int(rng.integers(0, 328 - nint + 1))
            out.append((t, "odf", (k0, nint)))
    return out


def serve_measure(w, lines, el, se, ss, n_burst=20, stream_s=20.0, load=0.7, seed=2024, drain_s=120.0):
    """Continuous batching against one request at a time, on the serving workload's request mix
    (90 % spectra of 40-120 depths over 1-500 nm windows at R = 5e5, 10 % ODFs of one composition
    over the 57 x 25 grid on 1-10 intervals).
      saturation: the same n_burst requests (the mix's proportions: 10 % ODFs) submitted at once;
        completed requests per second with 8 stream slots and with 1;
      latency: a Poisson stream offered at `load` times the one-slot saturation rate for
        stream_s seconds, served with 8 slots and with 1; p50 / p99 of completion - arrival.  Each
        run ends when every request has completed or drain_s seconds after the last arrival."""
    from paper_2105_13611_gb300 import binding
    N = binding.grid_size(w.grid.lam0_nm, w.grid.lam1_nm, w.grid.R)
    bounds_full = wl.equal_intervals(N, w.n_intervals)
    lnq = math.log1p(1.0 / w.grid.R)
    mus = [1.0, 0.8, 0.6, 0.4, 0.2]
    rows = np.arange(len(w.T), dtype=np.int32)

    def odf_args(k0, nint):
        j0, j1 = int(bounds_full[k0]), int(bounds_full[k0 + nint])
        lam_a = w.grid.lam0_nm * math.exp(j0 * lnq)
        g = wl.Grid(lam_a, lam_a * math.exp((j1 - j0 - 1) * lnq) * (1 + 1e-12), w.grid.R)
        n_sub = binding.grid_size(g.lam0_nm, g.lam1_nm, g.R)
        b = np.minimum(bounds_full[k0:k0 + nint + 1] - j0, n_sub)
        return rows, g, b, w.widths

    ctx = binding.Context(0)
    ctx.load_linelist(lines, se, ss)
    ctx.set_atmosphere_grid(el, w.T, w.P)

    def run(stream, max_inflight):
        srv = binding.Server(ctx, hbm_budget_bytes=int(120e9), max_inflight=max_inflight, rows_per_chunk=8)
        limit = (stream[-1][0] if stream else 0.0) + drain_s
        t0 = time.perf_counter()
        pending, lat, i = [], {"spectrum": [], "odf": []}, 0
        while time.perf_counter() - t0 < limit:
            now = time.perf_counter() - t0
            while i < len(stream) and stream[i][0] <= now:
                _, kind, a = stream[i]
                tk = srv.submit_spectrum(*a[:3], a[3], mus) if kind == "spectrum" else srv.submit_odf(*odf_args(*a))
                pending.append((tk, kind, stream[i][0]))
                i += 1
            still = []
            for tk, kind, t_arr in pending:
                try:
                    srv.wait(tk, timeout_ms=0)
                    lat[kind].append((time.perf_counter() - t0 - t_arr) * 1e3)
                except binding.MpsaError as e:
                    if e.code != binding.MPSA_ETIMEOUT:
                        raise
                    still.append((tk, kind, t_arr))
            pending = still
            if i >= len(stream) and not pending:
                break
            time.sleep(0.001)
        wall = time.perf_counter() - t0
        srv.cancel_queued()
        srv.close()
        done = sum(len(v) for v in lat.values())
        allv = lat["spectrum"] + lat["odf"]
        pct = lambda v, q: float(np.percentile(v, q)) if v else None
        return {"offered": len(stream), "completed": done, "wall_s": wall, "req_per_s": done / wall,
                "p50_ms": pct(allv, 50), "p99_ms": pct(allv, 99),
                "spectrum": {"n": len(lat["spectrum"]), "p50_ms": pct(lat["spectrum"], 50),
                             "p99_ms": pct(lat["spectrum"], 99)},
                "odf": {"n": len(lat["odf"]), "p50_ms": pct(lat["odf"], 50), "p99_ms": pct(lat["odf"], 99)}}

    # warm-up: one request of each kind
    run([(0.0, k, a) for k, a in [r[1:] for r in make_request_stream(50.0, 10.0, seed=seed + 7)][:1]] +
        [(0.0, "odf", (0, 1))], 1)
    pool_ = make_request_stream(1e6, 1e6, seed=seed, n_max=40 * n_burst)
    n_odf = max(1, round(0.1 * n_burst))
    burst = [r for r in pool_ if r[1] == "odf"][:n_odf] + [r for r in pool_ if r[1] == "spectrum"][:n_burst - n_odf]
    burst = [(0.0, k, a) for _, k, a in burst]
    sat8 = run(burst, 8)
    sat1 = run(burst, 1)
    rate = load * sat1["req_per_s"]
    stream = make_request_stream(rate, stream_s, seed=seed + 1)
    lat8 = run(stream, 8)
    lat1 = run(stream, 1)
    ctx.close()
    return {"mix": "90% spectra (40-120 depths, 1-500 nm at R=5e5, 5 mu) / 10% ODFs (57x25 grid, 1-10 intervals)",
            "saturation": {"requests": n_burst, "continuous_batching_8_slots": sat8, "one_at_a_time": sat1,
                           "speedup": sat8["req_per_s"] / sat1["req_per_s"]},
            "latency": {"offered_req_per_s": rate, "offered_load_vs_one_at_a_time_capacity": load,
                        "arrival_window_s": stream_s, "continuous_batching_8_slots": lat8, "one_at_a_time": lat1}}


def serve_arm(args):
    w = wl.config_table()
    lines = w.lines()
    el = wl.elements(w.n_metals)
    se, ss = wl.species_table(w.n_metals)
    out = {"mode": "serve", "metric": "requests/s and latency (continuous batching vs one at a time)",
           **serve_measure(w, lines, el, se, ss, stream_s=args.serve_seconds), "data": "synthetic"}
    print(json.dumps(out), flush=True)


def batch_measure(w, lines, el, se, ss, n_rows, n_windows, steps, seed=99, autotune=True):
    """64 compositions x 1425 (T, P) rows plus spectrum windows (1-500 nm at R = 5e5): a seeded
    sample of n_rows ODF rows and n_windows windows runs (a) point by point through
    synth_opacity / build_odf and (b) as one persistent graph-captured batch; same results,
    compared throughput (both timed from the host around `steps` runs, synchronised)."""
    import torch

    from paper_2105_13611_gb300 import binding
    ab = wl.abundance_scales(64, el.n, seed=77)
    ctx = binding.Context(0)
    ctx.load_linelist(lines, se, ss)
    ctx.set_atmosphere_grid(el, w.T, w.P, abund_scale=ab)
    nrows = 64 * len(w.T)
    rng = np.random.default_rng(seed)
    N = binding.grid_size(w.grid.lam0_nm, w.grid.lam1_nm, w.grid.R)
    bounds = wl.equal_intervals(N, w.n_intervals)
    groups = []
    odf_rows = rng.choice(nrows, n_rows, replace=False).astype(np.int32)
    groups.append(dict(grid=w.grid, sel=odf_rows, bounds=bounds, widths=w.widths, odf_on=True))
    for _ in range(n_windows):
        L = float(np.exp(rng.uniform(0.0, math.log(500.0))))
        lam0 = float(rng.uniform(9.0, 10000.0 - L))
        groups.append(dict(grid=wl.Grid(lam0, lam0 + L, 5e5), sel=np.array([rng.integers(0, nrows)], dtype=np.int32),
                           odf_on=False))
    for g in groups:
        n = binding.grid_size(g["grid"].lam0_nm, g["grid"].lam1_nm, g["grid"].R)
        g["kappa"] = torch.empty((len(g["sel"]), n), dtype=torch.float32, device="cuda")
        g["kappa_c"] = torch.empty(len(g["sel"]), dtype=torch.float32, device="cuda")
        g["evals"] = torch.empty(len(g["sel"]), dtype=torch.int64, device="cuda")
        if g["odf_on"]:
            g["odf"] = torch.empty((len(g["sel"]), w.n_intervals, 12), dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()

    def plain():
        for g in groups:
            for i, r in enumerate(g["sel"]):
                k = g["kappa"][i:i + 1]
                ctx.synth_opacity(g["grid"], [int(r)], k, g["kappa_c"][i:i + 1], g["evals"][i:i + 1], stream=st)
                if g["odf_on"]:
                    ctx.build_odf(k, g["bounds"], g["widths"], g["odf"][i:i + 1], stream=st)

    plain()
    torch.cuda.synchronize()
    evals = int(sum(int(g["evals"].sum()) for g in groups))
    ref = [g["kappa"].clone() for g in groups]
    t0 = time.perf_counter()
    for _ in range(steps):
        plain()
    torch.cuda.synchronize()
    t_plain = (time.perf_counter() - t0) / steps
    t0 = time.perf_counter()
    batch = binding.Batch(ctx, groups, autotune=autotune)
    t_create = time.perf_counter() - t0
    batch.run()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        batch.run(stream=st)
    torch.cuda.synchronize()
    t_batch = (time.perf_counter() - t0) / steps
    worst = 0.0
    for g, k_ref in zip(groups, ref):
        kb, kr = g["kappa"].double(), k_ref.double()
        kc = g["kappa_c"].double()[:, None]
        worst = max(worst, float(((kb - kr).abs() / (kr + kc)).max()))
    info = batch.info()
    batch.close()
    ctx.close()
    return {"metric": "line-evals/s, persistent graph-captured batch vs plain per-point path",
            "rows": {"odf_rows": len(odf_rows), "windows": n_windows, "compositions": 64},
            "evals_per_run": evals, "plain_s": t_plain, "batch_s": t_batch,
            "plain_evals_per_s": evals / t_plain, "batch_evals_per_s": evals / t_batch, "speedup": t_plain / t_batch,
            "batch_create_s": t_create, "max_rel_diff_vs_plain": worst, "autotune": info}


def batch_arm(args):
    w = wl.config_table()
    lines = w.lines()
    el = wl.elements(w.n_metals)
    se, ss = wl.species_table(w.n_metals)
    out = {"mode": "batch", **batch_measure(w, lines, el, se, ss, args.batch_rows, args.batch_windows, args.steps),
           "data": "synthetic"}
    print(json.dumps(out), flush=True)


def spectrum_arm(args):
    """One spectrum request of the serving workload's kind, timed alone: synth_spectrum over the
    5e6-line table list for the solar grey atmosphere (80 depths, Teff 5772 K, log g 4.44) on
    windows from 500 nm at R = 5e5 with 5 mu angles.  Each window: `warmup` untimed calls, then
    `steps` calls, each timed from the host around the call with a synchronize on both sides."""
    import torch
    from paper_2105_13611_gb300 import binding
    w = wl.config_table()
    lines = w.lines()
    se, ss = wl.species_table(w.n_metals)
    ctx = binding.Context(0)
    ctx.load_linelist(lines, se, ss)
    ctx.set_atmosphere_grid(wl.elements(w.n_metals), w.T, w.P)
    mus = [1.0, 0.8, 0.6, 0.4, 0.2]
    m, T, P = wl.grey_atmosphere(80, 5772.0, 4.44)
    res = []
    for length in [float(x) for x in args.spectrum_windows.split(",") if x]:
        g = wl.Grid(500.0, 500.0 + length, 5e5)
        N = binding.grid_size(g.lam0_nm, g.lam1_nm, g.R)
        I = torch.empty((len(mus), N), dtype=torch.float32, device="cuda")
        ts = []
        for it in range(args.warmup + args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.synth_spectrum(m, T, P, g, mus, I)
            torch.cuda.synchronize()
            if it >= args.warmup:
                ts.append((time.perf_counter() - t0) * 1e3)
        res.append({"window_nm": length, "N": N, "ms": ts, "ms_median": float(np.median(ts))})
    ctx.close()
    print(json.dumps({"mode": "spectrum", "metric": "ms per spectrum request (80 depths, 5 mu, 5e6 lines)",
                      "windows": res, "data": "synthetic"}), flush=True)


def bins_arm(args):
    """Module III through ODF tables (odf_intensity): emergent bin intensities of many 1D rays
    (grey atmospheres, 80 depths, 5 directions) from a seeded synthetic ODF table on the 57 x 25
    T-P grid with 328 bins x 12 sub-bins.  value = rays/s with the rays resident on the device;
    e2e adds the host->device copy of the rays and the device->host copy of the intensities."""
    import torch

    from paper_2105_13611_gb300 import binding
    from oracle import bin_intensity as obi
    nT, nP, K, ns, D = 57, 25, 328, 12, 80
    mus = [1.0, 0.8, 0.6, 0.4, 0.2]
    n = args.bin_rays
    lt, lp, odf, kc, lam = wl.odf_table_synthetic(nT, nP, K, ns, seed=1005)
    m, T, P = wl.ray_atmospheres(n, D, seed=1006)
    ctx = binding.Context(0)
    d_odf = torch.from_numpy(odf).cuda()
    d_kc = torch.from_numpy(kc).cuda()
    dm, dT, dP = (torch.from_numpy(a).cuda() for a in (m, T, P))
    out = torch.empty((n, len(mus), K), dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream()

    def step():
        ctx.odf_intensity(lt, lp, d_odf, d_kc, lam, wl.ODF_WIDTHS_12, dm, dT, dP, mus, out, stream=st)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = Clocks(0)
    clocks.start()
    ctx.profile_enable(True)
    ctx.profile_read(binding.KERNEL_BINS)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    steps = max(args.steps, 30)   # a timed region of about a second for the clock samples
    e0.record(st)
    for _ in range(steps):
        step()
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    k_ms, k_n = ctx.profile_read(binding.KERNEL_BINS)
    ctx.profile_enable(False)
    clk = clocks.stop()
    # end to end: rays from pinned host memory, intensities back to pinned memory
    hm, hT, hP = (torch.from_numpy(a).pin_memory() for a in (m, T, P))
    hout = torch.empty(out.shape, dtype=torch.float32).pin_memory()
    for _ in range(2):
        dm.copy_(hm, non_blocking=True)
        dT.copy_(hT, non_blocking=True)
        dP.copy_(hP, non_blocking=True)
        step()
        hout.copy_(out, non_blocking=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        dm.copy_(hm, non_blocking=True)
        dT.copy_(hT, non_blocking=True)
        dP.copy_(hP, non_blocking=True)
        step()
        hout.copy_(out, non_blocking=True)
    torch.cuda.synchronize()
    t_e2e = (time.perf_counter() - t0) / args.steps
    # oracle baseline on a bounded sample of rays
    t0 = time.perf_counter()
    done = 0
    while time.perf_counter() - t0 < 10.0 and done < 64:
        obi.bin_intensity(odf.reshape(nT, nP, K, ns), kc.reshape(nT, nP).astype(np.float64), lt, lp, lam,
                          wl.ODF_WIDTHS_12, m[done], T[done], P[done], mus)
        done += 1
    t_cpu = time.perf_counter() - t0
    updates = n * K * ns * (D - 1) * len(mus)
    out_line = {"mode": "bins", "metric": "rays/s (bin intensities from an ODF table)", "value": n / (ms / 1e3),
                "unit": "rays/s", "n_gpus": 1, "steps": steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"odf_table_57x25x{K}x{ns}_rays{n}_D{D}_mu5", "rays": n, "depth": D, "bins": K,
                           "sub_bins": ns, "mu": len(mus), "table_bytes": int(odf.nbytes + kc.nbytes)},
                "bin_intensities_per_s": n * K / (ms / 1e3),
                "layer_updates_per_s": updates / (ms / 1e3),
                "kernel_ms": k_ms / max(k_n, 1),
                "e2e": {"value": n / t_e2e, "unit": "rays/s", "h2d_bytes_per_step": int(3 * m.nbytes),
                        "d2h_bytes_per_step": int(hout.numel() * 4)},
                "cpu_baseline": {"value": done / t_cpu, "unit": "rays/s", "cores": 1, "kind": "oracle",
                                 "sample": f"{done} rays of the same table"},
                "gpu_launches": 3 * steps, "clocks": clk}
    print(json.dumps(out_line), flush=True)


_PREC_STATE = None


def _prec_worker_init(path):
    # the line list, memory-mapped from the arrays the parent saved
    global _PREC_STATE
    arrs = {f: np.load(os.path.join(path, f + ".npy"), mmap_mode="r") for f in
            ("lam_nm", "log_gf", "E_eV", "species", "log_gR", "log_gS", "log_gW")}
    _PREC_STATE = wl.LineList(**arrs)


def _prec_worker(job):
    from oracle import synthesis as sy
    r, T, P, js, lam0, lam1, R = job
    el = wl.elements(15)
    se, ss = wl.species_table(15)
    k, sl, kc = sy.kappa_at_chunked(_PREC_STATE, se, ss, el, T, P, wl.Grid(lam0, lam1, R), js)
    return r, k, sl, kc


def precision_arm(args):
    """Precision study: a 1e8-line list (same distributions, 9-10000 nm) on a 6 x 5 (T, P)
    subset of the table, synthesised on a 1 nm slice (300-301 nm at R = 2e6, every line of the
    list whose cut window reaches it) with the four precisions of the library.  Relative errors
    of the opacity against the FP64 oracle at 24 sampled grid points of every row (the oracle's
    chunked sampled synthesis over the whole list, in spawned processes: kappa_c from the median
    over all 1e8 lines), and of opacity and ODF steps against the all-FP64 GPU variant."""
    import multiprocessing as mp
    import shutil
    import torch

    from paper_2105_13611_gb300 import binding
    n_lines = int(os.environ.get("MPSA_PRECISION_LINES", "100000000"))
    t0 = time.perf_counter()
    lines = wl.linelist(n_lines, 30, 9.0, 10000.0, seed=1002)
    t_gen = time.perf_counter() - t0
    print(f"precision: generated {n_lines} lines in {t_gen:.1f} s", file=sys.stderr, flush=True)
    el = wl.elements(15)
    se, ss = wl.species_table(15)
    T, P = wl.tp_grid_dfsynthe()
    ti, pi = np.array([4, 14, 24, 34, 44, 54]), np.array([2, 7, 12, 17, 22])
    rows = (ti[:, None] * 25 + pi[None, :]).reshape(-1).astype(np.int32)
    ctx = binding.Context(0)
    t0 = time.perf_counter()
    ctx.load_linelist(lines, se, ss)
    t_load = time.perf_counter() - t0
    print(f"precision: loaded in {t_load:.1f} s", file=sys.stderr, flush=True)
    ctx.set_atmosphere_grid(el, T, P)
    g = wl.Grid(300.0, 301.0, 2e6)
    N = binding.grid_size(g.lam0_nm, g.lam1_nm, g.R)
    b = wl.equal_intervals(N, 4)
    res, times, evals = {}, {}, None
    names = {2: "fp64_all", 1: "fp32_naive_sums", 0: "fp32_kahan_sums", 3: "fp32_kahan_fp32_populations"}
    for prec in (2, 1, 0, 3):
        k = torch.empty((len(rows), N), dtype=torch.float32, device="cuda")
        kc = torch.empty(len(rows), dtype=torch.float32, device="cuda")
        ev = torch.empty(len(rows), dtype=torch.int64, device="cuda")
        o = torch.empty((len(rows), 4, 12), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(0, len(rows), 6):  # six rows per call: scratch is ~105 B per (row, line)
            ctx.synth_opacity(g, rows[i:i + 6], k[i:i + 6], kc[i:i + 6], ev[i:i + 6],
                              opts=binding.make_opts(1e-3, 1e-2, prec))
        ctx.build_odf(k, b, wl.ODF_WIDTHS_12, o)
        torch.cuda.synchronize()
        times[names[prec]] = time.perf_counter() - t0
        print(f"precision: {names[prec]} {times[names[prec]]:.1f} s", file=sys.stderr, flush=True)
        res[prec] = (k.double().cpu().numpy(), kc.double().cpu().numpy(), o.cpu().numpy())
        evals = int(ev.sum())
    ctx.close()
    # ---- the FP64 oracle at sampled points of every row
    rng = np.random.default_rng(5)
    lnq = math.log1p(1.0 / g.R)
    i0, i1 = np.searchsorted(lines.lam_nm, [g.lam0_nm, g.lam1_nm])
    strong = i0 + np.argsort(lines.log_gf[i0:i1])[-8:]
    centres = np.clip(np.round(np.log(lines.lam_nm[strong] / g.lam0_nm) / lnq).astype(np.int64), 0, N - 1)
    js = np.unique(np.r_[rng.integers(0, N, 16), centres])
    tmp = tempfile.mkdtemp(prefix="mpsa_lines_")
    t0 = time.perf_counter()
    try:
        for f in ("lam_nm", "log_gf", "E_eV", "species", "log_gR", "log_gS", "log_gW"):
            np.save(os.path.join(tmp, f + ".npy"), getattr(lines, f))
        del lines
        jobs = [(int(r), float(T[r]), float(P[r]), js, g.lam0_nm, g.lam1_nm, g.R) for r in rows]
        n_proc = min(len(jobs), max(1, (os.cpu_count() or 1)))
        with mp.get_context("spawn").Pool(n_proc, initializer=_prec_worker_init, initargs=(tmp,)) as pool:
            orc = {r: (k_, s_, kc_) for r, k_, s_, kc_ in pool.map(_prec_worker, jobs)}
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
    t_orc = time.perf_counter() - t0
    print(f"precision: oracle at {len(js)} points x {len(rows)} rows in {t_orc:.1f} s", file=sys.stderr, flush=True)
    kr, kcr, orf = res[2]
    out = {"mode": "precision", "lines": n_lines, "rows": "6 T x 5 P of the 57 x 25 grid", "slice_nm": [300.0, 301.0],
           "grid_points": N, "evals_per_variant": evals, "reference": "FP64 oracle at sampled points; fp64_all (GPU) dense",
           "oracle_points_per_row": len(js), "oracle_s": t_orc, "oracle_processes": n_proc,
           "generate_s": t_gen, "load_s": t_load, "seconds": times, "variants": {}}
    for prec in (2, 1, 0, 3):
        k, kc, o = res[prec]
        rel_o, viol, kc_dev = [], 0, 0.0
        for n, r in enumerate(rows):
            ko, so, kco = orc[int(r)]
            kg = k[n, js]
            rel_o.append(np.abs(kg - ko) / (ko + kco))
            viol += int(np.sum(np.abs(kg - ko) > 1e-4 * (ko + kco) + so * 1.001))
            kc_dev = max(kc_dev, abs(kc[n] / kco - 1))
        rel_o = np.concatenate(rel_o)
        v = {"opacity_vs_oracle_max_rel": float(rel_o.max()), "opacity_vs_oracle_p99_rel": float(np.quantile(rel_o, 0.99)),
             "points_beyond_1e-4_tolerance": viol, "points_checked": int(len(rel_o)), "kappa_c_vs_oracle_max_rel": kc_dev}
        if prec != 2:
            rel = np.abs(k - kr) / (kr + kcr[:, None])
            ro = np.abs(o - orf) / np.maximum(np.abs(orf), 1e-300)
            v.update({"opacity_vs_fp64_gpu_max_rel": float(rel.max()), "opacity_vs_fp64_gpu_p99_rel": float(np.quantile(rel, 0.99)),
                      "odf_vs_fp64_gpu_max_rel": float(ro.max()), "odf_vs_fp64_gpu_p99_rel": float(np.quantile(ro, 0.99))})
        out["variants"][names[prec]] = v
    print(json.dumps(out), flush=True)


def table_arm(args):
    """The whole ODF table once: every (T, P) row of the 57 x 25 grid through synth_opacity and
    build_odf, in chunks of 16 rows, timed with CUDA events per chunk (inputs resident: the
    line list and the population table).  Prints the wall time, the line-evaluation rate and
    the ODF (T, P) points per second of the whole table, and the slowest chunks."""
    import torch

    from paper_2105_13611_gb300 import binding
    w = wl.config_table()
    lines = w.lines()
    el = wl.elements(w.n_metals)
    se, ss = wl.species_table(w.n_metals)
    ctx = binding.Context(0)
    ctx.load_linelist(lines, se, ss)
    ctx.set_atmosphere_grid(el, w.T, w.P)
    N = binding.grid_size(w.grid.lam0_nm, w.grid.lam1_nm, w.grid.R)
    K = w.n_intervals
    bounds = wl.equal_intervals(N, K)
    chunk = 16
    rows = np.arange(len(w.T), dtype=np.int32)
    kap = torch.empty((chunk, N), dtype=torch.float32, device="cuda")
    kc = torch.empty(chunk, dtype=torch.float32, device="cuda")
    ev = torch.empty(chunk, dtype=torch.int64, device="cuda")
    odf = torch.empty((len(rows), K, len(w.widths)), dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()
    opts = binding.make_opts(w.cut, w.kc_factor)
    # warm-up on the first chunk
    ctx.synth_opacity(w.grid, rows[:chunk], kap, kc, ev, opts=opts, stream=st)
    ctx.build_odf(kap, bounds, w.widths, odf[:chunk], stream=st)
    torch.cuda.synchronize()
    clocks = Clocks(0)
    clocks.start()
    ctx.profile_enable(True)
    ctx.profile_read(binding.KERNEL_PROFILE)
    ctx.profile_read(binding.KERNEL_ODF)
    evs, per_chunk = 0, []
    t0 = time.perf_counter()
    for i in range(0, len(rows), chunk):
        sel = rows[i:i + chunk]
        n = len(sel)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        ctx.synth_opacity(w.grid, sel, kap[:n], kc[:n], ev[:n], opts=opts, stream=st)
        ctx.build_odf(kap[:n], bounds, w.widths, odf[i:i + n], stream=st)
        e1.record(st)
        e1.synchronize()
        per_chunk.append((int(sel[0]), int(sel[-1]), e0.elapsed_time(e1) / 1e3, int(ev[:n].sum())))
        evs += per_chunk[-1][3]
    wall = time.perf_counter() - t0
    tiles_ms, _ = ctx.profile_read(binding.KERNEL_PROFILE)
    odf_ms, _ = ctx.profile_read(binding.KERNEL_ODF)
    clk = clocks.stop()
    gpu_s = sum(c[2] for c in per_chunk)
    slow = sorted(per_chunk, key=lambda c: -c[2])[:5]
    out = {"mode": "table", "metric": "whole 57 x 25 ODF table: wall time, line-evals/s, ODF (T,P) points/s",
           "rows": len(rows), "grid_points": N, "intervals": K, "lines": len(lines), "chunk_rows": chunk,
           "wall_s": wall, "gpu_s": gpu_s, "evals": evs, "evals_per_s": evs / gpu_s,
           "odf_points_per_s": len(rows) / gpu_s, "k_tiles_s": tiles_ms / 1e3, "k_odf_s": odf_ms / 1e3,
           "slowest_chunks": [{"rows": [a, b], "s": t, "evals": e} for a, b, t, e in slow],
           "clocks": clk, "data": "synthetic"}
    print(json.dumps(out), flush=True)


def profile_value(name, key, kernel, sources):
    """A number recorded in a profiles/ summary (key: value), or None when the summary is missing
    or was taken on kernel sources that have changed since (SHA-1 of the files)."""
    import hashlib
    import re
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    text = open(path).read()
    h = hashlib.sha1()
    for f in sources:
        with open(os.path.join(ROOT, "paper_2105_13611_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    m_src = re.search(rf"^{kernel}_source_sha1: ([0-9a-f]+)$", text, re.M)
    m_val = re.search(rf"^{key}: ([0-9.eE+-]+)$", text, re.M)
    if not (m_src and m_val) or m_src.group(1) != h.hexdigest():
        return None
    return float(m_val.group(1))


def measured_traffic(kernel, sources, rows):
    """DRAM bytes (read + written) per launch of `kernel` from the ncu summary in
    profiles/traffic_table_workload.md, or None when that capture was taken on other rows
    or on kernel sources that have changed since (recorded as SHA-1 of the files)."""
    import hashlib
    import re
    path = os.path.join(ROOT, "profiles", "traffic_table_workload.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    h = hashlib.sha1()
    for f in sources:
        with open(os.path.join(ROOT, "paper_2105_13611_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    m_rows = re.search(r"^rows: ([0-9,]+)$", text, re.M)
    m_src = re.search(rf"^{kernel}_source_sha1: ([0-9a-f]+)$", text, re.M)
    m_val = re.search(rf"^{kernel}_bytes_per_launch: ([0-9]+)$", text, re.M)
    if not (m_rows and m_src and m_val):
        return None
    if [int(r) for r in m_rows.group(1).split(",")] != [int(r) for r in rows] or m_src.group(1) != h.hexdigest():
        return None
    return int(m_val.group(1))


def main():
    args = parse()
    if args.mode == "precision":
        precision_arm(args)
        return
    if args.mode == "batch":
        batch_arm(args)
        return
    if args.mode == "bins":
        bins_arm(args)
        return
    if args.mode == "table":
        table_arm(args)
        return
    if args.mode == "serve":
        serve_arm(args)
        return
    if args.mode == "spectrum":
        spectrum_arm(args)
        return
    if args.impl == "reference":
        reference_arm(args)
    else:
        native_arm(args)


if __name__ == "__main__":
    main()
