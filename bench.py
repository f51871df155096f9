#!/usr/bin/env python
"""Benchmark of the GB300 transmission-BEM hot path.

One step = one complete transmission solve of the at-scale sphere workload in the
mixed-precision mode (the headline), and the same solve in plain FP64 (the
comparison arm, reported under "fp64"):
grid intake of both grids, Galerkin assembly of V, K, T, D on both grids (regular
and Sauter-Schwab quadrature), mass and mortar matrices, plane-wave data, and
unrestarted GMRES on the mass-preconditioned multiple-traces system.

Workload (at scale): unit sphere; exterior grid = icosphere level 5 (10242
vertices, 20480 triangles); interior grid = icosphere level 5 rotated by a
Haar-random rotation (seed 2) with 1% tangential jitter; k_ext = 10, k_int = 15,
rho_int / rho_ext = 2; one unit plane wave along +z; GMRES tolerance 1e-8;
40968 unknowns, 8 dense operator blocks (6.7 GB complex64 in the mixed mode,
13.4 GB complex128 in FP64).  The headline "value" is the mixed-precision rate;
"accuracy" gives its traces' relative L2 error against a converged FP64 solve
(target <= 1e-6); "fp64" holds the plain-FP64 GPU arm.

Output (rank 0): one JSON line per section ({"section": name, ...}: autotune, mixed,
fp64, e2e, serving, field, formulations, screen, cuda_graphs, cube, batching,
uneven_instances, cpu_baseline), then, as the LAST line, the compact contract line
(metric, value, latency, accuracy, fp64 arm, rooflines, cpu_baseline, e2e, clocks,
launches; under 1.5 KB).  The headline steps are timed with CUDA events and no
profiler events; the rooflines come from separate profiled steps of the same workload.
`--impl reference` times the FP64 CPU oracle on a bounded sample of the same workload
on all host cores, extrapolated to one solve.  `--case` runs one small profiling case
(for ncu) instead.  With torchrun (N > 1) every rank solves its own copy (the method
has no data exchange between solves: replicas).
"""
from __future__ import annotations

import argparse
import re
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "Transmission solves/s + p50/p99 latency vs plain FP64 GPU at <=1e-6 rel. err"
UNIT = "solves/s"
WORKLOAD = dict(level_ext=5, level_int=5, seed=2, k_ext=10.0, k_int=15.0, rho=2.0, tol=1e-8)
WORKLOAD_NAME = ("at-scale sphere: icosphere L5 exterior (10242 vertices) + L5 interior rotated/jittered "
                 "(seed 2), k_ext=10, k_int=15, rho_int/rho_ext=2, 1 plane wave +z, GMRES tol 1e-8, "
                 "40968 unknowns")
L2_FLUSH_BYTES = 256 << 20
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12  # SMs x DFMA/clk/SM x 2 flops x max SM clock
# Algorithmic flops per point pair of the regular-pair assembly, counted from the
# oracle's formula (G, dG/dn(y), dG/dn(x) of Sec. 2.1 and the Galerkin sums of V, K, T,
# with D formed per triangle pair from V and the integral of G), FMA = 2, add/mul = 1,
# sqrt = rcp = 1, sincos = 2, summed over q first (the per-p outer sums amortised over
# the 6 points q of the trial triangle):
FLOP_COUNT_PER_POINT_PAIR = (
    ("d = x - y", 3),
    ("r^2 = d.d", 5),
    ("r = sqrt(r^2), 1/r", 2),
    ("phase k r", 1),
    ("cos, sin of the phase", 2),
    ("1 / (4 pi r)", 1),
    ("G = exp(i k r) / (4 pi r)", 2),
    ("F = G (1 - i k r) / r^2", 7),
    ("d.n(y), d.n(x)", 10),
    ("dG/dn(y) = F d.n(y), dG/dn(x) = -F d.n(x)", 4),
    ("sum over q of (w L_b)(q) x {G, dG/dn(y), dG/dn(x)}, b = 0..2", 36),
    ("sum over p of (w L_a)(p) x the three 3-vectors, per q", 18),
)
FLOP_PER_POINT_PAIR = sum(f for _, f in FLOP_COUNT_PER_POINT_PAIR)  # 91, FP64 and FP32 kernels alike

# Flops per point of the Sauter-Schwab singular-pair quadrature, counted from the oracle's
# formula the same way (each point carries its own x, y and all nine shape-value products):
FLOP_COUNT_PER_SINGULAR_POINT = (
    ("x = sum_m B_m(x^) X_m, y likewise (3 components each)", 30),
    ("kernel values G, dG/dn(y), dG/dn(x) as for a regular point pair", 37),
    ("per (a, b): w L_a L_b, then V, K, T accumulations (complex)", 126),
)
FLOP_PER_SINGULAR_POINT = sum(f for _, f in FLOP_COUNT_PER_SINGULAR_POINT)  # 193
SINGULAR_N = 4  # Gauss-Legendre points per axis (bem_solve_opts.n_singular default)


def singular_points(t, n=SINGULAR_N):
    """Quadrature points of the singular pairs of one grid: each unordered pair once
    (coincident: 6 regions, edge-adjacent: 4, vertex-adjacent: 2; n^4 points each)."""
    t = np.asarray(t)
    nv = int(t.max()) + 1
    vt = [[] for _ in range(nv)]
    for i, tri in enumerate(t):
        for v in tri:
            vt[v].append(i)
    shared = {}
    for i, tri in enumerate(t):
        for v in tri:
            for j in vt[v]:
                if j > i:
                    shared[(i, j)] = shared.get((i, j), 0) + 1
    edge = sum(1 for c in shared.values() if c == 2)
    vert = sum(1 for c in shared.values() if c == 1)
    return (6 * len(t) + 4 * edge + 2 * vert) * n ** 4


# Unit-cube efficiency benchmarks (Sec. 5.5): the physics of the paper's table of physical
# parameters (wavenumber 2 pi f / c of each medium; density ratio rho_int / rho_ext) and
# nonconforming grids with the node counts of its mesh table (N_ext, N_int), here structured
# cube grids with n nodes per cube edge, n chosen so that 6 n^2 + 2 is nearest to N; GMRES
# tolerance 1e-5 as in Sec. 5.1; plane wave along +x (eq. planewave).
CUBE_BENCHMARKS = (
    dict(name="standard", f=1.0, c_ext=0.3, c_int=1.1, rho_ext=1.0, rho_int=2.0, N_ext=2836, N_int=272),
    dict(name="high frequency", f=3.0, c_ext=0.3, c_int=1.1, rho_ext=1.0, rho_int=2.0, N_ext=25302, N_int=2072),
    dict(name="high contrast", f=1.0, c_ext=0.1, c_int=1.1, rho_ext=0.11, rho_int=2.0, N_ext=25302, N_int=272),
)
CUBE_TOL = 1e-5
CUBE_CENTER = (0.5, 0.5, 0.5)


def cube_edge_nodes(N):
    """n with 6 n^2 + 2 nearest to N (nodes of a structured cube grid)."""
    n = max(1, int(round(((N - 2) / 6.0) ** 0.5)))
    return min((m for m in (n - 1, n, n + 1) if m >= 1), key=lambda m: abs(6 * m * m + 2 - N))


def cube_case(b):
    """(grids, k_ext, k_int, rho) of one cube benchmark."""
    import bem_inputs as bi
    ve, te = bi.cube_grid(cube_edge_nodes(b["N_ext"]), jitter=0.3, seed=61)
    vi, ti = bi.cube_grid(cube_edge_nodes(b["N_int"]), jitter=0.3, seed=62)
    k_ext = 2.0 * np.pi * b["f"] / b["c_ext"]
    k_int = 2.0 * np.pi * b["f"] / b["c_int"]
    return (ve, te, vi, ti), k_ext, k_int, b["rho_int"] / b["rho_ext"]


def workload_inputs(w=WORKLOAD):
    import bem_inputs as bi
    return bi.transmission_pair(w["level_ext"], w["level_int"], w["seed"])


def regular_point_pairs(t):
    """Unordered triangle pairs without a common vertex, times 36 point pairs."""
    t = np.asarray(t)
    nt = len(t)
    nv = int(t.max()) + 1
    # singular unordered pairs (t < s sharing >= 1 vertex) via vertex -> triangle lists
    vt = [[] for _ in range(nv)]
    for i, tri in enumerate(t):
        for v in tri:
            vt[v].append(i)
    sing = set()
    for i, tri in enumerate(t):
        for v in tri:
            for j in vt[v]:
                if j > i:
                    sing.add((i, j))
    return (nt * (nt - 1) // 2 - len(sing)) * 36


# ----------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self, index=0):
        self.index = index
        self.lines = []
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------- CPU oracle sample
# GMRES iterations of one at-scale solve at tol 1e-8: the GPU path takes 205 in FP64 and
# 205 inner iterations in the mixed mode, and the oracle's GMRES matches the FP64 path's
# count within one (parity tests), so the extrapolated oracle solve uses the same count
# in both arms.
ORACLE_GMRES_ITERS = 205
ORACLE_MATVEC_ROWS = 512
_ORACLE_STATE = {}


def _oracle_init():
    """Pool worker set-up: the workload's grids, built once per worker process."""
    _ORACLE_STATE["grids"] = workload_inputs()


def _oracle_task(seed):
    """Oracle assembly of all four operators for the test triangles of one random row of
    each grid (the row's vertex star); returns (t_start, t_end, test triangles done)."""
    from oracle.helmholtz import assemble
    w = WORKLOAD
    if "grids" not in _ORACLE_STATE:
        _oracle_init()
    ve, te, vi, ti = _ORACLE_STATE["grids"]
    rng = np.random.default_rng(seed)
    t0 = time.monotonic()
    done = 0
    for (v, t, k) in ((ve, te, w["k_ext"]), (vi, ti, w["k_int"])):
        rows = rng.choice(len(v), 1, replace=False)
        done += int(np.count_nonzero(np.isin(np.asarray(t), rows).any(axis=1)))
        assemble(v, t, k, rows=rows)
    return t0, time.monotonic(), done


def oracle_sample_steps(steps, cores, seed=0):
    """Run `steps` bounded samples of the FP64 CPU oracle on `cores` host cores and
    extrapolate each to one at-scale solve.  Per sample: `cores` processes each assemble
    V, K, T, D for one random row of each grid (about 6 test triangles x 20480 trial
    triangles per grid); the wall time of that concurrent phase gives the oracle's
    assembly rate in test triangles per second on `cores` cores, scaled to both grids'
    40960 test triangles; then the dense strong-form matvec on a 512-row block of the
    40968 x 40968 system (BLAS on `cores` threads), scaled by rows and by the GMRES
    iteration count.  Mortar, mass, preconditioner and Arnoldi are not counted."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    ve, te, vi, ti = workload_inputs()
    n = 2 * len(ve) + 2 * len(vi)
    nt_total = len(te) + len(ti)
    rng = np.random.default_rng(seed)
    blk = ORACLE_MATVEC_ROWS
    A = (rng.standard_normal((blk, n)) + 1j * rng.standard_normal((blk, n)))
    z = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    out = []
    pool = None
    if cores > 1:
        # workers do their assembly on one thread each (they are the parallelism)
        for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[var] = "1"
        pool = ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn"), initializer=_oracle_init)
        list(pool.map(_oracle_task, [10_000 + i for i in range(cores)], chunksize=1))  # start + warm the workers
    try:
        for s in range(steps):
            t_step = time.monotonic()
            seeds = [1000 * (s + 1) + i for i in range(cores)]
            res = list(pool.map(_oracle_task, seeds, chunksize=1)) if pool else [_oracle_task(seeds[0])]
            wall = max(r[1] for r in res) - min(r[0] for r in res)
            tris = sum(r[2] for r in res)
            t_asm = wall / tris * nt_total
            t0 = time.monotonic()
            reps = 3
            for _ in range(reps):
                A @ z
            t_mv = (time.monotonic() - t0) / reps * (n / blk)
            total = t_asm + ORACLE_GMRES_ITERS * t_mv
            out.append({"value": 1.0 / total, "step_ms": 1e3 * (time.monotonic() - t_step),
                        "t_assembly_s": t_asm, "t_matvec_s": t_mv, "test_triangles": tris})
    finally:
        if pool:
            pool.shutdown()
    desc = (f"extrapolated: V,K,T,D of ~{out[-1]['test_triangles']} of {nt_total} test triangles "
            f"(x{nt_total / out[-1]['test_triangles']:.0f}) + a {blk}-row block of the {n}-row dense matvec "
            f"(x{n / blk:.0f}) x {ORACLE_GMRES_ITERS} GMRES iterations; mortar/mass/Arnoldi not counted")
    return out, desc


def run_oracle_child(steps, cores):
    """The oracle sample in a child process whose BLAS uses `cores` threads; returns
    dict(steps=[...], sample=..., cores=...) or None if it failed."""
    c = str(cores)
    env = dict(os.environ, OMP_NUM_THREADS=c, OPENBLAS_NUM_THREADS=c, MKL_NUM_THREADS=c)
    code = ("import json,sys; sys.path.insert(0,%r); import bench; r,d=bench.oracle_sample_steps(%d,%d); "
            "print(json.dumps({'steps':r,'sample':d}))" % (ROOT, steps, cores))
    p = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if p.returncode != 0:
        sys.stderr.write(p.stderr[-2000:])
        return None
    r = json.loads(p.stdout.strip().splitlines()[-1])
    r["cores"] = cores
    return r


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


# ----------------------------------------------------------------- reference arm
def run_reference(args, rank):
    """The FP64 CPU oracle as the reference arm: each step is one bounded sample of the
    at-scale workload on all host cores, extrapolated to one solve (value = median over
    the timed steps); a one-core sample is reported beside it."""
    if rank != 0:
        return
    t0 = time.perf_counter()
    cores = host_cores()
    r = run_oracle_child(args.warmup + args.steps, cores)
    one = run_oracle_child(1, 1)
    if r is None:
        print(json.dumps({"impl": "reference", "unavailable": "the CPU oracle sample failed to run"}))
        return
    timed = r["steps"][args.warmup:]
    value = statistics.median(s["value"] for s in timed)
    ms_step = statistics.mean(s["step_ms"] for s in timed)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "extrapolated": True,
        "ms_per_solve_extrapolated": 1e3 / value,
        "config": {"workload": WORKLOAD_NAME, "parallelism": "replicas"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": r["sample"],
                         "one_core_value": (one["steps"][0]["value"] if one else None)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": time.perf_counter() - t0,
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- GPU arm
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # SMs x FP32 lanes x 2 flops x max SM clock
HBM_PEAK_GBS = None


def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s"


def serving_stream(n, seed=50):
    """First n requests of the seeded serving stream (ellipsoids, levels 2-4, random
    wavenumbers, density ratios and 1-16 plane waves), grids built ahead of time."""
    import bem_inputs as bi
    reqs = bi.serving_requests(n, seed, rate=1.0)
    out = []
    for r in reqs:
        ve, te, vi, ti = bi.transmission_pair(r["level_ext"], r["level_int"], r["seed"], axes=r["axes"])
        out.append(dict(ve=ve, te=te, vi=vi, ti=ti, k_ext=r["k_ext"], k_int=r["k_int"], rho=r["rho_ratio"],
                        dirs=r["dirs"], arrival=r["arrival"]))
    return out


SERVE_STREAM_LENGTH = 2000  # requests of the whole seeded serving stream


def run_serving(bem, reqs, precision, rate=None, max_inflight=4, group_max=0):
    """Submit the requests (all at once when rate is None, else at Poisson arrival
    times scaled to `rate` per second); returns latencies (ms) and solves/s.
    group_max: the server's lockstep-group limit (0: its default; 1: every request
    alone)."""
    srv = bem.bem_serve_create(max_inflight=max_inflight, precision=precision, group_max=group_max)
    try:
        t0 = time.perf_counter()
        tickets = []
        base = reqs[0]["arrival"]
        for r in reqs:
            if rate is not None:
                due = t0 + (r["arrival"] - base) / rate
                wait = due - time.perf_counter()
                if wait > 0:
                    time.sleep(wait)
            tickets.append(bem.bem_serve_submit(srv, r["ve"], r["te"], r["vi"], r["ti"], r["k_ext"], r["k_int"],
                                                r["rho"], r["dirs"], precision=precision))
        infos = []
        for t in tickets:
            bem.bem_serve_wait(srv, t, 0.0)
            infos.append(bem.bem_serve_poll(srv, t))
        wall = time.perf_counter() - t0
        stats = bem.bem_serve_get_stats(srv)
    finally:
        bem.bem_serve_destroy(srv)
    lat = np.array([i["total_ms"] for i in infos])
    ok = sum(1 for i in infos if i["status"] == 0)
    return {"requests": len(reqs), "ok": ok, "solves_per_s": len(reqs) / wall,
            "rhs_per_s": sum(len(r["dirs"]) for r in reqs) / wall,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "wall_s": wall, "hbm_high_water_bytes": stats["hbm_high_water_bytes"],
            "lockstep_groups": stats["groups"], "requests_in_groups": stats["grouped"]}


BATCH_WORKLOAD = dict(level=4, seed=4, k_ext=5.0, k_int=7.5, rho=1.0, n_dirs=64, n_single=8)
TF32_PER_BF16 = 1.1 / 2.25  # nominal dense TF32 / BF16 tensor rates of GB300


def tf32_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            v = float(json.load(fh)["bf16_tflops"])
        return v * TF32_PER_BF16, "measured bf16 burst (MEASURED_PEAKS.json) x nominal TF32/BF16 ratio 1.1/2.25"
    except (OSError, KeyError, ValueError):
        return 1900.0 * TF32_PER_BF16, "fallback 1.9 PFLOP/s bf16 x nominal TF32/BF16 ratio"


def fp16_peak():
    """Dense FP16 tensor rate: the measured BF16 burst (FP16 and BF16 run at the same
    nominal rate on GB300)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["bf16_tflops"]), "measured bf16 burst (MEASURED_PEAKS.json), = fp16 rate"
    except (OSError, KeyError, ValueError):
        return 1900.0, "fallback 1.9 PFLOP/s bf16 (= fp16 rate)"


def run_batching(bem, ctx, precision, tensor_cores=2, batch_columns=0):
    """Many plane waves at one frequency: one call with all directions (solved in
    lockstep batches) against the same directions one call each; the batched call
    is profiled per kernel."""
    import torch
    import bem_inputs as bi
    b = BATCH_WORKLOAD
    ve, te, vi, ti = bi.transmission_pair(b["level"], b["level"], b["seed"])
    dirs = bi.plane_wave_directions(b["n_dirs"], seed=b["seed"] + 100)
    opts = {"precision": precision, "tensor_cores": tensor_cores, "batch_columns": batch_columns}
    ge = bem.bem_grid_create(ctx, ve, te)
    gi = bem.bem_grid_create(ctx, vi, ti)
    bem.bem_solve_transmission(ctx, ge, gi, b["k_int"], b["k_ext"], b["rho"], dirs[:16], opts=opts)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, rep = bem.bem_solve_transmission(ctx, ge, gi, b["k_int"], b["k_ext"], b["rho"], dirs, opts=opts)
    t_batch = time.perf_counter() - t0
    bem.bem_profile_reset()
    bem.bem_profile_enable(True)
    bem.bem_solve_transmission(ctx, ge, gi, b["k_int"], b["k_ext"], b["rho"], dirs, opts=opts)
    bem.bem_context_synchronize(ctx)
    bem.bem_profile_enable(False)
    prof = bem.bem_profile_table()
    single_solve_ms, single_wall = [], 0.0
    for r in range(b["n_single"]):
        t0 = time.perf_counter()
        _, r1 = bem.bem_solve_transmission(ctx, ge, gi, b["k_int"], b["k_ext"], b["rho"], dirs[r:r + 1], opts=opts)
        single_wall += time.perf_counter() - t0
        single_solve_ms.append(r1["t_solve_ms"])
    bem.bem_grid_destroy(ge)
    bem.bem_grid_destroy(gi)
    out = {"rhs_per_s_one_call": b["n_dirs"] / t_batch,
           "rhs_per_s_one_call_each": b["n_single"] / single_wall,
           "solve_ms_per_rhs_batched": rep["t_solve_ms"] / b["n_dirs"],
           "solve_ms_per_rhs_single": float(np.mean(single_solve_ms)),
           "iterations_per_rhs_batched": rep["iterations"] / b["n_dirs"],
           "assembly_ms": rep["t_assembly_ms"],
           "kernels": [{"name": p[0], "ms": p[1], "launches": p[2]} for p in prof[:8]]}
    tc = [p for p in prof if p[0] == "k_gemm_tc" or p[0].startswith("k_gemm_tc16")]
    if tc:
        name, ms, nl = tc[0]
        N = len(ve)  # both grids have the same level here
        rp = (b["n_dirs"] + 7) // 8 * 8 if batch_columns == 0 else (batch_columns + 7) // 8 * 8
        flops = 96.0 * rp * (N * N + len(vi) * len(vi))  # 3 split terms x 2 flops x K 4N x N_b x 2 RP, 4 block rows
        if name.startswith("k_gemm_tc16"):
            peak, kind = fp16_peak()
            kp = lambda n: (4 * n + 63) // 64 * 64
            nbytes = 2 * (N * kp(N) + len(vi) * kp(len(vi))) * 4  # hi + lo halves, padded rows, 4 block rows
        else:
            peak, kind = tf32_peak()
            nbytes = 8 * 4 * (N * N + len(vi) * len(vi))
        ach = flops / (ms / nl / 1e3) / 1e12
        # the three split terms are tensor work; the method's own product is one of them
        out["tensor_roofline"] = {"kernel": name, "bound": "tensor", "achieved": ach, "peak": peak,
                                  "unit": "TFLOP/s", "frac": ach / peak, "traffic": None, "peak_kind": kind,
                                  "flops_per_launch": flops, "method_flops_per_launch": flops / 3,
                                  "method_tflops": ach / 3, "avg_launch_ms": ms / nl, "bytes_per_launch": nbytes,
                                  "hbm_frac": nbytes / (ms / nl / 1e3) / 1e9 / hbm_peak()[0]}
    return out


BATCH_FULL_WORKLOAD = dict(level=4, seed=4, n_dirs=256, n_freq=8, k_lo=2.0, k_hi=8.0, ratio=1.5, rho=1.0)


def run_batching_full(bem, ctx):
    """The whole many-waves workload: 256 plane-wave directions uniform on S^2 at each
    of 8 frequencies (k_ext U[2, 8], k_int = 1.5 k_ext) on the icosphere L4 pair, one
    bem_solve_transmission call per frequency (operators assembled once per call, the
    256 waves in tensor-core batches of 64), mixed precision, host buffers; wall clock
    of the 8 calls."""
    import torch
    import bem_inputs as bi
    b = BATCH_FULL_WORKLOAD
    ve, te, vi, ti = bi.transmission_pair(b["level"], b["level"], b["seed"])
    dirs = bi.plane_wave_directions(b["n_dirs"], seed=b["seed"] + 200)
    ks = np.random.default_rng(b["seed"] + 300).uniform(b["k_lo"], b["k_hi"], b["n_freq"])
    ge = bem.bem_grid_create(ctx, ve, te)
    gi = bem.bem_grid_create(ctx, vi, ti)
    opts = {"precision": bem.BEM_PREC_MIXED}
    bem.bem_solve_transmission(ctx, ge, gi, b["ratio"] * ks[0], ks[0], b["rho"], dirs[:16], opts=opts)  # warm-up
    torch.cuda.synchronize()
    per, t_all = [], time.perf_counter()
    for k in ks:
        t0 = time.perf_counter()
        _, rep = bem.bem_solve_transmission(ctx, ge, gi, b["ratio"] * k, k, b["rho"], dirs, opts=opts)
        per.append({"k_ext": float(k), "seconds": time.perf_counter() - t0,
                    "iterations_per_rhs": rep["iterations"] / b["n_dirs"], "converged": bool(rep["converged"]),
                    "t_assembly_ms": rep["t_assembly_ms"]})
    wall = time.perf_counter() - t_all
    bem.bem_grid_destroy(ge)
    bem.bem_grid_destroy(gi)
    n = b["n_dirs"] * b["n_freq"]
    return {"workload": f"icosphere L{b['level']} pair (seed {b['seed']}), {b['n_dirs']} directions uniform on "
                        f"S^2 x {b['n_freq']} frequencies k_ext U[{b['k_lo']}, {b['k_hi']}], "
                        f"k_int = {b['ratio']} k_ext, rho {b['rho']}, mixed precision, tensor-core batches "
                        "of 64, one call per frequency, host buffers",
            "rhs": n, "seconds": wall, "rhs_per_s": n / wall, "all_converged": all(q["converged"] for q in per),
            "per_frequency": per}


def run_field(bem, ctx, w, ve, te, vi, ti, out):
    """Fields of the headline solve (mixed-precision traces) on a 100 x 100 grid of
    the plane z = 0 over [-2, 2]^2 (the paper evaluates its fields on a 100 x 100 plane
    grid): the interior field with the interior grid and the scattered field with the
    exterior grid, each at every point.  Their accuracy against the Mie series is
    checked in the tests; here only the throughput."""
    import torch
    g1 = np.linspace(-2.0, 2.0, 100)
    X, Y = np.meshgrid(g1, g1, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], axis=1)
    ge, gi = bem.bem_grid_create(ctx, ve, te), bem.bem_grid_create(ctx, vi, ti)
    host = {k: out[k][0].cpu().numpy() for k in out}
    bem.bem_field(ctx, gi, w["k_int"], pts[:64], phi=host["v_int"], psi=host["w_int"])  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    bem.bem_field(ctx, gi, w["k_int"], pts, phi=host["v_int"], psi=host["w_int"])
    bem.bem_field(ctx, ge, w["k_ext"], pts, phi=host["v_ext"], psi=host["w_ext"])
    t = time.perf_counter() - t0
    bem.bem_grid_destroy(ge)
    bem.bem_grid_destroy(gi)
    evals = len(pts) * 6 * (len(te) + len(ti))  # (point, quadrature point) pairs of both calls
    return {"points": len(pts), "plane": "z = 0, [-2, 2]^2, 100 x 100", "seconds": t,
            "evaluations_per_s": evals / t,
            "note": "interior and scattered fields of the at-scale traces, FP64 kernel, host buffers"}


UNEVEN_WORKLOAD = dict(count=32, seed=42)


def run_cube(bem, ctx, formulations=("mtf", "pmchwt_ext", "hc_ext_neu")):
    """The unit-cube efficiency benchmarks (CUBE_BENCHMARKS) with nonconforming grids, and the
    standard one also with conforming grids (the interior grid as fine as the exterior one):
    one mixed-precision solve per formulation, host buffers, times from the solve report
    (device events) and the wall clock."""
    import torch
    forms = {"mtf": bem.BEM_FORM_MTF, "pmchwt_ext": bem.BEM_FORM_PMCHWT, "muller_ext": bem.BEM_FORM_MULLER,
             "pmchwt_int": bem.BEM_FORM_PMCHWT_INT, "muller_int": bem.BEM_FORM_MULLER_INT,
             "hc_ext_neu": bem.BEM_FORM_HC_EXT_NEU, "hc_ext_dir": bem.BEM_FORM_HC_EXT_DIR,
             "hc_int_neu": bem.BEM_FORM_HC_INT_NEU, "hc_int_dir": bem.BEM_FORM_HC_INT_DIR}
    cases = [(b["name"], b) for b in CUBE_BENCHMARKS]
    cases.insert(1, ("standard (conforming)", dict(CUBE_BENCHMARKS[0], N_int=CUBE_BENCHMARKS[0]["N_ext"])))
    out = {"workload": "unit cube [0,1]^3, structured face grids with in-face jitter 0.3 (seeds 61/62), "
                       "plane wave +x, GMRES tol 1e-5, mixed precision, one solve each",
           "cases": []}
    for name, b in cases:
        (ve, te, vi, ti), k_ext, k_int, rho = cube_case(b)
        entry = {"benchmark": name, "k_ext": k_ext, "k_int": k_int, "rho_int_over_rho_ext": rho,
                 "N_ext": len(ve), "N_int": len(vi), "paper_N": [b["N_ext"], b["N_int"]]}
        for fname in formulations:
            opts = {"precision": bem.BEM_PREC_MIXED, "gmres_tol": CUBE_TOL, "gmres_maxiter": 6000,
                    "formulation": forms[fname], "center": CUBE_CENTER}
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ge, gi = bem.bem_grid_create(ctx, ve, te), bem.bem_grid_create(ctx, vi, ti)
            try:
                _, rep = bem.bem_solve_transmission(ctx, ge, gi, k_int, k_ext, rho, np.array([[1.0, 0.0, 0.0]]),
                                                    opts=opts)
            except bem.BemError as e:
                rep = e.report
            finally:
                bem.bem_grid_destroy(ge)
                bem.bem_grid_destroy(gi)
            wall = time.perf_counter() - t0
            entry[fname] = {"seconds": wall, "iterations": rep["iterations"], "converged": bool(rep["converged"]),
                            "residual": rep["residual"], "t_assembly_ms": rep["t_assembly_ms"],
                            "t_mortar_ms": rep["t_mortar_ms"], "t_solve_ms": rep["t_solve_ms"],
                            "ms_per_iteration": rep["t_solve_ms"] / max(1, rep["iterations"]),
                            "mortar_share_of_assembly": rep["t_mortar_ms"] / max(1e-9, rep["t_assembly_ms"])}
        out["cases"].append(entry)
    return out


# The screen benchmark of Sec. 5.7: the rectangle of bem_inputs.SCREEN_CORNERS, f = 15, c = 1
# (k = 94.2), plane wave along +x; a fine grid with the paper's 87,712 nodes (here a
# structured 300 x 291 grid, 87,892 nodes) and a coarse one with its 9934 (100 x 97, 9898).
SCREEN_WORKLOAD = dict(fine=(300, 291), coarse=(100, 97), f=15.0, c=1.0, tol=1e-5)


def run_screen(bem, ctx):
    """Mass-matrix, conforming and nonconforming opposite-order preconditioning of the
    Neumann screen at the paper's size, mixed precision, one solve each (host buffers):
    iterations and times from the report, and each opposite-order solution's distance
    from the mass-preconditioned one."""
    import torch
    import bem_inputs as bi
    w = SCREEN_WORKLOAD
    v, t = bi.screen_grid(*w["fine"], jitter=0.2, seed=71)
    vc, tc = bi.screen_grid(*w["coarse"], jitter=0.2, seed=72)
    k = 2.0 * np.pi * w["f"] / w["c"]
    gf, gc = bem.bem_grid_create(ctx, v, t), bem.bem_grid_create(ctx, vc, tc)
    out = {"workload": f"rectangular screen (corners as in the paper), fine {len(v)} nodes, coarse {len(vc)} nodes, "
                       f"k = {k:.1f}, plane wave +x, mixed precision, GMRES tol {w['tol']}", "runs": {}}
    phis = {}
    for name, coarse, pre in (("mass", None, bem.BEM_SCREEN_MASS), ("oo_conforming", gf, bem.BEM_SCREEN_OO),
                              ("oo_nonconforming", gc, bem.BEM_SCREEN_OO)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        try:
            phi, rep = bem.bem_solve_screen(ctx, gf, k, np.array([[1.0, 0.0, 0.0]]), coarse=coarse, precond=pre,
                                            opts={"precision": bem.BEM_PREC_MIXED, "gmres_tol": w["tol"]})
        except bem.BemError as e:
            phi, rep = e.outputs, e.report
        wall = time.perf_counter() - t0
        phis[name] = phi[0]
        out["runs"][name] = {"seconds": wall, "iterations": rep["iterations"], "converged": bool(rep["converged"]),
                             "t_assembly_ms": rep["t_assembly_ms"], "t_mortar_ms": rep["t_mortar_ms"],
                             "t_solve_ms": rep["t_solve_ms"],
                             "ms_per_iteration": rep["t_solve_ms"] / max(1, rep["iterations"])}
    ref = phis["mass"]
    for name in ("oo_conforming", "oo_nonconforming"):
        out["runs"][name]["rel_l2_vs_mass_preconditioned"] = float(np.linalg.norm(phis[name] - ref) /
                                                                   np.linalg.norm(ref))
    bem.bem_grid_destroy(gf)
    bem.bem_grid_destroy(gc)
    return out


def run_graphs(bem, ctx, reps=5):
    """Launch forms of the mass inverses (the 18-35 short kernels of each application):
    one launch per Chebyshev step, the same replayed as CUDA graphs (the default), and one
    cooperative launch per inverse (an exclusive context).  One mixed-precision solve
    (k_ext 10, k_int 15, rho 2, one wave) per grid level, wall time per solve with host
    buffers (median of reps), and the library's launch count."""
    import torch
    import bem_inputs as bi
    out = {"workload": "icosphere pair L/L (seed 2), k_ext=10, k_int=15, rho=2, one plane wave +z, mixed, "
                       "tol 1e-8; median of %d solves per setting" % reps, "levels": []}
    modes = (("steps", 0, 0), ("steps_graphs", 0, 1), ("fused", 1, 1))
    for L in (2, 3, 4):
        ve, te, vi, ti = bi.transmission_pair(L, L, seed=2)
        ge, gi = bem.bem_grid_create(ctx, ve, te), bem.bem_grid_create(ctx, vi, ti)
        entry = {"level": L, "unknowns": 2 * (len(ve) + len(vi))}
        for name, excl, g in modes:
            bem.bem_context_set_exclusive(ctx, bool(excl))
            opts = {"precision": bem.BEM_PREC_MIXED, "cuda_graphs": g}
            bem.bem_solve_transmission(ctx, ge, gi, 15.0, 10.0, 2.0, np.array([[0.0, 0.0, 1.0]]), opts=opts)
            ts, launches = [], 0
            for _ in range(reps):
                torch.cuda.synchronize()
                l0 = bem.bem_launch_count()
                t0 = time.perf_counter()
                _, rep = bem.bem_solve_transmission(ctx, ge, gi, 15.0, 10.0, 2.0, np.array([[0.0, 0.0, 1.0]]),
                                                    opts=opts)
                ts.append(time.perf_counter() - t0)
                launches = bem.bem_launch_count() - l0
            entry[name] = {"ms": 1e3 * statistics.median(ts), "iterations": rep["iterations"], "kernels": launches}
        bem.bem_context_set_exclusive(ctx, False)
        entry["speedup_graphs"] = entry["steps"]["ms"] / entry["steps_graphs"]["ms"]
        entry["speedup_fused"] = entry["steps"]["ms"] / entry["fused"]["ms"]
        bem.bem_grid_destroy(ge)
        bem.bem_grid_destroy(gi)
        out["levels"].append(entry)
    return out


def run_uneven(bem, ctx):
    """Uneven instances: ellipsoids with semi-axes U[0.5, 1.5], exterior and interior
    icosphere levels drawn from {2, 3, 4}, k_ext U[2, 8], k_int = 1.5 k_ext, density
    ratio 1, one random plane wave each; all in one bem_solve_many call against the
    same instances solved one call each (mixed precision)."""
    import torch
    import bem_inputs as bi
    u = UNEVEN_WORKLOAD
    rng = np.random.default_rng(u["seed"])
    probs, grids = [], []
    for i in range(u["count"]):
        axes = rng.uniform(0.5, 1.5, 3)
        le, li = int(rng.integers(2, 5)), int(rng.integers(2, 5))
        ve, te, vi, ti = bi.transmission_pair(le, li, seed=u["seed"] * 1000 + i, axes=axes)
        ge, gi = bem.bem_grid_create(ctx, ve, te), bem.bem_grid_create(ctx, vi, ti)
        grids += [ge, gi]
        k = float(rng.uniform(2.0, 8.0))
        d = bi.plane_wave_directions(1, seed=u["seed"] * 1000 + 500 + i)[0]
        probs.append(dict(ext=ge, intr=gi, k_ext=k, k_int=1.5 * k, rho=1.0, dir=d, levels=(le, li)))
    bem.bem_solve_many(ctx, probs[:4])  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, reps = bem.bem_solve_many(ctx, probs)
    t_many = time.perf_counter() - t0
    t0 = time.perf_counter()
    its_single = 0
    for p in probs:
        _, r1 = bem.bem_solve_transmission(ctx, p["ext"], p["intr"], p["k_int"], p["k_ext"], p["rho"],
                                           np.array([p["dir"]]), opts={"precision": bem.BEM_PREC_MIXED})
        its_single += r1["iterations"]
    t_single = time.perf_counter() - t0
    for g in grids:
        bem.bem_grid_destroy(g)
    return {"instances": u["count"], "levels": [p["levels"] for p in probs],
            "instances_per_s_one_call": u["count"] / t_many, "instances_per_s_one_call_each": u["count"] / t_single,
            "speedup": t_single / t_many, "iterations_one_call": int(sum(r["iterations"] for r in reps)),
            "iterations_one_call_each": int(its_single), "all_converged": all(r["converged"] for r in reps)}


def tiled_operator_bytes(N, entry_bytes):
    """Bytes of one grid's operators in the tiled storage that one product streams:
    V and D as the 64 x 64 tiles of their upper tile triangles, K as all tiles (T = K^T
    is not stored)."""
    nt = (N + 63) // 64
    return (nt * (nt + 1) + nt * nt) * 64 * 64 * entry_bytes


# DRAM bytes (read + write) per launch of the single-column FP32 tile product over the bytes
# it streams: ncu capture of the L4/L4 sphere solve (dram__bytes_read.sum 223,205,888 B +
# dram__bytes_write.sum 5,181,696 B over 223,019,008 B of tiles); the traffic grows with the
# tiles streamed, so the L5 launch's traffic is this ratio times its bytes
TILE_TRAFFIC_RATIO = 1.024


def kernel_roofline(name, ms, n, te, ti, Ne, Ni, pp_cache):
    """Roofline entry of one profiled kernel (per-launch averages)."""
    avg_s = ms / n / 1e3
    if name.startswith("k_tile<"):
        # the product streams the tiled operators of both grids once per launch
        peak, kind = hbm_peak()
        eb = 16 if "c128" in name else 8
        bytes_ = tiled_operator_bytes(Ne, eb) + tiled_operator_bytes(Ni, eb)
        ach = bytes_ / avg_s / 1e9
        traffic = bytes_ * TILE_TRAFFIC_RATIO if (TILE_TRAFFIC_RATIO and name == "k_tile<c64,f32,1>") else None
        return {"kernel": name, "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "traffic": traffic, "peak_kind": kind, "algorithmic_bytes_per_launch": bytes_,
                "bytes_note": "V, D upper tile triangles + K, 64 x 64 tiles, both grids (T = K^T not stored)",
                "avg_launch_ms": ms / n}
    if "k_singular" in name:
        if "sp" not in pp_cache:
            pp_cache["sp"] = (singular_points(te) + singular_points(ti)) / 2
        units = pp_cache["sp"]
        ach = FLOP_PER_SINGULAR_POINT * units / avg_s / 1e12
        return {"kernel": name, "bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / FP64_PEAK_TFLOPS, "traffic": None,
                "peak_kind": "derived FP64 FMA peak: 152 SMs x 2 DFMA/clk x 2 x 2.07 GHz (geometry and kernel "
                             "values on the FP64 pipe; the 54 sums run in double-float on the FP32 pipe)",
                "flop_per_point": FLOP_PER_SINGULAR_POINT, "points_per_launch": units, "avg_launch_ms": ms / n}
    if name.startswith("k_regular"):
        if "pp" not in pp_cache:
            pp_cache["pp"] = (regular_point_pairs(te) + regular_point_pairs(ti)) / 2
        units = pp_cache["pp"]
        fp32 = name.startswith("k_regular32")
        fpp = FLOP_PER_POINT_PAIR
        peak = FP32_PEAK_TFLOPS if fp32 else FP64_PEAK_TFLOPS
        ach = fpp * units / avg_s / 1e12
        return {"kernel": name, "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": None,
                "peak_kind": ("derived FP32 peak: 152 SMs x 128 lanes x 2 x 2.07 GHz" if fp32 else
                              "derived FP64 FMA peak: 152 SMs x 2 DFMA/clk x 2 x 2.07 GHz"),
                "flop_per_point_pair": fpp, "point_pairs_per_launch": units, "avg_launch_ms": ms / n}
    return {"kernel": name, "avg_launch_ms": ms / n}


def _r(x, nd=4):
    """x rounded to nd significant digits (keeps the contract line short)."""
    if x is None or isinstance(x, (bool, int, str)):
        return x
    return float(f"{x:.{nd}g}")


def _short_roof(r):
    if not r:
        return None
    keep = ("kernel", "bound", "achieved", "peak", "unit", "frac", "traffic", "avg_launch_ms")
    out = {k: _r(r.get(k)) for k in keep if k in r}
    if "algorithmic_bytes_per_launch" in r:
        out["bytes"] = _r(r["algorithmic_bytes_per_launch"])
    if "flop_per_point_pair" in r:
        out["flop_per_point_pair"] = r["flop_per_point_pair"]
    return out


CONTRACT_KEYS = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                 "scaling", "vs_baseline", "dtype", "data", "config", "latency_ms", "accuracy", "fp64",
                 "speedup_vs_fp64", "roofline", "roofline_second", "cpu_baseline", "e2e", "clocks",
                 "gpu_launches")
CONTRACT_MAX_BYTES = 1536


def contract_line(*, value, steps, warmup, world, times, clocks, launches, err=None, fp64=None, roof=None,
                  roof2=None, cpu=None, e2e=None):
    """The bench's last output line: the headline metric and its evidence, compact
    (numbers to 4 significant digits, short strings) so that it stays under
    CONTRACT_MAX_BYTES; the full sections are printed on earlier lines."""
    line = {
        "metric": METRIC, "value": _r(value), "unit": UNIT, "n_gpus": world, "steps": steps, "warmup": warmup,
        "ms_per_step": _r(sum(times) / len(times)), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_SHORT, "parallelism": "replicas" if world > 1 else "single",
                   "precision": "mixed: FP32 assembly/matvec (c64); FP64 or double-float singular/mass/mortar/refinement",
                   "l2": "inputs > L2 + 256 MB flush"},
        "latency_ms": {"p50": _r(float(np.percentile(times, 50))), "p99": _r(float(np.percentile(times, 99)))},
        "accuracy": (None if err is None else {"max": _r(max(err.values()), 3), "target": 1e-6,
                                               "ok": max(err.values()) <= 1e-6}),
        "fp64": (None if fp64 is None else {"value": _r(fp64["value"]),
                                            "ms_per_step": _r(sum(fp64["times"]) / len(fp64["times"]))}),
        "speedup_vs_fp64": _r(value / fp64["value"]) if fp64 else None,
        "roofline": _short_roof(roof),
        "roofline_second": _short_roof(roof2),
        "cpu_baseline": (None if cpu is None else {"value": _r(cpu["value"]), "unit": UNIT, "cores": cpu["cores"],
                                                   "kind": "oracle", "sample": cpu["sample_short"]}),
        "e2e": (None if e2e is None else {"value": _r(e2e["value"]), "unit": UNIT,
                                          "h2d_bytes_per_step": e2e["h2d_bytes_per_step"],
                                          "d2h_bytes_per_step": e2e["d2h_bytes_per_step"]}),
        "clocks": {"sm_mhz": clocks.get("sm_mhz"), "sm_max_mhz": clocks.get("sm_max_mhz"),
                   "reasons": clocks.get("reasons", [])},
        "gpu_launches": int(launches),
    }
    return line


def emit_section(name, obj):
    """One earlier output line per bench section."""
    print(json.dumps({"section": name, **(obj if isinstance(obj, dict) else {"data": obj})}), flush=True)


def emit_contract(line):
    s = json.dumps(line, separators=(",", ":"))
    if len(s) > CONTRACT_MAX_BYTES:  # never expected: drop the secondary evidence first
        for k in ("roofline_second", "fp64"):
            line[k] = None
            s = json.dumps(line, separators=(",", ":"))
            if len(s) <= CONTRACT_MAX_BYTES:
                break
    print(s, flush=True)


WORKLOAD_SHORT = ("icosphere L5 ext (10242 v) + L5 int rotated+jittered (seed 2), k_ext 10, k_int 15, "
                  "rho 2, 1 plane wave +z, GMRES tol 1e-8, 40968 unknowns")


def run_case(args):
    """Small standalone cases of the library's kernels for ncu captures (no timing, no
    JSON): one assembly, one mortar, one transmission solve or one screen solve on the
    synthetic icosphere grids."""
    import bem_inputs as bi
    import paper_2206_00708_gb300 as bem

    ctx = bem.bem_context_create(0)
    li = args.level if args.level_int is None else args.level_int
    ve, te, vi, ti = bi.transmission_pair(args.level, li, seed=2)
    ge = bem.bem_grid_create(ctx, ve, te)
    gi = bem.bem_grid_create(ctx, vi, ti)
    prec = bem.BEM_PREC_MIXED if args.mixed else bem.BEM_PREC_FP64
    for _ in range(args.repeat):
        if args.case == "assemble":
            m = bem.bem_assemble(ctx, bem.BEM_OP_V, args.k, ge, precision=prec)
            bem.bem_context_synchronize(ctx)
            bem.bem_matrix_destroy(m)
        elif args.case == "mortar":
            s = bem.bem_projection(ctx, gi, ge)
            bem.bem_sparse_destroy(s)
        elif args.case == "screen":
            vs, ts = bi.screen_grid(args.screen_cells, args.screen_cells, jitter=0.2, seed=71)
            c = max(2, args.screen_cells // 3)
            vc, tc = bi.screen_grid(c, c, jitter=0.2, seed=72)
            gs, gc = bem.bem_grid_create(ctx, vs, ts), bem.bem_grid_create(ctx, vc, tc)
            _, rep = bem.bem_solve_screen(ctx, gs, args.k, np.array([[1.0, 0.0, 0.0]]), coarse=gc,
                                          precond=bem.BEM_SCREEN_OO, opts={"precision": prec})
            bem.bem_grid_destroy(gs)
            bem.bem_grid_destroy(gc)
            print("iterations", rep["iterations"])
        else:
            dirs = np.array([[0.0, 0.0, 1.0]]) if args.rhs == 1 else bi.plane_wave_directions(args.rhs, seed=40)
            opts = {"precision": prec, "formulation": args.formulation}
            if args.dd_switch is not None:
                opts["dd_switch"] = args.dd_switch
            if args.tensor_cores is not None:
                opts["tensor_cores"] = args.tensor_cores
            _, rep = bem.bem_solve_transmission(ctx, ge, gi, 1.5 * args.k, args.k, 2.0, dirs, opts=opts)
            print("iterations", rep["iterations"])
    bem.bem_grid_destroy(ge)
    bem.bem_grid_destroy(gi)
    bem.bem_context_destroy(ctx)
    print("ok")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain-FP64 comparison arm")
    ap.add_argument("--no-accuracy", dest="accuracy", action="store_false",
                    help="skip the converged FP64 reference solve (profiling runs)")
    ap.add_argument("--no-field", dest="field", action="store_false", help="skip the field-evaluation section")
    ap.add_argument("--no-cube", dest="cube", action="store_false", help="skip the unit-cube benchmarks")
    ap.add_argument("--no-screen", dest="screen", action="store_false", help="skip the screen benchmark")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="keep the built-in launch shapes (no bem_autotune before the measured steps)")
    ap.add_argument("--no-graphs", dest="graphs", action="store_false",
                    help="skip the CUDA-graph on/off comparison")
    ap.add_argument("--no-formulations", dest="single_trace", action="store_false",
                    help="skip the section timing the other formulations (single-trace, high-contrast)")
    ap.add_argument("--no-batching", dest="batching", action="store_false",
                    help="skip the many-directions section")
    ap.add_argument("--serve-requests", type=int, default=96,
                    help="requests of the seeded serving stream to replay (0: skip serving)")
    ap.add_argument("--case", choices=["assemble", "solve", "mortar", "screen"], default=None,
                    help="run one small profiling case instead of the benchmark (for ncu)")
    ap.add_argument("--level", type=int, default=4, help="--case: exterior icosphere level")
    ap.add_argument("--level-int", type=int, default=None, help="--case: interior level (default: --level)")
    ap.add_argument("--k", type=float, default=10.0, help="--case: exterior wavenumber (interior 1.5 k)")
    ap.add_argument("--repeat", type=int, default=1, help="--case: repetitions")
    ap.add_argument("--mixed", action="store_true", help="--case: mixed precision instead of FP64")
    ap.add_argument("--rhs", type=int, default=1, help="--case solve: plane waves (batched)")
    ap.add_argument("--formulation", type=int, default=0, help="--case solve: BEM_FORM_* formulation")
    ap.add_argument("--tensor-cores", dest="tensor_cores", type=int, default=None,
                    help="--case solve: bem_solve_opts.tensor_cores (0 CUDA cores, 1 TF32 split, 2 FP16 split)")
    ap.add_argument("--dd-switch", dest="dd_switch", type=float, default=None,
                    help="--case solve: bem_solve_opts.dd_switch (0: double-float inner products throughout, "
                         "1: FP32 throughout)")
    ap.add_argument("--screen-cells", dest="screen_cells", type=int, default=60,
                    help="--case screen: cells per side of the fine grid")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank)
    if args.case:
        return run_case(args)

    import torch
    import torch.distributed as dist
    import paper_2206_00708_gb300 as bem

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    w = WORKLOAD
    ve, te, vi, ti = workload_inputs()
    dev = torch.device("cuda", local)
    xe = torch.from_numpy(np.ascontiguousarray(ve)).to(dev)
    tre = torch.from_numpy(np.ascontiguousarray(te, dtype=np.int32)).to(dev)
    xi = torch.from_numpy(np.ascontiguousarray(vi)).to(dev)
    tri_ = torch.from_numpy(np.ascontiguousarray(ti, dtype=np.int32)).to(dev)
    Ne, Ni = len(ve), len(vi)
    dirs = np.array([[0.0, 0.0, 1.0]])
    stream = torch.cuda.current_stream(dev)
    ctx = bem.bem_context_create(local, stream=stream)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def new_out():
        return {k: torch.zeros((1, n), dtype=torch.complex128, device=dev)
                for k, n in (("v_ext", Ne), ("w_ext", Ne), ("v_int", Ni), ("w_int", Ni))}

    def step(precision, out, tol, formulation=0):
        ge = bem.bem_grid_create(ctx, xe, tre)
        gi = bem.bem_grid_create(ctx, xi, tri_)
        _, rep = bem.bem_solve_transmission(ctx, ge, gi, w["k_int"], w["k_ext"], w["rho"], dirs,
                                            opts={"gmres_tol": tol, "precision": precision,
                                                  "formulation": formulation}, out=out, on_device=True)
        bem.bem_grid_destroy(ge)
        bem.bem_grid_destroy(gi)
        return rep

    def timed(precision, roof_steps):
        """Warm-up, then the timed steps (CUDA events around each solve on the launching
        stream, no profiler events inside), then untimed profiled steps: one with every
        launch bracketed (the kernel table) and `roof_steps` with only the four longest
        kernels bracketed (their average launch durations for the rooflines; the four
        longest, the first two in the contract line)."""
        out = new_out()
        for _ in range(args.warmup):
            step(precision, out, w["tol"])
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        times, reports = [], []
        l0 = bem.bem_launch_count()
        with ClockSampler(local) as clocks:
            for _ in range(args.steps):
                flush.zero_()  # L2 flush outside the timed events
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                reports.append(step(precision, out, w["tol"]))
                e1.record(stream)
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
        torch.cuda.synchronize()
        launches = bem.bem_launch_count() - l0
        barrier()
        total = sum(times)
        if world > 1:
            tt = torch.tensor([total], dtype=torch.float64, device=dev)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            total = float(tt.item())
        # profiled steps (not part of the timed region): the kernel table, then the four
        # longest kernels bracketed by events
        bem.bem_profile_select(None)
        bem.bem_profile_reset()
        bem.bem_profile_enable(True)
        flush.zero_()
        step(precision, out, w["tol"])
        torch.cuda.synchronize()
        bem.bem_profile_enable(False)
        table = bem.bem_profile_table()
        top = [p[0] for p in table[:4]]
        bem.bem_profile_reset()
        bem.bem_profile_select(top)
        for _ in range(roof_steps):
            flush.zero_()
            bem.bem_profile_enable(True)
            step(precision, out, w["tol"])
            torch.cuda.synchronize()
            bem.bem_profile_enable(False)
        prof = bem.bem_profile_table()
        bem.bem_profile_select(None)
        return dict(out=out, times=times, reports=reports, launches=launches, clocks=clocks.summary(),
                    value=world * args.steps / (total / 1e3), prof=prof, table=table)

    # launch shapes for this workload's sizes, timed once before any measured step
    if args.autotune:
        ge, gi = bem.bem_grid_create(ctx, xe, tre), bem.bem_grid_create(ctx, xi, tri_)
        t0 = time.perf_counter()
        bem.bem_autotune(ctx, ge, gi, 1)
        n_unk = 2 * (Ne + Ni)
        tuning = {"seconds": time.perf_counter() - t0,
                  "chosen": {f"{k}/{w_}": dict(zip(("block", "variant", "ms"), bem.bem_tune_get(k, w_, n_unk)))
                             for k, w_ in (("cheb", 1), ("cheb", 8))}}
        bem.bem_grid_destroy(ge)
        bem.bem_grid_destroy(gi)
        if rank == 0:
            emit_section("autotune", tuning)

    mixed = timed(bem.BEM_PREC_MIXED, args.steps)
    fp64 = None if args.no_fp64 else timed(bem.BEM_PREC_FP64, min(args.steps, 2))

    # accuracy: the mixed traces against a tightly converged FP64 solve of the same system
    err, err64 = None, None
    if args.accuracy:
        ref = new_out()
        step(bem.BEM_PREC_FP64, ref, 1e-12)
        torch.cuda.synchronize()
        err = {k: float(torch.linalg.norm(mixed["out"][k] - ref[k]) / torch.linalg.norm(ref[k])) for k in ref}
        err64 = ({k: float(torch.linalg.norm(fp64["out"][k] - ref[k]) / torch.linalg.norm(ref[k])) for k in ref}
                 if fp64 else None)

    pp_cache = {}
    roofs = [kernel_roofline(*p, te, ti, Ne, Ni, pp_cache) for p in mixed["prof"]]
    roof = roofs[0] if roofs else None
    roof2 = roofs[1] if len(roofs) > 1 else None
    roof64 = [kernel_roofline(*p, te, ti, Ne, Ni, pp_cache) for p in fp64["prof"]] if fp64 else None

    def solve_info(rep):
        return {k: rep[k] for k in ("iterations", "outer_iterations", "residual", "t_assembly_ms", "t_mortar_ms",
                                    "t_solve_ms")}

    def lat(times):
        return {"p50": float(np.percentile(times, 50)), "p99": float(np.percentile(times, 99))}

    if rank == 0:
        emit_section("mixed", {"workload": WORKLOAD_NAME, "value": mixed["value"], "unit": UNIT,
                               "times_ms": mixed["times"], "solve": solve_info(mixed["reports"][-1]),
                               "gpu_launches": mixed["launches"], "clocks": mixed["clocks"],
                               "accuracy": {"rel_l2_vs_fp64_converged": err, "target": 1e-6,
                                            "reference": "FP64 GPU solve of the same system at GMRES tol 1e-12 "
                                                         "(the FP64 path matches the CPU oracle to 1e-10)"},
                               "rooflines": roofs,
                               "kernels": [{"name": p[0], "ms": p[1], "launches": p[2]} for p in mixed["table"][:12]]})
        if fp64:
            emit_section("fp64", {"value": fp64["value"], "unit": UNIT, "times_ms": fp64["times"],
                                  "latency_ms": lat(fp64["times"]), "rel_l2_vs_fp64_converged": err64,
                                  "solve": solve_info(fp64["reports"][-1]), "rooflines": roof64,
                                  "gpu_launches": fp64["launches"], "clocks": fp64["clocks"],
                                  "kernels": [{"name": p[0], "ms": p[1], "launches": p[2]}
                                              for p in fp64["table"][:10]]})

    e2e = None
    if not args.no_e2e:
        # end to end through the public API with pinned host buffers (mixed precision)
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        hxe, hte, hxi, hti = pin(ve), pin(np.asarray(te, dtype=np.int32)), pin(vi), pin(np.asarray(ti, dtype=np.int32))
        hout = {k: torch.zeros((1, n), dtype=torch.complex128).pin_memory()
                for k, n in (("v_ext", Ne), ("w_ext", Ne), ("v_int", Ni), ("w_int", Ni))}
        e2e_times = []
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ge = bem.bem_grid_create(ctx, hxe, hte)
            gi = bem.bem_grid_create(ctx, hxi, hti)
            bem.bem_solve_transmission(ctx, ge, gi, w["k_int"], w["k_ext"], w["rho"], dirs,
                                       opts={"gmres_tol": w["tol"], "precision": bem.BEM_PREC_MIXED}, out=hout)
            bem.bem_grid_destroy(ge)
            bem.bem_grid_destroy(gi)
            e2e_times.append(time.perf_counter() - t0)
        h2d = sum(int(a.numel() * a.element_size()) for a in (hxe, hte, hxi, hti))
        d2h = sum(int(a.numel() * a.element_size()) for a in hout.values())
        e2e = {"value": world * args.steps / sum(e2e_times), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}
        if rank == 0:
            emit_section("e2e", dict(e2e, times_s=e2e_times,
                                     note="bem_grid_create + bem_solve_transmission from pinned host buffers, "
                                          "traces copied back to pinned host buffers, wall clock"))

    if args.serve_requests > 0:
        reqs = serving_stream(args.serve_requests)
        sat = {p: run_serving(bem, reqs, p) for p in (bem.BEM_PREC_FP64, bem.BEM_PREC_MIXED)}
        sat_alone = run_serving(bem, reqs, bem.BEM_PREC_MIXED, group_max=1)
        rate = 0.7 * sat[bem.BEM_PREC_FP64]["solves_per_s"]
        rep = {p: run_serving(bem, reqs, p, rate=rate) for p in (bem.BEM_PREC_FP64, bem.BEM_PREC_MIXED)}
        if rank == 0:
            emit_section("serving", {
                "workload": f"first {len(reqs)} of the {SERVE_STREAM_LENGTH} requests of the seeded serving "
                            "stream (seed 50): ellipsoids with semi-axes U[0.5,1.5], icosphere levels 2-4 per "
                            "grid, k_ext U[1,8], k_int/k_ext U[1.2,2], rho log-U[0.1,10], 1-16 plane waves; "
                            "4 requests in flight; small mixed-precision requests in lockstep groups of up to 8",
                "fraction_of_stream": len(reqs) / SERVE_STREAM_LENGTH,
                "saturated": {"fp64": sat[bem.BEM_PREC_FP64], "mixed": sat[bem.BEM_PREC_MIXED],
                              "mixed_every_request_alone": sat_alone},
                "poisson": {"rate_per_s": rate, "fp64": rep[bem.BEM_PREC_FP64], "mixed": rep[bem.BEM_PREC_MIXED]}})

    if args.field and rank == 0:
        emit_section("field", run_field(bem, ctx, w, ve, te, vi, ti, mixed["out"]))

    if args.single_trace and rank == 0:
        # the other formulations on the same workload: mixed-precision solves timed like the
        # headline, accuracy against each one's own converged FP64 solve, and the distance
        # of their exterior traces from the multiple-traces ones (discretisation)
        rn = lambda a, b: float(torch.linalg.norm(a - b) / torch.linalg.norm(b))
        single = {"note": "Sec. 2.2 single-trace and Sec. 2.3 high-contrast systems on the nonconforming pair, "
                          "discretised as eq. pmchwt:discrete: 2 unknowns per vertex of one grid; every product "
                          "applies that grid's operators and P M^-1 A M^-1 P of the other grid's (never formed)"}
        for name, form in (("pmchwt_ext", bem.BEM_FORM_PMCHWT), ("muller_ext", bem.BEM_FORM_MULLER),
                           ("pmchwt_int", bem.BEM_FORM_PMCHWT_INT), ("muller_int", bem.BEM_FORM_MULLER_INT),
                           ("hc_ext_neu", bem.BEM_FORM_HC_EXT_NEU), ("hc_ext_dir", bem.BEM_FORM_HC_EXT_DIR),
                           ("hc_int_neu", bem.BEM_FORM_HC_INT_NEU), ("hc_int_dir", bem.BEM_FORM_HC_INT_DIR)):
            pout = new_out()
            step(bem.BEM_PREC_MIXED, pout, w["tol"], form)
            ptimes, preps = [], []
            for _ in range(args.steps):
                flush.zero_()
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                preps.append(step(bem.BEM_PREC_MIXED, pout, w["tol"], form))
                e1.record(stream)
                e1.synchronize()
                ptimes.append(e0.elapsed_time(e1))
            entry = {"value": args.steps / (sum(ptimes) / 1e3), "unit": UNIT,
                     "ms_per_step": sum(ptimes) / args.steps, "precision": "mixed",
                     "solve": {k: preps[-1][k] for k in ("iterations", "outer_iterations", "residual",
                                                         "t_assembly_ms", "t_solve_ms")},
                     "exterior_traces_vs_mtf": {k: rn(pout[k], mixed["out"][k]) for k in ("v_ext", "w_ext")}}
            if args.accuracy:
                pref = new_out()
                step(bem.BEM_PREC_FP64, pref, 1e-12, form)
                torch.cuda.synchronize()
                perr = {k: rn(pout[k], pref[k]) for k in pref}
                entry["rel_l2_vs_fp64_converged"] = perr
                entry["max_err"] = max(perr.values())
            single[name] = entry
        emit_section("formulations", single)

    if args.screen and rank == 0:
        emit_section("screen", run_screen(bem, ctx))

    if args.graphs and rank == 0:
        emit_section("cuda_graphs", run_graphs(bem, ctx))

    if args.cube and rank == 0:
        emit_section("cube", run_cube(bem, ctx))

    if args.batching and rank == 0:
        bw = BATCH_WORKLOAD
        emit_section("batching", {
            "workload": f"unit sphere, icosphere L{bw['level']} on both grids (seed {bw['seed']}), "
                        f"k_ext={bw['k_ext']}, k_int={bw['k_int']}, rho={bw['rho']}, {bw['n_dirs']} plane "
                        f"waves in one call vs {bw['n_single']} of them one call each; mixed precision "
                        "with tensor-core products (one batch of 64; FP16 two-term split fed by TMA "
                        "bulk copies, the default; TF32 three-term split; BF16 two-term split) and with "
                        "CUDA-core products (batches of 8), FP64 (batches of 8)",
            "mixed_tensor_cores_fp16_split": run_batching(bem, ctx, bem.BEM_PREC_MIXED, 2, 0),
            "mixed_tensor_cores_tf32_split": run_batching(bem, ctx, bem.BEM_PREC_MIXED, 1, 0),
            "mixed_tensor_cores_bf16_split": run_batching(bem, ctx, bem.BEM_PREC_MIXED, 3, 0),
            "mixed_cuda_cores_8": run_batching(bem, ctx, bem.BEM_PREC_MIXED, 0, 8),
            "fp64": run_batching(bem, ctx, bem.BEM_PREC_FP64)})
        emit_section("batching_full", run_batching_full(bem, ctx))
        emit_section("uneven_instances", run_uneven(bem, ctx))

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = host_cores()
        r = run_oracle_child(1, cores)
        if r is not None:
            cpu = {"value": r["steps"][-1]["value"], "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": r["sample"],
                   "sample_short": (f"extrapolated from ~{r['steps'][-1]['test_triangles']} test triangles + "
                                    f"a {ORACLE_MATVEC_ROWS}-row matvec block x {ORACLE_GMRES_ITERS} iterations")}
            emit_section("cpu_baseline", cpu)

    if rank == 0:
        emit_contract(contract_line(value=mixed["value"], steps=args.steps, warmup=args.warmup, world=world,
                                    times=mixed["times"], clocks=mixed["clocks"], launches=mixed["launches"],
                                    err=err, fp64=fp64, roof=roof, roof2=roof2, cpu=cpu, e2e=e2e))
    bem.bem_context_destroy(ctx)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
