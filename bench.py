"""Benchmark: cells integrated to t_end per second at stated error, and NVECTOR
operation HBM bandwidth, on one B300 (or N GPUs, one process each).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step integrates the 100 000-cell mass-action workload (sizes drawn from
{3, 10, 32, 54}, 2 n reactions per cell, t in [0, 1e-3], rtol 1e-6, atol
1e-10) from its initial state to t_end through the library's public C ABI
(bdfb_init + bdfb_integrate), inputs resident in device memory.  Prints one
JSON line.  ``--impl reference`` times the CPU oracle on the host cores on a
bounded sample of the same workload (the reference arm).
"""
from __future__ import annotations

import argparse
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

NCELL = 100_000
TOUT = 1.0e-3
RTOL, ATOL = 1.0e-6, 1.0e-10
SIZES = (3, 10, 32, 54)
# DRAM bytes read + written by one timed step's k_cells launches (the four
# size classes of the 100 000-cell workload), from one single-pass ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum) of `bench.py --quick --steps 2
# --warmup 1` on the kernels of this source tree: a recorded figure, not
# measured by the run that prints it
K_CELLS_STEP_DRAM_BYTES = 462_835_968
# the FP64 pipe's activity on the 54-species launch (8192 cells), recorded from
# an ncu capture of that launch (sm__inst_executed_pipe_fp64, percent of peak
# while active)
K54_FP64_PIPE_PCT = 82.2
METRIC = "cells integrated to t_end per second at stated error; NVECTOR op HBM GB/s"
UNIT = "cells/s"
WORKLOAD = ("mass-action 100k: 100000 independent cells, n ~ U{3,10,32,54}, 2n reactions "
            "(2-4 distinct reactants/products), k log-U[1e-2,1e8], Dirichlet y0, t in [0,1e-3], "
            "rtol 1e-6, atol 1e-10, FP64")
FP64_NOMINAL_TFLOPS = 1.25  # nominal B300 FP64 rate: context only; the roofline divides by the measured DGEMM
L2_FLUSH_BYTES = 256 << 20


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0}, "fallback"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def rhs_flops(prob):
    """FP64 flops of one right-hand side per cell: per reaction m multiplies
    for the rate and 2 m additions into f."""
    m = (prob.reactants != 255).sum(axis=1) * 3
    return np.add.reduceat(m, prob.rxn_off[:-1])


def algorithmic_flops(prob, cs):
    """FP64 flops the method needs for the counters in cs (per-cell stats):
    per setup 2n^3/3 (LU) + 2 n^2 (M = I - gamma J) + Jacobian entries,
    per Newton iteration 2 n^2 (triangular solves) + 10 n (residual, norm,
    update), per RHS its reaction flops, per step (q+1)(q+2) n (predict and
    correct)."""
    n = prob.n.astype(np.float64)
    nsetup, nni, nfe, nst = cs[:, 2], cs[:, 3], cs[:, 1], cs[:, 0]
    q = np.clip(cs[:, 6], 1, 5).astype(np.float64)
    jac = 2.0 * rhs_flops(prob)              # m(m-1) products + 2m^2 scatter ~ 2x the RHS
    per = (nsetup * (2.0 * n ** 3 / 3.0 + 2.0 * n ** 2 + jac) + nni * (2.0 * n ** 2 + 10.0 * n)
           + nfe * rhs_flops(prob) + nst * (q + 1) * (q + 2) * n)
    return float(per.sum())


def cpu_oracle_rate(prob, seconds=10.0, threads=None):
    """oracle cells/s on a bounded sample of the workload (first cells: the
    size mix is uniform over the index)"""
    import oracle
    threads = threads or oracle.host_threads()
    n0 = min(prob.ncell, 1024)
    t = time.perf_counter()
    oracle.integrate_cells(prob.subset(np.arange(n0)), 0.0, TOUT, RTOL, ATOL, threads=threads)
    dt = time.perf_counter() - t
    ns = int(min(prob.ncell, max(n0, n0 * seconds / max(dt, 1e-3))))
    sub = prob.subset(np.arange(ns))
    t = time.perf_counter()
    _, st, _ = oracle.integrate_cells(sub, 0.0, TOUT, RTOL, ATOL, threads=threads)
    dt = time.perf_counter() - t
    return ns / dt, threads, ns, dt, int((st != 0).sum())


def oracle_rate(prob, sample):
    """the oracle (all host cores, cells spread over threads) on a subset of a
    workload at the run's tolerances: cells per second; cells are independent,
    so the rate carries over to the whole workload"""
    import oracle
    threads = oracle.host_threads()
    t = time.perf_counter()
    _, st, _ = oracle.integrate_cells(prob, 0.0, TOUT, RTOL, ATOL, threads=threads)
    dt = time.perf_counter() - t
    return {"cells_per_s": prob.ncell / dt, "seconds": dt, "cores": threads, "failed": int((st != 0).sum()),
            "sample": sample}


def accuracy(prob, y, ncheck=1024, seed=1):
    """weighted final-state error vs the oracle at rtol 1e-10 on a seeded sample"""
    import oracle
    cells = np.sort(np.random.default_rng(seed).choice(prob.ncell, min(ncheck, prob.ncell), replace=False))
    sub = prob.subset(cells)
    yt, _, _ = oracle.integrate_cells(sub, 0.0, TOUT, 1e-10, 1e-14, threads=oracle.host_threads())
    ys = np.concatenate([y[prob.y_off[c]:prob.y_off[c + 1]] for c in cells])
    w = np.abs(ys - yt) / (RTOL * np.abs(yt) + ATOL)
    e = np.maximum.reduceat(w, sub.y_off[:-1])
    return {"cells_checked": int(len(cells)), "truth": "oracle rtol 1e-10 atol 1e-14",
            "err_median": float(np.median(e)), "err_p99": float(np.percentile(e, 99)),
            "err_max": float(e.max()), "frac_within_10": float((e <= 10).mean())}


def nvector_bandwidth(torch, bdfb, n=1 << 25, reps=20):
    """achieved GB/s (algorithmic bytes / event time, mean over calls)"""
    dev = "cuda"
    g = torch.Generator(device=dev).manual_seed(3)
    v = [torch.rand(n, dtype=torch.float64, device=dev, generator=g) * 2 - 1 for _ in range(7)]
    out = torch.zeros(8, dtype=torch.float64, device=dev)
    work = bdfb.nv_work(n, 8)
    s = torch.cuda.current_stream()
    ops = {
        "linear_sum": (lambda: bdfb.nv_linear_sum(0.5, v[0], 0.25, v[1], v[2]), 24),
        "linear_sum_difference": (lambda: bdfb.nv_linear_sum(0.5, v[0], -1.0, v[1], v[2]), 24),
        "linear_combination_6": (lambda: bdfb.nv_linear_combination([0.1] * 6, v[:6], v[6]), 8 * 7),
        "scale_add_multi_3": (lambda: bdfb.nv_scale_add_multi([0.1] * 3, v[0], v[1:4], v[4:7]), 8 * 7),
        "dot_prod_multi_5": (lambda: bdfb.nv_dot_prod_multi(v[0], v[1:6], out, work), 8 * 6),
        "wrms_norm": (lambda: bdfb.nv_wrms_norm(v[0], v[1], out, work), 16),
    }
    res = {}
    for name, (fn, bpe) in ops.items():
        for _ in range(3):
            fn()
        times = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            fn()
            e1.record(s)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) * 1e-3)
        res[name] = round(bpe * n / statistics.mean(times) / 1e9, 1)
    res["n"] = n
    return res


# FP64 instructions per byte moved, per element of the benchmarked forms
# (DFMA/DMUL/DADD all issue on the FP64 pipe, 2 lanes per SM per cycle)
NV_FP64_INST_PER_BYTE = {"linear_sum": 2 / 24, "linear_sum_difference": 1 / 24, "linear_combination_6": 6 / 56,
                         "scale_add_multi_3": 3 / 56, "dot_prod_multi_5": 5 / 48, "wrms_norm": 2 / 16}


def dgemm_tflops(torch, n=8192, reps=3):
    """FP64 throughput a library GEMM reaches on this part (cuBLAS DGEMM,
    n x n x n): the measured counterpart of the nominal FP64 rate, for context
    beside the per-cell kernels' FP64 roofline"""
    a = torch.rand(n, n, dtype=torch.float64, device="cuda")
    b = torch.rand(n, n, dtype=torch.float64, device="cuda")
    c = torch.empty_like(a)
    torch.matmul(a, b, out=c)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        torch.matmul(a, b, out=c)
    e1.record()
    e1.synchronize()
    t = e0.elapsed_time(e1) * 1e-3 / reps
    del a, b, c
    return 2.0 * n ** 3 / t / 1e12


def nvector_ceilings(nv, hbm_gbs, sm_mhz):
    """per op: the lower of the HBM copy rate and the FP64 issue limit
    (148 SMs x 2 FP64 lanes per cycle / FP64 instructions per byte); on B300
    FP64 runs at 1:64 of FP32, so the reductions are co-limited by it"""
    mhz = sm_mhz or 2032.0
    inst_rate = 148 * 2 * mhz * 1e6
    out = {}
    for k, ipb in NV_FP64_INST_PER_BYTE.items():
        cap = min(hbm_gbs, inst_rate / ipb / 1e9)
        out[k] = {"achieved_gbs": nv[k], "fp64_limit_gbs": round(inst_rate / ipb / 1e9, 1),
                  "ceiling_gbs": round(cap, 1), "frac_of_ceiling": round(nv[k] / cap, 3),
                  "frac_of_hbm": round(nv[k] / hbm_gbs, 3)}
    return out


# the grid integrator's streaming vector operations (the NVECTOR kernels of the
# GMRES and error-norm path, and the fused history and Newton-update passes)
NVECTOR_KINDS = ("wrms_norm", "dot_prod_multi", "linear_combination", "linear_sum")
STREAM_KINDS = NVECTOR_KINDS + ("predict", "accept", "rescale", "error_weights", "newton_update", "unscale")


def op_bandwidth(prof, hbm_gbs):
    """per kind of the integrator's op profile: launches, GB/s (algorithmic
    bytes / summed event time), fraction of the measured HBM copy rate"""
    out = {}
    for k, (n, ms, gb) in prof.items():
        if n:
            out[k] = {"launches": n, "ms": round(ms, 3), "gb": round(gb, 3), "gbs": round(gb / (ms * 1e-3), 1),
                      "frac_of_hbm": round(gb / (ms * 1e-3) / hbm_gbs, 3)}
    for name, kinds in (("nvector_ops", NVECTOR_KINDS), ("all_streaming_ops", STREAM_KINDS)):
        gb = sum(prof[k][2] for k in kinds)
        ms = sum(prof[k][1] for k in kinds)
        if ms > 0:
            out[name] = {"gb": round(gb, 3), "ms": round(ms, 3), "gbs": round(gb / (ms * 1e-3), 1),
                         "frac_of_hbm": round(gb / (ms * 1e-3) / hbm_gbs, 3)}
    return out


def grid_workload(torch, bdfb, gen, nx=256, tout=1.0, reps=2, hbm_gbs=None):
    """The coupled-system workload: Brusselator reaction-diffusion on a
    periodic nx^3 grid (3 nx^3 unknowns), one shared step, Newton + GMRES
    (Krylov dimension 5) with the 3x3 reaction blocks as preconditioner;
    FP64 throughout, then with the preconditioner and the GMRES operator in
    FP32 (option precision 1), compared with the FP64 result.  A further run
    of each with option "profile" times every vector operation with events:
    achieved GB/s = algorithmic bytes / event time, per operation kind."""
    p = gen.brusselator3d(nx)
    y0 = torch.from_numpy(p.y0).cuda()
    y = torch.empty_like(y0)
    out, yref = {}, None
    for prec in (0, 1):
        ts = []
        with bdfb.Integrator(p, rtol=RTOL, atol=ATOL, maxl=5, precision=prec) as gi:
            for _ in range(reps + 1):
                gi.init(0.0, y0)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                r = gi.integrate(tout, y)
                torch.cuda.synchronize()
                ts.append(time.perf_counter() - t0)
                if r != 0:
                    raise RuntimeError(f"grid integrate returned {r}")
            gs = gi.cell_stats()[0]
            prof = None
            if hbm_gbs:
                gi.set_option("profile", 1)
                gi.init(0.0, y0)
                if gi.integrate(tout, y) != 0:
                    raise RuntimeError("profiled grid integrate failed")
                prof = op_bandwidth(gi.op_profile(), hbm_gbs)
        t = min(ts[1:])
        res = {"grid_points_per_s": nx ** 3 / t, "seconds": t, "steps": int(gs[0]),
               "ms_per_step": 1e3 * t / max(1, gs[0]), "newton_iters": int(gs[3]), "gmres_iters": int(gs[6]),
               "jacobian_setups": int(gs[2])}
        if prof:
            res["vector_ops"] = prof
        if prec == 0:
            yref = y.clone()
            out.update(res)
        else:
            d = ((y - yref).abs() / (RTOL * yref.abs() + ATOL)).max().item()
            out["fp32_preconditioner_and_operator"] = {**res, "max_weighted_diff_vs_fp64": d}
    out["workload"] = (f"Brusselator 3-D {nx}^3 x 3 = {3 * nx ** 3} unknowns, A=1, B=3, eps=5e-6, D=1e-2, "
                       f"t in [0,{tout}], rtol 1e-6, atol 1e-10, GMRES(5) + 3x3 block Jacobi")
    return out


class GridOracleLeg:
    """The oracle on a smaller grid of the same workload (nx^3, same t range,
    one host thread: one coupled system), run in a background thread while the
    GPU legs run: its rate in grid points per second and an rtol 1e-10 truth
    against which the GPU's final state at that size is measured."""

    def __init__(self, gen, nx=64, tout=1.0):
        import oracle
        self.nx, self.tout = nx, tout
        self.p = gen.brusselator3d(nx)
        self.res = {}

        def run():
            t0 = time.perf_counter()
            r, yo, so = oracle.bruss_integrate(self.p, 0.0, tout, RTOL, ATOL, maxl=5)
            dt = time.perf_counter() - t0
            rt, yt, _ = oracle.bruss_integrate(self.p, 0.0, tout, 1e-10, 1e-14, maxl=5)
            self.res = {"ret": int(r), "truth_ret": int(rt), "seconds": dt, "yo": yo, "so": so, "yt": yt}

        self.th = threading.Thread(target=run, daemon=True)
        self.th.start()

    def finish(self, torch, bdfb):
        """join; the GPU at the same size and tolerances in both precisions:
        counters against the oracle's, error against the truth"""
        self.th.join()
        R = self.res
        p, nx = self.p, self.nx
        w = RTOL * np.abs(R["yt"]) + ATOL
        eo = np.abs(R["yo"] - R["yt"]) / w
        out = {"oracle": {"points_per_s": nx ** 3 / R["seconds"], "seconds": R["seconds"], "cores": 1,
                          "steps": int(R["so"][0]), "ret": R["ret"],
                          "sample": f"{nx}^3 grid (same problem, same t range)",
                          "error_vs_truth": {"max": float(eo.max()), "rms": float(np.sqrt(np.mean(eo * eo)))}},
               "truth": f"oracle rtol 1e-10 atol 1e-14 at {nx}^3"}
        y0 = torch.from_numpy(p.y0).cuda()
        y = torch.empty_like(y0)
        for prec in (0, 1):
            with bdfb.Integrator(p, rtol=RTOL, atol=ATOL, maxl=5, precision=prec) as gi:
                gi.init(0.0, y0)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                r = gi.integrate(self.tout, y)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                gs = gi.cell_stats()[0]
            yg = y.cpu().numpy()
            eg = np.abs(yg - R["yt"]) / w
            out["fp64" if prec == 0 else "fp32_preconditioner_and_operator"] = {
                "ret": int(r), "points_per_s": nx ** 3 / dt, "steps": int(gs[0]),
                "counters_equal_oracle": bool(np.array_equal(gs[:8], R["so"][:8])),
                "max_weighted_diff_vs_oracle": float(np.max(np.abs(yg - R["yo"]) / (RTOL * np.abs(R["yo"]) + ATOL))),
                "error_vs_truth": {"max": float(eg.max()), "rms": float(np.sqrt(np.mean(eg * eg)))}}
        return out


def timed_integrations(torch, integ, y0, y, tout, reps, flush=None):
    """event-timed seconds of `reps` integrations from t = 0 (one untimed first)"""
    ts = []
    for i in range(reps + 1):
        if flush is not None:
            flush.fill_(float(i))
        integ.init(0.0, y0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = integ.integrate(tout, y)
        e1.record()
        e1.synchronize()
        if r != 0:
            raise RuntimeError(f"integrate returned {r}")
        if i >= 1:
            ts.append(e0.elapsed_time(e1) * 1e-3)
    return sum(ts) / len(ts)


def robertson_workload(torch, bdfb, gen, reps=3):
    """1000 Robertson cells (per-cell log-uniform rate factors in [0.5, 2]),
    t in [0, 40], rtol 1e-4, atol 1e-8; every cell checked against the oracle
    at rtol 1e-10, atol 1e-14; the oracle timed at the run's tolerances."""
    import oracle
    p = gen.robertson(1000)
    y0 = torch.from_numpy(p.y0).cuda()
    y = torch.empty_like(y0)
    with bdfb.Integrator(p, rtol=1e-4, atol=1e-8, autotune=1) as I:
        t = timed_integrations(torch, I, y0, y, 40.0, reps)
        st = I.stats()
        mp, _ = I.mapping()
    yh = y.cpu().numpy()
    yt, _, _ = oracle.integrate_cells(p, 0.0, 40.0, 1e-10, 1e-14, threads=oracle.host_threads())
    e = (np.abs(yh - yt) / (1e-4 * np.abs(yt) + 1e-8)).reshape(-1, 3).max(axis=1)
    t0 = time.perf_counter()
    oracle.integrate_cells(p, 0.0, 40.0, 1e-4, 1e-8, threads=oracle.host_threads())
    tc = time.perf_counter() - t0
    return {"workload": "Robertson 1000 cells, k scaled by log-U[0.5,2] per cell, t in [0,40], rtol 1e-4, atol 1e-8",
            "cells_per_s": 1000 / t, "ms": t * 1e3, "steps_per_cell": st["nsteps"] / 1000,
            "lanes_per_cell_and_nmax": [int(mp[0][0]), int(mp[0][1])],
            "sum_y_max_dev": float(np.abs(yh.reshape(-1, 3).sum(axis=1) - 1.0).max()),
            "accuracy": {"cells_checked": 1000, "err_median": float(np.median(e)),
                         "err_p99": float(np.percentile(e, 99)), "err_max": float(e.max()),
                         "frac_within_10": float((e <= 10).mean())},
            "oracle_cells_per_s": 1000 / tc, "oracle_cores": oracle.host_threads()}


def mixed54_workload(torch, bdfb, gen, ncell=262_144, reps=1, flush=None):
    """262 144 mass-action cells of 54 species: FP64 factorisation against
    FP32 factorisation with FP64 refinement, same GPU, same inputs."""
    p = gen.mass_action(ncell, sizes=(54,), seed=gen.DEFAULT_SEED + 7)
    y0 = torch.from_numpy(p.y0).cuda()
    y = torch.empty_like(y0)
    out = {"workload": f"mass-action {ncell} cells, n = 54, 108 reactions, t in [0,1e-3], rtol 1e-6, atol 1e-10"}
    for name, prec in (("fp64_lu", 0), ("fp32_lu_fp64_refinement", 1)):
        with bdfb.Integrator(p, rtol=RTOL, atol=ATOL, precision=prec) as I:
            t = timed_integrations(torch, I, y0, y, TOUT, reps, flush)
            st = I.stats()
        out[name] = {"cells_per_s": ncell / t, "s": t, "steps_per_cell": st["nsteps"] / ncell,
                     "accuracy": accuracy(p, y.cpu().numpy(), ncheck=256)}
        if prec:
            out[name]["refinement_sweeps_per_solve"] = st["nrefine"] / max(1, st["nniters"])
            out[name]["fp64_fallbacks"] = st["nrefine_fallback"]
    out["speedup_mixed_over_fp64"] = out["fp32_lu_fp64_refinement"]["cells_per_s"] / out["fp64_lu"]["cells_per_s"]
    return out


def learned_workload(torch, bdfb, gen, ncell=1_000_000, ntrain_pairs=10_000_000, train_steps=6000,
                     reps=1):
    """The learned-guess workload: one 10-species network shared by ncell
    cells (initial states differ), t in [0, 1e-3], rtol 1e-6.  Training pairs
    come from recorded plain runs of other cells of the same network (seed + 1;
    cells with index % 10 == 0 held out for validation); the network trains
    on the GPU (Adam, batch 4096); then the ncell cells are integrated with
    the plain zero start and with the guess, both one warp per cell."""
    NI, NO, NP = bdfb.MLP_NI, bdfb.MLP_NO, bdfb.MLP_NPARAM
    t_rec = time.perf_counter()
    src_cells = max(1000, int(ntrain_pairs / 200))
    src = gen.mass_action_shared(src_cells, seed=gen.DEFAULT_SEED + 1)
    cap = int(ntrain_pairs * 1.3)
    X = torch.zeros((cap, NI), device="cuda")
    T = torch.zeros((cap, NO), device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    with bdfb.Integrator(src, rtol=RTOL, atol=ATOL, mapping=32) as ri:
        ri.set_record(X, T, cnt)
        ri.init(0.0, torch.from_numpy(src.y0).cuda())
        ri.integrate(TOUT, torch.empty(src.y0.size, dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    npairs = min(int(cnt.item()), cap)
    t_rec = time.perf_counter() - t_rec
    # shuffle; hold out 10% for validation
    g = torch.Generator(device="cuda").manual_seed(5)
    perm = torch.randperm(npairs, device="cuda", generator=g)
    nval = npairs // 10
    Xv, Tv = X[perm[:nval]].contiguous(), T[perm[:nval]].contiguous()
    Xt, Tt = X[perm[nval:]].contiguous(), T[perm[nval:]].contiguous()
    del X, T
    rng = np.random.default_rng(7)
    p0 = np.zeros(NP, np.float32)
    sizes = [(64, 12), (64,), (64, 64), (64,), (10, 64), (10,)]
    o = 0
    for s in sizes:
        k = int(np.prod(s))
        fan_in = s[1] if len(s) == 2 else 1
        p0[o:o + k] = rng.standard_normal(k) * (np.sqrt(2.0 / fan_in) if len(s) == 2 else 0.0)
        o += k
    params = torch.from_numpy(p0).cuda()
    m, v = torch.zeros(NP, device="cuda"), torch.zeros(NP, device="cuda")
    pk, grad = bdfb.mlp_packed(), torch.zeros(NP, device="cuda")
    hist = torch.zeros(train_steps, device="cuda")

    def val_loss():
        vg = torch.zeros(NP, device="cuda")
        vl = torch.zeros(1, device="cuda")
        bdfb.mlp_loss_grad(Xv, Tv, pk, vg, vl)
        return float(vl.item())

    bdfb.mlp_pack(params, pk)
    v0 = val_loss()
    torch.cuda.synchronize()
    t_train = time.perf_counter()
    bdfb.mlp_train(Xt, Tt, params, m, v, pk, grad, hist, batch=4096, nsteps=train_steps, lr=1e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t_train
    v1 = val_loss()
    var_t = float(Tv.var().item())
    del Xt, Tt
    prob = gen.mass_action_shared(ncell, seed=gen.DEFAULT_SEED)
    y0 = torch.from_numpy(prob.y0).cuda()
    y = torch.empty_like(y0)
    out = {}
    for name, opts in (("plain_autotuned_tiles", {}), ("plain_warp_per_cell", {"mapping": 32}),
                       ("learned_warp_per_cell", {"mapping": 32, "predictor": 1})):
        with bdfb.Integrator(prob, rtol=RTOL, atol=ATOL, mapping=opts.get("mapping", 0),
                             autotune=0 if opts.get("mapping") else 1) as li:
            if opts.get("predictor"):
                li.load_mlp(pk)
                li.set_option("predictor", 1)
            ts = []
            for i in range(1 + reps):
                li.init(0.0, y0)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                r = li.integrate(TOUT, y)
                e1.record()
                e1.synchronize()
                if r != 0:
                    raise RuntimeError(f"{name}: integrate returned {r}")
                if i >= 1:
                    ts.append(e0.elapsed_time(e1) * 1e-3)
            s = li.stats()
            out[name] = {"cells_per_s": ncell / (sum(ts) / len(ts)),
                         "newton_iters_per_step": s["nniters"] / max(1, s["nsteps"]),
                         "rhs_per_step": s["nfevals"] / max(1, s["nsteps"]),
                         "steps_per_cell": s["nsteps"] / ncell,
                         "setups_per_cell": s["nlinsetups"] / ncell,
                         "accuracy": accuracy(prob, y.cpu().numpy(), ncheck=512)}
            if opts.get("predictor"):
                out[name]["guesses"] = s["nguess"]
                out[name]["guesses_redone_from_zero"] = s["nguess_fallback"]
    return {"workload": f"mass-action shared 10-species network, {ncell} cells, Dirichlet y0, t in [0,1e-3], "
                        "rtol 1e-6, atol 1e-10; MLP 12-64-64-10 BF16 MMA, FP32 accumulate",
            "training": {"pairs": npairs, "pairs_offered": int(cnt.item()), "source_cells": src_cells,
                         "record_s": t_rec, "train_s": t_train, "adam_steps": train_steps, "batch": 4096,
                         "val_loss_init": v0, "val_loss_final": v1, "target_variance": var_t},
            **out}


def shard_seed(seed, rank):
    """weak scaling: rank r integrates its own cells, drawn with seed + r (the
    ranks' workloads are disjoint and equally sized; no data-path exchange)"""
    return seed + rank


def slowest_rank_time(torch, dist, t, device):
    """the job's step time: the maximum over ranks (t itself on one rank)"""
    if not dist:
        return t
    tt = torch.tensor([t], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def line_workload(torch, bdfb, gen, nx=10_000_000, length=1000.0, tout=3.0, reps=1, oracle_points=50_000):
    """The paper's demonstration problem (Sec. 7) as one coupled system:
    Brusselator reactions (A = 1, B = 3.5, eps = 5e-6) advected with c = 0.01
    on a periodic line of nx points over [0, length) by first-order upwind
    differences, the paper's Gaussian-bump initial state, t in [0, tout];
    BDF with Newton + GMRES(5), 3x3 reaction blocks as preconditioner
    (advection implicit in the Newton operator); FP64, then with the
    preconditioner and the GMRES operator in FP32 (option precision 1)."""
    p = gen.brusselator1d(nx, length=length)
    y0 = torch.from_numpy(p.y0).cuda()
    y = torch.empty_like(y0)
    out, yref = {}, None
    for prec in (0, 1):
        ts = []
        with bdfb.Integrator(p, rtol=RTOL, atol=ATOL, maxl=5, precision=prec) as li:
            for _ in range(reps + 1):
                li.init(0.0, y0)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                r = li.integrate(tout, y)
                torch.cuda.synchronize()
                ts.append(time.perf_counter() - t0)
                if r != 0:
                    raise RuntimeError(f"line integrate returned {r}")
            gs = li.cell_stats()[0]
        t = min(ts[1:])
        res = {"points_per_s": nx / t, "seconds": t, "steps": int(gs[0]), "newton_iters": int(gs[3]),
               "gmres_iters": int(gs[6]), "jacobian_setups": int(gs[2])}
        if prec == 0:
            yref = y.clone()
            out.update(res)
        else:
            d = ((y - yref).abs() / (RTOL * yref.abs() + ATOL)).max().item()
            out["fp32_preconditioner_and_operator"] = {**res, "max_weighted_diff_vs_fp64": d, "y": y.clone()}
    # both against the same integration at rtol 1e-9 (the oracle cannot run 3e7 unknowns
    # in the bench's time): a global norm over 3e7 unknowns bounds neither run's
    # largest error, so report the largest and the RMS
    with bdfb.Integrator(p, rtol=1e-9, atol=1e-13, maxl=5) as li:
        li.init(0.0, y0)
        if li.integrate(tout, y) != 0:
            raise RuntimeError("reference line integrate failed")
    for tgt, yy in ((out, yref), (out["fp32_preconditioner_and_operator"], out["fp32_preconditioner_and_operator"].pop("y"))):
        w = (yy - y).abs() / (RTOL * y.abs() + ATOL)
        tgt["error_vs_rtol_1e-9_run"] = {"max": w.max().item(), "rms": (w * w).mean().sqrt().item()}
    if oracle_points:
        out["oracle"] = line_oracle_rate(gen, "bdf", nx, length, tout, oracle_points)
    out["workload"] = (f"Brusselator 1-D advection-reaction (the paper's demo) {nx} points x 3, length {length}, "
                       f"c 0.01, A 1, B 3.5, eps 5e-6, t in [0,{tout}], rtol 1e-6, atol 1e-10, GMRES(5) + 3x3 blocks")
    return out


def line_oracle_rate(gen, method, nx, length, tout, nsample):
    """the oracle (one host thread: one coupled system) on the first-order
    line with the workload's spacing and nsample points: points per second
    of the same integration"""
    import oracle
    ns = min(nx, nsample)
    p = gen.brusselator1d(ns, length=length * ns / nx)
    t0 = time.perf_counter()
    if method == "ark":
        r, _, st = oracle.bruss_ark_integrate(p, 0.0, tout, RTOL, ATOL)
    else:
        r, _, st = oracle.bruss_integrate(p, 0.0, tout, RTOL, ATOL)
    dt = time.perf_counter() - t0
    return {"points_per_s": ns / dt, "seconds": dt, "steps": int(st[0]), "ret": int(r), "cores": 1,
            "sample": f"{ns} points at the same spacing ({length * ns / nx:g} long), same t range"}


def imex_workload(torch, bdfb, gen, nx, length, tout=10.0, precisions=(0, 1), reps=1, oracle_points=None):
    """The paper's demonstration problem with its own integrator type (Sec. 7):
    IMEX additive Runge-Kutta (ARK3(2)4L[2]SA), first-order upwind advection
    explicit, Brusselator reactions implicit, every implicit stage solved by
    Newton on the 3x3 point blocks (one task per GPU), rtol 1e-6,
    atol 1e-10, t in [0, tout]."""
    p = gen.brusselator1d(nx, length=length)
    y0 = torch.from_numpy(p.y0).cuda()
    y = torch.empty_like(y0)
    out = {"workload": f"Brusselator 1-D advection-reaction {nx} points x 3, length {length}, c 0.01, "
                       f"A 1, B 3.5, eps 5e-6, t in [0,{tout}], rtol 1e-6, atol 1e-10, IMEX ARK3(2)4 + "
                       f"task-local Newton (3x3 blocks)"}
    for prec in precisions:
        ts = []
        with bdfb.Integrator(p, rtol=RTOL, atol=ATOL, imex=1, precision=prec) as li:
            for _ in range(reps + 1):
                li.init(0.0, y0)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                r = li.integrate(tout, y)
                torch.cuda.synchronize()
                ts.append(time.perf_counter() - t0)
                if r != 0:
                    raise RuntimeError(f"imex integrate returned {r}")
            cs = li.cell_stats()[0]
        t = min(ts[1:])
        name = "fp64" if prec == 0 else "fp32_blocks_fp64_residual"
        out[name] = {"seconds": t, "points_per_s": nx / t, "steps": int(cs[0]), "newton_iters": int(cs[3]),
                     "error_test_failures": int(cs[5]), "newton_failures": int(cs[4]),
                     "ms_per_step": 1e3 * t / max(1, int(cs[0]))}
    if oracle_points:
        out["oracle"] = line_oracle_rate(gen, "ark", nx, length, tout, oracle_points)
    return out


def shared_sparse_workload(torch, bdfb, gen, ncell=100_000, n=128, reps=1):
    """Cells sharing one sparse network (the submodel case with one pattern
    for every block, Sec. 5): a banded n-species mechanism (reactions within
    windows of 6 species), integrated as one grouped system with task-local
    Newton solves on the shared sparse LU (BDFB_MASSACTION_SHARED) and with
    per-cell step control on the same LU (option grouped 0); and the
    10-species shared network of the learned-guess leg on those paths and on
    the per-cell dense path."""
    out = {}
    for name, p in ((f"banded_{n}_species", gen.mass_action_banded(ncell, n=n)),
                    ("network_10_species", gen.mass_action_shared(ncell, n=10))):
        y0 = torch.from_numpy(bdfb.species_major(p)).cuda()
        y = torch.empty_like(y0)
        with bdfb.Integrator(p, rtol=RTOL, atol=ATOL, shared_network=True) as I:
            t = timed_integrations(torch, I, y0, y, TOUT, reps)
            st, row = I.stats(), I.cell_stats()[0]
        yc = bdfb.cell_major(p, y.cpu().numpy())
        # every cell with its own step size and order on the same sparse LU
        with bdfb.Integrator(p, rtol=RTOL, atol=ATOL, shared_network=True, grouped=0) as I:
            tp = timed_integrations(torch, I, y0, y, TOUT, reps)
            stp = I.stats()
        per_cell_sparse = {"cells_per_s": ncell / tp, "s": tp, "steps_per_cell": stp["nsteps"] / ncell,
                           "max_steps": stp["max_steps"],
                           "accuracy": accuracy(p, bdfb.cell_major(p, y.cpu().numpy()), ncheck=128)}
        out[name] = {"workload": f"{ncell} cells sharing one {int(p.n[0])}-species network "
                                 f"({int(p.rxn_off[1])} reactions), t in [0,1e-3], rtol 1e-6, atol 1e-10",
                     "cells_per_s": ncell / t, "s": t, "steps": st["max_steps"],
                     "newton_iters_per_cell": st["nniters"] / ncell,
                     "lu_entries_with_fill": int(row[6]), "matrix_entries": int(row[7]),
                     "accuracy": accuracy(p, yc, ncheck=128),
                     "per_cell_sparse": per_cell_sparse}
        if int(p.n[0]) <= 56:
            yd = torch.from_numpy(p.y0).cuda()
            yo = torch.empty_like(yd)
            with bdfb.Integrator(p, rtol=RTOL, atol=ATOL, autotune=1) as I:
                td = timed_integrations(torch, I, yd, yo, TOUT, max(reps, 2))
            out[name]["per_cell_dense_cells_per_s"] = ncell / td
        import oracle
        sub = p.subset(np.arange(min(128, ncell)))
        t0 = time.perf_counter()
        oracle.integrate_cells_grouped(sub, 0.0, TOUT, RTOL, ATOL)
        dt = time.perf_counter() - t0
        out[name]["oracle_grouped"] = {"cells_per_s": sub.ncell / dt, "cores": 1,
                                       "sample": f"first {sub.ncell} cells as one grouped system (dense LU)"}
    return out


def grouped_workload(torch, bdfb, gen, ncell=100_000, reps=1, flush=None):
    """The mass-action workload integrated as ONE system (option "grouped":
    one step size and order, error test over every species, task-local
    Newton solves per cell; the grouping of Sec. 2) against per-cell step
    control on the same cells: the cost of the stiffness caveat of Sec. 2."""
    p = gen.mass_action(ncell, sizes=SIZES)
    y0 = torch.from_numpy(p.y0).cuda()
    y = torch.empty_like(y0)
    out = {"workload": f"mass-action {ncell} cells (sizes {'/'.join(map(str, SIZES))}), t in [0,1e-3], "
                       f"rtol 1e-6, atol 1e-10"}
    for name, opts in (("per_cell", {}), ("grouped_task_local_newton", {"grouped": 1})):
        with bdfb.Integrator(p, rtol=RTOL, atol=ATOL, **opts) as I:
            t = timed_integrations(torch, I, y0, y, TOUT, reps, flush)
            st = I.stats()
        out[name] = {"cells_per_s": ncell / t, "s": t, "steps_per_cell": st["nsteps"] / ncell,
                     "max_steps": st["max_steps"], "newton_iters_per_cell": st["nniters"] / ncell,
                     "accuracy": accuracy(p, y.cpu().numpy(), ncheck=256)}
    out["per_cell_over_grouped"] = out["per_cell"]["cells_per_s"] / out["grouped_task_local_newton"]["cells_per_s"]
    import oracle
    sub = p.subset(np.arange(min(512, ncell)))
    t0 = time.perf_counter()
    oracle.integrate_cells_grouped(sub, 0.0, TOUT, RTOL, ATOL)
    dt = time.perf_counter() - t0
    out["oracle_grouped"] = {"cells_per_s": sub.ncell / dt, "cores": 1,
                             "sample": f"first {sub.ncell} cells as one grouped system"}
    return out


def run_reference(args):
    """reference arm: the CPU oracle as it stands, on the host cores"""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_2011_12984_b300 import gen
    prob = gen.mass_action(NCELL, sizes=SIZES)
    threads = oracle.host_threads()
    ns = 4096
    sub = prob.subset(np.arange(ns))
    for _ in range(args.warmup):
        oracle.integrate_cells(sub, 0.0, TOUT, RTOL, ATOL, threads=threads)
    t = time.perf_counter()
    for _ in range(args.steps):
        oracle.integrate_cells(sub, 0.0, TOUT, RTOL, ATOL, threads=threads)
    dt = (time.perf_counter() - t) / args.steps
    v = ns / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded generators)",
            "config": {"workload": WORKLOAD, "sample_cells_per_step": ns},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"first {ns} of the {NCELL} cells per step"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2011_12984_b300 import bdfb, gen
    # weak scaling: every rank integrates its own 100 000 cells (seed per rank)
    prob = gen.mass_action(NCELL, sizes=SIZES, seed=shard_seed(gen.DEFAULT_SEED, rank))
    y0 = torch.from_numpy(prob.y0).cuda()
    y = torch.empty_like(y0)
    st = torch.empty(prob.ncell, dtype=torch.int32, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    # the step's launch sequence (counter reset, one persistent launch per
    # kernel variant on forked streams, join) is captured in a CUDA graph on
    # the first integrate and replayed on every later one
    integ = bdfb.Integrator(prob, rtol=RTOL, atol=ATOL, mapping=args.mapping, precision=args.precision,
                            autotune=0 if args.no_autotune or args.mapping else 1, graph=0 if args.no_graph else 1)

    def step():
        integ.init(0.0, y0)
        r = integ.integrate(TOUT, y, st)
        if r != 0:
            raise RuntimeError(f"integrate returned {r}: {bdfb.strerror(r)}")

    for _ in range(args.warmup):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize()
    # one persistent launch per kernel variant in use (the autotuner may put
    # two size classes on one variant)
    mp, trial_ms = integ.mapping()
    launches_per_step = len({(int(g), int(nm)) for g, nm, c in mp if c})
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    step_s, kern_s = [], []
    phases = os.environ.get("BDFB_LIBRARY") == "phases"
    if phases:
        bdfb.phase_cycles(reset=True)      # the profiling build: count the timed steps only
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.fill_(float(len(step_s)))       # evict L2 between steps
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            step()
            e1.record(s)
            e1.synchronize()
            step_s.append(e0.elapsed_time(e1) * 1e-3)
            kern_s.append(integ.stats()["last_kernel_ms"] * 1e-3)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t_step = slowest_rank_time(torch, dist, sum(step_s) / len(step_s), "cuda")
    value = ws * NCELL / t_step
    cs = integ.cell_stats()
    yh = y.cpu().numpy()
    phase_line = None
    if phases:
        pc = bdfb.phase_cycles(reset=True)
        nst = args.steps * integ.stats()["nsteps"]      # every timed integration takes the same steps
        tot = sum(pc.values())
        phase_line = {"cycles_per_step": {k: v / nst for k, v in pc.items()},
                      "share": {k: v / tot for k, v in pc.items()}, "steps": nst}
    if args.quick:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
                              "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3,
                              "kernel_ms": 1e3 * sum(kern_s) / len(kern_s), "ncell": NCELL,
                              "mapping": args.mapping, "sizes": list(SIZES), "quick": True,
                              "precision": args.precision, "stats": integ.stats(),
                              "mapping_by_class": mp.tolist(), "autotune_trial_ms": trial_ms.tolist(),
                              "steps_per_cell": float(cs[:, 0].mean()),
                              "fp64_tflops_algorithmic": algorithmic_flops(prob, cs) / (sum(kern_s) / len(kern_s)) / 1e12,
                              "phases": phase_line}))
        integ.close()
        if dist:
            dist.destroy_process_group()
        return

    # end to end through the C ABI with host buffers in pinned memory (numpy
    # views of pinned torch tensors; the copies are inside the timed region)
    y0h = torch.from_numpy(prob.y0).pin_memory().numpy()
    yh2 = torch.empty(prob.y0.size, dtype=torch.float64, pin_memory=True).numpy()
    sth = torch.empty(prob.ncell, dtype=torch.int32, pin_memory=True).numpy()
    e2e_t = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        integ.init(0.0, y0h)
        r = integ.integrate(TOUT, yh2, sth)
        t1 = time.perf_counter()
        if r != 0:
            raise RuntimeError(f"integrate (host) returned {r}")
        if i >= args.warmup:
            e2e_t.append(t1 - t0)
    e2e_v = ws * NCELL / (sum(e2e_t) / len(e2e_t))

    if rank != 0:
        integ.close()
        if dist:
            dist.destroy_process_group()
        return
    pk, pk_kind = peaks()
    t_kern = sum(kern_s) / len(kern_s)
    flops = algorithmic_flops(prob, cs)
    achieved = flops / t_kern / 1e12
    # the coupled workload's oracle (one host thread) runs beside the GPU-only legs
    grid_leg = GridOracleLeg(gen) if not args.no_configs else None
    try:
        dgemm_tf = dgemm_tflops(torch)
    except RuntimeError:
        dgemm_tf = None
    nv = nvector_bandwidth(torch, bdfb)
    grid = grid_workload(torch, bdfb, gen, hbm_gbs=pk["hbm_gbs"])
    learned = learned_workload(torch, bdfb, gen, train_steps=20000) if not args.no_learned else None
    if grid_leg is not None:
        grid["oracle_64"] = grid_leg.finish(torch, bdfb)
    if learned is not None:
        learned["oracle"] = oracle_rate(gen.mass_action_shared(10_000, seed=gen.DEFAULT_SEED),
                                        "first 10000 of the 1000000 cells")
    configs = None
    if not args.no_configs:
        configs = {"robertson_1000": robertson_workload(torch, bdfb, gen),
                   "mixed_precision_262144x54": mixed54_workload(torch, bdfb, gen, flush=flush),
                   "advection_line_1e7": line_workload(torch, bdfb, gen),
                   "grouped_vs_per_cell_100k": grouped_workload(torch, bdfb, gen, ncell=NCELL, flush=flush),
                   # the paper's single-GPU demo sizes (Sec. 7.2: n_x = 1e7, b = 1000, t_f = 10) and
                   # its one-node Summit problem (Sec. 7.1: n_x = 6e5, b = 10, t_f = 10, run there on 6 GPUs)
                   "shared_sparse_network": shared_sparse_workload(torch, bdfb, gen, ncell=NCELL),
                   "imex_demo_1e7": imex_workload(torch, bdfb, gen, 10_000_000, 1000.0, oracle_points=20_000),
                   "imex_demo_6e5_b10": imex_workload(torch, bdfb, gen, 600_000, 10.0, precisions=(1,),
                                                      oracle_points=5_000)}
        configs["mixed_precision_262144x54"]["oracle"] = oracle_rate(
            gen.mass_action(10_000, sizes=(54,), seed=gen.DEFAULT_SEED + 7), "first 10000 of the 262144 cells")
    variants = {"batched_fp64": value}
    for name, opts in (("plain_fp64_warp_per_cell", {"mapping": 32}),
                       ("batched_fp64_gauss_jordan_inverse", {"lsolver": 1}),
                       ("batched_mixed_fp32_lu", {"precision": 1, "autotune": 1})):
        with bdfb.Integrator(prob, rtol=RTOL, atol=ATOL, **opts) as vi:
            ts = []
            for i in range(2 + max(1, min(args.steps, 3))):
                flush.fill_(float(i))
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(s)
                vi.init(0.0, y0)
                r = vi.integrate(TOUT, y, st)
                e1.record(s)
                e1.synchronize()
                if r != 0:
                    raise RuntimeError(f"{name}: integrate returned {r}")
                if i >= 2:
                    ts.append(e0.elapsed_time(e1) * 1e-3)
            variants[name] = ws * NCELL / (sum(ts) / len(ts))
            if name == "batched_mixed_fp32_lu":
                variants["mixed_accuracy"] = accuracy(prob, y.cpu().numpy())
                mst = vi.stats()
                # precision 1 factors in FP32 the cells of more than 32 species
                # (the others keep FP64 factors): sweeps per Newton solve of those
                big = np.diff(prob.y_off) > 32
                nni_big = int(vi.cell_stats()[:, 3][big].sum())
                variants["mixed_fp32_factored_cells"] = int(big.sum())
                variants["mixed_refine_sweeps_per_solve"] = mst["nrefine"] / max(1, nni_big)
                variants["mixed_fp64_fallbacks"] = mst["nrefine_fallback"]
    traffic = K_CELLS_STEP_DRAM_BYTES if (NCELL == 100_000 and SIZES == (3, 10, 32, 54) and not args.mapping
                                          and args.precision == 0) else None
    acc = accuracy(prob, yh)
    cpu_v, cpu_threads, cpu_ns, cpu_dt, cpu_fail = cpu_oracle_rate(prob)
    cpu1_v, _, cpu1_ns, cpu1_dt, _ = cpu_oracle_rate(prob, seconds=3.0, threads=1)
    st_sum = integ.stats()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded generators)",
        "config": {"workload": WORKLOAD, "ncell": NCELL,
                   "mapping": ("one warp per cell" if args.mapping else
                               "size-class tiles" + ("" if args.no_autotune else ", autotuned")),
                   "lanes_per_cell_and_nmax_by_class": [[int(g), int(nm)] if c else None for g, nm, c in mp],
                   "launch": ("per step: one CUDA graph replay (captured once) of the persistent launches, "
                              "one per kernel variant, on forked streams" if not args.no_graph else
                              "per step: the persistent launches, one per kernel variant, on forked streams"),
                   "graph_launches": int(st_sum["graph_launches"]), "graph_captures": int(st_sum["graph_captures"]),
                   "l2": "flushed between steps (256 MB write)", "parallelism": f"replicas x{ws}"},
        "accuracy": acc,
        "integrator_stats": {"steps_per_cell": st_sum["nsteps"] / NCELL,
                             "newton_per_step": st_sum["nniters"] / max(1, st_sum["nsteps"]),
                             "setups_per_cell": st_sum["nlinsetups"] / NCELL,
                             "failed_cells": st_sum["ncells_failed"]},
        "roofline": {"kernel": "k_cells (persistent BDF/Newton)", "bound": "alu", "achieved": achieved,
                     "peak": dgemm_tf, "unit": "TFLOP/s", "frac": achieved / dgemm_tf if dgemm_tf else None,
                     "traffic": traffic, "kernel_ms": t_kern * 1e3, "algorithmic_fp64_flops": flops,
                     "peak_source": "FP64 of measured: cuBLAS DGEMM 8192^3 timed in this run",
                     "traffic_source": "recorded: ncu DRAM bytes of one timed step's k_cells launches, "
                                       "single-pass capture of bench.py --quick at full size",
                     "fp64_nominal_tflops": FP64_NOMINAL_TFLOPS,
                     "frac_of_nominal": achieved / FP64_NOMINAL_TFLOPS,
                     "recorded": {"fp64_pipe_active_pct_54_species_launch": K54_FP64_PIPE_PCT,
                                  "how": "ncu sm__inst_executed_pipe_fp64 on one 8192-cell launch"}},
        "variants_cells_per_s": variants,
        "coupled_grid": grid,
        "learned_guess": learned,
        "other_workloads": configs,
        "nvector_gbs": nv,
        "nvector_roofline": {"bound": "hbm", "achieved": nv["linear_sum"], "peak": pk["hbm_gbs"],
                             "unit": "GB/s", "frac": nv["linear_sum"] / pk["hbm_gbs"],
                             "peak_source": f"hbm_gbs of {pk_kind}"},
        "nvector_ceilings": nvector_ceilings(nv, pk["hbm_gbs"], clk.summary().get("sm_mhz")),
        "cpu_baseline": {"value": cpu_v, "unit": UNIT, "cores": cpu_threads, "kind": "oracle",
                         "sample": f"first {cpu_ns} of the {NCELL} cells ({cpu_dt:.1f} s, {cpu_fail} failed)",
                         "single_thread": {"value": cpu1_v, "cores": 1,
                                           "sample": f"first {cpu1_ns} cells ({cpu1_dt:.1f} s)"}},
        "e2e": {"value": e2e_v, "unit": UNIT, "h2d_bytes_per_step": int(8 * y0h.size),
                "d2h_bytes_per_step": int(8 * y0h.size + 4 * prob.ncell), "host_memory": "pinned"},
        "gpu_launches": args.steps * launches_per_step,
        "clocks": clk.summary(),
    }
    print(json.dumps(line))
    integ.close()
    if dist:
        dist.destroy_process_group()


def run_part(args):
    """one leg alone (a profiling entry point); prints its JSON"""
    import torch
    from paper_2011_12984_b300 import bdfb, gen
    if args.part == "grid":
        out = grid_workload(torch, bdfb, gen, nx=args.grid_nx, tout=args.grid_tout, reps=max(1, args.steps),
                            hbm_gbs=peaks()[0]["hbm_gbs"])
    elif args.part == "nvector":
        out = nvector_bandwidth(torch, bdfb, reps=max(1, args.steps))
    elif args.part == "robertson":
        out = robertson_workload(torch, bdfb, gen, reps=max(1, args.steps))
    elif args.part == "mixed54":
        out = mixed54_workload(torch, bdfb, gen, reps=max(1, args.steps))
    elif args.part == "imex":
        out = imex_workload(torch, bdfb, gen, args.line_nx, args.line_length, tout=args.grid_tout,
                            precisions=(args.precision,), reps=max(1, args.steps))
    elif args.part == "shared":
        out = shared_sparse_workload(torch, bdfb, gen, ncell=args.ncell, reps=max(1, args.steps))
    elif args.part == "grouped":
        out = grouped_workload(torch, bdfb, gen, ncell=args.ncell, reps=max(1, args.steps))
    elif args.part == "line":
        out = line_workload(torch, bdfb, gen, nx=args.line_nx, tout=args.grid_tout, reps=max(1, args.steps),
                            oracle_points=0)
    else:
        out = learned_workload(torch, bdfb, gen, ncell=args.ncell, train_steps=20000)
    print(json.dumps({"part": args.part, **out}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ncell", type=int, default=NCELL, help="cells per GPU (default: the workload)")
    ap.add_argument("--mapping", type=int, default=0, choices=[0, 32],
                    help="0: size-class tiles; 32: one warp per cell in input order (plain form)")
    ap.add_argument("--quick", action="store_true",
                    help="time the device path only (no e2e, accuracy, CPU or vector legs)")
    ap.add_argument("--precision", type=int, default=0, choices=[0, 1],
                    help="0: FP64 factorisation; 1: FP32 factorisation + FP64 refinement")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch the step kernels directly instead of replaying a captured CUDA graph")
    ap.add_argument("--no-autotune", action="store_true",
                    help="run each size class on its own tiling instead of the autotuned one")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the Robertson, 262144 x 54 mixed-precision, 1-D demo and grouped legs")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the learned-guess leg (1M-cell shared network, training on the GPU)")
    ap.add_argument("--sizes", default=None,
                    help="comma-separated cell sizes (default 3,10,32,54: the workload)")
    ap.add_argument("--part", default="all",
                    choices=["all", "grid", "nvector", "learned", "robertson", "mixed54", "line", "grouped",
                             "imex", "shared"],
                    help="run one leg alone and print its JSON (for profiling); all: the benchmark")
    ap.add_argument("--grid-nx", type=int, default=256, help="--part grid: grid points per dimension")
    ap.add_argument("--grid-tout", type=float, default=1.0, help="--part grid / line: end time")
    ap.add_argument("--line-nx", type=int, default=10_000_000, help="--part line / imex: points on the line")
    ap.add_argument("--line-length", type=float, default=1000.0, help="--part imex: length of the line")
    args = ap.parse_args()
    globals()["NCELL"] = args.ncell
    if args.sizes:
        globals()["SIZES"] = tuple(int(s) for s in args.sizes.split(","))
    if args.impl == "reference":
        run_reference(args)
    elif args.part != "all":
        run_part(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
