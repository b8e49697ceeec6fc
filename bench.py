"""Benchmark of the corrector-step PCG path on GB300.

Workload (default): anisotropic porous block in a channel on a jittered
1024 x 1024-vertex triangular lattice (2,093,058 cells), CP2 matrix,
Dirichlet eta = 0 on the right edge, b = A_e N(0,1).  One step = one pass of
the hot path: assemble (geometry, transmissibilities, ELL pack, Jacobi
set-up) and one FP64 Jacobi-PCG solve to relative residual 1e-10.

value = PCG cell-iterations per second of the whole step (cells x iterations
/ step time), summed over ranks.  Extra keys report the mixed-precision and
IC(0) time-to-1e-10, the iteration roofline (the method's 108 B/cell/iter), the
CPU baseline (the oracle's PCG on all host cores, timed to tolerance), each
solve variant's error against the oracle, and compact summaries of the other
workloads: the 7,938-cell latency case, the 256-system ensemble, the 50-step
differentiable chain, the CP1 step and the 33.5M-cell sequence.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--n 1024]
    python bench.py --impl reference   # the CPU oracle on the host cores
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "PCG cell-iters/s (FP64 Jacobi-PCG to 1e-10, assemble+solve)"
UNIT = "cell-iters/s"
# Algorithmic bytes per cell per iteration of the Jacobi loop on the scaled
# matrix (neighbour gathers counted once):
#   FP64, three kernels: k_spmv_dot reads p, 3 values, 3 columns, writes q
#     (8 + 24 + 12 + 8 = 52); k_cg_b reads r, q, writes r (24); k_cg_c reads
#     y, p, r, writes y, p (40); every 8th k_cg_b also reads s (+1).
#   binary32, two kernels: k_cg_a reads r, p_old, y, 3 values, 3 columns and
#     writes p_new, q, y (4+4+4+12+12 + 4+4+4 = 48); k_cg_b 12; +0.5 for s.
BYTES_PER_CELL_ITER_FP64 = 52 + 24 + 40 + 1
BYTES_PER_CELL_ITER_MIXED = 48 + 12 + 0.5
#   FP64 single-reduction loop, two kernels: k_gear_update reads p, s, w, r, y
#     and writes p, s, y, r (72); k_gear_spmv reads r, 3 values, 3 columns and
#     writes w (8 + 24 + 12 + 8 = 52); every 8th SpMV also reads S (+1).  The
#     persistent single-reduction launch moves the same bytes.
BYTES_PER_CELL_ITER_FP64_1RED = 72 + 52 + 1
# The method's own unit, whatever loop runs it: one Jacobi-PCG iteration must
# stream the matrix once (diagonal 8 + three values 24 + three int32 columns
# 12 = 44 B) and read and write the state vectors x, r, p and q = A p once each
# (4 x 16 = 64 B): 108 B per cell per iteration.  The headline roofline
# fraction divides these bytes; the bytes the chosen loop moves (117 or 125,
# extra vectors of its recurrence included) are reported beside it.
BYTES_PER_CELL_ITER_METHOD = 44 + 64
# DRAM bytes (read + write) of one FP64 Jacobi iteration, measured by ncu on
# the 1024 x 1024 channel lattice for a fixed launch configuration of each
# loop (grids, block sizes, L2 window).  The line reports a figure only when
# the autotuner chose that same configuration, and says that it comes from a
# stored capture (the rows per thread per trip, which the tuner may set
# differently from box to box, do not change the bytes a kernel moves).
TRAFFIC_CAPTURES = [
    # textbook three-kernel loop, r, p, q in persisting L2
    ({"grid": [608, 152, 152], "block": [256, 1024, 1024], "l2_window": "vectors",
      "persistent": False, "cluster": False, "stream_single_reduction": False},
     (121.8 + 21.9 + 40.9) * 1e6),
    # single-reduction streaming loop (k_gear_update + k_gear_spmv), the five
    # vectors in persisting L2, update kernel on 152 x 1024 threads
    ({"grid": [608, 152, 152], "block": [256, 1024, 1024], "l2_window": "vectors5",
      "persistent": False, "cluster": False, "stream_single_reduction": True,
      "update_1red_grid_block": [152, 1024]},
     (108.3 + 124.5) * 1e6),
    # single-reduction persistent launch (k_persistent_gear, 152 x 1024, the
    # five vectors in persisting L2): 45.07 GB over a 200-iteration solve
    ({"l2_window": "vectors5", "persistent": True, "persistent_single_reduction": True,
      "cluster": False},
     (141.7 + 83.6) * 1e6),
]
# Algorithmic bytes per cell of the CP2 step kernels (each array counted once):
# mean flux: u 16, per side col 4 + area weight 8 + l n 16, Fbar out 24, B1 out 8;
# tangential: eta 8, per side col 4 + 4 weights 32 + 4 indices 16, tau out 24,
# B2 read and write 16; update: eta 8, per side col 4 + Fbar 8 + T 8 + tau 8,
# RT0 48, Mbar 24, u 16, g 16, flux out 24, u out 16, g out 16.
BYTES_PER_CELL_CP2 = {"mean_flux": 132, "tangential": 204, "update": 252}
# FP64 arithmetic instructions per cell of the same kernels, counted from the
# source (per side: mean flux 3 mul + 3 fma/add + 2 for the sum; tangential
# 4 x (sub + fma) + 1; update sub, fma, add and 2 fma; plus the cell terms).
# GB300 issues about 2 FP64 FMAs per SM per clock, which bounds these kernels
# before HBM does.
FP64_INSTR_PER_CELL_CP2 = {"mean_flux": 24, "tangential": 28, "update": 21}
FP64_INSTR_PER_SM_CLK = 2


def traffic_for(tf: dict, n: int):
    """ncu DRAM bytes per iteration of the loop the tuner chose, when a stored
    capture of that loop, grids, blocks and window exists (n = 1024)."""
    if n != 1024:
        return None
    tf = dict(tf, update_1red_grid_block=tf.get("update_1red", [0, 0, 0])[1:])
    for cfg, traffic in TRAFFIC_CAPTURES:
        if all(tf.get(k) == v for k, v in cfg.items()):
            return traffic
    return None


def loop_name(tf: dict) -> str:
    """The FP64 Jacobi loop the tuner chose, with its kernels."""
    if tf.get("persistent_single_reduction"):
        kname = ("k_persistent_gear (whole Jacobi-PCG solve in one cooperative launch, "
                 "Chronopoulos-Gear recurrences)")
    elif tf["persistent"]:
        kname = "k_persistent_cg (whole Jacobi-PCG solve in one cooperative launch)"
    elif tf["cluster"]:
        kname = {"single_reduction": "k_cluster_cg1 (whole Jacobi-PCG solve in one thread-block "
                                     "cluster, Chronopoulos-Gear recurrences)",
                 "pipelined": "k_cluster_cgp (whole Jacobi-PCG solve in one thread-block "
                              "cluster, pipelined Ghysels-Vanroose recurrences)",
                 "s_step2": "k_cluster_cgs<2> (whole Jacobi-PCG solve in one thread-block "
                            "cluster, s-step CG, s = 2)",
                 "s_step3": "k_cluster_cgs<3> (whole Jacobi-PCG solve in one thread-block "
                            "cluster, s-step CG, s = 3)"}.get(
            tf.get("cluster_recurrence"),
            "k_cluster_cg (whole Jacobi-PCG solve in one thread-block cluster)")
    elif tf["stream_single_reduction"]:
        kname = ("pcg_iteration_fp64_single_reduction (k_gear_update + k_gear_spmv, Jacobi, "
                 "Chronopoulos-Gear recurrences)")
    else:
        kname = "pcg_iteration_fp64 (k_spmv_dot + k_cg_b + k_cg_c, Jacobi)"
    if tf["l2_window"] != "none":
        kname += {"matrix": "; matrix in persisting L2",
                  "vectors": "; r, p, q in persisting L2",
                  "vectors5": "; r, p, s, y, w in persisting L2"}[tf["l2_window"]]
    return kname


def loop_bytes(tf: dict) -> int:
    """Bytes per cell per iteration the chosen FP64 Jacobi loop moves."""
    single = tf["stream_single_reduction"] or tf.get("persistent_single_reduction")
    return BYTES_PER_CELL_ITER_FP64_1RED if single else BYTES_PER_CELL_ITER_FP64


def roofline(tf: dict, nt: int, iters: int, seconds: float, peak: float, peak_kind: str,
             n: int) -> dict:
    """Roofline of one FP64 Jacobi-PCG iteration: achieved = the method's
    108 algorithmic bytes per cell x cells / (solve time / iterations); the
    solve time is the whole timed solve (start-up, stop tests and the final
    true residual included), so the per-iteration figure is a lower bound."""
    per_iter = seconds / max(iters, 1)
    bpc = loop_bytes(tf)
    achieved = BYTES_PER_CELL_ITER_METHOD * nt / per_iter / 1e9
    loop_achieved = bpc * nt / per_iter / 1e9
    traffic = traffic_for(tf, n)
    return {"bound": "hbm", "kernel": loop_name(tf),
            "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_kind": peak_kind, "bytes_per_cell_iter": BYTES_PER_CELL_ITER_METHOD,
            "algorithmic_bytes_per_iter": BYTES_PER_CELL_ITER_METHOD * nt,
            "us_per_iter": 1e6 * per_iter,
            "loop_bytes_per_cell_iter": bpc, "loop_achieved": loop_achieved,
            "loop_frac": loop_achieved / peak,
            "traffic": traffic,
            "traffic_unit": "bytes per iteration (DRAM read + write, ncu)",
            "traffic_source": ("stored ncu capture of this loop and launch configuration on "
                               "this workload" if traffic is not None else
                               "no capture of this loop and configuration")}


def workload_label(n: int, rtol: float) -> str:
    """The benchmark's workload, named the same way by both arms."""
    return f"channel-block-aniso lattice n={n} (CP2, Jacobi-PCG, rtol {rtol:g})"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--n", type=int, default=1024, help="lattice vertices per side")
    ap.add_argument("--rtol", type=float, default=1e-10)
    ap.add_argument("--impl", default="cps", choices=["cps", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="default line only: skip the config 0 latency, config 3 ensemble, "
                         "config 4 chain, CP1 step and config 2 sequence summaries")
    ap.add_argument("--batch", type=int, default=0,
                    help="ensemble mode: this many systems of log-uniform 2k-500k cells, "
                         "batched solve vs a loop of single solves (prints its own line)")
    ap.add_argument("--batch-max-cells", type=int, default=500000,
                    help="ensemble mode: largest member (log-uniform from 2k cells)")
    ap.add_argument("--batch-no-loops", action="store_true",
                    help="ensemble mode: batched designs only, no loop of single solves")
    ap.add_argument("--batch-one-launch-only", action="store_true",
                    help="ensemble mode: the one-launch batch (FP64 and mixed) only, for "
                         "profiling (no graph chunks, streams or loops)")
    ap.add_argument("--chain", type=int, default=0,
                    help="adjoint mode: this many chained log-permeability solves on the "
                         "--n lattice with checkpointed adjoint backward (own line)")
    ap.add_argument("--chain-rtol", type=float, default=1e-8,
                    help="relative residual of the chained forward and adjoint solves")
    ap.add_argument("--sequence", action="store_true",
                    help="sequence mode: warm-started solves to --rtol on one fixed matrix of "
                         "the --n lattice (4096: 33.5M cells), right-hand side redrawn each "
                         "step, --seq-solves per variant (own line)")
    ap.add_argument("--seq-iters", type=int, default=0,
                    help="sequence mode: iteration cap per solve (0: none, run to --rtol)")
    ap.add_argument("--seq-solves", default="reduced:3,jacobi:2,mixed:2,ic0:1",
                    help="sequence mode: solves per variant (reduced, jacobi, mixed, ic0)")
    ap.add_argument("--cp2-step", type=int, default=0,
                    help="CP2-step mode: this many timed CP2 steps (mean flux, two PCG solves, "
                         "tangential flux, RT0 velocity, eps grad Psi) on the --n lattice, "
                         "after --warmup untimed ones (own line)")
    ap.add_argument("--cp2-precond", default="jacobi", choices=["jacobi", "ic0", "reduced"],
                    help="preconditioner of the CP2-step mode's solves")
    ap.add_argument("--cp1-step", type=int, default=0,
                    help="CP1-step mode: this many timed CP1 steps (x and y systems coupled "
                         "through Mbar_12, outer iteration to --cp1-toll) on the --n lattice "
                         "with no-slip walls, after --warmup untimed ones (own line)")
    ap.add_argument("--cp1-toll", type=float, default=1e-4)
    ap.add_argument("--graded", type=int, default=0,
                    help="graded-mesh mode: FP64 Jacobi and IC(0) solves on the unstructured "
                         "graded Delaunay mesh of this lattice size (900: ~2.0M cells), Morton "
                         "and triangulation numbering (own line)")
    ap.add_argument("--latency", default="",
                    help="latency mode: FP64 Jacobi solves of the centred-block lattice of "
                         "--n vertices a side on the listed ways of running the loop (comma "
                         "separated: tuned, cluster_1red, cluster_pipelined, cluster_s_step2, "
                         "cluster_s_step3, cluster, stream_1red, stream, persistent_1red; "
                         "'all' for every one), own line")
    ap.add_argument("--pin", default="",
                    help="profiling run only: pin the FP64 Jacobi configuration instead of "
                         "tuning it (a profiler's replay skews the tuner), as "
                         "'U0,U1,U2/G0,G1,G2/B0,B1,B2/PATH' with PATH stream, stream_l2, "
                         "persistent, persistent_l2, stream_1red, stream_1red_l2, persistent_1red "
                         "or persistent_1red_l2 (for the "
                         "reduced system too)")
    ap.add_argument("--profile-iters", type=int, default=0,
                    help="profiling run: assemble, then FP64 and mixed solves bounded to this "
                         "many iterations (Jacobi and IC(0)); no timing output")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class ClockSampler:
    """nvidia-smi clock and throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def host_cores() -> int:
    """Cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(problem, b, seconds: float = 10.0) -> dict:
    """The CPU baseline on a bounded sample of the same workload: the oracle's
    assembly, then its Jacobi-PCG with OpenMP parallel loops on all the host's
    cores (oracle.pcg_jacobi_omp) for as many iterations as fill about
    `seconds` (sized from a 20-iteration calibration run).  The single-
    threaded oracle's rate on a shorter sample is reported beside it."""
    import oracle
    t0 = time.perf_counter()
    A = oracle.assemble_problem(problem)
    t1 = time.perf_counter()
    nt = problem.mesh.nt
    _, cal = oracle.pcg_jacobi_omp(A, b, rtol=0.0, maxit=20)
    t2 = time.perf_counter()
    per_iter = max((t2 - t1) / max(cal.iters, 1), 1e-6)
    iters = max(20, int(seconds / per_iter))
    _, st = oracle.pcg_jacobi_omp(A, b, rtol=0.0, maxit=iters)
    t3 = time.perf_counter()
    threads = oracle.omp_threads()
    one_iters = max(5, iters // (4 * threads))
    _, st1 = oracle.pcg(A, b, rtol=0.0, maxit=one_iters, precond=oracle.PC_JACOBI,
                        raise_on_error=False)
    t4 = time.perf_counter()
    return {"value": nt * st.iters / ((t3 - t2) + (t1 - t0)), "unit": UNIT, "cores": threads,
            "host_cores": host_cores(), "kind": "oracle",
            "sample": f"oracle assembly ({t1 - t0:.2f} s, single thread) + {st.iters} Jacobi-PCG "
                      f"iterations ({t3 - t2:.2f} s) of the oracle's PCG with OpenMP parallel "
                      f"loops on {threads} threads, same {nt}-cell system",
            "pcg_only_cell_iters_per_s": nt * st.iters / (t3 - t2),
            "single_thread_oracle_pcg_cell_iters_per_s": nt * st1.iters / (t4 - t3)}


def cpu_solve_to_tolerance(problem, b, rtol: float, ref_rtol: float = 1e-13):
    """The CPU baseline on the whole workload, timed to tolerance: the
    oracle's assembly and its Jacobi-PCG with OpenMP parallel loops on all the
    host's cores to rtol (value: cells x iterations / (assembly + solve)
    time, the GPU line's metric), then, untimed, the same PCG continued from
    that solution to ref_rtol: the reference solution against which the GPU
    solutions' errors are reported.  Returns (baseline dict, reference x)."""
    import oracle
    t0 = time.perf_counter()
    A = oracle.assemble_problem(problem)
    t1 = time.perf_counter()
    nt = problem.mesh.nt
    x, st = oracle.pcg_jacobi_omp(A, b, rtol=rtol, maxit=200000)
    t2 = time.perf_counter()
    xr, st_ref = oracle.pcg_jacobi_omp(A, b, x0=x, rtol=ref_rtol, maxit=200000)
    t3 = time.perf_counter()
    threads = oracle.omp_threads()
    one_iters = max(5, min(st.iters, 200) // threads)
    _, st1 = oracle.pcg(A, b, rtol=0.0, maxit=one_iters, precond=oracle.PC_JACOBI,
                        raise_on_error=False)
    t4 = time.perf_counter()
    out = {"value": nt * st.iters / (t2 - t0), "unit": UNIT, "cores": threads,
           "host_cores": host_cores(), "kind": "oracle",
           "sample": f"the whole workload to tolerance: oracle assembly ({t1 - t0:.2f} s, single "
                     f"thread) + Jacobi-PCG to rtol {rtol:g} ({st.iters} iterations, "
                     f"{t2 - t1:.2f} s) with OpenMP parallel loops on {threads} threads, "
                     f"{nt}-cell system",
           "time_to_rtol_s": t2 - t0, "iters": st.iters, "rel_res": st.rel_res,
           "pcg_only_cell_iters_per_s": nt * st.iters / (t2 - t1),
           "single_thread_oracle_pcg_cell_iters_per_s": nt * st1.iters / (t4 - t3),
           "reference_solution": {"rtol": ref_rtol, "extra_iters": st_ref.iters,
                                  "rel_res": st_ref.rel_res, "seconds": t3 - t2}}
    return out, xr


def run_reference(args):
    """--impl reference: the CPU baseline (the oracle's assembly and its
    Jacobi-PCG on all host cores) timed on the same workload and metric.
    Each step is a bounded sample sized so that warm-up plus timed steps take
    about two minutes."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    p = synth.channel_block_problem(args.n, seed=0)
    b = synth.rhs(p.mesh, seed=1)
    per_step = min(10.0, max(1.0, 120.0 / max(args.warmup + args.steps, 1)))
    vals = []
    for k in range(args.warmup + args.steps):
        r = cpu_baseline(p, b, seconds=per_step)
        if k >= args.warmup:
            vals.append(r)
    v = float(np.mean([r["value"] for r in vals]))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_label(args.n, args.rtol), "cells": p.mesh.nt},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": vals[0]["cores"],
                             "kind": "oracle", "sample": vals[0]["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def library_spmv(s, x, stream, reps: int = 20) -> dict:
    """Library comparison point: y = A x in FP64 through cps_matvec (the
    library's own FP64 SpMV) and through torch's CSR product (cuSPARSE) on
    the same matrix, exported from the system.  Mean time over `reps`."""
    import torch
    diag, col, val = s.export_matrix()
    nt = diag.shape[0]
    rows = torch.arange(nt, device=diag.device, dtype=torch.int64)
    live = col.to(torch.int64) != rows.unsqueeze(0)
    r_all = torch.cat([rows, rows.unsqueeze(0).expand(3, nt)[live]])
    c_all = torch.cat([rows, col.to(torch.int64)[live]])
    v_all = torch.cat([diag, val[live]])
    order = torch.argsort(r_all * nt + c_all)
    crow = torch.zeros(nt + 1, dtype=torch.int64, device=diag.device)
    crow[1:] = torch.cumsum(torch.bincount(r_all, minlength=nt), 0)
    A = torch.sparse_csr_tensor(crow, c_all[order], v_all[order], size=(nt, nt))
    xv = torch.randn(nt, dtype=torch.float64, device=diag.device)
    out = {}
    for name, fn in (("cps_matvec", lambda: s.matvec(xv)),
                     ("torch_csr_cusparse", lambda: A @ xv)):
        fn()
        t, _ = timed(lambda: [fn() for _ in range(reps)], stream)
        out[name + "_us"] = 1e6 * t / reps
    y1, y2 = s.matvec(xv), A @ xv
    out["max_rel_diff"] = float((y1 - y2).abs().max() / y2.abs().max())
    out["nnz"] = int(v_all.numel())
    return out


def timed(fn, stream):
    import torch
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / 1e3, out


def batch_summary(n_systems: int, rtol: float, reps: int, loops: bool = True,
                  mixed_loop: bool = True, max_cells: int = 500000,
                  one_launch_only: bool = False) -> dict:
    """Uneven ensemble (config 3): n_systems systems with sizes log-uniform in
    [2k, max_cells] cells, random-Fourier porosity in [0.3, 1], isotropic
    Kozeny-Carman K; FP64 and mixed Jacobi-PCG to rtol, batched (cps_solve_batch)
    against a loop of single solves (best of `reps`)."""
    import torch
    import paper_2309_03543_gb300 as cps
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    ctx = cps.Context(0)
    sizes = synth.ensemble_sizes(n_systems, 2000, max_cells, seed=2024)
    systems, bs = [], []
    t0 = time.perf_counter()
    for i, nt in enumerate(sizes):
        p = synth.ensemble_member_problem(int(nt), seed=5000 + i)
        m = p.mesh
        systems.append(ctx.assemble(m.xy, m.tri, m.dirichlet, p.eps, p.kinv, p.field_loc,
                                    cps.KIND_CP2, p.nu, p.dt))
        bs.append(torch.as_tensor(synth.rhs(m, 9000 + i), device=dev))
    setup = time.perf_counter() - t0
    cells = sum(s.nt for s in systems)
    xs = [torch.zeros_like(b) for b in bs]

    def loop(prec):
        its = 0
        for s, b, x in zip(systems, bs, xs):
            x.zero_()
            _, st = s.solve(b, x=x, rtol=rtol, precision=prec)
            its += st.iters * s.nt
        return its

    status = {}

    def batch(prec):
        for x in xs:
            x.zero_()
        st = cps.solve_batch(systems, bs, xs, rtol=rtol, precision=prec, check=False)
        status[prec] = {"members_not_converged": sum(1 for t in st if t.status != 0),
                        "max_rel_res": max(t.rel_res for t in st)}
        return sum(t.iters * s.nt for t, s in zip(st, systems))

    def batch_graph(prec):
        # FP64: one launch per phase in graph chunks; mixed: whole per-system
        # solves on worker streams (the designs the one launch replaces)
        ctx.set_batch_path(cps.BATCH_GRAPH)
        try:
            for x in xs:
                x.zero_()
            st = cps.solve_batch(systems, bs, xs, rtol=rtol, precision=prec, check=False)
            return sum(t.iters * s.nt for t, s in zip(st, systems))
        finally:
            ctx.set_batch_path(cps.BATCH_ONE_LAUNCH)

    if one_launch_only:
        loops = False
        batch(cps.FP64)   # warm-up
        batch(cps.MIXED)
        runs = [("batch_fp64", lambda: batch(cps.FP64)), ("batch_mixed", lambda: batch(cps.MIXED))]
    else:
        if loops:
            loop(cps.FP64)
        batch(cps.FP64)   # warm-up (autotuning, graph capture)
        batch_graph(cps.FP64)
        batch(cps.MIXED)
        batch_graph(cps.MIXED)
        runs = [("batch_fp64", lambda: batch(cps.FP64)),
                ("batch_fp64_graph", lambda: batch_graph(cps.FP64)),
                ("batch_mixed", lambda: batch(cps.MIXED)),
                ("batch_mixed_streams", lambda: batch_graph(cps.MIXED))]
    if loops:
        runs.append(("loop_fp64", lambda: loop(cps.FP64)))
        if mixed_loop:
            loop(cps.MIXED)
            runs.append(("loop_mixed", lambda: loop(cps.MIXED)))
    res = {}
    for name, fn in runs:
        best = None
        for _ in range(max(1, reps)):
            t, ci = timed(fn, stream)
            best = (t, ci) if best is None or t < best[0] else best
        res[name] = {"seconds": best[0], "cell_iters": best[1],
                     "cell_iters_per_s": best[1] / best[0]}
    for s in systems:
        s.free()
    ctx.close()
    out = {"systems": n_systems, "cells": cells, "rtol": rtol, "host_setup_s": setup,
           "variants": res, "fp64_status": status.get(cps.FP64),
           "mixed_status": status.get(cps.MIXED),
           "batch_mixed_vs_batch_fp64_seconds":
               res["batch_mixed"]["seconds"] / res["batch_fp64"]["seconds"]}
    if "batch_fp64_graph" in res:
        out["one_launch_speedup_vs_graph_chunks"] = \
            res["batch_fp64_graph"]["seconds"] / res["batch_fp64"]["seconds"]
        out["mixed_one_launch_speedup_vs_streams"] = \
            res["batch_mixed_streams"]["seconds"] / res["batch_mixed"]["seconds"]
    if "loop_fp64" in res:
        out["batch_speedup_vs_loop"] = res["loop_fp64"]["seconds"] / res["batch_fp64"]["seconds"]
    if "loop_mixed" in res:
        out["batch_mixed_speedup_vs_loop_mixed"] = \
            res["loop_mixed"]["seconds"] / res["batch_mixed"]["seconds"]
    return out


def run_batch(args):
    """--batch N: the ensemble as its own line."""
    r = batch_summary(args.batch, args.rtol, args.steps, loops=not args.batch_no_loops,
                      max_cells=args.batch_max_cells, one_launch_only=args.batch_one_launch_only)
    line = {"metric": "ensemble corrector solves: batched vs loop (FP64 Jacobi-PCG to rtol)",
            "value": r["variants"]["batch_fp64"]["cell_iters_per_s"], "unit": UNIT,
            "config": {"workload": f"{args.batch} systems, log-uniform 2k-"
                                   f"{args.batch_max_cells // 1000}k cells",
                       "cells": r["cells"], "rtol": args.rtol,
                       "host_setup_s": r["host_setup_s"]},
            **{k: v for k, v in r.items() if k not in ("systems", "cells", "rtol",
                                                        "host_setup_s")}}
    print(json.dumps(line), flush=True)


def chain_summary(n: int, steps: int, rtol: float) -> dict:
    """Differentiable chain (config 4): x_t = A(theta)^-1 (n_t + 0.1 |n_t|/|x_{t-1}|
    x_{t-1}), n_t = area N(0,1); loss = sum_t |x_t - x*_t|^2 with targets from
    theta* (seed + 1000); gradient by the adjoint with checkpoints every 10
    steps; forward, forward + backward and the same number of plain FP64
    solves, each timed once after a warm-up.  (With the unnormalised feedback
    0.1 x_{t-1} the chain grows by 0.1 / lambda_min(A) ~ 1e7 per step on this
    matrix and overflows.)"""
    import torch
    import paper_2309_03543_gb300 as cps
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    ctx = cps.Context(0)
    p, theta_np = synth.log_permeability_problem(n, seed=0)
    _, theta_star = synth.log_permeability_problem(n, seed=1000)
    m = p.mesh
    area = synth.triangle_areas(m)
    rhs = [torch.as_tensor(area * synth.normal_noise(m.nt, 100 + t), device=dev)
           for t in range(steps)]
    model = cps.LogPermeabilityCorrector(ctx, m.xy, m.tri, m.dirichlet, p.eps, p.nu, p.dt,
                                         rtol=rtol)
    with torch.no_grad():
        targets = [x.clone() for x in cps.chained_solve(
            model, torch.as_tensor(theta_star, device=dev), rhs, checkpoint_every=0,
            normalized=True)]
    theta = torch.as_tensor(theta_np, device=dev).requires_grad_(True)

    def fwd_only():
        with torch.no_grad():
            return cps.chained_solve(model, theta, rhs, checkpoint_every=0, normalized=True)

    def fwd_bwd():
        theta.grad = None
        xs = cps.chained_solve(model, theta, rhs, checkpoint_every=10, normalized=True)
        loss = sum(((x - t) ** 2).sum() for x, t in zip(xs, targets))
        loss.backward()
        return float(loss)

    sys_ = model.system(theta)

    def plain():
        its = 0
        x = torch.zeros(m.nt, dtype=torch.float64, device=dev)
        for t in range(steps):
            x.zero_()
            _, st = sys_.solve(rhs[t], x=x, rtol=rtol)
            its += st.iters
        return its

    fwd_only()
    fwd_bwd()
    t_plain, its = timed(plain, stream)
    t_fwd, _ = timed(fwd_only, stream)
    t_fb, loss = timed(fwd_bwd, stream)
    out = {"workload": f"log-permeability lattice n={n}", "cells": m.nt, "steps": steps,
           "rtol": rtol, "checkpoint_every": 10,
           "plain_fp64_solves_s": t_plain, "plain_iters": its, "forward_s": t_fwd,
           "forward_backward_s": t_fb, "backward_s": t_fb - t_fwd,
           "ratio_forward_backward_vs_plain": t_fb / t_plain, "loss": loss,
           "grad_norm": float(theta.grad.norm())}
    model.free()
    ctx.close()
    return out


def run_chain(args):
    """--chain T: the differentiable chain as its own line."""
    r = chain_summary(args.n, args.chain, args.chain_rtol)
    line = {"metric": "differentiable chained corrector solves (adjoint backward, checkpoint 10)",
            "value": r["forward_backward_s"], "unit": "s per forward+backward",
            "higher_is_better": False,
            "config": {"workload": r["workload"], "cells": r["cells"], "steps": r["steps"],
                       "rtol": r["rtol"]},
            **{k: v for k, v in r.items() if k not in ("workload", "cells", "steps", "rtol")}}
    print(json.dumps(line), flush=True)


def latency_summary(n: int, rtol: float, reps: int = 5, names=None) -> dict:
    """Config 0: the centred-block lattice of n x n vertices (7,938 cells at
    n = 64, isotropic Kozeny-Carman, Dirichlet on the right edge), FP64
    Jacobi-PCG to rtol from x = 0, on the tuned path and on each forced path;
    median of `reps` solve times.  At this size the system is cache-resident
    and the loop is latency-bound: the figures are microseconds per
    iteration, not bandwidth.  names: the subset of paths to run (all if
    None)."""
    import torch
    import paper_2309_03543_gb300 as cps
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    ctx = cps.Context(0)
    p = synth.centred_block_problem(n, seed=0)
    m = p.mesh
    s = ctx.assemble(m.xy, m.tri, m.dirichlet, p.eps, p.kinv, p.field_loc, cps.KIND_CP2,
                     p.nu, p.dt)
    b = torch.as_tensor(synth.rhs(m, seed=1), device=dev)
    x = torch.zeros_like(b)
    out = {"workload": f"centred-block lattice n={n}", "cells": m.nt, "rtol": rtol}
    for name, path in (("tuned", cps.PATH_AUTO), ("cluster_1red", cps.PATH_CLUSTER_1RED),
                       ("cluster_pipelined", cps.PATH_CLUSTER_PIPE),
                       ("cluster_s_step2", cps.PATH_CLUSTER_SSTEP2),
                       ("cluster_s_step3", cps.PATH_CLUSTER_SSTEP3),
                       ("cluster", cps.PATH_CLUSTER), ("stream_1red", cps.PATH_STREAM_1RED),
                       ("stream", cps.PATH_STREAM), ("persistent_1red", cps.PATH_PERSISTENT_1RED)):
        if names is not None and name not in names:
            continue
        try:
            s.set_solver_path(path)
        except cps.CpsError:
            continue
        x.zero_()
        s.solve(b, x=x, rtol=rtol)       # tuning / warm-up
        ts = []
        for _ in range(reps):
            x.zero_()
            ts.append(timed(lambda: s.solve(b, x=x, rtol=rtol)[1], stream))
        t, st = sorted(ts, key=lambda v: v[0])[len(ts) // 2]
        out[name] = {"time_to_rtol_s": t, "iters": st.iters,
                     "us_per_iter": 1e6 * t / max(st.iters, 1)}
        if path == cps.PATH_AUTO:
            tf = s.tuning(cps.FP64)
            out["tuned_path"] = loop_name(tf)
    s.free()
    ctx.close()
    return out


def sequence_summary(n: int, rtol: float, iters: int = 200) -> dict:
    """Config 2, compactly: the n x n channel-block lattice (33.5M cells at
    n = 4096), matrix assembled once.  FP64 Jacobi, mixed Jacobi and FP64
    IC(0) are timed per iteration over a fixed `iters`-iteration solve (each
    after one untimed solve that also tunes); the reduced system, the fastest
    FP64 solver here, is timed to rtol on a second right-hand side,
    warm-started from the first one's solution.  GB/s are the method's
    algorithmic bytes (108 B/cell/iter Jacobi, 60.5 mixed inner, 148 IC(0),
    80 reduced) over the measured copy bandwidth.  `bench.py --sequence`
    runs the longer sequence of solves to rtol."""
    import torch
    import paper_2309_03543_gb300 as cps
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    t0 = time.perf_counter()
    p = synth.channel_block_problem(n, seed=0)
    m = p.mesh
    nt = m.nt
    rhs = [torch.as_tensor(synth.rhs(m, seed=t), device=dev) for t in range(2)]
    ctx = cps.Context(0)
    s = ctx.assemble(m.xy, m.tri, m.dirichlet, p.eps, p.kinv, p.field_loc, cps.KIND_CP2,
                     p.nu, p.dt)
    setup = time.perf_counter() - t0
    peak, peak_kind = measured_peaks()
    x = torch.zeros(nt, dtype=torch.float64, device=dev)
    out = {"workload": f"channel-block-aniso lattice n={n}", "cells": nt, "rtol": rtol,
           "host_setup_s": setup, "peak": peak, "peak_kind": peak_kind,
           "per_iteration_over": iters}
    for name, pc, prec, bpc in (("jacobi_fp64", cps.PC_JACOBI, cps.FP64,
                                 BYTES_PER_CELL_ITER_METHOD),
                                ("jacobi_mixed", cps.PC_JACOBI, cps.MIXED,
                                 BYTES_PER_CELL_ITER_MIXED),
                                ("ic0_fp64", cps.PC_IC0, cps.FP64, BYTES_PER_CELL_ITER_METHOD + 40)):
        s.set_precond(pc)
        x.zero_()
        s.solve(rhs[0], x=x, rtol=rtol, max_iter=iters, precision=prec, check=False)
        x.zero_()
        t, st = timed(lambda: s.solve(rhs[0], x=x, rtol=rtol, max_iter=iters, precision=prec,
                                      check=False)[1], stream)
        gbs = bpc * nt * st.iters / t / 1e9
        out[name] = {"iters": st.iters, "us_per_iter": 1e6 * t / max(st.iters, 1),
                     "bytes_per_cell_iter": bpc, "algorithmic_gbs": gbs, "frac": gbs / peak}
        if name == "jacobi_fp64":
            out[name]["path"] = loop_name(s.tuning(cps.FP64))
    s.set_precond(cps.PC_REDUCED)
    x.zero_()
    s.solve(rhs[0], x=x, rtol=rtol, max_iter=iters, check=False)      # tunes its path
    t, st = timed(lambda: s.solve(rhs[1], x=x, rtol=rtol, check=False)[1], stream)
    gbs = 80 * nt * st.iters / t / 1e9
    out["reduced_fp64_to_rtol"] = {
        "time_to_rtol_s": t, "iters": st.iters, "rel_res": st.rel_res, "status": st.status,
        "warm_start": "from the solution of a capped solve of the first right-hand side",
        "us_per_iter": 1e6 * t / max(st.iters, 1), "bytes_per_cell_iter": 80,
        "algorithmic_gbs": gbs, "frac": gbs / peak}
    s.free()
    ctx.close()
    return out


def run_sequence(args):
    """Warm-started corrector sequence on one fixed matrix (config 2): the
    matrix is assembled once (Sec. 3.1: assembled and factored once, solved
    every step), b_t = area N(0,1) from seed t, and each solve starts from the
    previous solution and runs to --rtol.  At 33.5M cells a Jacobi solve to
    1e-10 takes tens of thousands of iterations, so every variant runs its own
    number of solves (--seq-solves, e.g. "reduced:3,jacobi:2,mixed:2,ic0:1"),
    stated in the line.  Per variant: seconds per solve to rtol, iterations,
    microseconds per iteration and the method's algorithmic bytes against the
    measured copy bandwidth (108 B/cell/iter for Jacobi; 148 for IC(0); the
    reduced system's own 160 B per black-row pair)."""
    import torch
    import paper_2309_03543_gb300 as cps
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    ctx = cps.Context(0)
    t0 = time.perf_counter()
    p = synth.channel_block_problem(args.n, seed=0)
    m = p.mesh
    nt = m.nt
    s = ctx.assemble(m.xy, m.tri, m.dirichlet, p.eps, p.kinv, p.field_loc, cps.KIND_CP2,
                     p.nu, p.dt)
    counts = {k: int(v) for k, v in (kv.split(":") for kv in args.seq_solves.split(","))}
    total = max(counts.values()) + 1
    rhs = [torch.as_tensor(synth.rhs(m, seed=t), device=dev) for t in range(total)]
    setup = time.perf_counter() - t0
    peak, peak_kind = measured_peaks()
    max_iter = args.seq_iters if args.seq_iters > 0 else 1_000_000
    # (name, preconditioner, precision, algorithmic bytes per cell per iteration)
    table = {"reduced": (cps.PC_REDUCED, cps.FP64, 160 / 2),
             "jacobi": (cps.PC_JACOBI, cps.FP64, BYTES_PER_CELL_ITER_METHOD),
             "mixed": (cps.PC_JACOBI, cps.MIXED, BYTES_PER_CELL_ITER_MIXED),
             "ic0": (cps.PC_IC0, cps.FP64, BYTES_PER_CELL_ITER_METHOD + 40)}
    out = {}
    for name, k in counts.items():
        pc, prec, bpc = table[name]
        s.set_precond(pc)
        x = torch.zeros(nt, dtype=torch.float64, device=dev)
        t_tot, it_tot, rel, status, per = 0.0, 0, [], [], []
        for t in range(k + 1):          # solve 0 also tunes: not timed
            dt_, st = timed(lambda: s.solve(rhs[t], x=x, rtol=args.rtol, max_iter=max_iter,
                                            precision=prec, check=False)[1], stream)
            if t == 0:
                continue
            t_tot += dt_
            it_tot += st.iters
            rel.append(st.rel_res)
            status.append(st.status)
            per.append(dt_)
        # reduced system: iterations run over the black half of the cells
        units = nt // 2 if pc == cps.PC_REDUCED else nt
        gbs = bpc * nt * it_tot / t_tot / 1e9
        out[name] = {"solves": k, "seconds_per_solve": t_tot / k, "seconds_each": per,
                     "iters": it_tot, "us_per_iter": 1e6 * t_tot / max(it_tot, 1),
                     "cell_iters_per_s": units * it_tot / t_tot, "algorithmic_gbs": gbs,
                     "bytes_per_cell_iter": bpc, "frac_of_peak": gbs / peak,
                     "rel_res_each": rel, "status_each": status,
                     "path": loop_name(s.tuning(cps.FP64)) if name == "jacobi" else None}
    s.free()
    ctx.close()
    first = out.get("jacobi") or next(iter(out.values()))
    line = {"metric": "warm-started corrector sequence: time per solve to rtol",
            "value": first["cell_iters_per_s"], "unit": "cell-iters/s",
            "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"channel-block-aniso lattice n={args.n}", "cells": nt,
                       "rtol": args.rtol, "solves": counts,
                       "rhs": "area N(0,1) from seed t, warm start from x_{t-1}",
                       "host_setup_s": setup},
            "peak": peak, "peak_kind": peak_kind, "variants": out}
    print(json.dumps(line), flush=True)


def run_cp2_step(args):
    """Whole CP2 steps on the channel-block workload: each step takes a new
    cell velocity u^{k+2/3} (seeded random-Fourier field plus a mean flow) and
    the previous step's eps grad(Psi); the line reports steps per second, the
    iterations of the two solves (the second warm-started from the first), the
    device time of each step kernel against the measured copy bandwidth, and
    the largest net cell flux left after the step."""
    import torch
    import paper_2309_03543_gb300 as cps
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    ctx = cps.Context(0)
    p = synth.channel_block_problem(args.n, seed=0)
    m = p.mesh
    nt = m.nt
    s = ctx.assemble(m.xy, m.tri, m.dirichlet, p.eps, p.kinv, p.field_loc, cps.KIND_CP2,
                     p.nu, p.dt)
    s.cp2_setup(m.xy, m.tri, p.eps, p.kinv)
    pc = {"jacobi": cps.PC_JACOBI, "ic0": cps.PC_IC0, "reduced": cps.PC_REDUCED}[args.cp2_precond]
    if pc != cps.PC_JACOBI:
        s.set_precond(pc)
    total = args.warmup + args.cp2_step
    us = [torch.as_tensor(synth.cell_vector_field(m, 100 + t, mean=(0.05, 0.01), scale=0.02),
                          device=dev) for t in range(total)]
    g = torch.as_tensor(synth.cell_vector_field(m, 12, scale=1e-3), device=dev)
    peak, peak_kind = measured_peaks()
    secs, iters, kms, imbalance = [], [], [], 0.0
    for t in range(total):
        dt_, out = timed(lambda: s.cp2_step(us[t], g, rtol=args.rtol), stream)
        g = out["g_next"]
        if t >= args.warmup:
            secs.append(dt_)
            iters.append([out["stats"][0].iters, out["stats"][1].iters])
            kms.append(s.cp2_kernel_times())
            q = out["flux"]
            imbalance = max(imbalance, float(q.sum(dim=0).abs().max() / q.abs().max()))
    kernels = {}
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak = sms * FP64_INSTR_PER_SM_CLK * 2070e6     # FP64 instructions/s at the max clock
    for k, name in enumerate(("mean_flux", "tangential", "update")):
        ms = sum(x[k] for x in kms) / len(kms)
        gbs = BYTES_PER_CELL_CP2[name] * nt / (ms * 1e-3) / 1e9
        ips = FP64_INSTR_PER_CELL_CP2[name] * nt / (ms * 1e-3)
        kernels[name] = {"ms": ms, "bytes_per_cell": BYTES_PER_CELL_CP2[name],
                         "achieved_gbs": gbs, "frac": gbs / peak,
                         "fp64_instr_per_cell": FP64_INSTR_PER_CELL_CP2[name],
                         "fp64_frac_of_issue_peak": ips / alu_peak}
    kernel_s = sum(v["ms"] for v in kernels.values()) * 1e-3
    t_step = sum(secs) / len(secs)
    s.free()
    line = {"metric": "CP2 steps per second (mean flux, two PCG solves to rtol, tangential "
                      "flux, RT0 velocity, eps grad Psi)",
            "value": 1.0 / t_step, "unit": "steps/s", "higher_is_better": True,
            "ms_per_step": 1e3 * t_step, "steps": args.cp2_step, "warmup": args.warmup,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"channel-block-aniso lattice n={args.n}", "cells": nt,
                       "rtol": args.rtol, "precond": args.cp2_precond,
                       "u23": "random-Fourier field + mean flow, seed 100+t",
                       "l2": "step working set ~1.2 GB, larger than L2"},
            "solve_iters": iters, "step_kernels": kernels,
            "step_kernels_share_of_step": kernel_s / t_step,
            "peak": peak, "peak_kind": peak_kind,
            "fp64_issue_peak_instr_per_s": alu_peak, "max_net_cell_flux_rel": imbalance}
    print(json.dumps(line), flush=True)


def cp1_summary(n: int, steps: int, warmup: int, toll: float, rtol: float) -> dict:
    """Whole CP1 steps on the channel-block workload with no-slip walls: each
    step takes a new predictor increment (seeded random-Fourier field) and
    runs the outer iteration of App. B to toll, in one launch (the default
    path) and as host-driven sweeps of single solves; per path ms per step,
    outer sweeps and PCG iterations per step."""
    import dataclasses
    import torch
    import paper_2309_03543_gb300 as cps
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    ctx = cps.Context(0)
    p = synth.channel_block_problem(n, seed=0)
    m = p.mesh
    nbr = side_neighbours(m.tri)
    e, j = np.nonzero(nbr < 0)
    m = dataclasses.replace(m, dirichlet=(e * 3 + j).astype(np.int32))
    nt = m.nt
    sx = ctx.assemble(m.xy, m.tri, m.dirichlet, p.eps, p.kinv, p.field_loc, cps.KIND_CP1_X,
                      p.nu, p.dt)
    sy = ctx.assemble(m.xy, m.tri, m.dirichlet, p.eps, p.kinv, p.field_loc, cps.KIND_CP1_Y,
                      p.nu, p.dt)
    cps.cp1_setup(sx, sy, m.xy, m.tri, p.eps, p.kinv)
    total = warmup + steps
    dus = [torch.as_tensor(synth.cell_vector_field(m, 200 + t, mean=(0.01, -0.02), scale=0.05),
                           device=dev) for t in range(total)]
    out = {"workload": f"channel-block-aniso lattice n={n}, no-slip walls", "cells": nt,
           "toll": toll, "rtol": rtol, "steps": steps,
           "du_breve": "random-Fourier field + mean, seed 200+t"}
    for name, path in (("one_launch", cps.CP1_ONE_LAUNCH), ("host_sweeps", cps.CP1_HOST)):
        cps.set_cp1_path(sx, path)
        secs, outer, iters, status = [], [], [], []
        for t in range(total):
            dt_, (du, st) = timed(lambda: cps.cp1_step(sx, sy, dus[t], toll=toll, rtol=rtol,
                                                       check=False), stream)
            if t >= warmup:
                secs.append(dt_)
                outer.append(st["outer"])
                iters.append(st["solve_iters"])
                status.append(st["status"])
        t_step = sum(secs) / len(secs)
        out[name] = {"ms_per_step": 1e3 * t_step, "outer_sweeps": outer, "solve_iters": iters,
                     "status": status,
                     "us_per_solve_iter": 1e6 * sum(secs) / max(sum(iters), 1)}
    out["one_launch_speedup"] = (out["host_sweeps"]["ms_per_step"]
                                 / out["one_launch"]["ms_per_step"])
    sx.free()
    sy.free()
    ctx.close()
    return out


def run_cp1_step(args):
    """--cp1-step K: the CP1 step as its own line (steps per second of the
    default one-launch path; the host-driven sweeps beside it)."""
    r = cp1_summary(args.n, args.cp1_step, args.warmup, args.cp1_toll, args.rtol)
    t_step = r["one_launch"]["ms_per_step"] / 1e3
    line = {"metric": "CP1 steps per second (x and y solves coupled through Mbar_12, outer "
                      "iteration of App. B)",
            "value": 1.0 / t_step, "unit": "steps/s", "higher_is_better": True,
            "ms_per_step": 1e3 * t_step, "steps": args.cp1_step, "warmup": args.warmup,
            "dtype": "f64", "data": "synthetic",
            "config": {k: r[k] for k in ("workload", "cells", "toll", "rtol", "du_breve")},
            "paths": {k: r[k] for k in ("one_launch", "host_sweeps")},
            "one_launch_speedup": r["one_launch_speedup"]}
    print(json.dumps(line), flush=True)


def run_graded(args):
    """Solves on an unstructured Delaunay mesh graded toward the porous
    block's interface (two levels of refinement, up to four colours): FP64
    Jacobi on its tuned path and multicolour IC(0) to --rtol, with the cells
    numbered along a Morton curve and as the triangulation left them."""
    import torch
    import paper_2309_03543_gb300 as cps
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    ctx = cps.Context(0)
    peak, peak_kind = measured_peaks()
    res = {}
    cells = 0
    for order in ("morton", "none"):
        p = synth.graded_problem(args.graded, seed=0, order=order)
        m = p.mesh
        cells = m.nt
        s = ctx.assemble(m.xy, m.tri, m.dirichlet, p.eps, p.kinv, p.field_loc, cps.KIND_CP2,
                         p.nu, p.dt)
        b = torch.as_tensor(synth.rhs(m, seed=1), device=dev)
        for name, pc in (("jacobi", cps.PC_JACOBI), ("ic0", cps.PC_IC0)):
            s.set_precond(pc)
            x = torch.zeros_like(b)
            s.solve(b, x=x, rtol=args.rtol, check=False)   # tuning, path probes
            ts = []
            for _ in range(max(args.steps, 1)):
                x.zero_()
                dt_, st = timed(lambda: s.solve(b, x=x, rtol=args.rtol, check=False)[1], stream)
                ts.append(dt_)
            t = sorted(ts)[len(ts) // 2]
            entry = {"seconds": t, "iters": st.iters, "us_per_iter": 1e6 * t / st.iters,
                     "rel_res": st.rel_res, "status": st.status}
            if name == "jacobi":
                tf = s.tuning(cps.FP64)
                bpc = loop_bytes(tf)
                gbs = BYTES_PER_CELL_ITER_METHOD * cells / (t / st.iters) / 1e9
                entry.update({"algorithmic_gbs": gbs, "frac": gbs / peak,
                              "bytes_per_cell_iter": BYTES_PER_CELL_ITER_METHOD,
                              "loop_bytes_per_cell_iter": bpc,
                              "loop_frac": bpc / BYTES_PER_CELL_ITER_METHOD * gbs / peak,
                              "path": tf})
            res[f"{order}_{name}"] = entry
        s.free()
    line = {"metric": "time to rtol on a graded unstructured Delaunay mesh",
            "value": res["morton_jacobi"]["seconds"], "unit": "s", "higher_is_better": False,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"graded-delaunay n={args.graded} levels=2 (channel-block "
                                   f"fields, anisotropic K)", "cells": cells, "rtol": args.rtol},
            "peak": peak, "peak_kind": peak_kind, **res}
    print(json.dumps(line), flush=True)


def side_neighbours(tri):
    """Neighbour across each local side (-1 on the boundary), by sorting the
    sides' vertex pairs; host-side set-up of the no-slip wall list."""
    nt = tri.shape[0]
    a = tri[:, [1, 2, 0]].astype(np.int64)
    b = tri[:, [2, 0, 1]].astype(np.int64)
    key = np.minimum(a, b) * (int(tri.max()) + 1) + np.maximum(a, b)
    flat = key.ravel()
    order = np.argsort(flat, kind="stable")
    sk = flat[order]
    nbr = np.full(3 * nt, -1, dtype=np.int64)
    same = np.flatnonzero(sk[1:] == sk[:-1])
    s0, s1 = order[same], order[same + 1]
    nbr[s0] = s1 // 3
    nbr[s1] = s0 // 3
    return nbr.reshape(nt, 3)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.batch:
        run_batch(args)
        return
    if args.chain:
        run_chain(args)
        return
    if args.sequence:
        run_sequence(args)
        return
    if args.cp2_step:
        run_cp2_step(args)
        return
    if args.cp1_step:
        run_cp1_step(args)
        return
    if args.graded:
        run_graded(args)
        return
    if args.latency:
        names = None if args.latency == "all" else args.latency.split(",")
        print(json.dumps({"latency": latency_summary(args.n, args.rtol, names=names)}),
              flush=True)
        return
    import torch
    import paper_2309_03543_gb300 as cps

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    def barrier():
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize()

    # Each rank solves its own independent instance (weak scaling, no
    # collective in the data path).
    seed = 1000 * rank
    p = synth.channel_block_problem(args.n, seed=seed)
    m = p.mesh
    b_np = synth.rhs(m, seed=seed + 1)
    nt = m.nt
    ctx = cps.Context(local)
    stream = torch.cuda.current_stream(dev)

    host = {"xy": torch.as_tensor(m.xy).pin_memory(), "tri": torch.as_tensor(m.tri).pin_memory(),
            "dir": torch.as_tensor(m.dirichlet).pin_memory(),
            "eps": torch.as_tensor(p.eps).pin_memory(),
            "kinv": torch.as_tensor(p.kinv).pin_memory(), "b": torch.as_tensor(b_np).pin_memory()}
    d = {k: v.to(dev) for k, v in host.items()}
    x = torch.zeros(nt, dtype=torch.float64, device=dev)
    x_host = torch.empty(nt, dtype=torch.float64).pin_memory()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    h2d_bytes = sum(v.numel() * v.element_size() for v in host.values())
    d2h_bytes = nt * 8

    if args.profile_iters:
        # every variant once (autotuning, path probes), then the FP64 Jacobi
        # solve again inside the NVTX range "cps_profile", the mixed Jacobi
        # solve inside "cps_profile_mixed", IC(0) inside "cps_profile_ic0" and
        # the reduced-system solve inside "cps_profile_reduced" (the launches a
        # profiler should select: ncu --nvtx --nvtx-include "cps_profile/")
        s = ctx.assemble(d["xy"], d["tri"], d["dir"], d["eps"], d["kinv"], cps.PER_VERTEX,
                         cps.KIND_CP2, p.nu, p.dt)
        if args.pin:
            u, g, b, path = args.pin.split("/")
            s.set_kernel_shapes(cps.FP64, *[[int(v) for v in f.split(",")] for f in (u, g, b)])
            s.set_solver_path({"stream": cps.PATH_STREAM, "stream_l2": cps.PATH_STREAM_L2,
                               "persistent": cps.PATH_PERSISTENT,
                               "persistent_l2": cps.PATH_PERSISTENT_L2,
                               "stream_1red": cps.PATH_STREAM_1RED,
                               "stream_1red_l2": cps.PATH_STREAM_1RED_L2,
                               "persistent_1red": cps.PATH_PERSISTENT_1RED,
                               "persistent_1red_l2": cps.PATH_PERSISTENT_1RED_L2}[path])
        for pc in (cps.PC_JACOBI, cps.PC_IC0):
            s.set_precond(pc)
            for prec in (cps.FP64, cps.MIXED):
                x.zero_()
                s.solve(d["b"], x=x, rtol=args.rtol, max_iter=args.profile_iters,
                        precision=prec, check=False)
        s.set_precond(cps.PC_JACOBI)
        x.zero_()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("cps_profile")
        s.solve(d["b"], x=x, rtol=args.rtol, max_iter=args.profile_iters, check=False)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        x.zero_()
        torch.cuda.nvtx.range_push("cps_profile_mixed")
        s.solve(d["b"], x=x, rtol=args.rtol, max_iter=args.profile_iters, precision=cps.MIXED,
                check=False)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        # IC(0) (tuned or pinned loop), marked "cps_profile_ic0"
        s.set_precond(cps.PC_IC0)
        x.zero_()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("cps_profile_ic0")
        s.solve(d["b"], x=x, rtol=args.rtol, max_iter=args.profile_iters, check=False)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        # the reduced system: first solve tunes its path, the second is marked
        try:
            s.set_precond(cps.PC_REDUCED)
        except cps.CpsError:
            pass
        else:
            for mark in (False, True):
                x.zero_()
                torch.cuda.synchronize()
                if mark:
                    torch.cuda.nvtx.range_push("cps_profile_reduced")
                s.solve(d["b"], x=x, rtol=args.rtol, max_iter=args.profile_iters, check=False)
                torch.cuda.synchronize()
                if mark:
                    torch.cuda.nvtx.range_pop()
        tuned = s.tuning(cps.FP64)
        s.free()
        print(json.dumps({"profile_run": True, "n": args.n, "cells": nt,
                          "max_iter": args.profile_iters, "fp64_tuning": tuned}))
        return

    def step(src, precision=cps.FP64):
        s = ctx.assemble(src["xy"], src["tri"], src["dir"], src["eps"], src["kinv"],
                         cps.PER_VERTEX, cps.KIND_CP2, p.nu, p.dt)
        x.zero_()
        _, st = s.solve(src["b"], x=x, rtol=args.rtol, precision=precision)
        launches = s.info()["setup_launches"] + st.launches
        s.free()
        return st, launches

    # warm-up
    for _ in range(args.warmup):
        step(d)
    barrier()

    # ---- timed region: device-resident inputs
    sampler = ClockSampler(local)
    sampler.start()
    times, iters, launches = [], [], 0
    for _ in range(args.steps):
        flush.zero_()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, nl = step(d)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
        iters.append(st.iters)
        launches += nl
        assert st.rel_res <= args.rtol, st
    barrier()
    clocks = sampler.stop()
    t_total = sum(times)
    cell_iters = nt * sum(iters)
    from paper_2309_03543_gb300.dist import aggregate
    t_max, total_cell_iters = aggregate(t_total, cell_iters, device=dev)
    value = total_cell_iters / t_max

    # ---- e2e: host buffers in, host result out, through the public API
    e2e_times = []
    for _ in range(max(2, min(args.steps, 3))):
        flush.zero_()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        src = {k: v.to(dev, non_blocking=True) for k, v in host.items()}
        st, _ = step(src)
        x_host.copy_(x, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_times.append((e0.elapsed_time(e1) / 1e3, st.iters))
    e2e_value = world * nt * sum(i for _, i in e2e_times) / sum(t for t, _ in e2e_times)

    # ---- solve loop alone (matrix assembled): FP64 vs mixed, Jacobi vs IC(0)
    s = ctx.assemble(d["xy"], d["tri"], d["dir"], d["eps"], d["kinv"], cps.PER_VERTEX,
                     cps.KIND_CP2, p.nu, p.dt)
    peak, peak_kind = measured_peaks()
    variants, solutions = {}, {}
    for pc_name, pc in (("jacobi", cps.PC_JACOBI), ("ic0", cps.PC_IC0),
                        ("reduced", cps.PC_REDUCED)):
        try:
            s.set_precond(pc)
        except cps.CpsError:
            continue
        for prec_name, prec in (("fp64", cps.FP64), ("mixed", cps.MIXED)):
            if pc == cps.PC_REDUCED and prec != cps.FP64:
                continue
            ts = []
            for _ in range(2):
                x.zero_()
                flush.zero_()
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                _, st = s.solve(d["b"], x=x, rtol=args.rtol, precision=prec)
                e1.record(stream)
                e1.synchronize()
                ts.append((e0.elapsed_time(e1) / 1e3, st))
            t, st = min(ts, key=lambda v: v[0])
            variants[f"{pc_name}_{prec_name}"] = {
                "time_to_rtol_s": t, "iters": st.iters, "refinements": st.refinements,
                "rel_res": st.rel_res, "us_per_iter": 1e6 * t / max(st.iters, 1)}
            solutions[f"{pc_name}_{prec_name}"] = x.cpu().numpy().copy()
    tuning = {"fp64": s.tuning(cps.FP64), "mixed": s.tuning(cps.MIXED)}
    # each way of running the loop, forced: streaming kernels, the one-launch
    # cluster solve (small systems), the persistent grid-synchronised launch
    for pc_name, pc in (("jacobi", cps.PC_JACOBI), ("reduced", cps.PC_REDUCED),
                        ("ic0", cps.PC_IC0)):
        try:
            s.set_precond(pc)
        except cps.CpsError:
            continue
        for path_name, path in (("stream", cps.PATH_STREAM), ("cluster", cps.PATH_CLUSTER),
                                ("persistent", cps.PATH_PERSISTENT),
                                ("stream_1red", cps.PATH_STREAM_1RED),
                                ("stream_1red_l2", cps.PATH_STREAM_1RED_L2),
                                ("persistent_1red", cps.PATH_PERSISTENT_1RED),
                                ("persistent_1red_l2", cps.PATH_PERSISTENT_1RED_L2)):
            if pc == cps.PC_REDUCED and path in (cps.PATH_CLUSTER, cps.PATH_STREAM_1RED,
                                                 cps.PATH_STREAM_1RED_L2):
                continue
            if pc == cps.PC_IC0 and path not in (cps.PATH_STREAM, cps.PATH_PERSISTENT_1RED,
                                                 cps.PATH_PERSISTENT_1RED_L2):
                continue
            try:
                s.set_solver_path(path)
            except cps.CpsError:
                continue
            ts = []
            for _ in range(3):
                x.zero_()
                ts.append(timed(lambda: s.solve(d["b"], x=x, rtol=args.rtol)[1], stream))
            t, st = min(ts, key=lambda v: v[0])
            variants[f"{pc_name}_fp64_{path_name}_path"] = {
                "time_to_rtol_s": t, "iters": st.iters, "us_per_iter": 1e6 * t / max(st.iters, 1)}
        s.set_solver_path(cps.PATH_AUTO)
    library = library_spmv(s, x, stream)
    s.free()
    jf = variants["jacobi_fp64"]
    roof = roofline(tuning["fp64"], nt, jf["iters"], jf["time_to_rtol_s"], peak, peak_kind,
                    args.n)
    jm = variants["jacobi_mixed"]
    jm["inner_gbs"] = BYTES_PER_CELL_ITER_MIXED * nt * jm["iters"] / jm["time_to_rtol_s"] / 1e9

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_label(args.n, args.rtol),
                   "cells": nt, "iters_per_step": int(np.mean(iters)),
                   "l2": "256 MB buffer written between steps",
                   "parallelism": f"replicas x{world}"},
        "roofline": roof,
        "solve_variants": variants,
        "autotuned": tuning,
        "library_spmv": library,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d_bytes,
                "d2h_bytes_per_step": d2h_bytes},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    # the other workloads, compactly (each in its own context, after the
    # headline measurement): config 0 latency, config 3 ensemble (batched
    # FP64 and mixed against a loop of FP64 single solves), config 4 chain,
    # the CP1 step on the headline lattice (one launch and host sweeps), and
    # config 2 (33.5M cells: per-iteration rates, a reduced solve to rtol)
    if rank == 0 and world == 1 and not args.no_extras:
        extras = (("n64_latency", lambda: latency_summary(64, args.rtol)),
                  ("batch", lambda: batch_summary(256, args.rtol, 1, loops=True,
                                                  mixed_loop=False)),
                  ("chain", lambda: chain_summary(512, 50, 1e-8)),
                  ("cp1_step", lambda: cp1_summary(args.n, 3, 2, 1e-4, args.rtol)),
                  ("n4096_sequence", lambda: sequence_summary(4096, args.rtol)))
        for key, fn in extras:
            t0 = time.perf_counter()
            try:
                line[key] = fn()
            except Exception as e:      # an extra must not cost the headline line
                line[key] = {"error": repr(e)[:400]}
            line[key]["wall_s"] = time.perf_counter() - t0
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle's PCG on all host cores, timed to tolerance on the whole
        # workload; its solution (continued to 1e-13) gives every solve
        # variant's error against the oracle
        cb, x_oracle = cpu_solve_to_tolerance(p, b_np, args.rtol)
        line["cpu_baseline"] = cb
        nref = float(np.linalg.norm(x_oracle))
        for k, xs in solutions.items():
            variants[k]["rel_err_vs_oracle"] = float(np.linalg.norm(xs - x_oracle)) / nref
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.barrier()
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
