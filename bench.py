#!/usr/bin/env python
"""Throughput of the stabilized implicit u-p MPM load step on GB300.

One "step" is one load step of the whole hot path (bin + sort, shape
functions, Stage-1 P2G, sparsity, Newton with residual / Jacobian assembly and
FGMRES to the paper's 1e-8 residual test, G2P + convection).  The default
workload is the largest single-GPU one, the 3D slope: a 12.8 x 12.8 x 6.4 m box
of 128 x 128 x 64 cells at h = 0.1 m, the cells below a 30 degree ground
surface filled with 2 x 2 x 2 points (4,208,640), GIMP, quasi-static implicit
Euler, dt = 10 s, gravity from t = 0 with a hydrostatic pore pressure below a
water table at mid-height, k = 1e-12 m^2.  `value` is FP64; `mixed` is the
same steps in the mixed-precision mode with its error against the FP64 run.
Inputs are synthetic (seeded), resident in HBM for `value`; `e2e` goes
through the C-ABI with host buffers.  --workload footing | block3d |
terzaghi | harmonic | batch select the other configurations.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun, one process per GPU) every rank steps its own
independent replica of the problem ("replicas only": the path has no exchange
step at this size); value = all ranks' particle updates / max rank time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# The oracle legs (cpu_baseline and --impl reference) are reported as one core:
# keep the BLAS / OpenMP thread pools of numpy and scipy at one thread (set
# before numpy is imported).
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ[_v] = "1"

METRIC = "implicit u–p MPM steps/s and particle-updates/s at 1e-8 residual, FP64 vs mixed"
UNIT = "particle-updates/s"
L2_FLUSH_BYTES = 512 << 20


def max_over_ranks(x, world, device):
    """The largest of the ranks' values of x (a time: the whole job is as slow
    as its slowest rank); x itself on a single process."""
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="slope")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--batch-sample", type=int, default=4)
    ap.add_argument("--precond-lag", type=int, default=2,
                    help="Newton iterations served by one preconditioner set-up")
    ap.add_argument("--profile", default="jacobian",
                    help="kernel classes timed with CUDA events inside the timed steps")
    ap.add_argument("--breakdown-steps", type=int, default=3,
                    help="extra steps, after the timed ones, with every kernel class timed")
    ap.add_argument("--schur-order", type=int, default=None, help="0 upper, 1 lower triangular")
    ap.add_argument("--mg-sweeps", type=int, default=None, help="V(k,k) smoothing sweeps")
    ap.add_argument("--mg-omega", type=float, default=None, help="block-Jacobi damping")
    ap.add_argument("--precond-reuse", type=int, default=None,
                    help="steps served by one Galerkin product of the multigrid coarse levels")
    ap.add_argument("--autotune", type=int, default=1,
                    help="1: the library times its Jacobian kernel configurations at the first "
                         "assembly of each context (a warm-up step) and keeps the fastest")
    return ap.parse_args()


def solver_opts(args):
    """Preconditioner options given on the command line (library defaults otherwise)."""
    o = {"autotune": int(args.autotune)}
    if args.schur_order is not None:
        o["schur_order"] = args.schur_order
    if args.mg_sweeps is not None:
        o["mg_sweeps"] = args.mg_sweeps
    if args.mg_omega is not None:
        o["mg_omega"] = args.mg_omega
    if args.precond_reuse is not None:
        o["precond_reuse"] = args.precond_reuse
    return o


def make_workload(name):
    """A named configuration; 'block3d-jit:AxBxC' is the 3D block on A x B x C
    cells with its points jittered (the small case of the profiles)."""
    from paper_1905_00671_gb300 import inputs as I

    if name.startswith("block3d-jit:"):
        body = tuple(int(x) for x in name.split(":", 1)[1].split("x"))
        return I.jittered(I.consolidation_block(body=body), seed=5, frac=0.15, shuffle=False, logk_spread=0.0)
    if name == "footing":
        return I.strip_footing()
    if name == "terzaghi":
        return I.terzaghi_column()
    if name == "block3d":
        return I.consolidation_block()
    if name == "slope":
        return I.slope_3d()
    if name == "harmonic":
        return I.harmonic_footing()
    raise SystemExit(f"unknown workload {name}")


def workload_label(w):
    if w.name.startswith("slope-") and not w.name.startswith("slope-piece"):
        return f"{w.name}: 3D slope under gravity (30 degrees, water table at mid-height)"
    if w.name.startswith("footing-"):
        return f"{w.name}: 2D plane-strain dynamic strip footing"
    return w.name


def workload_config(w):
    return {"workload": workload_label(w),
            "grid_cells": list(w.ncell[:w.dim]), "h_m": w.h, "points": w.n,
            "shape": "GIMP" if w.shape == 1 else "original MPM",
            "scheme": "Newmark" if w.dynamic else "quasi-static implicit Euler",
            "dt_s": w.dt, "newton_rtol": 1e-8, "krylov_rtol": 1e-8,
            "l2": "flushed between timed steps (512 MiB write)"}


# --------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) >= 9:
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------- helpers
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


KERNEL_SOURCE = {"k_bsr_spmv": "mpm_solver.cu", "k_jacobian": "mpm_assemble.cu"}


def kernel_source_hash(kernel):
    """Hash of the sources a kernel is built from (its file and the shared
    header): a committed ncu figure counts only for the source it was taken on."""
    h = hashlib.sha256()
    for f in (KERNEL_SOURCE[kernel], "mpm_internal.cuh"):
        with open(os.path.join(ROOT, "paper_1905_00671_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` on `workload` (its name) from the
    committed ncu summary, if the summary was taken on that workload and on the
    current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    src = kernel_source_hash(kernel)
    for ln in lines:
        parts = ln.split()
        if (len(parts) >= 5 and not ln.startswith("#") and parts[0] == kernel and parts[1] == src
                and parts[2] == workload):
            return float(parts[4])
    return None


# Algorithmic FP64 flops of the Jacobian assembly (Eqs. jacobian-system-
# stabilized-ppp, newmark-linearization as evaluated per point), counted by
# hand (an FMA is 2 flops) from the staged form: the per-(point, node) vectors
# (g_a = F^-T grad S_a, S_a, S_a - S0_a, tau' g_a, g_a.w, g_a.grad v) and their
# products with the point's coefficients of the block terms are formed once per
# node (G per (point, node)); the blocks (a, b) and (b, a) are assembled as one
# symmetric pair (A and C once, B1 and B2 for both), so a (point, a, b) term
# with a != b costs F_pair per unordered pair and a diagonal term F_diag:
#   F_diag = 2 (2d^2 + 6d + 1) + 1       (+ 2 (d + 1), Newmark)
#   F_pair = F_diag + 6d                 (+ 2 (2d + 1) over F_pair's QS value, Newmark)
# (the pair adds the d + 2d FMAs of the second block's B1 and B2; the grad p
# part of B2, (p7 g_a.g_b) grad p, is accumulated once for both blocks, and the
# d = h_a.g_b part of A's diagonal into one sum subtracted once per pair).
# {(dim, dynamic): (F_pair, F_diag, G)}.
JAC_FLOPS = {(2, False): (55, 43, 43), (2, True): (65, 49, 52), (3, False): (93, 75, 77),
             (3, True): (107, 83, 96)}
# Hencky elasticity adds, per pair and per diagonal term, the d^3 FMAs of
# sum_l U_a,ikl g_b,l and, per (point, node), the staged U of its spectral
# tangent: gh_A = g.n_A (d^2 FMAs), w_Akl = kappa_A gh_A n_Ak n_Al + sum_{B != A}
# theta_AB gh_B (n_Ak n_Bl + n_Bk n_Al) (3 + 6 (d - 1) flops each, d^3 of
# them) and U_ikl = -cs (1 + cv) (lambda g_i delta_kl + sum_A n_Ai w_Akl)
# (2 d + 1 flops each, d^3 of them).  {dim: (per pair or diagonal term, G)}
JAC_FLOPS_HENCKY = {2: (16, 120), 3: (54, 612)}


def jacobian_flops(dim, dynamic, hencky, terms, point_nodes):
    """Algorithmic flops of one assembly: terms = sum over points of n_p^2
    (ordered (a, b) pairs of the point's active support nodes), point_nodes =
    sum of n_p; (terms - point_nodes) / 2 unordered pairs a != b and
    point_nodes diagonal terms."""
    fp, fd, g = JAC_FLOPS[(dim, dynamic)]
    if hencky:
        h, gh = JAC_FLOPS_HENCKY[dim]
        fp, fd, g = fp + h, fd + h, g + gh
    return fp * (terms - point_nodes) / 2 + (fd + g) * point_nodes
# FP64 peak from unit counts and clocks: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2070 MHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2070e6 / 1e12


def spmv_bytes(nnodes, nnzb, nb, word=8):
    """Algorithmic bytes of one block-CSR SpMV: values + column indices + row
    pointers, x read once, y written once (word = 8 for FP64, 4 for FP32)."""
    return nnzb * (nb * nb * word + 4) + (nnodes + 1) * 4 + 2 * nnodes * nb * word


# FP32 peak from unit counts and clocks: 152 SMs x 128 FP32 FMA lanes x 2 flop x 2070 MHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2070e6 / 1e12


def jacobian32_bytes(n, nnzb, nnodes, dim, dynamic, hencky=False):
    """Algorithmic bytes of one FP32 Jacobian assembly: every point's data the
    tangent needs read once (dF^-1, tau', grad p - rho_f (g - a), grad p, nine
    scalar coefficients, the 1D basis S, dS, S0 in 4 slots per axis; Newmark:
    the mass and grad v; Hencky: the principal directions, kappa_A and
    theta_AB), the sparsity read once (coupling mask, row pointers, block
    columns) and every (d+1)^2 block written once, 4-byte words."""
    per_point = 2 * dim * dim + 2 * dim + 9 + 3 * dim * 4 + (1 + dim * dim if dynamic else 0)
    if hencky:
        per_point += dim * dim + dim + dim * (dim - 1) // 2
    nb = dim + 1
    return 4 * per_point * n + nnzb * (nb * nb * 4 + 4) + nnodes * (6 * 8 + 4)


def nvtx_push(name):
    try:
        import torch
        torch.cuda.nvtx.range_push(name)
    except Exception:
        pass


def nvtx_pop():
    try:
        import torch
        torch.cuda.nvtx.range_pop()
    except Exception:
        pass


# --------------------------------------------------------------- our arm
def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_1905_00671_gb300 import build as B
    from paper_1905_00671_gb300 import mpm

    torch.cuda.set_device(local_rank)
    if not B.up_to_date():
        B.build()
    mpm.load()
    w = make_workload(args.workload)
    # a dedicated stream: the library launches on it (CUDA-graph capture needs a
    # non-default stream) and the timing events are recorded on it
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    prof_bits = 0
    for k in args.profile.split(","):
        if k and k != "none":
            prof_bits |= 1 << mpm.PROF[k]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # ---- device-resident throughput
    sopts = solver_opts(args)
    sim = mpm.Simulation(w, stream=stream.cuda_stream, profile=prof_bits, precond_lag=args.precond_lag, **sopts)
    for _ in range(args.warmup):
        sim.step(resident=True)
    barrier()
    clocks = ClockSampler(local_rank)
    clocks.start()
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    newton = krylov = launches = 0
    prof_ms = {k: 0.0 for k in mpm.PROF}
    prof_n = {k: 0 for k in mpm.PROF}
    nnzb = []
    terms = []
    for i in range(args.steps):
        flush.zero_()                       # evict L2 between timed steps (not timed)
        nvtx_push("timed")                  # lets a profiler select the timed steps
        ev0[i].record(stream)
        st = sim.step(resident=True)
        ev1[i].record(stream)
        nvtx_pop()
        newton += st["newton_iters"]
        krylov += st["krylov_total"]
        launches += st["kernel_launches"]
        nnzb.append(st["nnzb"])
        terms.append((st["jac_terms"], st["jac_point_nodes"]))
        jac_cfg = {"config": st["jac_config"][0], "tuned": st["jac_tuned"][0],
                   "candidates_ms": [round(x, 3) for x in st["jac_tune_ms"][0]]}
        for k in mpm.PROF:
            prof_ms[k] += st["prof_ms"][k]
            prof_n[k] += st["prof_launches"][k]
    barrier()
    clk = clocks.stop()
    step_ms = sum(a.elapsed_time(b) for a, b in zip(ev0, ev1))
    total_ms = max_over_ranks(step_ms, world, "cuda")
    sim.close()

    # ---- per-class breakdown: events around every kernel class cost time and
    # break the overlap of dependent launches, so they run in a separate pass
    # of a few steps after the timed ones (same workload, fresh context)
    bd_ms = {k: 0.0 for k in mpm.PROF}
    bd_n = {k: 0 for k in mpm.PROF}
    bd_nnzb = []
    if args.breakdown_steps > 0:
        all_bits = sum(1 << v for v in mpm.PROF.values())
        sim_b = mpm.Simulation(w, stream=stream.cuda_stream, profile=all_bits, precond_lag=args.precond_lag,
                               **sopts)
        sim_b.step(resident=True)
        for _ in range(args.breakdown_steps):
            flush.zero_()
            st = sim_b.step(resident=True)
            bd_nnzb.append(st["nnzb"])
            for k in mpm.PROF:
                bd_ms[k] += st["prof_ms"][k]
                bd_n[k] += st["prof_launches"][k]
        sim_b.close()
        barrier()

    final64 = None

    # ---- mixed precision (FP32 Jacobian / preconditioner / Krylov in the FP64
    # Newton loop): same steps, same timing rules, error against the FP64 run
    mixed = None
    if not args.no_mixed:
        sim_m = mpm.Simulation(w, stream=stream.cuda_stream, precision=mpm.MPM_MIXED,
                               newton_max=60, profile=prof_bits, precond_lag=args.precond_lag, **sopts)
        sim_r = mpm.Simulation(w, stream=stream.cuda_stream, **sopts)   # FP64 twin for the error
        for _ in range(args.warmup):
            sim_m.step(resident=True)
            sim_r.step(resident=True)
        barrier()
        ms = 0.0
        newton_m = krylov_m = 0
        prof_m = {k: 0.0 for k in mpm.PROF}
        prof_nm = {k: 0 for k in mpm.PROF}
        terms_m, nnzb_m = [], []
        for i in range(args.steps):
            flush.zero_()
            nvtx_push("timed_mixed")
            ev0[i].record(stream)
            st = sim_m.step(resident=True)
            ev1[i].record(stream)
            nvtx_pop()
            newton_m += st["newton_iters"]
            krylov_m += st["krylov_total"]
            jac_cfg_m = {"config": st["jac_config"][1], "tuned": st["jac_tuned"][1],
                         "candidates_ms": [round(x, 3) for x in st["jac_tune_ms"][1]]}
            terms_m.append((st["jac_terms"], st["jac_point_nodes"]))
            nnzb_m.append(st["nnzb"])
            for k in mpm.PROF:
                prof_m[k] += st["prof_ms"][k]
                prof_nm[k] += st["prof_launches"][k]
            sim_r.step(resident=True)
            torch.cuda.synchronize()
            ms += ev0[i].elapsed_time(ev1[i])
        barrier()
        a, b = sim_m.read(("u", "p")), sim_r.read(("u", "p"))
        errs = {k: float(np.abs(a[k] - b[k]).max() / max(np.abs(b[k]).max(), 1e-300)) for k in a}
        ms = max_over_ranks(ms, world, "cuda")
        mixed = {"value": world * w.n * args.steps / (ms * 1e-3), "unit": UNIT,
                 "ms_per_step": ms / args.steps, "dtype": "f32 solve / f64 Newton residual",
                 "newton_iters_per_step": newton_m / args.steps,
                 "krylov_iters_per_step": krylov_m / args.steps,
                 "class_ms_per_step": {k: round(v / args.steps, 3) for k, v in prof_m.items() if v > 0},
                 "rel_error_vs_fp64": errs, "jacobian_kernel": jac_cfg_m}
        sim_m.close()
        sim_r.close()
        # FP32 rooflines: the Jacobian from the live events of the timed steps,
        # the SpMV from a separate pass with events around every class
        peaks_m, peak_src_m = measured_peaks()
        hbm = float(peaks_m["hbm_gbs"])
        roof_m = {}
        if prof_nm["jacobian"] > 0:
            avg_ms = prof_m["jacobian"] / prof_nm["jacobian"]
            nz = sum(nnzb_m) / len(nnzb_m)
            hk = w.model == mpm.MPM_MODEL_HENCKY
            byt = jacobian32_bytes(w.n, nz, w.nnodes, w.dim, w.dynamic, hk)
            fl = sum(jacobian_flops(w.dim, w.dynamic, hk, t, pn) for t, pn in terms_m) / len(terms_m)
            ach = byt / (avg_ms * 1e-3) / 1e9
            roof_m["jacobian"] = {
                "kernel": "k_jacobian_direct" if jac_cfg_m["config"] < 1000 else "k_point_nodes + k_jacobian (FP32)",
                "bound": "hbm", "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(ach / hbm, 4), "algorithmic_bytes": int(byt),
                "avg_launch_us": round(avg_ms * 1e3, 3), "peak_source": peak_src_m + " hbm_gbs",
                "fp32_tflops": round(fl / (avg_ms * 1e-3) / 1e12, 3),
                "fp32_frac": round(fl / (avg_ms * 1e-3) / 1e12 / FP32_PEAK_TFLOPS, 4),
                "fp32_peak_source": "FP32 from unit counts and clocks (152 SMs x 128 lanes x 2 x 2070 MHz)"}
        if args.breakdown_steps > 0:
            all_bits = sum(1 << v for v in mpm.PROF.values())
            sim_mb = mpm.Simulation(w, stream=stream.cuda_stream, precision=mpm.MPM_MIXED, newton_max=60,
                                    profile=all_bits, precond_lag=args.precond_lag, **sopts)
            sim_mb.step(resident=True)
            bdm, bdn, bnz = {k: 0.0 for k in mpm.PROF}, {k: 0 for k in mpm.PROF}, []
            for _ in range(args.breakdown_steps):
                flush.zero_()
                st = sim_mb.step(resident=True)
                bnz.append(st["nnzb"])
                for k in mpm.PROF:
                    bdm[k] += st["prof_ms"][k]
                    bdn[k] += st["prof_launches"][k]
            sim_mb.close()
            if bdn["spmv"] > 0:
                nb = w.dim + 1
                byt = spmv_bytes(w.nnodes, sum(bnz) / len(bnz), nb, word=4)
                avg_ms = bdm["spmv"] / bdn["spmv"]
                ach = byt / (avg_ms * 1e-3) / 1e9
                roof_m["spmv"] = {"kernel": "k_bsr_spmv (FP32)", "bound": "hbm", "achieved": round(ach, 1),
                                  "peak": hbm, "unit": "GB/s", "frac": round(ach / hbm, 4),
                                  "algorithmic_bytes": int(byt), "avg_launch_us": round(avg_ms * 1e3, 3),
                                  "peak_source": peak_src_m + " hbm_gbs"}
            mixed["class_ms_per_step_breakdown"] = {k: round(v / args.breakdown_steps, 3)
                                                    for k, v in bdm.items() if bdn[k] > 0}
        mixed["roofline"] = roof_m

    # ---- end to end through the C-ABI with host buffers
    e2e = None
    if not args.no_e2e:
        n, d = w.n, w.dim
        pin = lambda shape: torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()
        trac_h = pin((max(w.n_surf, 1), d))
        outs = {"x": pin((n, d)), "u": pin((n, d)), "p": pin(n)}
        sim2 = mpm.Simulation(w, stream=stream.cuda_stream, **sopts)
        for _ in range(args.warmup):
            trac_h[:w.n_surf] = w.traction(sim2.t + w.dt)
            sim2.step(traction=trac_h[:w.n_surf])
        barrier()
        e2e_s = 0.0
        import ctypes as C
        o = mpm.mpm_particles_out(x=outs["x"].ctypes.data_as(C.c_void_p),
                                  u=outs["u"].ctypes.data_as(C.c_void_p),
                                  p=outs["p"].ctypes.data_as(C.c_void_p))
        for i in range(args.steps):
            flush.zero_()
            trac_h[:w.n_surf] = w.traction(sim2.t + w.dt)   # the step's input, in pinned memory
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sim2.step(traction=trac_h[:w.n_surf])          # H2D copy of the loads inside
            rc = sim2.lib.mpm_read(sim2.ctx, C.byref(o))    # D2H of the step's result
            e2e_s += time.perf_counter() - t0
            if rc != 0:
                raise RuntimeError("mpm_read failed")
        barrier()
        sim2.close()
        e2e_total = max_over_ranks(e2e_s, world, "cuda")
        e2e = {"value": world * w.n * args.steps / e2e_total, "unit": UNIT,
               "h2d_bytes_per_step": int(w.n_surf * d * 8),
               "d2h_bytes_per_step": int(n * (2 * d + 1) * 8),
               "steps_per_s": world * args.steps / e2e_total}

    # ---- roofline of the dominant kernel (the Jacobian assembly: the largest
    # single kernel of the step, bound by GB300's FP64 pipe) with the SpMV
    # beside it (HBM and FP64 fractions); live CUDA-event times on the
    # library's stream
    peaks, peak_src = measured_peaks()
    shares = {k: bd_ms[k] for k in bd_ms if bd_n[k] > 0}
    dominant = max(shares, key=shares.get) if shares else None
    nbd = max(args.breakdown_steps, 1)
    roofline = None
    if prof_n.get("jacobian", 0) > 0:
        hk = w.model == mpm.MPM_MODEL_HENCKY
        flops = sum(jacobian_flops(w.dim, w.dynamic, hk, t, pn) for t, pn in terms) / len(terms)
        avg_ms = prof_ms["jacobian"] / prof_n["jacobian"]
        ach = flops / (avg_ms * 1e-3) / 1e12
        roofline = {"kernel": "k_jacobian", "bound": "alu", "achieved": round(ach, 4),
                    "peak": round(FP64_PEAK_TFLOPS, 4), "unit": "TFLOP/s",
                    "frac": round(ach / FP64_PEAK_TFLOPS, 4),
                    "traffic": ncu_traffic("k_jacobian", w.name),
                    "peak_source": "FP64 from unit counts and clocks (152 SMs x 2 FMA/clk x 2070 MHz)",
                    "algorithmic_flops": int(flops), "jac_terms": int(sum(t for t, _ in terms) / len(terms)),
                    "avg_launch_us": round(avg_ms * 1e3, 3),
                    "dominant_class": dominant,
                    "class_ms_per_step": {k: round(v / nbd, 3) for k, v in shares.items()},
                    "class_launches_per_step": {k: bd_n[k] / nbd for k in shares},
                    "class_source": f"separate pass of {args.breakdown_steps} steps with events "
                                    "around every kernel class"}
    if "spmv" in shares and bd_n["spmv"] > 0:
        nb = w.dim + 1
        avg_nnzb = sum(bd_nnzb) / len(bd_nnzb)
        bytes_launch = spmv_bytes(w.nnodes, avg_nnzb, nb)
        avg_ms = bd_ms["spmv"] / bd_n["spmv"]
        ach = bytes_launch / (avg_ms * 1e-3) / 1e9
        peak = float(peaks["hbm_gbs"])
        fl = 2 * avg_nnzb * nb * nb / (avg_ms * 1e-3) / 1e12
        # one FMA per stored FP64 value: on GB300 the FP64 pipe (2 FMA/clk/SM)
        # binds before HBM does (ncu: FP64 pipe ~87% busy at ~50% of DRAM
        # peak), so the bound is the ALU; the HBM fraction is kept beside it
        spmv = {"kernel": "k_bsr_spmv", "bound": "alu", "achieved": round(fl, 4),
                "peak": round(FP64_PEAK_TFLOPS, 4), "unit": "TFLOP/s", "frac": round(fl / FP64_PEAK_TFLOPS, 4),
                "traffic": ncu_traffic("k_bsr_spmv", w.name),
                "peak_source": "FP64 from unit counts and clocks (152 SMs x 2 FMA/clk x 2070 MHz)",
                "algorithmic_flops": int(2 * avg_nnzb * nb * nb),
                "algorithmic_bytes": int(bytes_launch), "avg_launch_us": round(avg_ms * 1e3, 3),
                "hbm_gbs": round(ach, 1), "hbm_peak_gbs": peak, "hbm_frac": round(ach / peak, 4),
                "hbm_peak_source": peak_src + " hbm_gbs"}
        if roofline is None:
            roofline = spmv
        else:
            roofline["spmv"] = spmv

    value = world * w.n * args.steps / (total_ms * 1e-3)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
            "config": dict(workload_config(w), parallelism=f"replicas x{world}"),
            "steps_per_s": world * args.steps / (total_ms * 1e-3),
            "newton_iters_per_step": newton / args.steps, "krylov_iters_per_step": krylov / args.steps,
            "gpu_launches": launches, "clocks": clk, "roofline": roofline, "e2e": e2e,
            "mixed": mixed}
    line["jacobian_kernel"] = jac_cfg   # threads per block + 1000 if staged; tuned = chosen by timing
    if sopts:
        line["solver_options"] = sopts
    return line, w


# --------------------------------------------------------------- oracle
# largest workload the oracle steps whole in bounded time (a direct sparse solve)
CPU_BASELINE_MAX_POINTS = 100_000
# the slope piece: 24 x 16 x 12 cells at the same h, the slope geometry (toe,
# crest, water table) scaled by 24/128 so that the 30 degree face is kept
SLOPE_PIECE_CELLS = (24, 16, 12)


def oracle_piece(w):
    """(workload, description) of the bounded piece of workload `w` that the
    oracle legs time: the workload itself when it is small, else a piece of
    the same kind at the same h, material, loading and time step."""
    from paper_1905_00671_gb300 import inputs as I

    if w.name.startswith("slope-"):
        s = 128.0 / SLOPE_PIECE_CELLS[0]
        nc = SLOPE_PIECE_CELLS
        p = I.slope_3d(ncell=nc, z_toe=1.2 / s, z_crest=5.2 / s, x_toe=2.9 / s,
                       name="slope-piece-{}x{}x{}".format(*nc))
        return p, (f"a {nc[0]}x{nc[1]}x{nc[2]}-cell, {p.n}-point piece of the slope (same h, "
                   "material, gravity, dt and 30 degree face; toe, crest and water table scaled "
                   f"by {nc[0]}/128)")
    if w.name.startswith("block-") and w.n > CPU_BASELINE_MAX_POINTS:
        p = I.consolidation_block(body=(16, 16, 8), name="block-piece-16x16x8")
        return p, f"a 16x16x8-cell, {p.n}-point piece of the 3D block (same h, material, load, dt)"
    if w.name.startswith("footing-") and w.n > 40_000:
        p = I.strip_footing(body=(140, 70), seed=2)
        return p, (f"a 140x70-cell, {p.n}-point piece of the footing (same h, material, load, dt)")
    return w, f"the full {w.n}-point {w.name}"


def run_cpu_baseline(w, min_seconds=10.0, max_steps=3):
    """The oracle as it stands on one host core: consecutive load steps from
    t = 0 of the full workload (when small) or of its piece, until about
    min_seconds of CPU work (at most max_steps steps)."""
    from oracle import oracle as O

    if w.n <= CPU_BASELINE_MAX_POINTS:
        piece, desc = w, f"the full {w.n}-point {w.name}"
        max_steps = 1
    else:
        piece, desc = oracle_piece(w)
    o = O.Oracle(piece, newton_rtol=1e-8)
    sec, steps, its = 0.0, 0, []
    while steps < max_steps and (steps == 0 or sec < min_seconds):
        t0 = time.perf_counter()
        info = o.step()
        sec += time.perf_counter() - t0
        steps += 1
        its.append(info.newton_iters)
    return {"value": piece.n * steps / sec, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{steps} oracle load step(s) from t = 0 ({sum(its)} Newton iterations) of "
                      f"{desc}, C loops + SuperLU, single thread",
            "seconds": round(sec, 2)}


def run_reference(args, rank, world):
    """The reference arm: the oracle (this project's reference is a paper; its
    CPU restatement is the oracle) on one host core, each step one oracle load
    step of the workload's bounded piece, stepped on from t = 0; the warm-up
    steps are stepped but not timed."""
    if rank != 0:
        return None
    from oracle import oracle as O

    w = make_workload(args.workload)
    piece, desc = oracle_piece(w)
    o = O.Oracle(piece, newton_rtol=1e-8)
    secs = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        o.step()
        if i >= args.warmup:
            secs.append(time.perf_counter() - t0)
    total = sum(secs)
    value = piece.n * args.steps / total
    sample = f"each step: one oracle load step of {desc}, continuing from t = 0"
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded)",
            "config": dict(workload_config(piece), parallelism="cpu", l2="host CPU: not applicable",
                           sample_of=workload_label(w)),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# --------------------------------------------------------------- batched instances
def run_batch(args, rank, world, local_rank):
    """Batched stepping of many independent instances (256 uneven 2D problems,
    Terzaghi-type and footing-type alternating): the two kinds (different
    shape functions, time scheme and step) are two batched contexts; one timed
    step advances every instance once, in mixed precision and in FP64.  Beside
    it, a sample of the instances stepped one at a time in FP64 (each its own
    context), extrapolated to all instances by kind."""
    import numpy as np
    import torch

    from paper_1905_00671_gb300 import build as B
    from paper_1905_00671_gb300 import inputs as I
    from paper_1905_00671_gb300 import mpm

    torch.cuda.set_device(local_rank)
    if not B.up_to_date():
        B.build()
    mpm.load()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ws = I.batch_instances(count=args.batch_count, seed=5)
    kinds = {"terzaghi": [w for w in ws if w.name.startswith("terzaghi")],
             "footing": [w for w in ws if w.name.startswith("footing")]}
    npts = sum(w.n for w in ws)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    sopts = solver_opts(args)

    def timed(precision):
        bs = [mpm.Batch(v, stream=stream.cuda_stream, precision=precision, newton_max=60, **sopts)
              for v in kinds.values() if v]
        for _ in range(args.warmup):
            for b in bs:
                b.step()
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        ms = 0.0
        newton = []
        launches = 0
        clocks = ClockSampler(local_rank)
        clocks.start()
        for _ in range(args.steps):
            flush.zero_()
            e0.record(stream)
            for b in bs:
                st = b.step()
                newton.append(st["newton_iters"])
                launches += st["kernel_launches"]
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
        clk = clocks.stop()
        out = [b.read(("u", "p")) for b in bs]
        pi = 0 if precision == mpm.MPM_FP64 else 1
        jac = []
        for name, b in zip([k for k, v in kinds.items() if v], bs):
            st = b.stats()
            jac.append({"context": name, "config": st["jac_config"][pi], "tuned": st["jac_tuned"][pi],
                        "candidates_ms": [round(x, 3) for x in st["jac_tune_ms"][pi]]})
        for b in bs:
            b.close()
        info = {"kernel_launches_per_step": launches / args.steps, "jacobian_kernel": jac}
        return max_over_ranks(ms, world, "cuda"), newton, out, clk, info

    ms_mixed, newton_mixed, res_mixed, clk_mixed, info_mixed = timed(mpm.MPM_MIXED)
    ms_fp64, newton_fp64, res_fp64, clk_fp64, info_fp64 = timed(mpm.MPM_FP64)
    # one at a time, FP64: a sample of each kind, same number of steps
    sample = {k: v[:args.batch_sample] for k, v in kinds.items() if v}
    per_kind_ms = {}
    errs = []
    for ki, (k, v) in enumerate(sample.items()):
        tot = 0.0
        for j, w in enumerate(v):
            sim = mpm.Simulation(w, stream=stream.cuda_stream, newton_max=60)
            for _ in range(args.warmup):
                sim.step(resident=True)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            for _ in range(args.steps):
                e0.record(stream)
                sim.step(resident=True)
                e1.record(stream)
                torch.cuda.synchronize()
                tot += e0.elapsed_time(e1)
            ref = sim.read(("u", "p"))
            kidx = list(kinds).index(k)
            got = res_mixed[kidx][j]
            errs.append(max(float(np.abs(got[f] - ref[f]).max() / max(np.abs(ref[f]).max(), 1e-300))
                            for f in ("u", "p")))
            sim.close()
        per_kind_ms[k] = tot / len(v)          # per instance, all timed steps
    one_ms = max_over_ranks(sum(per_kind_ms[k] * len(kinds[k]) for k in per_kind_ms), world, "cuda")
    # every rank steps its own replica of the batch: whole-job points over the slowest rank's time
    value = world * npts * args.steps / (ms_mixed * 1e-3)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_mixed / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 solve / f64 Newton residual",
            "data": "synthetic (seeded)",
            "config": {"workload": f"batch-{len(ws)}: independent 2D instances 16-128 x 32-64 cells, "
                                   "Terzaghi-type (original MPM, quasi-static, dt 1 s) and footing-type "
                                   "(GIMP, Newmark, dt 1e-3 s) alternating, 2x2 points per cell",
                       "instances": len(ws), "points": npts, "contexts": len(sample),
                       "l2": "flushed between timed steps (512 MiB write)", "parallelism": f"replicas x{world}"},
            "newton_iters_per_context_step": float(np.mean(newton_mixed)),
            "clocks": clk_mixed,
            "gpu_launches": int(info_mixed["kernel_launches_per_step"] * args.steps),
            "kernel_launches_per_step": info_mixed["kernel_launches_per_step"],
            "jacobian_kernel": info_mixed["jacobian_kernel"],
            "solver_options": sopts,
            "fp64_batched": {"value": world * npts * args.steps / (ms_fp64 * 1e-3), "unit": UNIT,
                             "ms_per_step": ms_fp64 / args.steps, "clocks": clk_fp64,
                             "newton_iters_per_context_step": float(np.mean(newton_fp64)),
                             "kernel_launches_per_step": info_fp64["kernel_launches_per_step"],
                             "jacobian_kernel": info_fp64["jacobian_kernel"]},
            "one_by_one_fp64": {"value": world * npts * args.steps / (one_ms * 1e-3), "unit": UNIT,
                                "ms_per_step": one_ms / args.steps,
                                "sample": f"{sum(len(v) for v in sample.values())} instances stepped alone "
                                          "(first of each kind), extrapolated per kind to all instances",
                                "max_rel_error_of_batched_mixed": max(errs) if errs else None}}
    return line


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line), flush=True)
        return
    if world > 1:
        import torch

        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    if args.workload == "batch":
        line = run_batch(args, rank, world, local_rank)
        if rank == 0:
            print(json.dumps(line), flush=True)
        return
    line, w = run_ours(args, rank, world, local_rank)
    if rank == 0:
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = run_cpu_baseline(w)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch

        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
