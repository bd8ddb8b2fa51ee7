"""Benchmark of the Schwarz neural-operator FGMRES solve (one JSON line).

Workload: a synthetic 4096 x 4096 freeform-dielectric problem (eps in
{1, 12.25}, lambda/dx = 30, 20-cell PML, unit line source at the centre).
Preconditioner: the two-level Schwarz sweep (restriction, batched neural
local solves, restricted prolongation, Robin traces, Galerkin coarse solve
and correction).

* A step is one outer FGMRES(60) iteration of the whole hot path:
  preconditioner, stencil matvec, CGS orthogonalisation, FP64 Hessenberg
  update.  `value` = Mcell-iterations per second = cells x steps / device
  time of K steps after W warm-up steps.
* `time_to_1e-6`: full solves from a zero initial guess to true relative
  residual 1e-6 (median of repeats, CUDA events, set-up excluded and
  reported separately), for the Schwarz neural-operator FGMRES and for
  Jacobi-GMRES(60) on the same GPU; Jacobi-GMRES runs under a time cap and
  reports the residual it reached.
* `--impl reference` times the FP64 CPU oracle's FGMRES (as it stands) on a
  bounded sample of the same recipe.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to rel-resid 1e-6 @4096^2: Schwarz-NO FGMRES vs plain GMRES; Mcell-it/s"
HBM_FALLBACK = 6800.0
BF16_FALLBACK = 1900.0


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", HBM_FALLBACK), d.get("bf16_tflops", BF16_FALLBACK), \
            d.get("bf16_tflops_sustained", BF16_FALLBACK), "measured"
    return HBM_FALLBACK, BF16_FALLBACK, 1700.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, out):
        self.out = out
        self.p = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.out, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(int(os.environ.get("LOCAL_RANK", "0")))],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
            self.f.close()

    def summary(self):
        if not self.p or not os.path.exists(self.out):
            return None
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.out):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# Algorithmic HBM bytes per window (80 x 80, 6400 pixels) of each neural-
# operator stage: what it must read and write once (bf16 activations of 32
# channels = 64 B per pixel, complex64 fields = 8 B per cell).
WIN_BYTES = {
    "nno_pack": 6400 * 8,                     # residual in (window RMS)
    "nno_lift": 6400 * (8 + 4) + 160 * 512 * 2,  # residual + eps in, block 0's T1 out (X is not stored)
    "nno_dft_x": 6400 * 64 + 160 * 512 * 2,   # activation in, half-spectrum along x out
    "nno_dft_y": 160 * 512 * 2 + 512 * 64 * 2,
    "nno_mix": 512 * 64 * 2 * 2,              # spectrum in and out (weights amortised)
    "nno_idft_y": 512 * 64 * 2 + 80 * 32 * 32 * 2,
    "nno_idft_x_mix_act": 6400 * 64 * 2 + 80 * 32 * 32 * 2,   # + T1 out in blocks 0..2 (below)
    "nno_proj": 6400 * 64 + 4096 * 8,         # activation in, core field out
}
G5_T1_BYTES = 160 * 512 * 2                   # next block's half-spectrum, written by blocks 0..2
# With per-window inputs (the local NN-FGMRES steps) the window RMS pass also
# writes the 16 BF16 input channels per pixel as tiles, and the lift and
# block 0 read those instead of gathering the residual and eps; the
# projection writes whole windows instead of cores.
WIN_BYTES_PACKED = {"nno_pack": 6400 * (8 + 4 + 32), "nno_lift": 6400 * 32 + 160 * 512 * 2,
                    "nno_proj": 6400 * 64 + 6400 * 8}  # the local steps' output is the whole window
BLOCK0_INPUT_BYTES = {False: 6400 * 12, True: 6400 * 32}
# DRAM bytes (read + write) per window of one launch of a neural stage, from
# one-kernel ncu captures of a smaller case of the same recipe, scaled to a
# launch by the number of windows it processes (TRAFFIC_SAMPLE names the
# case).  Empty while no capture of the current kernels exists.
TRAFFIC_SAMPLE = "freeform 2048^2 (1024 windows), one kernel per capture, caches flushed"
# Keyed by whether the inputs were packed (per-window inputs: the local
# NN-FGMRES steps); None where no capture of the current kernels exists.
SMALL_CASE_TRAFFIC = {
    "nno_proj": {False: 452800, True: None},            # (global output; the local steps write whole windows)
    "nno_idft_x_mix_act": {False: None, True: 919329},  # block 0 (881,333) and blocks 1-3 (988,546 /
                                                        # 985,683 / 821,754, the last writes no T1)
    "nno_lift": {False: None, True: 327850},            # packed tiles in, T1 out (partly still in L2)
    "nno_pack": {False: None, True: 258716},            # residual + eps in, packed tiles out (partly in L2)
}
# Useful FLOPs per window of each stage (padding excluded).
NNO_FLOP_PER_WIN = {
    "nno_lift": 6400 * 32 * 15 * 2 + 2560 * 32 * 80 * 2, "nno_dft_x": 2560 * 32 * 80 * 2, "nno_dft_y": 512 * 64 * 160 * 2,
    "nno_mix": 512 * 64 * 64 * 2, "nno_idft_y": 512 * 160 * 64 * 2, "nno_idft_x_mix_act": 80 * 80 * 32 * 64 * 2,
    "nno_proj": 6400 * (128 * 32 + 2 * 128) * 2,
}
KERNEL_NAMES = {"stencil": "stencil_c64", "cgs_dots": "cgs_dots_kernel", "cgs_update": "cgs_update_kernel",
                "residual64": "residual64", "nno_pack": "rho_kernel (window RMS)",
                "nno_lift": "g5_kernel<lift> (input channels + lift + block-0 DFT-x)",
                "nno_dft_x": "gemm_kernel<32,80,MN> (G1Op)", "nno_dft_y": "gemm_kernel<64,160,MN> (G2Op; operand tiles by TMA or gather, autotuned)",
                "nno_mix": "g3_kernel (spectral mixing)", "nno_idft_y": "gemm_kernel<160,64> (G4Op, bulk-copied swizzled operand)",
                "nno_idft_x_mix_act": "g5_kernel (block 0) + g5f_kernel (blocks 1-3, inverse DFT-y fused)", "nno_proj": "proj_kernel", "rhs_norm": "residual64 (x = 0)",
                "coarse": "galerkin_rhs + sweep_t/gemv_rows (row sweeps over S_b^-1) + correction_kernel"}


def coarse_bytes_per_apply(N, k):
    """Coarse solve and correction, per application on an n x n grid: both
    row sweeps stream every inverted Schur complement (complex half:
    2 (n/64) D^2 x 4 B, D = (n/64) k), the correction reads every basis
    field's core (complex half, n_win k 4096 x 4 B) and updates the field
    (16 B per cell), the right-hand side reads the trial vectors
    (n_win k 320 x 8 B)."""
    nw1 = int(round((N ** 0.5) / 64))
    D = nw1 * k
    nc = nw1 * nw1 * k
    return 2.0 * nw1 * D * D * 4 + nc * 4096 * 4 + 16.0 * N + nc * 320 * 8


def algorithmic_bytes(cls, launches, N, steps, k=0, coarse_launches_per_apply=0, packed=False):
    """Bytes the kernel class must move over the timed region."""
    nwin = N // 4096
    if cls == "coarse":
        if not k or not coarse_launches_per_apply:
            return None
        return coarse_bytes_per_apply(N, k) * (launches / coarse_launches_per_apply)
    if cls == "stencil":
        return 20.0 * N * launches
    if cls in ("cgs_dots", "cgs_update"):
        js = [s % RESTART for s in range(steps)]
        extra = 8 if cls == "cgs_dots" else 16
        return float(sum((8 * (j + 1) + extra) * N for j in js))
    if cls == "residual64":
        return 36.0 * N * launches
    if cls == "rhs_norm":
        return 16.0 * N * launches
    if cls in WIN_BYTES:
        table = WIN_BYTES_PACKED if packed and cls in WIN_BYTES_PACKED else WIN_BYTES
        per = table[cls] * nwin + (512 * 64 * 64 * 2 if cls == "nno_mix" else 0)
        extra = 0
        if cls == "nno_idft_x_mix_act":  # blocks 0..2 write T1; block 0 reads the packed inputs, not X;
            # blocks 1..3 compute T3 themselves from the mixed spectrum (65,536 B / window)
            extra = (G5_T1_BYTES * 3 - (6400 * 64 - BLOCK0_INPUT_BYTES[packed])
                     - 3 * (80 * 32 * 32 * 2 - 512 * 64 * 2)) * nwin * (launches // 4)
        return float(per) * launches + extra
    return None


TRAINED = os.path.join(ROOT, "paper_2509_03622_gb300", "weights", "nno_trained.npy")
# Coarse basis vectors per window and NN-FGMRES steps per local solve of the
# bench's two-level preconditioner (Galerkin coarse space; 64 plane-wave
# trials per window are what the binary eps {1, 12.25} medium needs).
K_COARSE_DEFAULT = 64
INNER_DEFAULT = 2
# FGMRES restart of both arms: on the 4096^2 workload both stall near relres
# 1e-2, and a restart of 60 lowers that plateau for both (1.30e-2 / 1.31e-2
# against 1.75e-2 / 1.77e-2 at 30); the Krylov space then holds 121 vectors
# (16 GB at 4096^2).
RESTART = 60


def load_weights(path=None):
    """Trained FNO blob if available, else the seeded initialisation."""
    import numpy as np
    from paper_2509_03622_gb300 import workloads as wl
    p = path or (TRAINED if os.path.exists(TRAINED) else None)
    if p:
        return np.load(p), os.path.relpath(p, ROOT)
    return wl.pack_weights(wl.nno_weights(0)), "seeded init (seed 0)"


def max_over_ranks(x: float, world: int, device) -> float:
    """The job's time is its slowest rank's: MAX all-reduce of a per-rank float."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, cells: int, steps: int, seconds: float) -> float:
    """Whole-job Mcell-iterations/s: every rank solves its own replica of `cells`."""
    return world * cells * steps / seconds / 1e6


def make_problem(n, seed_off=0):
    from paper_2509_03622_gb300 import workloads as wl
    lam = 1.55e-6
    dx = lam / 30
    eps = wl.freeform_eps(n, n, seed=2000 + n + seed_off)
    J = wl.point_source(n, n)
    return eps, J, dx, lam


def cpu_oracle_rate(n_sample, iters, precond, weights=None, k_coarse=0, inner=0, budget_s=None, ritz_tol=0.0):
    """Mcell-it/s of the FP64 oracle FGMRES (as it stands) on an n_sample^2
    grid of the same recipe, `iters` Arnoldi steps (with budget_s, at most
    as many as fit in about that many seconds after a 2-step probe)."""
    from oracle import fdfd as OF, krylov as OK
    eps, J, dx, lam = make_problem(n_sample)
    t0 = time.perf_counter()
    A = OF.assemble_operator(eps, dx, lam, 20)
    b = OF.source_rhs(J, dx, lam)
    if precond == "jacobi":
        d = A.diagonal()
        M = lambda v: v / d
    else:
        from oracle import schwarz as OS
        M = OS.Schwarz(eps, dx, lam, 20, weights=weights, k_coarse=k_coarse, inner=inner,
                       ritz_tol=ritz_tol if k_coarse > 0 else 0.0)
    t1 = time.perf_counter()
    if budget_s:
        OK.fgmres(lambda v: A @ v, b, precond=M, restart=RESTART, tol=1e-14, max_iters=2)
        per = (time.perf_counter() - t1) / 2
        iters = int(max(2, min(iters, budget_s / max(per, 1e-6))))
        t1 = time.perf_counter()
    _, info = OK.fgmres(lambda v: A @ v, b, precond=M, restart=RESTART, tol=1e-14, max_iters=iters)
    t2 = time.perf_counter()
    iters = info["iters"]
    return n_sample * n_sample * iters / (t2 - t1) / 1e6, t2 - t1, iters


def workload_name(n, precond):
    return (f"freeform{n}: {n}x{n} grid, lambda/dx=30, eps {{1,12.25}}, npml 20, "
            f"{'two-level Schwarz-NNO FGMRES' if precond == 'schwarz' else 'Jacobi-GMRES'}({RESTART})")


def design_bench(iters, blob, dev):
    """Inverse-design iterations on the three-port demultiplexer (512^2,
    200 x 200 design square, wavelengths 1.50 / 1.55 / 1.60 um routed to the
    three output guides): density -> filter/projection -> forward solve per
    wavelength -> mode overlaps -> adjoint solves -> dF/drho -> Adam step.
    The figure of merit is the sum of |overlap|^2 with a Gaussian profile
    of each output guide; every solve runs to relres 1e-6 with the
    two-level preconditioner."""
    import numpy as np
    import torch
    from paper_2509_03622_gb300 import fdfd as F
    from paper_2509_03622_gb300 import workloads as wl
    from paper_2509_03622_gb300.autograd import fdfd_field, mode_overlap, last_stats
    from paper_2509_03622_gb300.design import Adam, Design, density_to_eps
    n, dx = 512, 1.55e-6 / 30
    base, mask, src_x, yin, port_x, port_rows = wl.demux_layout(n)
    ys, xs = np.nonzero(mask)
    x0, y0, w, h = int(xs.min()), int(ys.min()), int(xs.max() - xs.min() + 1), int(ys.max() - ys.min() + 1)
    J = np.zeros((n, n), np.complex64)
    J[yin[0] - 4:yin[1] + 4, src_x] = 1.0
    lams = [1.50e-6, 1.55e-6, 1.60e-6]
    solvers = [F.Solver(torch.from_numpy(base).to(dev), dx, lam, npml=20) for lam in lams]
    D = Design(solvers[0], x0, y0, w, h, radius=3.0, beta=8.0)
    rho = torch.full((h, w), 0.5, dtype=torch.float32, device=dev)
    opt = Adam(solvers[0], (h, w), lr=0.005)  # Adam moves every density by about lr in its first step
    Jd, bd = torch.from_numpy(J).to(dev), torch.from_numpy(base).to(dev)
    modes = []
    for (r0, r1) in port_rows:
        yy = np.arange(r0 - 8, r1 + 8)
        modes.append((int(r0 - 8), torch.from_numpy(np.exp(-((yy - (r0 + r1 - 1) / 2) / 4.0) ** 2)
                                                    .astype(np.complex64)).to(dev)))
    foms, relres, adj_relres, f0 = [], [], [], None
    for it in range(iters + 1):  # the first iteration is the warm-up (set-up, graph capture)
        if it == 1:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
        r = rho.clone().requires_grad_(True)
        eps = density_to_eps(D, r, bd)
        fom = 0.0
        for S, (my0, m) in zip(solvers, modes):
            E = fdfd_field(S, eps, Jd, blob, restart=30, max_iters=3000, tol=1e-6, precond=F.PRECOND_SCHWARZ,
                           k_coarse=64, inner=16)
            c = mode_overlap(E, port_x, m, my0, dx)
            fom = fom + c.abs() ** 2
            relres.append(last_stats["forward"]["relres_true"])
        fom.backward()
        adj_relres.append(last_stats["adjoint"]["relres_true"])
        fv = float(fom.detach())
        f0 = f0 or fv
        foms.append(fv / f0)
        opt.step(rho, r.grad, scale=1.0 / f0)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3 / max(iters, 1)
    return {"grid": n, "design": [h, w], "wavelengths": len(lams), "iters": iters, "ms_per_iter": ms,
            "fom_rel": foms, "max_forward_relres": max(relres), "last_adjoint_relres": adj_relres[-1],
            "note": "per iteration: 3 forward + 3 adjoint two-level Schwarz-NO FGMRES(30) solves to relres 1e-6 "
                    "(k = 64, 16 inner steps; coarse set-up redone for each new eps), filter/projection, chain "
                    "rule and Adam on the GPU; FoM relative to the first"}


def oracle_preconditioner(args):
    """The oracle counterpart of the arm's preconditioner configuration."""
    from paper_2509_03622_gb300 import workloads as wl
    if args.precond != "schwarz":
        return None, 0, 0
    blob, _ = load_weights(args.weights)
    kc = args.k_coarse if args.k_coarse >= 0 else K_COARSE_DEFAULT
    return wl.unpack_weights(blob), kc, args.inner


def run_reference(args):
    """The oracle's FGMRES(RESTART) with the arm's preconditioner configuration,
    as it stands, on an n_sample^2 grid of the same recipe: K consecutive
    Arnoldi steps of one solve (so later steps pay for their growing
    Gram-Schmidt), at most as many as fit in about a minute, timed
    together; set-up excluded."""
    n_s = args.cpu_sample
    w, k, inner = oracle_preconditioner(args)
    rate, t, iters = cpu_oracle_rate(n_s, args.steps, args.precond, w, k, inner, budget_s=60.0,
                                     ritz_tol=args.ritz_tol)
    cores = os.cpu_count()
    sample = (f"{n_s}x{n_s} grid of the same freeform recipe and preconditioner configuration "
              f"(k_coarse {k}, inner {inner}), {iters} consecutive FGMRES({RESTART}) steps of one solve "
              f"({args.precond}), {t:.1f} s")
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": "Mcell-it/s", "n_gpus": args.gpus,
            "steps": iters, "warmup": args.warmup, "ms_per_step": t / max(iters, 1) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_name(args.n, args.precond), "grid": args.n,
                                            "sample_grid": n_s},
            "cpu_baseline": {"value": rate, "unit": "Mcell-it/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": rate, "unit": "Mcell-it/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def batch_problems(n_prob=64, seed=3000):
    """The batching workload: n_prob square grids n = 64 U{4..24} (256^2 to
    1536^2) drawn from the seed, the freeform recipe, each at 1.31 / 1.55 /
    1.80 um with a fixed dx = 1.55 um / 30."""
    import numpy as np
    from paper_2509_03622_gb300 import workloads as wl
    g = wl.rng(seed)
    sizes = (64 * g.integers(4, 25, size=n_prob)).tolist()
    dx = 1.55e-6 / 30
    out = []
    for p, n in enumerate(sizes):
        eps = wl.freeform_eps(n, n, seed=seed + 1 + p)
        J = wl.point_source(n, n)
        for lam in (1.31e-6, 1.55e-6, 1.80e-6):
            out.append((eps, J, dx, lam))
    return out


def batch_bench(args):
    """Lock-step solves of the batching workload: one neural pass over the
    windows of all still-active problems per Arnoldi step, each problem with
    its own two-level preconditioner.  Reports the throughput of K steps and
    the time until every problem reaches relres 1e-6 (or the cap)."""
    import numpy as np
    import torch
    from paper_2509_03622_gb300 import fdfd as F
    dev = torch.device("cuda")
    probs = batch_problems(args.batch)
    blob, wsrc = load_weights(args.weights)
    kc = args.k_coarse if args.k_coarse >= 0 else 32
    solvers, Js = [], []
    t0 = time.perf_counter()
    for eps, J, dx, lam in probs:
        S = F.Solver(torch.from_numpy(eps).to(dev), dx, lam, npml=20)
        S.schwarz_setup(blob, k_coarse=kc, inner_iters=args.inner)
        solvers.append(S)
        Js.append(torch.from_numpy(J).to(dev))
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    B = F.Batch(solvers)
    Es = [torch.zeros_like(J) for J in Js]
    cells = sum(int(J.numel()) for J in Js)
    B.solve(Js, Es, restart=30, max_iters=args.warmup, tol=1e-30, precond=F.PRECOND_SCHWARZ)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(solvers[0].stream)
    rc, stats = B.solve(Js, Es, restart=30, max_iters=args.steps, tol=1e-30, precond=F.PRECOND_SCHWARZ)
    ev1.record(solvers[0].stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    steps = max(st["iters"] for st in stats)
    for E in Es:
        E.zero_()
    torch.cuda.synchronize()
    ev0.record(solvers[0].stream)
    rc, stats2 = B.solve(Js, Es, restart=30, max_iters=args.tts_max_iters, tol=1e-6, precond=F.PRECOND_SCHWARZ)
    ev1.record(solvers[0].stream)
    torch.cuda.synchronize()
    ms_tts = ev0.elapsed_time(ev1)
    rel = [st["relres_true"] for st in stats2]
    line = {"metric": METRIC, "value": cells * steps / (ms / 1e3) / 1e6, "unit": "Mcell-it/s", "n_gpus": 1,
            "steps": steps, "warmup": args.warmup, "ms_per_step": ms / max(steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic (seeded freeform eps)",
            "config": {"workload": f"batch of {len(probs)} problems: {args.batch} grids 64*U{{4..24}} "
                                   "(256^2..1536^2) x 3 wavelengths (1.31/1.55/1.80 um), dx = 1.55 um/30, "
                                   "lock-step two-level Schwarz-NNO FGMRES(30)",
                       "cells": cells, "k_coarse": kc, "inner_iters": args.inner, "weights": wsrc,
                       "setup_s": t_setup},
            "time_to_1e-6": {"ms": ms_tts, "iters_max": max(st["iters"] for st in stats2),
                             "converged": sum(st["status"] == F.OK for st in stats2), "problems": len(stats2),
                             "relres_max": max(rel), "relres_median": float(np.median(rel)),
                             "max_iters": args.tts_max_iters}}
    B.close()
    for S in solvers:
        S.close()
    print(json.dumps(line))


def cpu_baseline(argd):
    """The oracle's FGMRES with the arm's preconditioner configuration on a
    bounded sample (about 10 s of steps after its set-up)."""
    global RESTART
    RESTART = argd.get("restart", RESTART)  # a spawned worker starts from the module default
    args = argparse.Namespace(**argd)
    w, kc_o, inner_o = oracle_preconditioner(args)
    ns = args.cpu_sample if args.precond == "schwarz" else 1024
    rate, t, it = cpu_oracle_rate(ns, 60, args.precond, w, kc_o, inner_o, budget_s=10.0, ritz_tol=args.ritz_tol)
    return {"value": rate, "unit": "Mcell-it/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{ns}x{ns} grid, same recipe and preconditioner configuration (k_coarse {kc_o}, "
                      f"inner {inner_o}), {it} consecutive FGMRES({RESTART}) steps ({args.precond}), {t:.1f} s; "
                      f"run in a separate process while the GPU work ran"}


def timed_solve(S, Jd, E, precond, max_iters):
    """One full solve from E = 0 to true relative residual 1e-6 (FGMRES(RESTART)),
    device time by CUDA events on the solver's stream."""
    import torch
    from paper_2509_03622_gb300 import fdfd as F
    E.zero_()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(S.stream)
    try:
        rc, st = S.solve(Jd, E, restart=RESTART, max_iters=max_iters, tol=1e-6, precond=precond)
    except F.FDFDError as ex:  # a hard error ends this solve; report it instead of the numbers
        torch.cuda.synchronize()
        return {"ms": None, "iters": None, "relres": None, "status": str(ex), "converged": False}
    ev1.record(S.stream)
    torch.cuda.synchronize()
    return {"ms": ev0.elapsed_time(ev1), "iters": st["iters"], "relres": st["relres_true"],
            "status": F.status_string(rc), "converged": rc == F.OK}


def time_to_solution(S, Jd, E, precond, args):
    """Time to relres 1e-6 of the arm's preconditioner (median of repeats)
    and of Jacobi-GMRES(RESTART) on the same handle and GPU, the latter capped at
    max(20 x the Schwarz time, 30 s) but at most --jacobi-cap-s."""
    import statistics
    from paper_2509_03622_gb300 import fdfd as F
    out = {}
    if precond == F.PRECOND_SCHWARZ:
        runs = [timed_solve(S, Jd, E, precond, args.tts_max_iters) for _ in range(max(args.tts_repeats, 1))]
        if any(r["ms"] is None for r in runs):
            return {"schwarz_nno_fgmres": runs[-1]}
        med = statistics.median(r["ms"] for r in runs)
        out["schwarz_nno_fgmres"] = dict(runs[-1], ms=med, ms_runs=[r["ms"] for r in runs],
                                         repeats=len(runs), max_iters=args.tts_max_iters)
        cap_s = min(max(20.0 * med / 1e3, 30.0), args.jacobi_cap_s)
    else:
        cap_s = args.jacobi_cap_s
    probe = timed_solve(S, Jd, E, F.PRECOND_JACOBI, 300)  # per-iteration cost of the baseline
    per_it = probe["ms"] / max(probe["iters"], 1)
    cap_it = int(cap_s * 1e3 / per_it)
    jr = timed_solve(S, Jd, E, F.PRECOND_JACOBI, cap_it)
    out["jacobi_gmres"] = dict(jr, cap_s=cap_s, cap_iters=cap_it, ms_per_iter=per_it)
    if "schwarz_nno_fgmres" in out:
        s_ = out["schwarz_nno_fgmres"]
        out["speedup_vs_jacobi"] = (jr["ms"] / s_["ms"]) if (s_["converged"] and jr["converged"]) else None
        out["note"] = ("Jacobi-GMRES stopped at its cap or by stagnation; its time is a lower bound"
                       if not jr["converged"] else "both converged")
    return out


def main():
    global RESTART
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precond", default="schwarz", choices=["schwarz", "jacobi"])
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--k-coarse", type=int, default=-1)
    ap.add_argument("--restart", type=int, default=RESTART,
                    help="FGMRES restart length of every solve the bench runs (1..64)")
    ap.add_argument("--inner", type=int, default=INNER_DEFAULT,
                    help="NN-FGMRES steps per local solve (0 = one network application)")
    ap.add_argument("--design", type=int, default=0,
                    help="also time this many inverse-design iterations (512^2 demultiplexer, 3 wavelengths)")
    ap.add_argument("--ritz-tol", type=float, default=0.0,
                    help="Rayleigh-Ritz truncation of the coarse space: keep |eta| >= this (0 = off)")
    ap.add_argument("--weights", default=None, help="weight blob (.npy); default the trained blob if present")
    ap.add_argument("--cpu-sample", type=int, default=256)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-tts", action="store_true", help="skip the time-to-1e-6 solves")
    ap.add_argument("--tts-repeats", type=int, default=3, help="full Schwarz solves to 1e-6 (median reported)")
    ap.add_argument("--tts-max-iters", type=int, default=3000, help="iteration cap of each Schwarz solve")
    ap.add_argument("--jacobi-cap-s", type=float, default=60.0,
                    help="time cap of the Jacobi-GMRES solve to 1e-6 (at least 20x the Schwarz time, "
                         "at most this)")
    ap.add_argument("--stationary", type=int, default=0,
                    help="also time this many iterations of the stationary Schwarz loop (Algorithm 3)")
    ap.add_argument("--batch", type=int, default=0,
                    help="bench the batching workload instead: this many grids x 3 wavelengths in lock step")
    ap.add_argument("--nno-precision", default="bf16", choices=["bf16", "fp8"],
                    help="neural-operator activations: BF16, or E4M3 with per-channel scales")
    args = ap.parse_args()
    if not 1 <= args.restart <= 64:
        ap.error("--restart must be in 1..64")
    RESTART = args.restart
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return
    if args.batch > 0:
        if rank == 0:
            batch_bench(args)
        return
    cpu_job = cpu_pool = None
    if rank == 0 and not args.no_cpu:
        # the oracle baseline runs in a process of its own (spawned before
        # any CUDA call) while this process does the GPU work
        import multiprocessing as mp
        cpu_pool = mp.get_context("spawn").Pool(1)
        cpu_job = cpu_pool.apply_async(cpu_baseline, (vars(args),))
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2509_03622_gb300 import fdfd as F
    from paper_2509_03622_gb300 import workloads as wl
    if world > 1:
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    dev = torch.device("cuda")
    n = args.n
    # independent replica per rank (weak scaling): different seed per rank
    eps, J, dx, lam = make_problem(n, seed_off=rank)
    S = F.Solver(torch.from_numpy(eps).to(dev), dx, lam, npml=20, max_restart=RESTART)
    precond = F.PRECOND_SCHWARZ if args.precond == "schwarz" else F.PRECOND_JACOBI
    kc = args.k_coarse if args.k_coarse >= 0 else K_COARSE_DEFAULT
    prec_nno = args.nno_precision
    if precond == F.PRECOND_SCHWARZ:
        blob, wsrc = load_weights(args.weights)
        t0 = time.perf_counter()
        S.schwarz_setup(blob, k_coarse=kc, precision=F.PREC_FP8 if prec_nno == "fp8" else F.PREC_BF16,
                        inner_iters=args.inner, ritz_tol=args.ritz_tol if kc > 0 else 0.0)
        t_setup = time.perf_counter() - t0
    Jd = torch.from_numpy(J).to(dev)
    E = torch.zeros((n, n), dtype=torch.complex64, device=dev)
    # warm-up: W Arnoldi steps
    S.solve(Jd, E, restart=RESTART, max_iters=args.warmup, tol=1e-30, precond=precond)
    torch.cuda.synchronize()
    import tempfile
    clk = Clocks(os.path.join(tempfile.gettempdir(), f"fdfd_bench_clocks_rank{rank}_{os.getpid()}.csv"))
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with clk:
        S.profile_start()
        torch.cuda.profiler.start()  # (a launch-list capture with --profile-from-start off sees this region only)
        ev0.record(S.stream)
        rc, st = S.solve(Jd, E, restart=RESTART, max_iters=args.steps, tol=1e-30, precond=precond)
        ev1.record(S.stream)
        prof = S.profile_stop()
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1), world, dev)
    if world > 1:
        dist.barrier()
    steps = st["iters"]
    value = job_rate(world, n * n, steps, ms / 1e3)
    # the same steps replayed as CUDA graphs (profiling off), for comparison
    S.use_graphs = True
    S.solve(Jd, E, restart=RESTART, max_iters=min(args.steps, RESTART), tol=1e-30, precond=precond)  # capture
    torch.cuda.synchronize()
    ev0.record(S.stream)
    S.solve(Jd, E, restart=RESTART, max_iters=args.steps, tol=1e-30, precond=precond)
    ev1.record(S.stream)
    torch.cuda.synchronize()
    ms_graph = ev0.elapsed_time(ev1)
    # end to end through the host-buffer entry point
    Jh = np.ascontiguousarray(J.astype(np.complex64))
    Eh = np.zeros_like(Jh)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    S.solve_host(Jh, Eh, restart=RESTART, max_iters=args.steps, tol=1e-30, precond=precond)
    t_e2e = max_over_ranks(time.perf_counter() - t0, world, dev)
    e2e_value = job_rate(world, n * n, args.steps, t_e2e)
    hbm, bf16, bf16s, src = peaks()
    # rooflines per kernel class (algorithmic bytes of the timed region)
    cls_ms = prof["ms"]
    N = n * n
    roofs = {}
    for cls, ms_c in cls_ms.items():
        nl = prof["launches"][cls]
        if ms_c <= 0 or nl == 0:
            continue
        nw1 = n // 64
        byts = algorithmic_bytes(cls, nl, N, steps, k=kc if precond == F.PRECOND_SCHWARZ else 0,
                                 coarse_launches_per_apply=1 + (2 * nw1 - 1) + 2 * (nw1 - 1) + 1,
                                 packed=precond == F.PRECOND_SCHWARZ and args.inner > 0)
        if byts is None:
            continue
        ach = byts / (ms_c / 1e3) / 1e9
        r = {"bound": "hbm", "kernel": KERNEL_NAMES.get(cls, cls), "achieved": ach, "peak": hbm, "unit": "GB/s",
             "frac": ach / hbm, "traffic": None, "launches": nl, "ms": ms_c, "peak_source": src}
        fl = NNO_FLOP_PER_WIN.get(cls)
        if fl:
            r["tflops"] = fl * (N / 4096.0) * nl / (ms_c / 1e3) / 1e12
        roofs[cls] = r
    packed = precond == F.PRECOND_SCHWARZ and args.inner > 0
    for cls, by_mode in SMALL_CASE_TRAFFIC.items():
        per_win = by_mode[packed]
        if per_win and cls in roofs and precond == F.PRECOND_SCHWARZ and prec_nno == "bf16":
            roofs[cls]["traffic"] = per_win * (N / 4096.0)  # bytes per launch: per window x windows
            roofs[cls]["traffic_note"] = f"ncu capture of {TRAFFIC_SAMPLE}, scaled by windows"
    dom = max(roofs, key=lambda c: roofs[c]["ms"]) if roofs else None
    roof = dict(roofs[dom]) if dom else None
    line = {"metric": METRIC, "value": value, "unit": "Mcell-it/s", "n_gpus": world, "steps": steps,
            "warmup": args.warmup, "ms_per_step": ms / max(steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64",
            "data": "synthetic (seeded freeform eps, point source)",
            "config": {"workload": workload_name(n, args.precond),
                       "grid": n, "precond": args.precond, "k_coarse": kc if precond == F.PRECOND_SCHWARZ else None,
                       "inner_iters": args.inner if precond == F.PRECOND_SCHWARZ else None,
                       "weights": wsrc if precond == F.PRECOND_SCHWARZ else None,
                       "setup_s": t_setup if precond == F.PRECOND_SCHWARZ else None,
                       "ritz_tol": args.ritz_tol if precond == F.PRECOND_SCHWARZ and kc > 0 else None,
                       "n_coarse_kept": S.info()["n_coarse_kept"] if precond == F.PRECOND_SCHWARZ else None,
                       "nno_precision": prec_nno if precond == F.PRECOND_SCHWARZ else None,
                       "restart": RESTART,
                       "l2": "inputs larger than L2 (each Krylov vector 134 MB; V, Z 16 GB)",
                       "parallelism": f"replicas x{world}"},
            "roofline": roof, "rooflines": roofs, "gpu_launches": prof["total_launches"],
            "e2e": {"value": e2e_value, "unit": "Mcell-it/s", "h2d_bytes_per_step": N * 8 // args.steps,
                    "d2h_bytes_per_step": N * 8 // args.steps},
            "clocks": clk.summary(), "relres_after_steps": st["relres_true"],
            "class_ms_per_step": {c: v / max(steps, 1) for c, v in cls_ms.items() if v > 0},
            "autotuned": {k: v for k, v in S.info().items() if k.startswith("tuned_")},
            "graphs": {"ms_per_step": ms_graph / max(steps, 1),
                       "note": "same solve with each Arnoldi step replayed as a CUDA graph, unprofiled"}}
    if cpu_job is not None:
        line["cpu_baseline"] = cpu_job.get(timeout=1800)
        cpu_pool.close()
    if args.stationary > 0 and precond == F.PRECOND_SCHWARZ:
        # Algorithm 3 on the same workload; the loop is linear in b, so the
        # source field itself serves as the right-hand side
        U = torch.empty_like(E)
        S.schwarz_stationary(Jd, U, max_iters=2, tol=0.0, momentum=0.5)  # warm-up
        torch.cuda.synchronize()
        ev0.record(S.stream)
        it_s, rr_s = S.schwarz_stationary(Jd, U, max_iters=args.stationary, tol=0.0, momentum=0.5)
        ev1.record(S.stream)
        torch.cuda.synchronize()
        ms_s = max_over_ranks(ev0.elapsed_time(ev1), world, dev)
        line["stationary"] = {"iters": it_s, "ms_per_iter": ms_s / max(it_s, 1), "momentum": 0.5,
                              "value": job_rate(world, n * n, it_s, ms_s / 1e3), "unit": "Mcell-it/s",
                              "relres": rr_s, "note": "each iteration includes its FP64 true residual"}
    if args.design > 0 and rank == 0 and precond == F.PRECOND_SCHWARZ:
        line["design"] = design_bench(args.design, blob, dev)
    if not args.no_tts and rank == 0:
        line["time_to_1e-6"] = time_to_solution(S, Jd, E, precond, args)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
