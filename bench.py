#!/usr/bin/env python
"""Benchmark of the non-Hermitian FEAST hot path on one GB300 per rank.

Workload: 2D convection-diffusion, 5-point upwind finite differences on a
300 x 300 grid (n = 90 000, 448 800 nonzeros, Peclet 10), B = I, an ellipse
(axis ratio 0.5) around 30 interior eigenvalues, m0 = 64, ne = 16 trapezoid
nodes, seeded N(0,1) start blocks.  One step = one full solve (factorisation
of the 16 shifted matrices, contour integrations, Rayleigh-Ritz, convergence
test, output) from the same start blocks; the metric is converged eigenpairs
(eq. res <= 1e-10) per second.

--impl reference times the CPU oracle (the plain FP64 algorithm, scipy
SuperLU per node) on complete solves of the same workload, its shifted solves
spread over the host cores by node.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "eigenpairs/s at residual <=1e-10 (chosen vs plain FP64 form); SpMM HBM GB/s"
UNIT = "eigenpairs/s"
WORKLOAD = ("convdiff2d N=300 (n=90000, nnz=448800), Pe=10 upwind, B=I, ellipse ratio 0.5 around 30 "
            "eigenvalues, m0=64, ne=16")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--form", choices=["chosen", "plain"], default="chosen")
    p.add_argument("--N", type=int, default=300)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-plain", action="store_true", help="skip the plain FP64 comparison solve")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--workload", choices=["convdiff", "batched", "kernels"], default="convdiff",
                   help="convdiff: the 300 x 300 convection-diffusion solve (default); batched: 64 random sparse "
                        "problems of uneven size in one batched solve")
    p.add_argument("--only", default="",
                   help="--workload kernels: comma list of spmm_f32, conv, batch, proj (default: all)")
    p.add_argument("--nprob", type=int, default=64)
    p.add_argument("--nmax", type=int, default=200000)
    p.add_argument("--max-iter", type=int, default=30, help="outer iteration cap of the batched solve")
    p.add_argument("--inner-tol", type=float, default=None, help="inner refinement tolerance (default: the library's)")
    return p.parse_args()


def rank_info():
    r = int(os.environ.get("RANK", "0"))
    w = int(os.environ.get("WORLD_SIZE", "1"))
    lr = int(os.environ.get("LOCAL_RANK", "0"))
    return r, w, lr


def combine_ranks(total_ms, pairs, world, device):
    """Whole-job figures of a replicas run: the slowest rank's timed total and
    the converged pairs of all ranks (every rank solves its own problem)."""
    import torch
    t = torch.tensor([float(total_ms), float(pairs)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        tt = [torch.zeros_like(t) for _ in range(world)]
        dist.all_gather(tt, t)
        return max(float(x[0]) for x in tt), sum(float(x[1]) for x in tt)
    return float(total_ms), float(pairs)


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.p = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------
def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    from paper_1506_04463_gb300 import feast_nh as F
    from paper_1506_04463_gb300 import workloads as wl

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    wk = wl.config2(N=args.N)
    prec = F.PREC_FP32_IR if args.form == "chosen" else F.PREC_FP64
    stream = torch.cuda.current_stream(dev)
    extra = {} if args.inner_tol is None else {"inner_tol": args.inner_tol}
    # the chosen form takes the tensor-core Rayleigh-Ritz products, the plain form FP64 throughout
    proj = F.PROJ_TENSOR if args.form == "chosen" else F.PROJ_FP64
    ctx = F.FeastNH(wk.A, None, wk.contour, wk.m0, device=dev, precision=prec, projection=proj, timing=1, **extra)
    Y0 = torch.from_numpy(np.ascontiguousarray(wk.Y0)).to(dev)
    Yh0 = torch.from_numpy(np.ascontiguousarray(wk.Yh0)).to(dev)
    # L2 flush buffer (256 MB > 129 MB L2), written between timed steps
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    for _ in range(args.warmup):
        out = ctx.solve(Y0, Yh0)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()

    clk = Clocks(local_rank)
    clk.start()
    launches0 = F.kernel_launches()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    infos, ms_found = [], []
    for k in range(args.steps):
        flush.fill_(float(k))
        starts[k].record(stream)
        out = ctx.solve(Y0, Yh0)
        ends[k].record(stream)
        infos.append(out["info"])
        ms_found.append(out["m"])
    torch.cuda.synchronize()
    launches = F.kernel_launches() - launches0
    clocks = clk.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = sum(step_ms)
    # correctness of the timed result (closed-form spectrum of the operator)
    lam = np.sort(out["lam"].cpu().numpy().real)
    exact = np.sort(wk.exact.real)
    eig_err = float(np.max(np.abs(lam - exact) / np.abs(exact))) if lam.size == exact.size else None
    max_res = float(out["res"].max().item()) if out["m"] else None
    pairs = sum(ms_found)
    total_max, pairs_all = combine_ranks(total_ms, pairs, world, dev)
    value = pairs_all / (total_max / 1e3)

    # ---- dominant kernel and its roofline ----
    inf = infos[-1]
    solve_ms = sum(i["t_solve_kernel_ms"] for i in infos)
    resid_ms = sum(i["t_resid_kernel_ms"] for i in infos)
    n_solve = sum(i["n_solve_launches"] for i in infos)
    n_resid = sum(i["n_resid_launches"] for i in infos)
    fac_ms = sum(i["t_factor_ms"] for i in infos)
    n, m, ne, kl, ku = wk.A.shape[0], wk.m0, wk.contour.ne, inf["kl"], inf["ku"]
    peaks = load_peaks()
    sm_mhz = clocks.get("sm_max_mhz") or 2070.0
    # one banded solve launch: both sides, every node, every column:
    # n*(kl+ku) complex multiply-adds (8 real flops) plus n divisions, per column
    solve_flops = 2 * ne * m * (n * (kl + ku)) * 8.0
    fp32_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12       # TFLOP/s at the max SM clock
    fp64_peak = 1.25                                          # nominal FP64 TFLOP/s of the part
    # DRAM bytes (read + write) per k_band_solve_tma launch at N = 300: the
    # mean over the 5 launches of one solve in an ncu capture of the current
    # kernel (dram__bytes_read.sum + dram__bytes_write.sum); None for other
    # sizes or forms, where no capture was taken
    solve_traffic = 29.11e9 if (n == 90000 and prec == F.PREC_FP32_IR) else None
    roof = None
    if n_solve:
        avg = solve_ms / n_solve
        ach = solve_flops / (avg / 1e3) / 1e12
        peak = fp32_peak if prec == F.PREC_FP32_IR else fp64_peak
        roof = {"kernel": "k_band_solve_tma" if prec == F.PREC_FP32_IR else "k_band_solve",
                "bound": "alu", "achieved": round(ach, 3), "peak": round(peak, 2), "unit": "TFLOP/s",
                "frac": round(ach / peak, 4), "traffic": solve_traffic,
                "traffic_source": "ncu capture of this kernel (dram bytes read+write per launch), not this run",
                "avg_launch_ms": round(avg, 3),
                "launches": n_solve, "flops_per_launch": solve_flops,
                "peak_note": ("FP32 FMA: 152 SMs x 128 lanes x 2 flop x max SM clock" if prec == F.PREC_FP32_IR
                              else "FP64 nominal 1.25 TFLOP/s")}
    # multi-shift residual: algorithmic bytes per launch (one side)
    xs = ne * n * m * 16
    resid_bytes = xs + n * m * 16 + ne * n * m * 8 + wk.A.nnz * 12 + (n + 1) * 4
    spmm = None
    if n_resid:
        avg = resid_ms / n_resid
        gbs = resid_bytes / (avg / 1e3) / 1e9
        hbm = peaks.get("hbm_gbs", 6786.6)
        # FP64 work per launch: every (node, column) pair forms z_j x (4 FMA)
        # and the real A's products (2 FMA per entry) on every row
        resid_flops = ne * m * (8.0 * n + 4.0 * wk.A.nnz)
        tf = resid_flops / (avg / 1e3) / 1e12
        spmm = {"kernel": "k_multishift_residual", "bound_note": "FP64 arithmetic (GB300 FP64 ~1 TFLOP/s)",
                "achieved_gbs": round(gbs, 1), "peak_gbs": hbm, "frac_of_measured_hbm": round(gbs / hbm, 4),
                "frac_of_8tbs": round(gbs / 8000.0, 4), "bytes_per_launch": resid_bytes,
                "fp64_flops_per_launch": resid_flops, "achieved_fp64_tflops": round(tf, 3),
                "frac_of_fp64_nominal": round(tf / 1.25, 4), "fp64_peak_note": "FP64 nominal 1.25 TFLOP/s",
                "avg_launch_ms": round(avg, 3), "launches": n_resid}
    # FP32 multi-shift operator of the Krylov sweeps on the same matrix and
    # block shape (ne = 16 nodes x 64 columns): HBM-bound, 16-byte loads
    spmm_f32 = spmm_f32_measure(ctx, wk, dev, F, torch, peaks)
    kernel_times = {"factor_ms": round(fac_ms / len(infos), 2), "band_solve_ms": round(solve_ms / len(infos), 2),
                    "multishift_residual_ms": round(resid_ms / len(infos), 2),
                    "filter_ms": round(sum(i["t_filter_ms"] for i in infos) / len(infos), 2),
                    "rr_ms": round(sum(i["t_rr_ms"] for i in infos) / len(infos), 2)}

    # ---- end-to-end through the C ABI with host buffers ----
    e2e = None
    if not args.no_e2e:
        e2e = e2e_measure(args, wk, dev, prec, F, torch)

    # ---- plain FP64 form, same workload, one solve ----
    plain = None
    if args.form == "chosen" and not args.no_plain:
        ctxp = F.FeastNH(wk.A, None, wk.contour, wk.m0, device=dev, precision=F.PREC_FP64, projection=F.PROJ_FP64)
        ctxp.solve(Y0, Yh0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        o = ctxp.solve(Y0, Yh0)
        e1.record(stream)
        torch.cuda.synchronize()
        pms = e0.elapsed_time(e1)
        plain = {"eigenpairs_per_s": round(o["m"] / (pms / 1e3), 3), "ms_per_solve": round(pms, 1), "m": o["m"],
                 "_lam": o["lam"].cpu().numpy(), "_res": o["res"].cpu().numpy(),
                 "max_res": float(o["res"].max().item()) if o["m"] else None,
                 "speedup_chosen_over_plain": round(value / world / (o["m"] / (pms / 1e3)), 3)}
        ctxp.close()

    cpu, pairs_err = None, None
    if rank == 0 and not args.no_cpu_baseline:
        cpu, ref = cpu_baseline(wk)
        pairs_err = {"chosen": per_pair_errors(out["lam"].cpu().numpy(), out["res"].cpu().numpy(), ref)}
        if plain is not None:
            pairs_err["plain_fp64"] = per_pair_errors(plain.pop("_lam"), plain.pop("_res"), ref)
    if plain is not None:
        plain.pop("_lam", None)
        plain.pop("_res", None)

    ctx.close()
    if rank != 0:
        return None
    line = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_max / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": ("c64 solves + c128 refinement/RR; RR products as exact bf16-digit tensor-core sums"
                  if prec == F.PREC_FP32_IR else "c128"),
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "nnz": int(wk.A.nnz), "m0": m, "ne": ne,
                   "form": ("chosen: FP32 banded LU + FP64 iterative refinement; Rayleigh-Ritz products on the tensor cores "
                            "(FP64-accurate exact digit products)") if prec == F.PREC_FP32_IR
                   else "plain FP64 banded LU", "parallelism": f"replicas x{world}",
                   "l2": "256 MB buffer written between timed steps; working set > L2"},
        "e2e": e2e, "gpu_launches": int(launches), "roofline": roof, "spmm": spmm, "spmm_f32": spmm_f32,
        "kernel_ms_per_step": kernel_times,
        "cpu_baseline": cpu, "clocks": clocks, "plain_fp64": plain,
        "per_eigenpair_vs_fp64_oracle": pairs_err,
        "check": {"m": int(ms_found[-1]), "iterations": inf["iterations"], "max_res": max_res,
                  "inner_steps_last_filter": inf["inner_steps"], "inner_res": inf["inner_res"],
                  "max_rel_eig_err_vs_closed_form": eig_err},
    }
    return line


def spmm_f32_measure(ctx, wk, dev, F, torch, peaks, reps=20):
    """CUDA-event time of feast_nh_multishift_spmm (V_j = (z_j I - A) P_j in
    complex FP32 for all ne nodes x m columns) on the bench matrix; the block
    (ne * n * m * 8 bytes each way) is larger than L2."""
    n, m, ne = wk.A.shape[0], wk.m0, wk.contour.ne
    g = torch.Generator(device=dev).manual_seed(11)
    P = torch.randn((ne, n, m), dtype=torch.complex64, device=dev, generator=g)
    V = torch.empty_like(P)
    stream = torch.cuda.current_stream(dev)
    for _ in range(3):
        ctx.multishift_spmm(P, 0, out=V)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        ctx.multishift_spmm(P, 0, out=V)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    nbytes = 2 * ne * n * m * 8 + wk.A.nnz * 12 + (n + 1) * 4
    gbs = nbytes / (ms / 1e3) / 1e9
    hbm = peaks.get("hbm_gbs", 6786.6)
    return {"kernel": "k_multishift_spmm_f32", "bound": "hbm", "achieved_gbs": round(gbs, 1), "peak_gbs": hbm,
            "frac_of_measured_hbm": round(gbs / hbm, 4), "frac_of_8tbs": round(gbs / 8000.0, 4),
            "bytes_per_launch": int(nbytes), "avg_launch_ms": round(ms, 4), "launches": reps,
            "shape": f"ne={ne} nodes x m={m} columns, n={n}, complex64"}


def e2e_measure(args, wk, dev, prec, F, torch):
    """Same metric through the public API with pinned host buffers: H2D of the
    CSR matrix and start blocks, init, solve, D2H of eigenvalues, residuals and
    both eigenvector blocks, destroy -- all inside the timed region."""
    A = wk.A.tocsr()
    rp = torch.from_numpy(A.indptr.astype(np.int32)).pin_memory()
    ci = torch.from_numpy(A.indices.astype(np.int32)).pin_memory()
    va = torch.from_numpy(A.data.real.astype(np.float64)).pin_memory()
    Y0 = torch.from_numpy(np.ascontiguousarray(wk.Y0)).pin_memory()
    Yh0 = torch.from_numpy(np.ascontiguousarray(wk.Yh0)).pin_memory()
    n, m0 = A.shape[0], wk.m0
    h_lam = torch.empty(m0, dtype=torch.complex128).pin_memory()
    h_res = torch.empty(m0, dtype=torch.float64).pin_memory()
    h_X = torch.empty((n, m0), dtype=torch.complex128).pin_memory()
    h_Xh = torch.empty((n, m0), dtype=torch.complex128).pin_memory()
    h2d = rp.numel() * 4 + ci.numel() * 4 + va.numel() * 8 + 2 * Y0.numel() * 16
    d2h = 0
    times, found = [], 0
    reps = max(1, min(args.steps, 3))
    for k in range(reps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d_rp, d_ci, d_va = rp.to(dev, non_blocking=True), ci.to(dev, non_blocking=True), va.to(dev, non_blocking=True)
        dY0, dYh0 = Y0.to(dev, non_blocking=True), Yh0.to(dev, non_blocking=True)
        ctx = F.FeastNH((d_rp, d_ci, d_va, F.R64, n, A.nnz), None, wk.contour, m0, device=dev, precision=prec,
                        projection=F.PROJ_TENSOR if prec == F.PREC_FP32_IR else F.PROJ_FP64)
        out = ctx.solve(dY0, dYh0)
        mm = out["m"]
        h_lam[:mm].copy_(out["lam"], non_blocking=True)
        h_res[:mm].copy_(out["res"], non_blocking=True)
        h_X[:, :mm].copy_(out["X"], non_blocking=True)
        h_Xh[:, :mm].copy_(out["Xh"], non_blocking=True)
        torch.cuda.synchronize()
        ctx.close()
        t1 = time.perf_counter()
        if k > 0:  # first repetition is a warm-up
            times.append(t1 - t0)
            found += mm
            d2h = mm * (16 + 8) + 2 * n * mm * 16
    return {"value": round(found / sum(times), 4), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": round(1e3 * sum(times) / len(times), 2),
            "includes": "H2D CSR + start blocks, init (transposed CSR, workspace), solve, D2H results, destroy"}


# ----------------------------------------------------------------------------
# CPU oracle leg: the oracle's complete solve (Fig. alg:three, FP64), with its
# shifted solves spread over the host cores: one spawned worker process per
# group of nodes keeps that group's SuperLU factors (the saved-factorisation
# option of Sec. 4.1) and solves the right-hand sides it is sent through shared
# memory; the oracle itself sums the solutions in node order and runs the
# Rayleigh-Ritz step with numpy's threaded BLAS.
# ----------------------------------------------------------------------------
def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True,
                             timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def _node_worker(conn, nodes, a_parts, b_parts, z, rhs_name, out_name, n, m0, ne):
    import numpy as _np
    import scipy.sparse as _sp
    from multiprocessing import shared_memory
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    from oracle import feast_nh as OF
    A = _sp.csr_matrix(tuple(a_parts[:3]), shape=a_parts[3])
    B = None if b_parts is None else _sp.csr_matrix(tuple(b_parts[:3]), shape=b_parts[3])
    rhs_shm = shared_memory.SharedMemory(name=rhs_name)
    out_shm = shared_memory.SharedMemory(name=out_name)
    rhs_all = _np.ndarray((n * m0,), _np.complex128, buffer=rhs_shm.buf)
    out_all = _np.ndarray((ne, n * m0), _np.complex128, buffer=out_shm.buf)
    solvers = {}
    try:
        while True:
            msg = conn.recv()
            if msg[0] == "factor":
                for j in nodes:
                    solvers[j] = OF.NodeSolver(A, B, z[j], dense=False)
                conn.send("ok")
            elif msg[0] == "solve":
                _, m, herm = msg
                rhs = rhs_all[: n * m].reshape(n, m)
                for j in nodes:
                    out_all[j, : n * m].reshape(n, m)[...] = solvers[j].solve(rhs, herm=herm)
                conn.send("ok")
            else:
                break
    finally:
        del rhs_all, out_all
        rhs_shm.close()
        out_shm.close()


class ParallelNodeSolvers:
    """The oracle's per-node solvers (scipy SuperLU, FP64) in `workers` spawned
    processes; solve_all(rhs, herm) returns every node's solution in node order
    (views into shared memory, valid until the next call)."""

    def __init__(self, A, B, z, m0, workers=None):
        import multiprocessing as mp
        from multiprocessing import shared_memory
        ne, n = len(z), A.shape[0]
        self.ne, self.n, self.m0 = ne, n, m0
        self.workers = max(1, min(ne, workers or host_cores()))
        self.rhs_shm = shared_memory.SharedMemory(create=True, size=n * m0 * 16)
        self.out_shm = shared_memory.SharedMemory(create=True, size=ne * n * m0 * 16)
        self.rhs = np.ndarray((n * m0,), np.complex128, buffer=self.rhs_shm.buf)
        self.out = np.ndarray((ne, n * m0), np.complex128, buffer=self.out_shm.buf)
        A = A.tocsr()
        a_parts = (A.data, A.indices, A.indptr, A.shape)
        b_parts = None if B is None else (B.tocsr().data, B.tocsr().indices, B.tocsr().indptr, B.shape)
        ctx = mp.get_context("spawn")
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        os.environ.update(OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
        self.procs, self.conns = [], []
        try:
            for k in range(self.workers):
                nodes = list(range(k, ne, self.workers))
                a, b = ctx.Pipe()
                p = ctx.Process(target=_node_worker, args=(b, nodes, a_parts, b_parts, np.asarray(z),
                                                           self.rhs_shm.name, self.out_shm.name, n, m0, ne),
                                daemon=True)
                p.start()
                self.procs.append(p)
                self.conns.append(a)
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        self.t_solve = 0.0

    def _all(self, msg):
        for c in self.conns:
            c.send(msg)
        for c in self.conns:
            if c.recv() != "ok":
                raise RuntimeError("oracle worker failed")

    def factor(self):
        self._all(("factor",))

    def solve_all(self, rhs, herm=False):
        t0 = time.perf_counter()
        n, m = rhs.shape
        self.rhs[: n * m].reshape(n, m)[...] = rhs
        self._all(("solve", m, bool(herm)))
        self.t_solve += time.perf_counter() - t0
        return [self.out[j, : n * m].reshape(n, m) for j in range(self.ne)]

    def close(self):
        for c in self.conns:
            try:
                c.send(("stop",))
            except Exception:
                pass
        for p in self.procs:
            p.join(timeout=30)
        del self.rhs, self.out
        self.rhs_shm.close()
        self.rhs_shm.unlink()
        self.out_shm.close()
        self.out_shm.unlink()


def oracle_full_solve(wk, pool):
    """One complete oracle solve of the workload (factorisations included)."""
    from oracle import feast_nh as OF
    pool.t_solve = 0.0
    t0 = time.perf_counter()
    pool.factor()
    t1 = time.perf_counter()
    out = OF.feast_nh(wk.A, wk.B, wk.contour, wk.m0, wk.Y0, wk.Yh0, solvers=pool)
    t2 = time.perf_counter()
    phases = {"factor_s": round(t1 - t0, 3), "shifted_solves_s": round(pool.t_solve, 3),
              "rayleigh_ritz_and_rest_s": round(t2 - t1 - pool.t_solve, 3), "total_s": round(t2 - t0, 3)}
    return out, phases


def threads_used():
    try:
        from threadpoolctl import threadpool_info
        return max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline(wk):
    """The oracle's complete solve of the bench workload on the host cores."""
    pool = ParallelNodeSolvers(wk.A, wk.B, __import__("oracle.contour", fromlist=["x"]).contour_nodes(wk.contour)[0],
                               wk.m0)
    try:
        out, ph = oracle_full_solve(wk, pool)
    finally:
        pool.close()
    T = ph["total_s"]
    line = {"value": round(out["m"] / T, 5), "unit": UNIT, "cores": pool.workers, "kind": "oracle",
            "sample": (f"full oracle solve of the same workload (FP64, scipy SuperLU per node, {out['iterations']} "
                       f"outer iterations, m={out['m']}): {pool.workers} worker processes hold the ne="
                       f"{wk.contour.ne} node factorisations and run the shifted solves in parallel; Rayleigh-Ritz "
                       f"with numpy BLAS ({threads_used()} threads)"),
            "per_phase_s": ph, "nproc": host_cores(), "cpu_model": cpu_model(), "iterations": out["iterations"]}
    return line, out


def per_pair_errors(lam_gpu, res_gpu, ref):
    """|lambda_gpu - lambda_oracle| / |lambda_oracle| per eigenpair after an
    optimal one-to-one matching, with each pair's eq. (res) residual."""
    from scipy.optimize import linear_sum_assignment
    lam_gpu, lo = np.asarray(lam_gpu), np.asarray(ref["lam"])
    if lam_gpu.size == 0 or lo.size == 0:
        return None
    C = np.abs(lam_gpu[:, None] - lo[None, :])
    r, c = linear_sum_assignment(C)
    order = np.argsort(lo[c].real)
    r, c = r[order], c[order]
    err = C[r, c] / np.abs(lo[c])
    return {"n_gpu": int(lam_gpu.size), "n_oracle": int(lo.size), "max_rel_err": float(err.max()),
            "rel_err": [float(f"{e:.3g}") for e in err],
            "res_gpu": [float(f"{v:.3g}") for v in np.asarray(res_gpu)[r]],
            "res_oracle": [float(f"{v:.3g}") for v in np.asarray(ref["res"])[c]]}


def run_reference(args, rank, world):
    from oracle.contour import contour_nodes
    from paper_1506_04463_gb300 import workloads as wl
    if rank != 0:
        return None
    wk = wl.config2(N=args.N)
    pool = ParallelNodeSolvers(wk.A, wk.B, contour_nodes(wk.contour)[0], wk.m0)
    vals, phases, timed = [], None, 0
    budget_s, t_start = 240.0, time.perf_counter()
    try:
        for k in range(args.warmup + args.steps):
            out, ph = oracle_full_solve(wk, pool)
            if k >= args.warmup:
                vals.append(out["m"] / ph["total_s"])
                phases = ph
                timed += 1
            # each step is a complete solve; stop early rather than overrun the budget
            if time.perf_counter() - t_start > budget_s and timed >= 1:
                break
    finally:
        pool.close()
    value = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "steps_timed": timed, "warmup": args.warmup,
            "ms_per_step": round(1e3 * out["m"] / value, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": {"workload": WORKLOAD, "form": "CPU oracle (plain FP64 algorithm)", "parallelism": "host cores"},
            "cpu_baseline": {"value": round(value, 5), "unit": UNIT, "cores": pool.workers, "kind": "oracle",
                             "sample": (f"each step: one complete oracle solve ({out['iterations']} outer iterations, "
                                        f"m={out['m']}), the ne={wk.contour.ne} SuperLU factorisations and shifted "
                                        f"solves spread over {pool.workers} worker processes"),
                             "per_phase_s": phases, "nproc": host_cores(), "cpu_model": cpu_model()},
            "e2e": {"value": round(value, 5), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    return line


def run_batched(args, rank, world, local_rank):
    """Many random sparse problems of uneven size (log-uniform n in [5000,
    nmax], 9 entries per row, diagonal + U(0, 4)), each with a circle at the
    right edge of its spectrum, m0 = 48, ne = 8: one batched solve per step."""
    from paper_1506_04463_gb300 import workloads as wl
    def log(msg):
        print(f"[bench batched] {msg}", file=sys.stderr, flush=True)
    t0 = time.perf_counter()
    bw = wl.config4(nprob=args.nprob, nmax=args.nmax, seed=rank, workers=host_cores())
    t_gen = time.perf_counter() - t0
    log(f"workload: {args.nprob} problems, sum n = {sum(a.shape[0] for a in bw.A)}, {t_gen:.1f} s")
    import torch
    from paper_1506_04463_gb300 import feast_nh as F
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    prec = F.PREC_FP32_IR if args.form == "chosen" else F.PREC_FP64
    t0 = time.perf_counter()
    b = F.FeastBatch(bw.A, bw.contours, bw.m0, device=dev, precision=prec, max_iter=args.max_iter,
                     projection=F.PROJ_TENSOR if args.form == "chosen" else F.PROJ_FP64)
    t_init = time.perf_counter() - t0
    log(f"batch init (transposes, workspace, launch-shape tuner): {t_init:.1f} s")
    Y0 = torch.from_numpy(bw.Y0).to(dev)
    Yh0 = torch.from_numpy(bw.Yh0).to(dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        t1 = time.perf_counter()
        out = b.solve(Y0, Yh0)
        torch.cuda.synchronize()
        log(f"warm-up solve {time.perf_counter() - t1:.1f} s: {json.dumps(out['info'])}")
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    clk = Clocks(local_rank)
    clk.start()
    l0 = F.kernel_launches()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    found = []
    for k in range(args.steps):
        starts[k].record(stream)
        out = b.solve(Y0, Yh0)
        ends[k].record(stream)
        # pairs at eq. (res) <= 1e-10 (a problem stopped by the iteration cap
        # may carry pairs above it)
        found.append(sum(int((pb["res"] <= 1e-10).sum().item()) for pb in out["problems"]))
    torch.cuda.synchronize()
    launches = F.kernel_launches() - l0
    clocks = clk.stop()
    total_ms = sum(s_.elapsed_time(e_) for s_, e_ in zip(starts, ends))
    total_max, pairs_all = combine_ranks(total_ms, sum(found), world, dev)
    value = pairs_all / (total_max / 1e3)
    inf = out["info"]
    sizes = [a.shape[0] for a in bw.A]
    exact_ok = sum(int(pb["m"] == len(ex)) for pb, ex in zip(out["problems"], bw.exact))
    max_res = max((float(pb["res"].max()) for pb in out["problems"] if pb["m"]), default=None)
    b.close()
    if rank != 0:
        return None
    return {"metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(total_max / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "c64 Krylov sweeps + c128 refinement/RR" if prec == F.PREC_FP32_IR else "c128",
            "data": "synthetic",
            "config": {"workload": (f"{args.nprob} random sparse nonsymmetric problems, n log-uniform in [5000, "
                                    f"{args.nmax}] (sum {sum(sizes)}), 9 nnz/row, diag + U(0,4), B=I, circle at "
                                    "the right spectral edge holding 16-40 eigenvalues each, m0=48, ne=8"),
                       "form": ("batched: one persistent launch for all problems' contour integration (FP32 "
                                "Jacobi-BiCGStab + FP64 refinement), per-problem Rayleigh-Ritz concurrently")
                       if prec == F.PREC_FP32_IR else "batched, plain FP64 Jacobi-BiCGStab",
                       "parallelism": f"replicas x{world}", "l2": "working set far above L2"},
            "gpu_launches": int(launches), "clocks": clocks,
            "check": {"pairs_per_solve": found[-1], "problems_converged": inf["converged_problems"],
                      "iterations_per_problem": [pb["iterations"] for pb in out["problems"]],
                      "problems_with_m_equal_edge_count": exact_ok, "max_res": max_res,
                      "iterations": inf["iterations"], "krylov_iterations": inf["krylov_iterations"],
                      "refine_steps": inf["refine_steps"], "inner_fail": inf["inner_fail"]},
            "autotune": {"threads": inf["threads"], "tile_rows": inf["tile_rows"], "grid": inf["grid"],
                         "t_autotune_ms": round(inf["t_autotune_ms"], 1)},
            "phase_ms_last_solve": {"filter": round(inf["t_filter_ms"], 1), "rr": round(inf["t_rr_ms"], 1),
                                    "total": round(inf["t_total_ms"], 1)},
            "setup_s": {"workload_generation": round(t_gen, 1), "batch_init": round(t_init, 1)}}


def run_kernels(args, rank, world, local_rank):
    """The hot kernels added beside the banded path, each on a small case whose
    operands exceed L2 (the cases the ncu captures use), timed with CUDA
    events: the FP32 multi-shift operator (convection-diffusion, N = args.N),
    one tensor-core convolution layer of the learned preconditioner's network
    (512 images of 64 x 64, 32 channels), and the batched contour integration
    (8 random sparse problems, n <= 20000)."""
    import torch
    from paper_1506_04463_gb300 import feast_nh as F
    from paper_1506_04463_gb300 import workloads as wl
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    peaks = load_peaks()
    hbm = peaks.get("hbm_gbs", 6786.6)
    res = {}
    only = set(args.only.split(",")) if args.only else {"spmm_f32", "conv", "batch", "proj"}
    # FP32 multi-shift SpMM
    wk = wl.config2(N=args.N)
    if "spmm_f32" in only or "proj" in only:
        ctx = F.FeastNH(wk.A, None, wk.contour, wk.m0, device=dev, precision=F.PREC_FP32_IR)
        if "spmm_f32" in only:
            res["spmm_f32"] = spmm_f32_measure(ctx, wk, dev, F, torch, peaks, reps=10)
        if "proj" in only:
            res["proj"] = proj_measure(ctx, wk.m0, dev, F, torch, reps=10)
        ctx.close()
    if "conv" in only:
        res["conv3x3_tc"] = conv_measure(dev, F, torch, stream)
    if "batch" in only:
        # batched contour integration, one refinement step on a fixed input
        bw = wl.config4(nprob=8, nmin=5000, nmax=20000, seed=3, workers=host_cores())
        b = F.FeastBatch(bw.A, bw.contours, bw.m0, device=dev, precision=F.PREC_FP32_IR, max_iter=2)
        t0 = time.perf_counter()
        out = b.solve(torch.from_numpy(bw.Y0).to(dev), torch.from_numpy(bw.Yh0).to(dev))
        torch.cuda.synchronize()
        res["batch"] = {"problems": 8, "sum_n": int(sum(a.shape[0] for a in bw.A)), "outer_iterations": 2,
                        "wall_s": round(time.perf_counter() - t0, 3), "info": out["info"]}
        b.close()
    if rank != 0:
        return None
    return {"workload": "kernels", "hbm_gbs_measured_peak": hbm, "results": res}


def proj_measure(ctx, m, dev, F, torch, reps=10):
    """The Rayleigh-Ritz products at the solve's shapes (n x m blocks, m x m
    matrices): G = X^H Y and Z = X S on the tensor cores (exact digit
    products) and in FP64 on the CUDA cores, CUDA events per call through the
    C ABI (each call ends with a stream synchronisation)."""
    g = torch.Generator(device=dev).manual_seed(0)
    n = ctx.n
    X = torch.randn((n, m), dtype=torch.complex128, device=dev, generator=g)
    Y = torch.randn((n, m), dtype=torch.complex128, device=dev, generator=g)
    S = torch.randn((m, m), dtype=torch.complex128, device=dev, generator=g)
    out = {"n": n, "m": m}
    for meth, name in ((F.PROJ_TENSOR, "tensor"), (F.PROJ_FP64, "fp64")):
        for op, f in (("gram", lambda: ctx.gram(X, Y, meth)), ("block", lambda: ctx.block_product(X, S, meth))):
            for _ in range(3):
                f()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(ctx.stream)
            for _ in range(reps):
                f()
            e1.record(ctx.stream)
            torch.cuda.synchronize()
            out[f"{op}_{name}_ms"] = round(e0.elapsed_time(e1) / reps, 4)
    G1, G2 = ctx.gram(X, Y, F.PROJ_TENSOR), ctx.gram(X, Y, F.PROJ_FP64)
    out["gram_rel_diff"] = float(torch.linalg.norm(G1 - G2) / torch.linalg.norm(G2))
    return out


def conv_measure(dev, F, torch, stream):
    """One convolution layer (forward of a 1-layer network: conv + bias)."""
    N, nimg = 64, 512
    net = F.Net(1, N, nimg, device=dev)
    rng = np.random.default_rng(0)
    net.set_params(np.concatenate([rng.standard_normal(9 * 32 * 32) * 0.05, np.zeros(32)]).astype(np.float32))
    x = torch.randn((nimg, N, N, 32), dtype=torch.float32, device=dev)
    for _ in range(2):
        net.forward(x)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    reps = 5
    for _ in range(reps):
        net.forward(x)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps  # includes the FP32 -> BF16 input conversion and the output copy
    flops = 2.0 * nimg * N * N * 32 * 288
    net.close()
    return {"kernel": "k_conv3x3_tc", "images": nimg, "grid": N, "ms_per_forward": round(ms, 4),
            "tflops_incl_conversions": round(flops / (ms / 1e3) / 1e12, 2)}


def main():
    args = parse()
    rank, world, local_rank = rank_info()
    if args.impl == "reference":
        line = run_reference(args, rank, world)
    else:
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group("nccl")
        if args.workload == "batched":
            line = run_batched(args, rank, world, local_rank)
        elif args.workload == "kernels":
            line = run_kernels(args, rank, world, local_rank)
        else:
            line = run_ours(args, rank, world, local_rank)
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
            dist.destroy_process_group()
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
