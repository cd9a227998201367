#!/usr/bin/env python
"""Benchmark of the GB300 spectral-element Poisson solve.

Workload (default): the 32^3-element deformed unit cube of order N = 7
(32,768 hex elements, lx = 8, 16,777,216 local points), nodes displaced by
0.05 h sin(2 pi x) sin(2 pi y) sin(2 pi z), h1 = 1 + 0.5 sin(4 pi x) cos(2 pi y),
six geometric factors stored per point, seeded N(0,1) right-hand side per
global node, Dirichlet on all faces.  Synthetic, generated by ``workloads``.

One step = one complete solve of that problem to a relative residual of 1e-10
(true FP64 residual ||b - A x|| / ||b||), with the selected solver (default:
FP64 iterative refinement around an FP32 inner Jacobi-PCG; ``--solver fp64``
for plain FP64 Jacobi-PCG).  Metric: Poisson GDOF/s = n_local x CG iterations
/ solve time (the paper counts E (N+1)^3 points).  Inputs are resident in HBM
and larger than L2 (the FP64 factors alone are 805 MB).

Prints ONE JSON line.  ``--impl reference`` times the FP64 CPU oracle instead
(on the host cores, a bounded sample of the same workload).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "Poisson GDOF/s (FP64 vs mixed, to 1e-10 rel. residual); ax_helm % HBM peak"
UNIT = "GDOF/s"
L2_NOTE = "inputs larger than L2 (FP64 factors 805 MB, FP32 factors 403 MB); no flush"


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--solver", choices=["mixed", "fp64", "fp64_pair", "gmres"], default="mixed",
                    help="mixed refinement (default), FP64 PCG with the native operator, FP64 PCG in "
                         "FP32-pair arithmetic (SEM_FP64_PAIR), or the mixed GMRES + Schwarz solve")
    ap.add_argument("--n", type=int, default=32, help="elements per direction of the cube")
    ap.add_argument("--order", type=int, default=7)
    ap.add_argument("--no-extras", action="store_true", help="skip the comparison solves and ax-only bench")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--variant", type=int, default=None,
                    help="pin the operator kernel variant (SEM_FLAG_VARIANT) instead of autotuning")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle sample")
    ap.add_argument("--tc-split", action="store_true",
                    help="mixed solver: inner operator on the tensor cores (SEM_TC_SPLIT)")
    ap.add_argument("--suite", action="store_true",
                    help="also measure the cube (FP64 and mixed), the 256-member batch and the annulus")
    return ap.parse_args()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def combine_ranks(ms: float, units: float, dist=None, device=None):
    """Whole-job figures over ranks: time = max over ranks, units = sum.
    Each rank solves its own replica (no data-path collective)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return ms, units
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[q] for r in rows for q in range(4) if r[5 + q].lower() == "active"})
        power = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(power) if power else None}


# mixed refinement of the deformed-cube workload: FP32 inner CG to 1e-2 with its
# direction kept across the FP64 refinement steps (residual replacement).  On
# this workload it reaches 1e-10 14% sooner than the library's default
# refinement (restarts, inner tolerance 1e-5, timed beside it in the extras);
# on the ill-conditioned annulus restarting is the faster of the two.
MIXED_OPTS = {"inner_tol": 1e-2, "ir_carry": 1}

def _workload(args):
    m, h1, b = W.deformed_cube(args.n, args.order, seed=2)
    name = f"deformed cube {args.n}^3 hex, N={args.order}, h1 wavy, random RHS"
    return m, h1, b, name


def _config(args, m, extra=None):
    c = {"workload": f"deformed_cube_{args.n}^3_N{args.order}", "elements": m.E, "lx": m.lx,
         "n_local": m.n_local, "tol": 1e-10,
         "solver": {"mixed": "mixed_ir", "fp64": "fp64_pcg", "fp64_pair": "fp64_pair_pcg",
                    "gmres": "mixed_fgmres_schwarz"}[args.solver],
         "preconditioner": ("two-level additive Schwarz: element-interior fast-diagonalisation solves, point "
                            "Jacobi on shared nodes, corner coarse grid (10 Jacobi-PCG iterations)"
                            if args.solver == "gmres" else "point Jacobi (exact assembled diagonal)"),
         "l2": L2_NOTE}
    if extra:
        c.update(extra)
    return c


def _oracle_sample(m, h1, b, target_s: float):
    """Time the FP64 CPU oracle on a bounded number of PCG iterations of the
    full workload.  Returns (GDOF/s, iterations, seconds, threads, setup_s)."""
    import oracle
    t0 = time.perf_counter()
    P = oracle.Problem(m, h1)
    setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    P.pcg(b, tol=1e-30, max_iter=1)
    t1 = time.perf_counter() - t0
    k = max(1, int(round(target_s / max(t1, 1e-3))))
    t0 = time.perf_counter()
    _, info = P.pcg(b, tol=1e-30, max_iter=k)
    dt = time.perf_counter() - t0
    return m.n_local * info["iters"] / dt / 1e9, info["iters"], dt, oracle.threads(), setup


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    m, h1, b, _ = _workload(args)
    import oracle
    P = oracle.Problem(m, h1)
    t0 = time.perf_counter()
    P.pcg(b, tol=1e-30, max_iter=1)
    t1 = time.perf_counter() - t0
    budget = 150.0 / max(1, args.steps + args.warmup)
    k = max(1, int(budget / max(t1, 1e-3)))
    for _ in range(args.warmup):
        P.pcg(b, tol=1e-30, max_iter=k)
    t0 = time.perf_counter()
    its = 0
    for _ in range(args.steps):
        _, info = P.pcg(b, tol=1e-30, max_iter=k)
        its += info["iters"]
    dt = time.perf_counter() - t0
    val = m.n_local * its / dt / 1e9
    sample = f"{k} FP64 Jacobi-PCG iterations of the full workload per step (oracle, plain C loops)"
    out = {"metric": METRIC, "value": val, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": _config(args, m, {"solver": "oracle_fp64_pcg_sample"}),
           "cpu_baseline": {"value": val, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def ka_bytes_per_point(solver: str) -> int:
    """Algorithmic bytes per local point of the fused CG operator kernel (K-A):
    z, p and the six h1-folded factors read, p and w written, ten values of
    the solve's inner precision (4 B for the FP32 inner solves of the mixed
    and GMRES modes, 8 B otherwise)."""
    reads, writes = 2 + 6, 2
    return (reads + writes) * (4 if solver in ("mixed", "gmres") else 8)


def _traffic_for(kernel: str, workload: str):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu
    summaries (a `traffic-record:` line in profiles/*.md), if the kernel's
    source file is unchanged since the capture (else None)."""
    import glob
    import hashlib
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        try:
            lines = open(path).read().splitlines()
        except OSError:
            continue
        for line in lines:
            line = line.strip().strip("`")
            if not line.startswith("traffic-record:"):
                continue
            rec = dict(kv.split("=", 1) for kv in line[len("traffic-record:"):].split())
            if rec.get("kernel") != kernel or rec.get("workload") != workload:
                continue
            try:
                src = os.path.join(ROOT, rec["source"])
                h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
            except (KeyError, OSError):
                return None
            return float(rec["bytes_per_launch"]) if h == rec.get("source_sha") else None
    return None


def run_ours(args):
    import torch
    import paper_2207_07098_gb300 as S

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    S.load()
    m, h1, b, _ = _workload(args)
    n = m.n_local
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    # SEM_FLAG_SCHWARZ: the handle also carries the GMRES preconditioner (timed in the extras)
    h = S.sem_setup(m.E, m.lx, m.coords, m.gid, m.mask, h1,
                    S.SEM_FLAG_SCHWARZ | (0 if args.variant is None else S.SEM_FLAG_VARIANT(args.variant)))
    setup_s = time.perf_counter() - t0
    info = S.sem_get_info(h)
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros(n, dtype=torch.float64, device="cuda")
    mode = {"mixed": S.SEM_MODE_MIXED_IR, "gmres": S.SEM_MODE_GMRES}.get(args.solver, S.SEM_MODE_FP64)
    opts = {"mode": mode, "tol": 1e-10, **(MIXED_OPTS if args.solver == "mixed" else {})}
    if args.solver == "fp64_pair":
        opts["precision"] = S.SEM_FP64_PAIR
    if args.solver == "gmres":  # the paper's pressure solver, FP32 cycles inside FP64 restarts
        opts["precision"] = S.SEM_FP32
    if args.tc_split:
        opts["tc_split"] = 1

    def step():
        xd.zero_()
        return S.sem_cg_solve(h, xd, bd, opts)

    for _ in range(max(3, args.warmup)):
        st = step()
    assert st["status"] == S.SEM_OK and st["relres"] <= 1e-10, st
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    stats = [step() for _ in range(args.steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms_local = ev0.elapsed_time(ev1)
    iters = sum(s["iterations"] for s in stats)
    launches = sum(s["kernel_launches"] for s in stats)
    worst = max(s["relres"] for s in stats)
    ms, units = combine_ranks(ms_local, float(n * iters), dist, "cuda")
    value = units / (ms * 1e-3) / 1e9

    # e2e: the same solves through the C ABI with pinned host buffers (copies inside)
    xh = torch.zeros(n, dtype=torch.float64).pin_memory()
    bh = torch.from_numpy(b).pin_memory()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    e_it = 0
    for _ in range(args.steps):
        xh.zero_()
        s = S.sem_cg_solve(h, xh, bh, opts)
        e_it += s["iterations"]
    torch.cuda.synchronize()
    e_dt = time.perf_counter() - t0
    if dist:
        dist.barrier()
    e_ms, e_units = combine_ranks(e_dt * 1e3, float(n * e_it), dist, "cuda")  # max time, summed work
    e2e = {"value": e_units / (e_ms * 1e-3) / 1e9, "unit": UNIT, "h2d_bytes_per_step": 2 * 8 * n,
           "d2h_bytes_per_step": 8 * n}

    peak, peak_kind = _peaks()
    # dominant kernel: the fused p-update + ax_helm launch (K-A) of the CG loop
    samples = [s["ax_ms"] for s in stats if s["ax_samples"] > 0]
    ax_ms = statistics.mean(samples) if samples else None
    ka_bytes = ka_bytes_per_point(args.solver) * n
    achieved = ka_bytes / (ax_ms * 1e-3) / 1e9 if ax_ms else None
    variant = stats[-1].get("ax_variant", 0)
    tname = "float" if args.solver in ("mixed", "gmres") else "double"
    cfgs = {1: (1, 3), 2: (2, 2), 3: (2, 3), 4: (4, 2)}
    kname = (f"ax_kernel<{tname},{m.lx},true>" if variant == 0 else
             f"ax_df_kernel<{m.lx},true>" if variant == 5 else
             f"ax_dfl_kernel<{m.lx},true>" if variant == 6 else
             "ax_tc_kernel<true>" if variant == 8 else
             f"ax_ln_kernel<{m.lx},true>" if variant == 9 else
             f"ax_bulk_kernel<{tname},{m.lx},{cfgs[variant][0]},{cfgs[variant][1]},true>")
    traffic = _traffic_for(kname, f"deformed_cube_{args.n}^3_N{args.order}")
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak if achieved else None,
                "traffic": traffic, "kernel": kname, "algorithmic_bytes_per_launch": ka_bytes,
                "launch_ms": ax_ms, "peak_kind": peak_kind}
    if args.solver == "gmres":  # no live per-kernel sample in this mode: see the GMRES launch-list summary
        roofline = {"bound": "hbm", "achieved": None, "peak": peak, "unit": "GB/s", "frac": None, "traffic": None,
                    "kernel": "gm_lagged_update_kernel<float>", "peak_kind": peak_kind,
                    "note": "GMRES iterations are not CG iterations: value counts points x GMRES iterations"}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": max(3, args.warmup), "ms_per_step": ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": {"mixed": "f32+f64", "fp64": "f64", "fp64_pair": "f32x2+f64", "gmres": "f32+f64"}[args.solver],
           "data": "synthetic",
           "config": _config(args, m, {"inner_tol": MIXED_OPTS["inner_tol"] if args.solver == "mixed" else None,
                                       "refinement": ("inner CG direction kept across FP64 refinement steps"
                                                      if args.solver == "mixed" else None),
                                       "n_unique_free": info["n_free"], "parallelism": f"replicas x{ws}",
                                       "operator_variant": "autotuned" if args.variant is None else args.variant}),
           "iterations_per_solve": iters / args.steps, "outer_per_solve": stats[-1]["outer_iterations"],
           "relres_max": worst, "gpu_launches": launches, "e2e": e2e, "roofline": roofline, "clocks": clk,
           "setup_s": setup_s}

    if rank == 0 and not args.no_extras:
        out["extras"] = _extras(S, torch, h, m, bd, n, args, peak, stats, ms)
        sv = out["extras"]["solves_to_1e-10"]
        # the FP64 arm the mixed solve is compared with, on the same GPU and mesh
        out["fp64_arm"] = {
            "fp64_native_time_ms": sv["fp64"]["time_ms"], "fp64_native_iterations": sv["fp64"]["iterations"],
            "fp64_pair_time_ms": sv["fp64_pair"]["time_ms"], "fp64_pair_iterations": sv["fp64_pair"]["iterations"],
            "mixed_time_ms": ms / args.steps,
            "speedup_mixed_vs_fp64_native": sv["fp64"]["time_ms"] / (ms / args.steps),
            "speedup_mixed_vs_fp64_pair": sv["fp64_pair"]["time_ms"] / (ms / args.steps),
            "note": ("FP64 Jacobi-PCG to the same true 1e-10: native FP64 operator and vectors (SEM_FP64), and "
                     "the FP32-pair operator and vectors (SEM_FP64_PAIR, 48-bit), both with the true residual "
                     "recomputed by the native operator")}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        v, k, dt, thr, osetup = _oracle_sample(m, h1, b, args.cpu_seconds)
        out["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": thr, "kind": "oracle",
                               "sample": f"{k} FP64 Jacobi-PCG iterations of the full workload "
                                         f"({dt:.1f} s; oracle set-up {osetup:.1f} s not counted)"}
    S.sem_destroy(h)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


def _extras(S, torch, h, m, bd, n, args, peak, stats, ms_timed):
    """FP64 vs mixed solves, 200 FP64 CG iterations, and the ax_helm-only bench."""
    ex = {}
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    res = {}
    for name, mode, prec, extra in (("fp64", S.SEM_MODE_FP64, S.SEM_FP64, {}),
                                    ("fp64_pair", S.SEM_MODE_FP64, S.SEM_FP64_PAIR, {}),
                                    ("mixed", S.SEM_MODE_MIXED_IR, S.SEM_FP64, MIXED_OPTS),
                                    ("mixed_restart_1e-5", S.SEM_MODE_MIXED_IR, S.SEM_FP64,
                                     {"inner_tol": 1e-5, "ir_carry": 0}),
                                    ("mixed_tc_split", S.SEM_MODE_MIXED_IR, S.SEM_FP64, {**MIXED_OPTS, "tc_split": 1})):
        x.zero_()
        st = S.sem_cg_solve(h, x, bd, {"mode": mode, "precision": prec, "tol": 1e-10, **extra})
        res[name] = {"time_ms": st["time_ms"], "iterations": st["iterations"], "outer": st["outer_iterations"],
                     "relres": st["relres"], "status": st["status"],
                     "gdof_s": n * st["iterations"] / (st["time_ms"] * 1e-3) / 1e9, "ax_ms": st["ax_ms"],
                     "ax_variant": st["ax_variant"]}
    res["speedup_mixed_vs_fp64"] = res["fp64"]["time_ms"] / res["mixed"]["time_ms"]
    res["speedup_mixed_vs_fp64_pair"] = res["fp64_pair"]["time_ms"] / res["mixed"]["time_ms"]
    ex["solves_to_1e-10"] = res
    # the paper's pressure solver on the same handle: restarted FGMRES + two-level Schwarz
    gm = {}
    for name, extra in (("gmres_mixed", {"precision": S.SEM_FP32}),
                        ("gmres_fp64_pair_pc32", {"precision": S.SEM_FP64_PAIR, "precond_precision": S.SEM_FP32}),
                        ("gmres_fp64", {})):
        for _ in range(2):  # the first solve allocates the Krylov basis
            x.zero_()
            st = S.sem_cg_solve(h, x, bd, {"mode": S.SEM_MODE_GMRES, "tol": 1e-10, **extra})
        gm[name] = {"time_ms": st["time_ms"], "iterations": st["iterations"], "restarts": st["outer_iterations"],
                    "relres": st["relres"], "status": st["status"]}
    gm["speedup_gmres_mixed_vs_mixed_pcg"] = res["mixed"]["time_ms"] / gm["gmres_mixed"]["time_ms"]
    gm["speedup_gmres_fp64_vs_fp64_pcg"] = res["fp64"]["time_ms"] / gm["gmres_fp64"]["time_ms"]
    ex["gmres_schwarz_to_1e-10"] = gm
    for name, prec in (("cg200_fp64", S.SEM_FP64), ("cg200_fp64_pair", S.SEM_FP64_PAIR)):
        x.zero_()
        st = S.sem_cg_solve(h, x, bd, {"mode": S.SEM_MODE_FP64, "precision": prec, "tol": 1e-30, "max_iter": 200})
        ex[name] = {"time_ms": st["time_ms"], "iterations": st["iterations"],
                    "gdof_s": n * st["iterations"] / (st["time_ms"] * 1e-3) / 1e9}
    # ax_helm-only: plain local operator, back-to-back launches, CUDA events on the launching stream
    stream = torch.cuda.current_stream()
    axr = {}
    for name, prec, dt, bpp in (("fp64", S.SEM_FP64, torch.float64, 64), ("fp64_pair", S.SEM_FP64_PAIR, torch.float64, 64),
                                ("fp32", S.SEM_FP32, torch.float32, 32), ("fp32_tc_split", S.SEM_TC_SPLIT, torch.float32, 32)):
        u = torch.randn(n, dtype=dt, device="cuda")
        w = torch.empty_like(u)
        for _ in range(3):
            S.sem_ax(h, w, u, prec, 0)
        reps = 20
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            S.sem_ax(h, w, u, prec, 0)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / reps
        gbs = bpp * n / (t * 1e-3) / 1e9
        axr[name] = {"ms": t, "gb_s": gbs, "frac_hbm": gbs / peak, "bytes_per_point": bpp}
    axr["accuracy"] = ("fp64: native FP64 arithmetic, 1e-12 of the oracle on every field tested; fp64_pair: "
                       "FP32-pair arithmetic (unit roundoff 2^-48), 1e-12 on rough fields, a few 1e-12 on "
                       "smooth cancelling ones; fp32_tc_split: BF16 three-slice tensor-core contractions, "
                       "FP32 accuracy class")
    ex["ax_helm_only"] = axr
    # every operator variant (pinned at set-up), plain ax_helm: 0..4 native FP64 and FP32, 5..6 FP32-pair,
    # 8 tensor-core FP32, 9 native FP64 line transforms
    var = {}
    for v in (0, 1, 2, 3, 4, 5, 6, 8, 9):
        if (v == 8 and m.lx != 8) or (v == 9 and m.lx % 2):
            continue
        hv = S.sem_setup(m.E, m.lx, m.coords, m.gid, m.mask, None, S.SEM_FLAG_VARIANT(v))
        row = {}
        kinds = ((("fp64", S.SEM_FP64, torch.float64, 64), ("fp32", S.SEM_FP32, torch.float32, 32)) if v <= 4 else
                 (("fp32", S.SEM_FP32, torch.float32, 32),) if v == 8 else
                 (("fp64", S.SEM_FP64, torch.float64, 64),) if v == 9 else
                 (("fp64_pair", S.SEM_FP64_PAIR, torch.float64, 64),))
        for name, prec, dt, bpp in kinds:
            u = torch.randn(n, dtype=dt, device="cuda")
            w = torch.empty_like(u)
            for _ in range(3):
                S.sem_ax(hv, w, u, prec, 0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(10):
                S.sem_ax(hv, w, u, prec, 0)
            e1.record(stream)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / 10
            row[name] = {"ms": t, "gb_s": bpp * n / (t * 1e-3) / 1e9}
        S.sem_destroy(hv)
        var[str(v)] = row
    ex["ax_variants"] = var
    return ex


def _timed_solve(S, torch, h, b_dev, n, opts, reps=3):
    """Best-of-reps solve time (CUDA events inside the library) and its stats."""
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    S.sem_cg_solve(h, x, b_dev, opts)
    best = None
    for _ in range(reps):
        x.zero_()
        st = S.sem_cg_solve(h, x, b_dev, opts)
        if best is None or st["time_ms"] < best["time_ms"]:
            best = st
    return x, best


def _solve_report(st, n_local, n_free):
    t = st["time_ms"] * 1e-3
    return {"time_ms": st["time_ms"], "iterations": st["iterations"], "outer": st["outer_iterations"],
            "relres": st["relres"], "status": st["status"], "gdof_s_local": n_local * st["iterations"] / t / 1e9,
            "gdof_s_unique_free": n_free * st["iterations"] / t / 1e9, "cg_iter_s": st["iterations"] / t,
            "ax_variant": st["ax_variant"]}


def run_suite(args):
    """The other synthetic workloads: unit cube 4^3, N=7 (FP64 and mixed,
    error vs the exact solution and, in the CPU-baseline leg, vs the oracle),
    the 256-member batch (FP64 and mixed), and the rotor-like annulus (FP64 vs
    mixed, ax_helm timings).  Prints one JSON line."""
    import torch
    import paper_2207_07098_gb300 as S
    S.load()
    out = {"suite": "sem_poisson", "data": "synthetic"}
    # mixed: the library's default refinement (restarts); mixed_carry: the kept direction
    modes = (("fp64", {"mode": S.SEM_MODE_FP64, "tol": 1e-10}),
             ("fp64_pair", {"mode": S.SEM_MODE_FP64, "precision": S.SEM_FP64_PAIR, "tol": 1e-10}),
             ("mixed", {"mode": S.SEM_MODE_MIXED_IR, "tol": 1e-10}),
             ("mixed_carry", {"mode": S.SEM_MODE_MIXED_IR, "tol": 1e-10, **MIXED_OPTS}),
             ("mixed_carry_capped", {"mode": S.SEM_MODE_MIXED_IR, "tol": 1e-10, **MIXED_OPTS, "max_iter": 100}))
    # --- cube, manufactured solution
    m, f = W.cube_sines(4, 7)
    h = S.sem_setup(m.E, m.lx, m.coords, m.gid, m.mask, None)
    info = S.sem_get_info(h)
    fd = torch.from_numpy(f).cuda()
    bd = torch.empty_like(fd)
    S.sem_mass(h, bd, fd, S.SEM_FP64, 1)
    exact = W.exact_sines(m)
    cube = {"workload": "cube 4^3 hex, N=7, f = 3 pi^2 sin sin sin, h1 = 1", "n_local": m.n_local,
            "n_unique_free": info["n_free"]}
    xs = {}
    for name, o in modes:
        x, st = _timed_solve(S, torch, h, bd, m.n_local, o)
        xs[name] = x.cpu().numpy()
        r = _solve_report(st, m.n_local, info["n_free"])
        r["max_error_vs_exact"] = float(np.max(np.abs(xs[name] - exact)))
        cube[name] = r
    d = xs["mixed"] - xs["fp64"]
    cube["mixed_vs_fp64_gpu_rel_l2"] = float(np.linalg.norm(d) / np.linalg.norm(xs["fp64"]))
    cube["speedup_mixed_vs_fp64"] = cube["fp64"]["time_ms"] / cube["mixed"]["time_ms"]
    cube["speedup_mixed_vs_fp64_pair"] = cube["fp64_pair"]["time_ms"] / cube["mixed"]["time_ms"]
    cube["speedup_mixed_carry_vs_fp64"] = cube["fp64"]["time_ms"] / cube["mixed_carry"]["time_ms"]
    cube["speedup_mixed_carry_capped_vs_fp64"] = cube["fp64"]["time_ms"] / cube["mixed_carry_capped"]["time_ms"]
    # CPU-baseline leg: the oracle's own solve (timed) and the GPU error against it
    import oracle
    P = oracle.Problem(m)
    bo = P.mass(f, assemble=True)
    t0 = time.perf_counter()
    xo, oi = P.pcg(bo, tol=1e-10)
    dt = time.perf_counter() - t0
    cube["cpu_baseline"] = {"value": m.n_local * oi["iters"] / dt / 1e9, "unit": UNIT, "cores": oracle.threads(),
                            "kind": "oracle", "sample": f"full FP64 PCG solve ({oi['iters']} iterations, {dt:.2f} s)",
                            "iterations": oi["iters"]}
    for name in xs:
        cube[name]["rel_l2_error_vs_oracle"] = float(np.linalg.norm(xs[name] - xo) / np.linalg.norm(xo))
    S.sem_destroy(h)
    out["cube_4^3_N7"] = cube
    # --- batch of 256 independent boxes
    t0 = time.perf_counter()
    members = [W.batch_member_case(p) for p in W.batch_params()]
    gen_s = time.perf_counter() - t0
    hb = S.sem_setup_batch([(mm.E, mm.lx, mm.coords, mm.gid, mm.mask, None) for mm, _ in members])
    binfo = S.sem_get_info(hb)
    bcat = torch.from_numpy(np.concatenate([bb for _, bb in members])).cuda()
    nb = len(members)
    batch = {"workload": "256 boxes, nx,ny,nz ~ U{2..16}, N ~ U{5,7,9}, amp ~ U(0,0.08), random RHS (seed 4)",
             "n_local": binfo["n_local"], "elements": binfo["E"], "generation_s": gen_s}
    for name, o in modes:
        x = torch.zeros_like(bcat)
        S.sem_cg_solve_batch(hb, x, bcat, nb, o)
        x.zero_()
        sts = S.sem_cg_solve_batch(hb, x, bcat, nb, o)
        t = sts[0]["time_ms"] * 1e-3
        dofit = sum(mm.n_local * st["iterations"] for (mm, _), st in zip(members, sts))
        its = [st["iterations"] for st in sts]
        batch[name] = {"time_ms": sts[0]["time_ms"], "gdof_s_local": dofit / t / 1e9,
                       "cg_iter_s_summed_over_solves": sum(its) / t, "iterations_max": max(its),
                       "iterations_mean": float(np.mean(its)), "all_converged": all(st["status"] == 0 for st in sts),
                       "relres_max": max(st["relres"] for st in sts), "launches": sts[0]["kernel_launches"],
                       "launches_per_iteration": sts[0]["launches_per_iteration"],
                       "operator_variants": sorted({st["ax_variant"] for st in sts})}
    batch["speedup_mixed_vs_fp64"] = batch["fp64"]["time_ms"] / batch["mixed"]["time_ms"]
    batch["speedup_mixed_vs_fp64_pair"] = batch["fp64_pair"]["time_ms"] / batch["mixed"]["time_ms"]
    batch["speedup_mixed_carry_vs_fp64"] = batch["fp64"]["time_ms"] / batch["mixed_carry"]["time_ms"]
    batch["speedup_mixed_carry_capped_vs_fp64"] = batch["fp64"]["time_ms"] / batch["mixed_carry_capped"]["time_ms"]
    S.sem_destroy(hb)
    del bcat, members
    torch.cuda.empty_cache()
    out["batch_256"] = batch
    # --- annulus
    t0 = time.perf_counter()
    m, f = W.annulus_case()
    gen_s = time.perf_counter() - t0
    h = S.sem_setup(m.E, m.lx, m.coords, m.gid, m.mask, None)
    info = S.sem_get_info(h)
    fd = torch.from_numpy(f).cuda()
    bd = torch.empty_like(fd)
    S.sem_mass(h, bd, fd, S.SEM_FP64, 1)
    ann = {"workload": "O-grid annulus r in [0.5, 8], 64x32x24 elements (ratio 1.1), N=7, periodic span 4, "
                       "Fourier RHS |k| <= 4 (seed 5)", "n_local": m.n_local, "n_unique_free": info["n_free"],
           "generation_s": gen_s}
    for name, o in modes:
        _, st = _timed_solve(S, torch, h, bd, m.n_local, o, reps=2)
        ann[name] = _solve_report(st, m.n_local, info["n_free"])
    ann["speedup_mixed_vs_fp64"] = ann["fp64"]["time_ms"] / ann["mixed"]["time_ms"]
    ann["speedup_mixed_vs_fp64_pair"] = ann["fp64_pair"]["time_ms"] / ann["mixed"]["time_ms"]
    ann["speedup_mixed_carry_vs_fp64"] = ann["fp64"]["time_ms"] / ann["mixed_carry"]["time_ms"]
    ann["speedup_mixed_carry_capped_vs_fp64"] = ann["fp64"]["time_ms"] / ann["mixed_carry_capped"]["time_ms"]
    peak, _ = _peaks()
    stream = torch.cuda.current_stream()
    for name, prec, dt_, bpp in (("ax_fp64", S.SEM_FP64, torch.float64, 64),
                                 ("ax_fp64_pair", S.SEM_FP64_PAIR, torch.float64, 64),
                                 ("ax_fp32", S.SEM_FP32, torch.float32, 32)):
        u = torch.randn(m.n_local, dtype=dt_, device="cuda")
        w = torch.empty_like(u)
        for _ in range(3):
            S.sem_ax(h, w, u, prec, 0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(10):
            S.sem_ax(h, w, u, prec, 0)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 10
        ann[name] = {"ms": t, "gb_s": bpp * m.n_local / (t * 1e-3) / 1e9,
                     "frac_hbm": bpp * m.n_local / (t * 1e-3) / 1e9 / peak}
    S.sem_destroy(h)
    out["annulus_64x32x24_N7"] = ann
    out["helmholtz_velocity"] = _helmholtz_suite(S, torch)
    out["gmres_schwarz"] = _gmres_suite(S, torch)
    out["time_step"] = _timestep_suite(S, torch)
    print(json.dumps(out), flush=True)


def _gmres_suite(S, torch):
    """The paper's pressure solver (Sec. II-B): restarted flexible GMRES with
    the two-level Schwarz preconditioner, on the 4^3 cube and the 32^3
    deformed cube, to 1e-10: FP64 (native operator and preconditioner), FP64
    with the pair operator and an FP32 preconditioner, and the mixed form
    (FP32 cycles inside FP64 restarts), beside Jacobi-PCG (FP64) and the
    mixed CG refinement on the same handle."""
    res = {}
    for name, (m, h1, b) in (("cube_4^3_N7", _cube_problem()), ("deformed_cube_32^3_N7", W.deformed_cube(32, 7, seed=2))):
        h = S.sem_setup(m.E, m.lx, m.coords, m.gid, m.mask, h1, S.SEM_FLAG_SCHWARZ)
        info = S.sem_get_info(h)
        bd = torch.from_numpy(b).cuda()
        row = {"n_local": m.n_local}
        for mode, o in (("gmres_fp64", {"mode": S.SEM_MODE_GMRES, "tol": 1e-10}),
                        ("gmres_fp64_pair_pc32", {"mode": S.SEM_MODE_GMRES, "tol": 1e-10,
                                                  "precision": S.SEM_FP64_PAIR, "precond_precision": S.SEM_FP32}),
                        ("gmres_mixed", {"mode": S.SEM_MODE_GMRES, "tol": 1e-10, "precision": S.SEM_FP32}),
                        ("fp64_pcg", {"mode": S.SEM_MODE_FP64, "tol": 1e-10}),
                        ("mixed_pcg", {"mode": S.SEM_MODE_MIXED_IR, "tol": 1e-10, **MIXED_OPTS})):
            _, st = _timed_solve(S, torch, h, bd, m.n_local, o, reps=2)
            row[mode] = _solve_report(st, m.n_local, info["n_free"])
        row["speedup_gmres_fp64_vs_fp64_pcg"] = row["fp64_pcg"]["time_ms"] / row["gmres_fp64"]["time_ms"]
        row["speedup_gmres_mixed_vs_mixed_pcg"] = row["mixed_pcg"]["time_ms"] / row["gmres_mixed"]["time_ms"]
        S.sem_destroy(h)
        torch.cuda.empty_cache()
        res[name] = row
    return res


def _timestep_suite(S, torch):
    """The rest of a time step's solver work on the 32^3 deformed cube:
    projection onto previous solutions over a sequence of 30 time-correlated
    pressure right-hand sides (space of 20, the paper's reset interval on
    GPUs), pipelined against standard FP64 PCG, and the pressure right-hand
    side -div(vhat)/dt + (1/Re) div(curl(omega)) with the gradient kernels."""
    m, h1, _ = W.deformed_cube(32, 7, seed=2)
    h = S.sem_setup(m.E, m.lx, m.coords, m.gid, m.mask, h1, S.SEM_FLAG_METRICS | S.SEM_FLAG_SCHWARZ)
    n = m.n_local
    x, y, z = m.xyz()
    res = {"workload": "32^3 deformed cube, N=7; b_k = mask QQ^T B f(t_k), f = sin(pi(x+t)) sin(pi y) sin(pi z)(1+xy)"
                       " + 0.3 cos(3 pi (y-t)) z, t_k = 0.03 k, k < 30", "n_local": n}
    fd = torch.empty(n, dtype=torch.float64, device="cuda")
    bs = []
    for k in range(30):
        t = 0.03 * k
        f = np.sin(np.pi * (x + t)) * np.sin(np.pi * y) * np.sin(np.pi * z) * (1.0 + x * y) \
            + 0.3 * np.cos(3 * np.pi * (y - t)) * z
        fd.copy_(torch.from_numpy(f))
        bk = torch.empty_like(fd)
        S.sem_mass(h, bk, fd, S.SEM_FP64, 1)
        bs.append(bk)
    xd = torch.zeros(n, dtype=torch.float64, device="cuda")
    for name, o in (("mixed", {"mode": S.SEM_MODE_MIXED_IR, "tol": 1e-10}),
                    ("mixed_projection_20", {"mode": S.SEM_MODE_MIXED_IR, "tol": 1e-10, "projection": 20}),
                    ("fp64_pair", {"mode": S.SEM_MODE_FP64, "precision": S.SEM_FP64_PAIR, "tol": 1e-10}),
                    ("fp64_pair_projection_20", {"mode": S.SEM_MODE_FP64, "precision": S.SEM_FP64_PAIR,
                                                 "tol": 1e-10, "projection": 20}),
                    ("gmres_mixed", {"mode": S.SEM_MODE_GMRES, "precision": S.SEM_FP32, "tol": 1e-10}),
                    ("gmres_mixed_projection_20", {"mode": S.SEM_MODE_GMRES, "precision": S.SEM_FP32, "tol": 1e-10,
                                                   "projection": 20})):
        S.sem_projection_reset(h)
        xd.zero_()
        S.sem_cg_solve(h, xd, bs[0], {**o, "projection": 0})  # warm-up (autotune, graphs)
        its, ms, starts, ok = [], 0.0, [], True
        for k in range(30):
            xd.zero_()
            st = S.sem_cg_solve(h, xd, bs[k], o)
            its.append(st["iterations"])
            starts.append(st["relres_start"])
            ms += st["time_ms"]
            ok = ok and st["status"] == S.SEM_OK and st["relres"] <= 1e-10
        res[name] = {"total_ms": ms, "mean_iterations": float(np.mean(its)), "iterations": its,
                     "start_residual_last": starts[-1], "all_converged": ok}
    S.sem_projection_reset(h)
    res["speedup_projection_mixed"] = res["mixed"]["total_ms"] / res["mixed_projection_20"]["total_ms"]
    res["speedup_projection_fp64_pair"] = res["fp64_pair"]["total_ms"] / res["fp64_pair_projection_20"]["total_ms"]
    res["speedup_projection_gmres_mixed"] = res["gmres_mixed"]["total_ms"] / res["gmres_mixed_projection_20"]["total_ms"]
    # pipelined PCG against the standard loop (both native FP64)
    pipe = {}
    for name, o in (("fp64_pcg", {"mode": S.SEM_MODE_FP64, "tol": 1e-10}),
                    ("fp64_pipelined", {"mode": S.SEM_MODE_FP64, "tol": 1e-10, "pipelined": 1})):
        _, st = _timed_solve(S, torch, h, bs[5], n, o, reps=1)
        pipe[name] = {"time_ms": st["time_ms"], "iterations": st["iterations"], "relres": st["relres"],
                      "status": st["status"]}
    res["pipelined"] = pipe
    # pressure right-hand side and gradient (one call each, CUDA events, best of 10)
    v = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in
         (np.sin(np.pi * x) * np.cos(np.pi * y), np.cos(np.pi * y) * z, x * y * z)]
    w = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (y * z, np.sin(np.pi * z), x * x)]
    out = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(3)]
    b = torch.empty(n, dtype=torch.float64, device="cuda")

    def best_ms(fn):
        fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        best = None
        for _ in range(10):
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1)
            best = t if best is None else min(best, t)
        return best

    res["pressure_rhs_ms"] = best_ms(lambda: S.sem_pressure_rhs(h, *v, *w, 2e-5, 30000.0, b))
    res["grad_ms"] = best_ms(lambda: S.sem_grad(h, v[0], *out))
    res["grad_gb_s"] = n * (8 + 72 + 24) / (res["grad_ms"] * 1e-3) / 1e9
    S.sem_destroy(h)
    torch.cuda.empty_cache()
    return res


def _cube_problem():
    m, f = W.cube_sines(4, 7)
    import oracle
    return m, None, oracle.Problem(m).mass(f, assemble=True)


def _helmholtz_suite(S, torch):
    """The velocity solve of a time step (Sec. II-B: P-CG with a Jacobi-type
    preconditioner, tolerance 1e-8): the Helmholtz operator h1 K + h2 B with
    h1 = 1/Re (Re = 30000) and h2 = gamma_0 / dt (BDF3, gamma_0 = 11/6,
    dt = 2e-5, the rotor case's time step) on the 32^3 deformed cube, random
    right-hand side, FP64 and mixed."""
    m, _, b = W.deformed_cube(32, 7, seed=2)
    h1 = np.full(m.n_local, 1.0 / 30000.0)
    h2 = np.full(m.n_local, (11.0 / 6.0) / 2e-5)
    h = S.sem_setup(m.E, m.lx, m.coords, m.gid, m.mask, h1)
    S.sem_set_helmholtz(h, h2)
    info = S.sem_get_info(h)
    bd = torch.from_numpy(b).cuda()
    res = {"workload": "32^3 deformed cube, N=7, Helmholtz h1 = 1/30000, h2 = (11/6)/2e-5, random RHS, tol 1e-8",
           "n_local": m.n_local}
    for name, o in (("fp64", {"mode": S.SEM_MODE_FP64, "tol": 1e-8}),
                    ("fp64_pair", {"mode": S.SEM_MODE_FP64, "precision": S.SEM_FP64_PAIR, "tol": 1e-8}),
                    ("mixed", {"mode": S.SEM_MODE_MIXED_IR, "tol": 1e-8})):
        _, st = _timed_solve(S, torch, h, bd, m.n_local, o)
        res[name] = _solve_report(st, m.n_local, info["n_free"])
    res["speedup_mixed_vs_fp64"] = res["fp64"]["time_ms"] / res["mixed"]["time_ms"]
    S.sem_destroy(h)
    return res


def main():
    args = _args()
    if args.impl == "reference":
        run_reference(args)
    elif args.suite:
        run_suite(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
