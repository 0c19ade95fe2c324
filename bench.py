"""Benchmark: leftmost eigenpairs/s to residual 1e-8 on GB300.

Workload (one "step"): eig_leftmost(N = 500, tol = 1e-8) on the symmetric
kNN graph Laplacian (k = 10, weights exp(-d^2/sigma^2)) of 200,000 points
sampled area-uniformly on a torus (R = 1, r = 0.3) with 1e-3 Gaussian jitter,
plus 1e-6 I, FP64 CSR (seeded, synthetic).  The decomposition is built once
outside the timed region (its time is reported as build_s); each timed step
is one full eigensolve with the matrix and levels resident in HBM.  L2 is
flushed (a 512 MB write) before every timed step.

``--precision`` picks the timed form (fp64 = MMD_FP64, mixed = MMD_MIXED:
FP32 PCG on the coarse levels inside FP64 refinement, mixed_all =
MMD_MIXED_ALL: FP32 level-0 CG with FP64 reliable updates as well).  The other
of fp64 / mixed is then timed for ONE step on the same handle and reported
under ``compare`` with its per-eigenpair error against the timed form
(skipped, and said so, when the time budget would be exceeded); the mixed form
runs there with mg_refine = 0, its level-0 refinement block in the wide
double-float kernel.

Also reported:
  * t_level_ms -- wall time per level of the last timed step;
  * e2e     -- the same metric through the public API with host buffers:
               mmd_build from a host CSR + eig_leftmost into host outputs,
               one run;
  * spmv    -- standalone FP64 SELL SpMV GB/s on the 128^3 7-point operator
               (14.6M nnz, larger than L2);
  * roofline of the dominant kernel (the persistent CG/PCG solver) from its
               event-timed launches inside the timed steps;
  * reference_eigs -- the eigenvalues against an independent shift-invert
               Lanczos (scipy ARPACK) result stored with its input hash;
  * cpu_baseline -- the CPU oracle on a bounded sample of the same workload.

Expected wall time at --steps 20 --warmup 5 (one step ~24 s): about 12 minutes;
the optional legs are skipped once the run would pass --budget-s.
``--impl reference`` times the CPU oracle instead (the reference arm).
Multi-GPU (torchrun): replicas only -- every rank solves its own copy of the
workload, no data-path collective; value = total eigenpairs / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = {"workload": "torus_knn_200k", "n": 200000, "k": 10, "N": 500, "tol": 1e-8,
            "matrix": "torus kNN Laplacian + 1e-6 I, FP64 CSR", "l2": "flushed before each step"}
# bounded oracle sample of the same workload kind: the same generator at 5,000 points, N = 20
SAMPLE = {"npts": 5000, "N": 20, "tol": 1e-8}
FALLBACK_HBM = 6800.0
PRECISIONS = {"fp64": 0, "mixed": 1, "mixed_all": 2}  # MMD_FP64, MMD_MIXED, MMD_MIXED_ALL
# FP64 peak of the GB300: 152 SMs x 1.68 FP64 FMA per clock per SM (measured: chains of
# independent FMAs on one SM, 4+ warps, timed with clock64) x 2 flops x 2.070 GHz
FP64_FMA_PER_CLK_SM = 1.68
FP64_PEAK_TFLOPS = 152 * FP64_FMA_PER_CLK_SM * 2 * 2.070e9 / 1e12  # 1.057
FP64_NOMINAL_TFLOPS = 1.25
# DRAM bytes (read + write) per launch of the level-0 Operator OP kernel, solve_kernel<1, double, 0>,
# from the ncu capture summarised in profiles/solve_kernel_op_torus_knn_200k_level0.md (32.63 MB read +
# 0.81 MB written: the 30 MB level-0 matrix and the vectors once, every iteration after the first from L2)
TRAFFIC_PER_LAUNCH = 33.44e6
REF_EIGS = os.path.join(ROOT, "tests", "golden", "torus_knn_200k_eigs.json")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            for k in ("hbm_gbs", "hbm_GBs", "hbm"):
                if k in d:
                    return float(d[k]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) >= 9:
                for nm, v in zip(names, r[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


# ------------------------------------------------------------------ oracle (CPU) leg
def oracle_sample_worker(steps: int):
    """Run in a fresh single-threaded process: time the oracle on the bounded sample."""
    import workloads as W
    from oracle import eig as OE
    from oracle import mmd as OM

    A = W.torus_knn(SAMPLE["npts"], seed=W.BASE_SEED + 1)
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        D = OM.build(A, OM.BuildOpts())
        OE.eig_leftmost(D, SAMPLE["N"], SAMPLE["tol"])
        times.append(time.perf_counter() - t0)
    print(json.dumps({"times": times}))


def run_oracle(steps: int, threads: int = 1) -> dict:
    t = str(max(1, threads))
    env = dict(os.environ, OMP_NUM_THREADS=t, OPENBLAS_NUM_THREADS=t, MKL_NUM_THREADS=t,
               CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-worker", str(steps)],
                       capture_output=True, text=True, env=env, cwd=ROOT)
    if r.returncode != 0:
        raise RuntimeError("oracle worker failed: " + r.stderr[-2000:])
    times = json.loads(r.stdout.strip().splitlines()[-1])["times"]
    return {"times": times, "value": SAMPLE["N"] / float(np.median(times))}


def sample_desc(threads: int = 1):
    return (f"oracle (numpy/scipy FP64, BLAS/OpenMP threads limited to {threads}): build + eig_leftmost "
            f"N={SAMPLE['N']} tol={SAMPLE['tol']} on the same generator at {SAMPLE['npts']} points (a bounded "
            f"sample of the 200k workload)")


# ------------------------------------------------------------------ GPU arm
def input_hash(A) -> str:
    """sha256 of the CSR bytes (row pointers, columns, values) of a workload."""
    import hashlib

    hsh = hashlib.sha256()
    for arr in (A.rowptr, A.col, A.val):
        hsh.update(np.ascontiguousarray(arr).tobytes())
    return hsh.hexdigest()


def reference_check(A, lam) -> dict | None:
    """Relative eigenvalue errors against the stored independent reference
    (scipy eigsh shift-invert) when its input hash matches this matrix."""
    if not os.path.exists(REF_EIGS):
        return None
    ref = json.load(open(REF_EIGS))
    import hashlib

    hp = hashlib.sha256()
    for arr in (A.rowptr, A.col):
        hp.update(np.ascontiguousarray(arr).tobytes())
    same = (hp.hexdigest() == ref.get("pattern_sha256")
            and abs(float(np.sum(A.val ** 2)) - ref["val_sq_sum"]) <= 1e-12 * ref["val_sq_sum"])
    if not same:
        return {"error": "the matrix differs from the stored reference's", "sha256": input_hash(A)}
    r = np.asarray(ref["eigenvalues"][:len(lam)])
    lam = np.asarray(lam)
    rel = np.abs(lam - r) / np.abs(r)
    # the 1e-6-shifted zero mode is compared in absolute terms against ||A|| (its relative
    # accuracy is bounded by u ||A|| / lambda_1)
    absn = np.abs(lam - r) / float(ref["norm_A_inf"])
    return {"source": ref["method"], "pairs": int(len(r)), "max_rel_err": float(rel.max()),
            "max_rel_err_excl_first": float(rel[1:].max()) if len(rel) > 1 else None,
            "max_abs_err_over_normA": float(absn.max()), "worst_index": int(np.argmax(rel))}


def gpu_arm(args, rank, world):
    import torch

    import paper_1804_03415_gb300 as G
    import workloads as W

    t_start = time.perf_counter()
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    A = W.torus_knn(WORKLOAD["n"], k=WORKLOAD["k"], seed=W.BASE_SEED + 1)
    N, tol = WORKLOAD["N"], WORKLOAD["tol"]
    t0 = time.perf_counter()
    h = G.MMD(A.rowptr, A.col, A.val)
    build_s = time.perf_counter() - t0
    lam = torch.zeros(N, dtype=torch.float64, device="cuda")
    V = torch.zeros((N, A.n), dtype=torch.float64, device="cuda")
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    prec = PRECISIONS[args.precision]

    def step(profile, precision=prec, out=(lam, V), mg_refine=None):
        return h.eig_leftmost(N, tol, out=out, allow_noconv=True, stream=sptr, profile=profile,
                              precision=precision, mg_op=args.mg_op,
                              mg_refine=args.mg_refine if mg_refine is None else mg_refine)[2]

    def timed(steps, precision, out=(lam, V), mg_refine=None):
        ev, sts = [], []
        for _ in range(steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            sts.append(step(1, precision, out, mg_refine))
            e1.record(stream)
            torch.cuda.synchronize()
            ev.append(e0.elapsed_time(e1))
        return ev, sts

    for _ in range(args.warmup):
        step(0)
    dist_barrier(world)
    clk = ClockSampler(dev)
    clk.start()
    ev, stats = timed(args.steps, prec)
    clocks = clk.stop()
    ms_local = float(np.sum(ev))
    ms = dist_max(ms_local, world)
    value = job_value(world, N, args.steps, ms)
    lam_main = lam.cpu().numpy().copy()
    step_s = ms_local / 1e3 / args.steps
    # the other precision on the same handle: one step, with its per-eigenpair
    # difference from the timed form; skipped when it would overrun the budget
    compare = None
    if not args.no_compare:
        other = "fp64" if args.precision != "fp64" else "mixed"
        projected = (time.perf_counter() - t_start) + 3.5 * step_s + build_s + 60
        if projected > args.budget_s:
            compare = {"precision": other, "skipped": f"time budget: projected {projected:.0f} s > {args.budget_s} s"}
        else:
            lam2 = torch.zeros_like(lam)
            V2 = torch.zeros_like(V)
            dist_barrier(world)
            # the mixed form with its double-float refinement (all columns in one wide launch)
            mg2 = 0 if other == "mixed" else args.mg_refine
            ev2, st2 = timed(1, PRECISIONS[other], out=(lam2, V2), mg_refine=mg2)
            ms2 = dist_max(float(np.sum(ev2)), world)
            l2 = lam2.cpu().numpy()
            rel = np.abs(l2 - lam_main) / np.abs(lam_main)
            # subspace agreement: smallest singular value of V_main^T V_other per cluster is
            # summarised by the worst column's |cos| (clusters of near-equal values included)
            cosines = torch.linalg.svdvals(V.to(torch.float64) @ V2.T.to(torch.float64)).cpu().numpy()
            compare = {"precision": other, "mg_refine": mg2, "steps": 1, "value": job_value(world, N, 1, ms2),
                       "unit": "eigenpairs/s",
                       "ms_per_step": ms2,
                       "residual": {"max_rel": st2[-1]["max_rel_residual"], "n_converged": st2[-1]["n_converged"]},
                       "vs_timed_form": {"max_rel_eig_diff": float(rel.max()),
                                         "max_rel_eig_diff_excl_first": float(rel[1:].max()),
                                         "min_subspace_cos": float(cosines.min())},
                       "t_level_ms": st2[-1]["t_level_ms"], "pcg_iters": st2[-1]["pcg_iters"],
                       "refine_pcg_iters": st2[-1]["refine_pcg_iters"]}
            del V2
    # Section 8's comparison: IRLM with plain CG and no decomposition (MMD_IRLM_CG)
    # on the same handle, one step, when the budget allows
    irlm = None
    if not args.no_irlm:
        projected = (time.perf_counter() - t_start) + 3.0 * step_s + build_s + 60
        if projected > args.budget_s:
            irlm = {"skipped": f"time budget: projected {projected:.0f} s > {args.budget_s} s"}
        else:
            lam3 = torch.zeros_like(lam)
            V3 = torch.zeros_like(V)
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st3 = h.eig_leftmost(N, tol, out=(lam3, V3), allow_noconv=True, stream=sptr, method=1,
                                 precision=PRECISIONS["fp64"])[2]
            e1.record(stream)
            torch.cuda.synchronize()
            ms3 = dist_max(e0.elapsed_time(e1), world)
            l3 = lam3.cpu().numpy()
            irlm = {"method": "IRLM-CG (implicitly restarted Lanczos, plain CG solves, no decomposition)",
                    "steps": 1, "value": job_value(world, N, 1, ms3), "unit": "eigenpairs/s", "ms_per_step": ms3,
                    "hierarchical_speedup": ms3 / (ms / args.steps),
                    "residual": {"max_rel": st3["max_rel_residual"], "n_converged": st3["n_converged"]},
                    "max_rel_eig_diff_vs_timed_form": float((np.abs(l3 - lam_main) / np.abs(lam_main)).max()),
                    "counters": {k: st3[k] for k in ("op_calls", "pcg_iters", "restarts", "lanczos_steps")}}
            del V3
    # end to end: host CSR in, host outputs out, through the public API (one run)
    import ctypes as C

    lam_h = np.zeros(N)
    V_h = np.zeros((N, A.n))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h2 = G.MMD(A.rowptr, A.col, A.val)
    o2 = G.eig_opts(stream=sptr, precision=prec)
    s2 = G._lib.mmd_eig_stats()
    rc = h2._lib.eig_leftmost(h2.h, N, tol, C.byref(o2), lam_h.ctypes.data, V_h.ctypes.data, 0, C.byref(s2))
    torch.cuda.synchronize()
    e2e_s = dist_max(time.perf_counter() - t0, world)
    h2.close()
    if rc not in (0, -3):
        raise RuntimeError(f"e2e eig_leftmost failed: {rc}")
    h2d = A.nnz * 12 + (A.n + 1) * 4
    d2h = N * A.n * 8 + N * 8
    # roofline of the solver kernel
    pcg_ms = sum(s["pcg_ms"] for s in stats)
    pcg_bytes = sum(s["pcg_bytes"] for s in stats)
    pcg_flops = sum(s["pcg_flops"] for s in stats)
    pcg_launches = sum(s["pcg_launches"] for s in stats)
    op_ms = sum(s["op0_ms"] for s in stats)
    op_bytes = sum(s["op0_bytes"] for s in stats)
    op_flops = sum(s["op0_flops"] for s in stats)
    op_launches = sum(s["op0_launches"] for s in stats)
    op_iters = sum(s["op0_iters"] for s in stats)
    peak, src = peaks()
    gbs = (pcg_bytes / (pcg_ms / 1e3) / 1e9) if pcg_ms > 0 else None
    tflops = (pcg_flops / (pcg_ms / 1e3) / 1e12) if pcg_ms > 0 else None
    op_gbs = (op_bytes / (op_ms / 1e3) / 1e9) if op_ms > 0 else None
    op_tflops = (op_flops / (op_ms / 1e3) / 1e12) if op_ms > 0 else None
    st0 = stats[-1]
    spmv = spmv_bench(G, W, torch, sptr, peak)
    out = {
        "metric": "leftmost eigenpairs/sec to residual 1e-8", "value": value, "unit": "eigenpairs/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
        "config": dict(WORKLOAD, precision=args.precision, mg_refine=args.mg_refine, mg_op=args.mg_op,
                       parallelism=f"replicas{world}"),
        "build_s": build_s,
        "residual": {"max_rel": st0["max_rel_residual"], "n_converged": st0["n_converged"]},
        "reference_eigs": reference_check(A, lam_main),
        "t_level_ms": st0["t_level_ms"],
        "compare": compare,
        "irlm_cg": irlm,
        "counters": {k: st0[k] for k in ("op_calls", "pcg_iters", "inner_iters", "b_iters", "refine_pcg_calls",
                                         "refine_pcg_iters", "restarts", "lanczos_steps", "refine_iters",
                                         "n_levels")},
        "e2e": {"value": world * N / e2e_s, "unit": "eigenpairs/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "includes": "mmd_build from host CSR + eig_leftmost to host, one run"},
        "gpu_launches": int(sum(s["kernel_launches"] for s in stats)),
        "roofline": {"kernel": "solve_kernel<1, double, 0> (level-0 Operator OP: CG on A, one column)",
                     "bound": "alu", "achieved": op_tflops, "peak": FP64_PEAK_TFLOPS,
                     "peak_source": "derived: 152 SMs x 1.68 FP64 FMA/clk/SM (measured on one SM) x 2 x 2.07 GHz; "
                                    f"nominal {FP64_NOMINAL_TFLOPS}",
                     "unit": "TFLOP/s", "frac": (op_tflops / FP64_PEAK_TFLOPS) if op_tflops else None,
                     "traffic": TRAFFIC_PER_LAUNCH if args.precision == "fp64" else None,
                     "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch "
                                       "(profiles/solve_kernel_op_torus_knn_200k_level0.md)",
                     "launches": op_launches, "iterations": op_iters,
                     "algorithmic_flops_per_launch": (op_flops / op_launches) if op_launches else None,
                     "share_of_step": op_ms / max(ms_local, 1e-9),
                     "note": "latency bound (grid barriers, reduction rounds, L2 gathers of the SpMV): the 30 MB "
                             "level-0 matrix stays in L2 across iterations; algorithmic flops per iteration "
                             "2 nnz(A) + 10 n",
                     "hbm_view": {"achieved": op_gbs, "peak": peak, "peak_source": src, "unit": "GB/s",
                                  "frac": (op_gbs / peak) if op_gbs else None,
                                  "bytes": "12 nnz + 4 n per iteration (matrix) + 72 n (vectors)"}},
        "solver_all": {"kernel": "solve_kernel, every instance (OP, refinement tiles, coarse levels)",
                       "achieved_tflops": tflops, "frac_of_fp64_peak": (tflops / FP64_PEAK_TFLOPS) if tflops else None,
                       "achieved_gbs": gbs, "launches": pcg_launches, "share_of_step": pcg_ms / max(ms_local, 1e-9),
                       "note": "the refinement's tiles run on four concurrent lanes, so their event-timed "
                               "durations overlap"},
        "spmv": spmv,
        "clocks": clocks,
        "wall_s": time.perf_counter() - t_start,
    }
    h.close()
    return out


def spmv_bench(G, W, torch, sptr, peak):
    """Standalone FP64 SELL SpMV on the 128^3 7-point operator (175 MB of
    matrix, above L2): 20 back-to-back kernels between two events, checked
    bit-identical to the public mmd_level_spmv."""
    A = W.fd3d(128, seed=W.BASE_SEED + 2)
    h = G.MMD(A.rowptr, A.col, A.val, k_max=0)
    x = torch.rand(A.n, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    y2 = torch.empty_like(x)
    ms = h.level_spmv_timed(0, 0, x, y, reps=20, stream=sptr)
    h.level_spmv(0, 0, x, y2, stream=sptr)
    torch.cuda.synchronize()
    same = bool(torch.equal(y, y2))
    byts = 12.0 * A.nnz + 20.0 * A.n
    gbs = byts / (ms / 1e3) / 1e9
    variant, vms = h.spmv_tuning(0, 0)
    h.close()
    return {"matrix": "fd3d 128^3 7-point, n=2097152, nnz=14581760, FP64", "ms": ms, "GB_s": gbs,
            "frac_of_hbm": gbs / peak, "bytes_per_call": byts, "bit_identical_to_level_spmv": same,
            "bytes": "12 nnz + 20 n (values, columns, row pointers, x once, y)",
            "autotune": {"chosen_variant": variant, "ms_per_variant": vms,
                         "variants": "entries in flight / block size / min blocks per SM: 4/128/10, 4/256/5, "
                                     "8/128/8, 8/256/4, 8/512/2, 16/128/4"}}


# ------------------------------------------------------------------ distributed helpers
def dist_init(backend: str = "nccl"):
    """Replica group from the torchrun environment (one process per GPU; gloo
    for the CPU tests of this path)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist

        if backend == "nccl":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group(backend)
    return rank, world


def dist_barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def dist_max(v, world):
    """Maximum of v over the replicas (the job time is the slowest rank's)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, n_eig: int, steps: int, max_ms: float) -> float:
    """Whole-job eigenpairs/s: every replica solves its own copy, so the
    units are world * N * steps over the slowest rank's time (weak scaling)."""
    return world * n_eig * steps / (max_ms / 1e3)


def kernel_case(which: str, streams: int = 8):
    """Small fixed launches for ncu captures: 'op' = three Operator OP solves on
    level 0 of the torus 200k workload (one solver launch each), 'block' =
    three 8-column OP solves there (two of the refinement's 4-column tiles each), 'eig' = one full
    eig_leftmost of the workload (the launch list of a step), 'spmv' = three
    FP64 SpMVs on the 128^3 operator."""
    import torch

    import paper_1804_03415_gb300 as G
    import workloads as W

    if which == "op":
        A = W.torus_knn(WORKLOAD["n"], k=WORKLOAD["k"], seed=W.BASE_SEED + 1)
        h = G.MMD(A.rowptr, A.col, A.val, k_max=1)
        x = torch.rand(A.n, dtype=torch.float64, device="cuda")
        y = torch.empty_like(x)
        its, ms = [], []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            its.append(h.level_op(0, x, y, 1e-6))
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        print(json.dumps({"kernel_case": "op", "iters": its, "ms": ms,
                          "us_per_iter": [1e3 * t / i for t, i in zip(ms, its)]}))
    elif which == "eig":
        A = W.torus_knn(WORKLOAD["n"], k=WORKLOAD["k"], seed=W.BASE_SEED + 1)
        h = G.MMD(A.rowptr, A.col, A.val)
        st = h.eig_leftmost(WORKLOAD["N"], WORKLOAD["tol"], allow_noconv=True)[2]
        print(json.dumps({"kernel_case": "eig", "kernel_launches": st["kernel_launches"],
                          "n_converged": st["n_converged"]}))
    elif which == "vcycle":
        # V-cycle preconditioner of the level-0 refinement on the torus 200k levels:
        # 20 applications to 4 columns, event-timed, and one warm-started refinement-type
        # PCG solve of 4 columns with and without it
        A = W.torus_knn(WORKLOAD["n"], k=WORKLOAD["k"], seed=W.BASE_SEED + 1)
        h = G.MMD(A.rowptr, A.col, A.val)
        R = torch.rand((4, A.n), dtype=torch.float64, device="cuda")
        Z = torch.empty_like(R)
        h.level_vcycle(R, Z)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(20):
            h.level_vcycle(R, Z)
        e1.record()
        torch.cuda.synchronize()
        print(json.dumps({"kernel_case": "vcycle", "ms_per_vcycle_4cols": e0.elapsed_time(e1) / 20}))
    elif which == "batch":
        # the batched workload: 64 random geometric graphs (sizes log-uniform 2k-50k, mean degree 8,
        # unit weights, Laplacian + 1e-6 I), N = 20 leftmost eigenpairs each, tol 1e-8, one call
        mats = W.rgg_batch()
        t0 = time.perf_counter()
        hs = [G.MMD(A.rowptr, A.col, A.val) for A in mats]
        build_s = time.perf_counter() - t0
        Ns = [20] * len(mats)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = G.eig_leftmost_batched(hs, Ns, 1e-8, streams=streams, allow_noconv=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        worst = max(r[2]["max_rel_residual"] for r in res)
        conv = sum(r[2]["n_converged"] for r in res)
        print(json.dumps({"kernel_case": "batch", "streams": streams, "problems": len(mats),
                          "sum_n": int(sum(A.n for A in mats)),
                          "build_s": build_s, "solve_s": dt, "eigenpairs_per_s": sum(Ns) / dt,
                          "n_converged": conv, "worst_rel_residual": worst}))
        for x in hs:
            x.close()
        return
    elif which == "alpha":
        # Section 7's alpha sweep: beta = 1, alpha in [3, 5], on the paper-shaped SwissRoll point cloud
        # (20,000 points, kNN k = 10, weights exp(-r^2 / 0.1)); per level the most iterations one PCG
        # call on A^(k) took, alone and over log(1 / eps^(k)) with eps^(k) the level's PCG tolerance
        A = W.swissroll(20_000)
        h = G.MMD(A.rowptr, A.col, A.val)
        K = h.num_levels
        eps = [h.level(k)["eps"] for k in range(1, K + 1)]
        rows = []
        for alpha in (3.0, 3.5, 4.0, 4.5, 5.0):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = h.eig_leftmost(500, 1e-8, alpha=alpha, beta=1.0, allow_noconv=True)[2]
            torch.cuda.synchronize()
            mu1 = st["mu1"]
            # the PCG tolerance of level k >= 1 is 0.1 eps_k / mu_1 (relative), level 0 0.1 tol
            tol_k = [1e-9] + [min(0.1, max(1e-14, 0.1 * e / mu1)) for e in eps[:-1]]
            mx = st["max_pcg_iters"]
            rows.append({"alpha": alpha, "s": time.perf_counter() - t0, "max_pcg_iters": mx,
                         "max_pcg_iters_over_log": [m / np.log(1.0 / t) if t < 1 else None for m, t in zip(mx, tol_k)],
                         "n_converged": st["n_converged"], "refine_iters": st["refine_iters"],
                         "lanczos_steps": st["lanczos_steps"]})
        print(json.dumps({"kernel_case": "alpha", "workload": "swissroll_20k", "levels": K, "eps": eps,
                          "rows": rows}))
    elif which == "block":
        A = W.torus_knn(WORKLOAD["n"], k=WORKLOAD["k"], seed=W.BASE_SEED + 1)
        h = G.MMD(A.rowptr, A.col, A.val, k_max=1)
        X = torch.rand((8, A.n), dtype=torch.float64, device="cuda")
        Y = torch.empty_like(X)
        its = [h.level_op_block(0, X, Y, 1e-6) for _ in range(3)]
        print(json.dumps({"kernel_case": "block", "iters": its}))
    else:
        A = W.fd3d(128, seed=W.BASE_SEED + 2)
        h = G.MMD(A.rowptr, A.col, A.val, k_max=0)
        x = torch.rand(A.n, dtype=torch.float64, device="cuda")
        y = torch.empty_like(x)
        for _ in range(3):
            h.level_spmv(0, 0, x, y)
        torch.cuda.synchronize()
        print(json.dumps({"kernel_case": "spmv"}))
    h.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--oracle-worker", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", choices=sorted(PRECISIONS), default="fp64")
    ap.add_argument("--no-compare", action="store_true", help="skip timing the other precision")
    ap.add_argument("--no-irlm", action="store_true", help="skip the IRLM-CG baseline step")
    ap.add_argument("--mg-refine", type=int, default=2,
                    help="Chebyshev degree of the V-cycle preconditioning the level-0 refinement (0: plain CG)")
    ap.add_argument("--mg-op", type=int, default=0,
                    help="Chebyshev degree of the V-cycle preconditioning the level-0 Lanczos OP solves (0: plain CG)")
    ap.add_argument("--budget-s", type=float, default=1500.0,
                    help="wall-clock budget of the run; optional legs are skipped past it")
    ap.add_argument("--kernel-case", choices=["op", "block", "eig", "spmv", "vcycle", "batch", "alpha"], default=None)
    ap.add_argument("--streams", type=int, default=8, help="concurrent streams of the batch kernel case")
    args = ap.parse_args()
    if args.oracle_worker:
        oracle_sample_worker(args.oracle_worker)
        return
    if args.kernel_case:
        kernel_case(args.kernel_case, args.streams)
        return
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        rank = int(os.environ.get("RANK", "0"))
        if rank != 0:
            return
        nc = os.cpu_count() or 1
        o = run_oracle(args.warmup + args.steps, nc)
        t = o["times"][args.warmup:]
        val = SAMPLE["N"] * len(t) / float(np.sum(t))
        line = {"impl": "reference", "metric": "leftmost eigenpairs/sec to residual 1e-8", "value": val,
                "unit": "eigenpairs/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * float(np.mean(t)), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": dict(WORKLOAD, precision="fp64", parallelism="cpu",
                               sample=dict(SAMPLE, workload=f"torus_knn_{SAMPLE['npts']}",
                                           note="each step times the oracle on this bounded sample, not the "
                                                "200k workload: the ratio to the GPU arm compares unlike sizes")),
                "cpu_baseline": {"value": val, "unit": "eigenpairs/s", "cores": nc, "host_cores": nc,
                                 "kind": "oracle", "sample": sample_desc(nc)},
                "e2e": {"value": val, "unit": "eigenpairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return
    # the oracle leg runs first, in a child process, before any CUDA call in this one
    cpu = None
    rank0 = int(os.environ.get("RANK", "0")) == 0
    if rank0 and int(os.environ.get("WORLD_SIZE", "1")) == 1 and not args.no_cpu_baseline:
        nc = os.cpu_count() or 1
        try:
            o = run_oracle(1, nc)
            o1 = run_oracle(1, 1)
            cpu = {"value": o["value"], "unit": "eigenpairs/s", "cores": nc, "host_cores": nc,
                   "kind": "oracle", "sample": sample_desc(nc),
                   "one_thread": {"value": o1["value"], "cores": 1, "sample": sample_desc(1)}}
        except Exception as e:  # reported, never silently replaced
            cpu = {"value": None, "unit": "eigenpairs/s", "cores": nc, "kind": "oracle", "error": str(e)[-300:]}
    rank, world = dist_init()
    out = gpu_arm(args, rank, world)
    out["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
