"""Benchmark of the PHSVDS hot path on one GB300 (or N replicas).

One step = one complete PHSVDS solve (stage 1 GD+k on A^T A, switch test,
Rayleigh-Ritz post-process, stage 2 refined projection on the augmented matrix,
final residuals) of the synthetic workload, through the C ABI.  The default
workload is the random sparse 1,000,000 x 500,000 matrix (Poisson(12) entries
per row, log-normal(2) values with random signs, + 1e-3 [I; 0], seed 3), k = 20
largest triplets to 1e-14 ||A||, block 8, mixed precision against plain FP64.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--workload c3|grid] [--grid G] [--precision mixed|fp64|both]

Prints one JSON line (rank 0).  ``value`` = whole-job triplets/s with the CSR
already resident in device memory; ``e2e`` = the same solve through the same
call with pinned host buffers (host->device copy of A and device->host copy of
the singular triplets inside the timed region).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import re
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("smallest-k triplets/s to ‖r‖≤1e-14‖A‖ (mixed vs FP64); "
          "fused AᵀA SpMM GB/s")
TOL = 1e-14


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--c3s-steps", type=int, default=2,
                   help="timed mixed-precision solves of the full-size smallest-triplet workloads (C3's k=20 "
                        "smallest, the 512x512 grid's k=10 smallest; 0: skip)")
    p.add_argument("--c3s-mixed-inner", type=int, default=2,
                   help="opts.mixed_inner of those mixed solves (2: Jacobi-Davidson in the FP32 stage too)")
    p.add_argument("--workload", default="c3", choices=["c3", "grid"],
                   help="c3: random sparse 1e6 x 5e5, k=20 largest (default); grid: weighted grid gradient, "
                        "k=10 smallest")
    p.add_argument("--grid", type=int, default=64, help="grid side of the weighted gradient workload")
    p.add_argument("--sigma-log", type=float, default=1.0)
    p.add_argument("--k", type=int, default=0, help="triplets (0: the workload's own, 20 for c3, 10 for grid)")
    p.add_argument("--block", type=int, default=0, help="block size (0: the workload's own, 8 for c3, 4 for grid)")
    p.add_argument("--precision", default="both", choices=["mixed", "fp64", "both"])
    p.add_argument("--precond", default="none", choices=["none", "jacobi"])
    p.add_argument("--jd", action="store_true",
                   help="solve the workload by the Jacobi-Davidson path (Jacobi preconditioner, scaled inner solves "
                        "in stage 1, JDQMR in stage 2, ||A|| estimated)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-forms", action="store_true", help="skip the small runs of the preconditioned forms")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=15.0, help="bound of each oracle sample (CPU baseline)")
    p.add_argument("--ref-iters", type=int, default=0,
                   help="oracle outer iterations per reference-arm step (0: 4 for c3, 1000 for grid)")
    p.add_argument("--oracle-sample", action="store_true", help=argparse.SUPPRESS)
    p.add_argument("--spmm-only", action="store_true", help="only the full-size fused A^T A SpMM timings")
    p.add_argument("--kernel", default="", choices=["", "cgs", "tall"],
                   help="time one tall-skinny kernel at the 1e6 x 5e5 solve's shape: cgs = block Gram-Schmidt pass "
                        "(55 basis columns against 8), tall = V Y (35 columns to 21)")
    p.add_argument("--kernel-dtype", default="f64", choices=["f64", "f32"])
    p.add_argument("--kernel-reps", type=int, default=10)
    p.add_argument("--spmm-cases", default="c2,c3",
                   help="full-size SpMM workloads: c2 (512^2 grid), c3 (1e6 x 5e5), or none")
    p.add_argument("--spmm-reps", type=int, default=10)
    p.add_argument("--spmm-sweep", action="store_true", help="time every group width around the automatic one")
    p.add_argument("--batched", action="store_true",
                   help="batched workload: many uneven random sparse matrices, batched mixed vs sequential FP64")
    p.add_argument("--batch-count", type=int, default=64)
    p.add_argument("--batch-nlo", type=int, default=2000)
    p.add_argument("--batch-nhi", type=int, default=60000)
    p.add_argument("--batch-k", type=int, default=5)
    p.add_argument("--batch-concurrency", type=int, default=4)
    p.add_argument("--batch-no-seq", action="store_true", help="skip the sequential FP64 reference solves")
    p.add_argument("--learned", action="store_true",
                   help="learned-preconditioner workload: train, then none / Jacobi / network on held-out operators")
    p.add_argument("--learned-grid", type=int, default=32)
    p.add_argument("--learned-train", type=int, default=200)
    p.add_argument("--learned-test", type=int, default=10)
    p.add_argument("--learned-epochs", type=int, default=100)
    p.add_argument("--learned-cg-steps", type=int, default=3)
    p.add_argument("--learned-stall", type=int, default=200, help="stall window of the learned correction")
    a = p.parse_args()
    if a.k <= 0:
        a.k = 20 if a.workload == "c3" else 10
    if a.block <= 0:
        a.block = 8 if a.workload == "c3" else 4
    if a.ref_iters <= 0:
        a.ref_iters = 4 if a.workload == "c3" else 1000
    return a


def workload(a):
    """The synthetic matrix and the JSON config of the benchmark workload."""
    from paper_1408_5535_gb300 import synth
    if a.workload == "c3":
        A = synth.random_sparse(1000000, 500000, 12.0, 3)
        cfg = {"workload": f"random sparse 1000000x500000, Poisson(12) entries per row at uniform columns, "
                           f"log-normal(sigma=2) values with random signs, + 1e-3 [I; 0] (seed 3), nnz={A.nnz}; "
                           f"k={a.k} largest, block {a.block}, tol 1e-14*||A||, precond {a.precond}",
               "matrix": "random_sparse(1000000, 500000, 12.0, 3)", "target": "largest", "golden": "c3_largest",
               "m": A.m, "n": A.n, "nnz": A.nnz, "k": a.k, "block": a.block, "tol": TOL, "precond": a.precond,
               "l2": "inputs larger than L2 (CSR 150 MB + CSC copy), and a 256 MiB buffer written between "
                     "timed steps"}
        return A, cfg
    A = synth.grid_gradient(a.grid, a.sigma_log, 2)
    cfg = {"workload": f"weighted Dirichlet grid gradient {a.grid}x{a.grid} (log-normal sigma_log={a.sigma_log}, "
                       f"seed 2), m={A.m}, n={A.n}, nnz={A.nnz}; k={a.k} smallest, block {a.block}, "
                       f"tol 1e-14*||A||, precond {a.precond}",
           "matrix": f"grid_gradient({a.grid}, {a.sigma_log}, 2)", "target": "smallest", "golden": f"grid{a.grid}",
           "grid": a.grid, "m": A.m, "n": A.n, "nnz": A.nnz, "k": a.k, "block": a.block, "tol": TOL,
           "precond": a.precond, "l2": "256 MiB buffer written between timed steps"}
    return A, cfg


def dist_init(a):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if a.impl == "ours" else "gloo"
        dist.init_process_group(backend)
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p is not None:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    except Exception:
        return 6800.0, "fallback"


def spmm_bytes(m, n, nnz, b, p):
    """Algorithmic bytes of one fused A^T A SpMM launch set: one read of the CSR
    (values p bytes, column indices 4), the row offsets, X read and Y written."""
    return nnz * (p + 4) + 4 * (m + 1) + 2 * p * n * b


def spmm_lanes(avg):
    """Threads per sparse row (or CSC column) for a mean length avg: the
    group width the benchmark times by default."""
    return 1 if avg <= 2.5 else 2 if avg <= 6 else 4 if avg <= 16 else 8


def spmm_full(a):
    """Fused A^T A SpMM (products with C) on the full-size configurations:
    both schedules, FP64 and FP32, over the group widths (threads per sparse
    row: the automatic choice and its neighbours); CUDA events around each
    launch set on the library's stream, a 256 MiB L2 flush before each."""
    import numpy as np
    import torch
    from paper_1408_5535_gb300 import native, synth
    dev = torch.cuda.current_device()
    stream = torch.cuda.Stream(device=dev)
    h = native.Handle(dev, stream.cuda_stream)
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")
    hbm, _ = peaks()
    out = []
    cases = {"c2": ("weighted grid gradient 512x512 (sigma_log=1, seed 2)", lambda: synth.grid_gradient(512, 1.0, 2), 4),
             "c3": ("random 1e6 x 5e5, Poisson(12)/row, lognormal(2) +-, +1e-3[I;0], seed 3",
                    lambda: synth.random_sparse(1000000, 500000, 12.0, 3), 8)}

    def around(l0):
        return [x for x in (l0 // 2, l0, 2 * l0) if 1 <= x <= 16]

    with torch.cuda.stream(stream):
        for key in [c for c in a.spmm_cases.split(",") if c and c != "none"]:
            name, gen, b = cases[key]
            A = gen()
            rp = torch.from_numpy(A.row_ptr.astype(np.int32)).cuda()
            ci = torch.from_numpy(A.col).cuda()
            va = torch.from_numpy(A.val).cuda()
            cp = torch.empty(A.n + 1, dtype=torch.int32, device="cuda")
            ri = torch.empty(A.nnz, dtype=torch.int32, device="cuda")
            cv = torch.empty(A.nnz, dtype=torch.float64, device="cuda")
            native.phsvds_csr_to_csc(h, A.m, A.n, A.nnz, rp, ci, va, cp, ri, cv)
            native.phsvds_sync(h)
            la0, lt0 = spmm_lanes(A.nnz / A.m), spmm_lanes(A.nnz / A.n)
            for fp32 in (True, False):
                vt = torch.float32 if fp32 else torch.float64
                v1, v2 = (va.float(), cv.float()) if fp32 else (va, cv)
                X = torch.rand((A.n, b), dtype=vt, device="cuda")
                Y = torch.empty((A.n, b), dtype=vt, device="cuda")
                Z = torch.empty((A.m, b), dtype=vt, device="cuda")
                alg = spmm_bytes(A.m, A.n, A.nnz, b, 4 if fp32 else 8)
                plans = [(1, l, 0) for l in around(la0)] + [(2, l, lt0) for l in around(la0)] + \
                        [(2, la0, l) for l in around(lt0) if l != lt0]
                plans += [(1, -la0, 0), (2, -la0, -lt0)]
                if not a.spmm_sweep:
                    plans = [(1, la0, 0), (2, la0, lt0)]
                for sch, la, lt in plans:
                    def run():
                        native.phsvds_ata_spmm(h, sch, A.m, A.n, A.nnz, rp, ci, v1, cp, ri, v2, b, X, Y, Z,
                                               fp32=fp32, lanes_a=la, lanes_at=lt)
                    for _ in range(3):
                        run()
                    ts = []
                    for _ in range(a.spmm_reps):
                        flush.fill_(1.0)
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        run()
                        e1.record(stream)
                        stream.synchronize()
                        ts.append(e0.elapsed_time(e1))
                    ms = float(np.mean(ts))
                    gbs = alg / (ms * 1e-3) / 1e9
                    out.append({"case": key, "workload": name, "m": A.m, "n": A.n, "nnz": A.nnz, "b": b,
                                "dtype": "f32" if fp32 else "f64",
                                "schedule": "fused-atomic" if sch == 1 else "two-phase (Z=AX, CSC)",
                                "lanes_a": la, "lanes_at": lt if sch == 2 else None,
                                "avg_launch_ms": ms, "min_launch_ms": float(np.min(ts)), "alg_bytes": alg,
                                "GBps": gbs, "frac_of_hbm": gbs / hbm})
            del A
    h.close()
    return out


def kernel_only(a):
    """One tall-skinny kernel at the full-size solve's shape (n = 500,000),
    through the kernel-level entry points, timed with CUDA events on the
    library's stream over --kernel-reps launches after 3 warm-up launches; the
    inputs (about 240 MB) exceed L2, and a 256 MiB buffer is written between
    timed launches.  cgs: T <- T - P Gsub and Gout = P^T T, P = 55 columns (20
    locked + 35 basis), T = 8 columns (the second pass of stage 1's CGS2);
    tall: Out = V Y, V 35 columns, Y 35 x 21 (a thick restart)."""
    import numpy as np
    import torch
    from paper_1408_5535_gb300 import native
    n = 500000
    dt = torch.float64 if a.kernel_dtype == "f64" else torch.float32
    fp32 = a.kernel_dtype == "f32"
    esz = 8 if not fp32 else 4
    stream = torch.cuda.Stream()
    h = native.Handle(0, stream.cuda_stream)
    g = torch.Generator(device="cuda").manual_seed(1)
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")
    if a.kernel == "cgs":
        p1, p2, q = 20, 35, 8
        P = torch.rand((p1 + p2, n), dtype=dt, device="cuda", generator=g)
        T = torch.rand((q, n), dtype=dt, device="cuda", generator=g)
        Gs = torch.rand(((p1 + p2) * q,), dtype=torch.float64, device="cuda", generator=g) * 1e-6
        Gout = torch.zeros(((p1 + p2) * q,), dtype=torch.float64, device="cuda")

        def run():
            native.phsvds_block_cgs(h, n, P[:p1], n, p1, T, n, q, Gsub=Gs, Gout=Gout, P2=P[p1:], ld2=n, p2=p2,
                                    fp32=fp32)
        p = p1 + p2
        flops = 4.0 * n * p * q
        byts = esz * n * (p + 2 * q)
        shape = f"n={n}, p={p} ({p1} locked + {p2} basis), q={q}, Gsub and Gout"
    else:
        p, r = 35, 21
        P = torch.rand((p, n), dtype=dt, device="cuda", generator=g)
        Y = torch.rand((p * r,), dtype=torch.float64, device="cuda", generator=g)
        O = torch.empty((r, n), dtype=dt, device="cuda")

        def run():
            native.phsvds_tall_small(h, n, P, n, p, Y, p, r, O, n, fp32=fp32)
        flops = 2.0 * n * p * r
        byts = esz * n * (p + r)
        shape = f"n={n}, p={p}, r={r}"
    with torch.cuda.stream(stream):
        for _ in range(3):
            run()
        ts = []
        for _ in range(a.kernel_reps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            run()
            e1.record(stream)
            stream.synchronize()
            ts.append(e0.elapsed_time(e1))
    h.close()
    hbm, kind = peaks()
    ms = float(np.mean(ts))
    out = {"kernel": a.kernel, "dtype": a.kernel_dtype, "shape": shape, "avg_launch_ms": ms,
           "min_launch_ms": float(np.min(ts)), "alg_flops": flops, "alg_bytes": byts,
           "TFLOPs": flops / ms / 1e9, "GBps": byts / ms / 1e6, "frac_fp64_peak": flops / ms / 1e9 / 1.25,
           "frac_hbm": byts / ms / 1e6 / hbm, "hbm_peak": hbm, "hbm_peak_kind": kind}
    return out


def run_forms():
    """Small measured runs of the forms of Sec. 4 (GPU solves through the C
    ABI, CUDA events on the library's stream, median of 3, Table 1 once):
    * the two-stage demonstration of Sec. 5.1 with the caller's M ~ A
      (A = diag([1:10, 1000:100:1e6]), M = A + diag(1e4 rand), k = 1
      smallest): stage 1 alone and both stages;
    * the stage-2 preconditioner [0 A M; M A^T 0], M = diag(C)^{-1}, against
      plain GD in stage 2, on a 300 x 150 random matrix with columns scaled
      over two decades (k = 4 smallest, block 2, Jacobi in stage 1);
    * the JDQMR correction of stage 2 against GD on the 32 x 32 weighted
      grid, and on the paper's Table 1 (clustered tiny values, delta 1e-15)."""
    import numpy as np
    import scipy.sparse as sp
    import torch
    from paper_1408_5535_gb300 import native, synth
    stream = torch.cuda.Stream()
    h = native.Handle(0, stream.cuda_stream)

    def timed(A, k, prec, o, **kw):
        out = None
        ts = []
        for _ in range(3):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = native.phsvds_solve(h, A.m, A.n, A.row_ptr, A.col, A.val, k, native.SMALLEST, TOL, prec, o, **kw)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return out, float(np.median(ts))

    res = {}
    A, M = synth.e3_diag()
    for name, o in (("stage1_only", native.default_opts(stage2=0)), ("two_stages", native.default_opts())):
        (sig, U, V, rs, st, _), ms = timed(A, 1, native.PREC_GIVEN, o, precond_M=M)
        res[f"e3_{name}"] = {"ms": ms, "sigma": float(sig[0]), "resid_over_normA": float(rs[0] / 1e6),
                             "iters_stage1": st["iters_stage1"], "iters_stage2": st["iters_stage2"]}
    A0 = synth.random_sparse(300, 150, 6.0, 21, values="gaussian", shift=0.05)
    S = sp.csr_matrix((A0.val, A0.col, A0.row_ptr), shape=(A0.m, A0.n))
    S = (S @ sp.diags(10.0 ** (-2.0 * synth.uniform(31, 1, 150)))).tocsr()
    S.sort_indices()
    B = synth.Csr(S.shape[0], S.shape[1], S.indptr.astype(np.int64), S.indices.astype(np.int32), S.data)
    for sp2 in (0, 1):
        (sig, U, V, rs, st, _), ms = timed(B, 4, native.PREC_JACOBI, native.default_opts(block_size=2,
                                                                                       stage2_precond=sp2))
        res[f"stage2_precond_{sp2}"] = {"ms": ms, "iters_stage1": st["iters_stage1"],
                                        "iters_stage2": st["iters_stage2"],
                                        "max_resid_over_normA": float(np.max(rs) / st["norm_A_est"])}
    # JDQMR in stage 2 against GD in stage 2 (the weighted 32 x 32 grid, k = 10
    # smallest, block 4), and the paper's Table 1 (delta = 1e-15, block 2)
    G = synth.grid_gradient(32, 1.0, 2)
    for inner in (0, 1):
        (sig, U, V, rs, st, _), ms = timed(G, 10, native.PREC_NONE, native.default_opts(block_size=4,
                                                                                         stage2_inner=inner))
        res[f"grid32_stage2_{'jdqmr' if inner else 'gd'}"] = {
            "ms": ms, "iters_stage1": st["iters_stage1"], "iters_stage2": st["iters_stage2"],
            "inner_steps": st["inner2_steps"], "matvecs_A": st["matvecs_A"],
            "max_resid_over_normA": float(np.max(rs) / st["norm_A_est"])}
    T = synth.diag_matrix(synth.table1_sigma())
    exact = np.sort(synth.table1_sigma())[:10]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sig, U, V, rs, st, status = native.phsvds_solve(h, T.m, T.n, T.row_ptr, T.col, T.val, 10, native.SMALLEST, 1e-15,
                                                    native.PREC_NONE, native.default_opts(block_size=2,
                                                                                          stage2_inner=1),
                                                    raise_on_error=False)
    e1.record(stream)
    torch.cuda.synchronize()
    res["table1_jdqmr"] = {"ms": e0.elapsed_time(e1), "status": status, "sigma": sig.tolist(),
                           "max_abs_err": float(np.max(np.abs(sig - exact))), "max_resid": float(np.max(rs)),
                           "iters_stage1": st["iters_stage1"], "iters_stage2": st["iters_stage2"],
                           "inner_steps": st["inner2_steps"]}
    h.close()
    res["workloads"] = ("e3: diag([1:10, 1000:100:1e6]) with M = A + diag(1e4 rand) (seed 9), k=1 smallest; "
                        "stage2_precond: random_sparse(300, 150, 6, 21, gaussian, 0.05) with columns scaled "
                        "by 10^(-2u), k=4 smallest, block 2, Jacobi in stage 1; grid32: weighted 32x32 grid "
                        "gradient, k=10 smallest, block 4, GD vs JDQMR in stage 2; table1: diag(1e-14, 1e-12, "
                        "1e-8:1e-8:4e-8, 1e-3:1e-3:1), k=10 smallest, delta 1e-15, block 2, JDQMR")
    return res


def golden(a):
    """The oracle's recorded run of this workload (tests/golden/oracle_counts.json,
    written by tests/golden/make_oracle_counts.py from oracle/ only), or None."""
    try:
        with open(os.path.join(ROOT, "tests", "golden", "oracle_counts.json")) as f:
            gd = json.load(f)
    except Exception:
        return None
    key = "c3_largest" if a.workload == "c3" else f"grid{a.grid}"
    g = gd.get(key)
    if not g or g["k"] != a.k or g["block"] != a.block or a.precond != "none":
        return None
    if a.workload == "grid" and abs(a.sigma_log - 1.0) > 0:
        return None
    return g


def golden_iters(a):
    """The oracle's own outer-iteration count (stage 1 + stage 2) on this workload, or None."""
    g = golden(a)
    return g["iters_stage1"] + g["iters_stage2"] if g else None


def oracle_sample(a):
    """Runs the oracle (plain CPU FP64 PHSVDS, as it stands) on the workload in
    THIS process until it finishes, or has run --cpu-seconds, or (reference
    arm) --ref-iters outer iterations; prints {"seconds", "iters", "finished"}.
    Matrix generation is outside the timed region."""
    from oracle import phsvds_ref as R
    A, cfg = workload(a)

    class Stop(Exception):
        pass

    state = {"it": 0, "t0": None}
    cap_it = a.ref_iters if a.impl == "reference" else 0

    def tr(stage, it, d):
        state["it"] += 1
        if (cap_it and state["it"] >= cap_it) or time.perf_counter() - state["t0"] > a.cpu_seconds:
            raise Stop()

    o = R.Opts(block=a.block, precond=a.precond, trace=tr)
    state["t0"] = time.perf_counter()
    try:
        R.phsvds(A, cfg["k"], largest=cfg["target"] == "largest", delta=TOL, o=o)
        done = True
    except Stop:
        done = False
    el = time.perf_counter() - state["t0"]
    print(json.dumps({"seconds": el, "iters": max(state["it"], 1), "finished": done}), flush=True)


def _oracle_subprocess(a, threads, extra=()):
    """oracle_sample in a child process whose BLAS pools have `threads` threads
    (set before numpy loads), so the thread count reported is the one used."""
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[v] = str(threads)
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--oracle-sample", "--workload", a.workload,
           "--grid", str(a.grid), "--sigma-log", str(a.sigma_log), "--k", str(a.k), "--block", str(a.block),
           "--precond", a.precond, "--cpu-seconds", str(a.cpu_seconds), "--ref-iters", str(a.ref_iters), *extra]
    r = subprocess.run(cmd, env=env, capture_output=True, text=True, cwd=ROOT)
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    if r.returncode != 0 or not lines:
        raise RuntimeError("oracle sample failed: " + r.stderr[-500:])
    return json.loads(lines[-1])


def _scaled(a, k, smp, fallback_iters):
    """Triplets/s of a whole oracle solve from a sample: its time per outer
    iteration times the oracle's recorded iteration count for the workload."""
    gi = golden_iters(a)
    total = gi if gi else fallback_iters
    est = smp["seconds"] if smp["finished"] else smp["seconds"] / smp["iters"] * total
    return k / est, est, total, gi is not None


def cpu_baseline(a, k, fallback_iters):
    """The oracle on the host cores, on bounded samples of the same solve (at
    most --cpu-seconds each): with all host cores as BLAS threads (the value)
    and single-threaded.  An unfinished sample is scaled to a whole solve by
    the oracle's own recorded iteration count (else the GPU's) and labelled
    extrapolated."""
    ncpu = os.cpu_count() or 1
    out = {}
    for key, th in (("all", ncpu), ("one", 1)):
        smp = _oracle_subprocess(a, th)
        v, est, total, gold = _scaled(a, k, smp, fallback_iters)
        out[key] = dict(value=v, threads=th, seconds=smp["seconds"], iters=smp["iters"], finished=smp["finished"],
                        whole_solve_s=est, iters_whole=total)
    al, one = out["all"], out["one"]

    def text(d):
        if d["finished"]:
            return f"the whole oracle solve ({d['iters']} outer iterations) in {d['seconds']:.1f} s"
        return (f"EXTRAPOLATED: {d['iters']} of the oracle's {d['iters_whole']} outer iterations in "
                f"{d['seconds']:.1f} s, scaled to {d['whole_solve_s']:.0f} s per solve")

    return {"value": al["value"], "unit": "triplets/s", "cores": al["threads"], "kind": "oracle",
            "sample": text(al) + f"; {al['threads']} BLAS threads (scipy sparse products single-threaded)",
            "extrapolated": not al["finished"], "seconds": al["seconds"], "iterations_sampled": al["iters"],
            "single_thread": {"value": one["value"], "cores": 1, "sample": text(one),
                              "extrapolated": not one["finished"]}}


def _pinned_solve(native, h, A, cfg, target, prec_id, opts):
    """One solve through the C ABI from pinned host buffers: the CSR is copied
    host -> device and the triplets device -> host inside the call."""
    import ctypes as C
    import numpy as np
    import torch
    k = cfg["k"]
    if not hasattr(_pinned_solve, "buf"):
        pin = lambda x: torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
        _pinned_solve.buf = dict(rp=pin(A.row_ptr), ci=pin(A.col), va=pin(A.val),
                                 sigma=torch.zeros(k, dtype=torch.float64).pin_memory(),
                                 U=torch.zeros(k * A.m, dtype=torch.float64).pin_memory(),
                                 V=torch.zeros(k * A.n, dtype=torch.float64).pin_memory(),
                                 resid=torch.zeros(k, dtype=torch.float64).pin_memory())
    b = _pinned_solve.buf
    st = native.Stats()
    status = native.lib().phsvds_solve(h.h, A.m, A.n, A.nnz, b["rp"].data_ptr(), b["ci"].data_ptr(),
                                       b["va"].data_ptr(), 0, k, target, TOL, prec_id, C.byref(opts),
                                       b["sigma"].data_ptr(), b["U"].data_ptr(), b["V"].data_ptr(),
                                       b["resid"].data_ptr(), C.byref(st))
    h.check(status)
    return b["sigma"].numpy().copy(), st.as_dict()


def run_ours(a, rank, world):
    import numpy as np
    import torch
    from paper_1408_5535_gb300 import native
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    A, cfg = workload(a)
    if a.jd:
        cfg["path"] = ("Jacobi-Davidson: Jacobi preconditioner, scaled inner solves in stage 1 (FP32 MINRES, "
                       f"opts.mixed_inner = {a.c3s_mixed_inner}, in the mixed form; FP64 MINRES, "
                       "opts.stage1_inner = 1, in the FP64 form), JDQMR in stage 2, ||A|| estimated")
    target = native.LARGEST if cfg["target"] == "largest" else native.SMALLEST
    stream = torch.cuda.Stream(device=dev)
    h = native.Handle(dev, stream.cuda_stream)
    rp = torch.from_numpy(A.row_ptr).cuda()
    ci = torch.from_numpy(A.col).cuda()
    va = torch.from_numpy(A.val).cuda()
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")
    precs = {"mixed": [native.MIXED], "fp64": [native.FP64], "both": [native.MIXED, native.FP64]}[a.precision]
    prec_id = native.PREC_JACOBI if (a.precond == "jacobi" or a.jd) else native.PREC_NONE
    g = golden(a)
    results = {}
    for pi, prec in enumerate(precs):
        head = pi == 0                 # the headline precision; the second is the comparison leg
        steps = a.steps if head else max(2, min(a.steps, 5))
        # --jd: the Jacobi-Davidson path of the smallest-triplet blocks (Jacobi
        # preconditioner, scaled inner solves in stage 1, JDQMR in stage 2,
        # ||A|| estimated)
        jdo = {}
        if a.jd:
            jdo = dict(stage2_inner=1, norm_A=-1.0)
            jdo.update(dict(mixed_inner=a.c3s_mixed_inner) if prec == native.MIXED else dict(stage1_inner=1))
        o = native.default_opts(block_size=a.block, precision=prec, profile=0, **jdo)
        op = native.default_opts(block_size=a.block, precision=prec, profile=1, **jdo)

        def solve(opts, vectors=False):
            return native.phsvds_solve(h, A.m, A.n, rp, ci, va, cfg["k"], target, TOL, prec_id, opts,
                                       on_device=True, want_vectors=vectors)

        for _ in range(a.warmup):
            solve(o)
        times, launches, last = [], 0, None
        with Clocks(dev) as clk:
            for _ in range(steps):
                flush.fill_(1.0)
                torch.cuda.synchronize()
                barrier(world)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                last = solve(o)
                e1.record(stream)
                torch.cuda.synchronize()
                barrier(world)
                times.append(e0.elapsed_time(e1))
                launches += last[4]["kernel_launches"]
        sig, _, _, resid, st, _ = last
        ms = max_over_ranks(float(np.mean(times)), world)
        # per-class device times of one profiled solve (CUDA events inside the library)
        prof = solve(op)[4]
        # end to end: pinned host CSR in, host triplets out, through the same call
        e2e = None
        if not a.no_e2e:
            ee = []
            for _ in range(2):
                flush.fill_(1.0)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                _pinned_solve(native, h, A, cfg, target, prec_id, o)
                ee.append((time.perf_counter() - t0) * 1e3)
            e_ms = max_over_ranks(float(np.mean(ee)), world)
            h2d = 8 * (A.m + 1) + 4 * A.nnz + 8 * A.nnz
            d2h = 8 * cfg["k"] * (2 + A.m + A.n)
            e2e = {"value": world * cfg["k"] / (e_ms / 1e3), "unit": "triplets/s", "h2d_bytes_per_step": h2d,
                   "d2h_bytes_per_step": d2h, "ms_per_step": e_ms, "host_buffers": "pinned"}
        err = None
        if g:
            ref = np.asarray(g["sigma"])
            err = (np.abs(sig - ref) / ref).tolist()
        results[prec] = dict(ms=ms, times=times, sigma=sig.tolist(), resid_rel=(resid / st["norm_A_est"]).tolist(),
                             stats=st, prof=prof, e2e=e2e, clocks=clk.summary(), launches=launches, steps=steps,
                             err_vs_oracle=err)
    h.close()
    return A, cfg, results


# FP64 peak of one GB300: nominal 1.25 TFLOP/s (the recipe's table), i.e.
# 152 SMs x 2 FP64 FMA per clock x 2 flop x ~2.06 GHz.
FP64_PEAK_GFLOPS = 1250.0
JACOBI_CTAS = 8

CLASS_NAMES = ["fused A^T A SpMM (FP64)", "Gram / CGS passes (FP64)", "basis transforms / Ritz vectors (FP64)",
               "refined vector of stage 2 (inverse iteration on R)", "A / A^T products (FP64)",
               "projected eigensolvers (Jacobi)",
               "fused A^T A SpMM (FP32)", "Gram / CGS passes (FP32)", "basis transforms / Ritz vectors (FP32)",
               "inner MINRES vector kernels (FP32)", "A / A^T products (FP32)", "(unused FP32 Jacobi)"]
CLASS_KERNELS = {0: "k_csr_rows / k_ata_fused <double>", 1: "k_cgs_pass<double>", 2: "k_tall_small<double>",
                 4: "k_csr_rows<double, 1>", 6: "k_csr_rows / k_ata_fused <float>", 7: "k_cgs_pass<float>",
                 8: "k_tall_small<float>", 9: "k_jd_lanczos / k_jd_update / k_col_dots", 10: "k_csr_rows<float, 1>"}


# the stage-1 projected eigensolve of a call: the FP32 pass and the FP64
# clean-up of the target pairs, with the device helpers they call
JACOBI_FUNCS = ["rr_pair", "rot_params", "rot_params_small", "k_jacobi_eig", "k_jacobi_targets"]
# the block Gram-Schmidt pass (its ncu capture: profiles/cgs_pass_f64_1e6x5e5.txt)
CGS_FUNCS = ["cp_async16", "cp_async_wait_all", "stage_cols", "lds_vec", "reduce_scatter_step", "k_cgs_pass"]
# the row kernel of the two-phase SpMM (its capture: profiles/spmm_csr_rows_c3_f32.txt)
SPMM_FUNCS = ["load_row_256", "l2_evict_first_policy", "ld_stream", "gather_rows", "load_slots", "k_csr_rows"]
SPMM_FUSED_FUNCS = ["load_row_256", "l2_evict_first_policy", "ld_stream", "gather_rows", "load_slots",
                    "k_ata_fused"]


def kernel_source_sha256(kernel_file, names):
    """sha256 of the source text of the named functions of a .cu file (each
    from the line that declares it to its closing brace in column 0, every
    overload), so that edits elsewhere in the file do not invalidate a
    capture."""
    import hashlib
    try:
        lines = open(os.path.join(ROOT, "paper_1408_5535_gb300", "csrc", kernel_file)).read().splitlines()
    except OSError:
        return None
    h = hashlib.sha256()
    for name in names:
        pat = re.compile(r"\b" + re.escape(name) + r"\(")
        starts = [i for i, l in enumerate(lines) if re.match(r"(__global__|__device__)\b", l)
                  and (pat.search(l) or (i + 1 < len(lines) and pat.search(lines[i + 1])))]
        if not starts:
            return None
        for i in starts:                  # every overload, in file order
            while i < len(lines) and lines[i] != "}":
                h.update(lines[i].encode() + b"\n")
                i += 1
    return h.hexdigest()


def measured_traffic(kernel_file, names, summary, key):
    """A figure from a committed ncu summary, if the captured kernels' source
    is unchanged since the capture (the summary records its sha256)."""
    try:
        txt = open(os.path.join(ROOT, "profiles", summary)).read()
    except OSError:
        return None
    kv = dict(l.split(":", 1) for l in txt.splitlines() if ":" in l and not l.startswith("#"))
    if kv.get("kernel_sha256", "").strip() != kernel_source_sha256(kernel_file, names):
        return None
    try:
        return float(kv[key])
    except (KeyError, ValueError):
        return None


def roofline_for(A, prof, dom, hbm, peak_kind):
    """Roofline of the dominant kernel class of one profiled solve.

    * Projected eigensolve (class 5): algorithmic flops per call = 18 j per
      rotation (rows and columns of H and the columns of S, 6 j each) x
      rotations per call, against the FP64 peak.
    * FP64 classes (0-4: products with C or B, Gram/CGS passes, basis
      transforms): the algorithmic flops the library counts at each launch
      (stats.class_flops) over the class's device time, against the FP64
      peak.  At these shapes they do >= 1.7 flop per algorithmic byte, far
      above GB300's FP64 ridge (1.25 TFLOP/s / 6.7 TB/s = 0.19 flop/B), so the
      FP64 pipe, not HBM, bounds them.
    * FP32 classes (6-10, the mixed-precision stage 1): the algorithmic bytes
      (stats.class_bytes: each operand read once, each result written once)
      over the class's time, against the measured HBM copy rate; their
      <= 4 flop/B lies below the FP32 ridge (~10 flop/B)."""
    calls = prof["n_class"][dom]
    t_ms = prof["t_class_ms"][dom]
    if dom in (5, 11) and calls and prof["jacobi_calls"]:
        jc = prof["jacobi_calls"]
        j_avg = prof["jacobi_dim_sum"] / jc
        rot = prof["jacobi_rotations"] / jc
        flops = 18.0 * j_avg * rot
        per_call_ms = t_ms / jc
        ach = flops / (per_call_ms * 1e-3) / 1e9
        tr = measured_traffic("k_small.cu", JACOBI_FUNCS, "jacobi_fp32_targets_grid32.txt", "dram_bytes_per_call")
        return {"bound": "alu", "kernel": "stage-1 projected eigensolve (Jacobi kernels of k_small.cu)",
                "achieved": ach / 1e3, "peak": FP64_PEAK_GFLOPS / 1e3, "unit": "TFLOP/s",
                "frac": ach / FP64_PEAK_GFLOPS, "traffic": tr,
                "peak_source": "nominal FP64 rate of the GPU (152 SMs x 2 FMA/clk)",
                "flops_per_solve_call": flops, "ms_per_solve_call": per_call_ms,
                "launches_per_call": calls / jc, "j_avg": j_avg, "rotations_per_call": rot}
    fl = prof.get("class_flops", [0.0] * 12)[dom]
    by = prof.get("class_bytes", [0.0] * 12)[dom]
    avg_ms = t_ms / calls if calls else None
    out = {"kernel": CLASS_KERNELS.get(dom, CLASS_NAMES[dom]), "avg_launch_ms": avg_ms, "launches": calls,
           "flops_per_launch": fl / calls if calls else None, "bytes_per_launch": by / calls if calls else None,
           "traffic": None}
    if dom in (1, 7):
        out["traffic"] = measured_traffic("k_tall.cu", CGS_FUNCS, "cgs_pass_%s_1e6x5e5.txt" % ("f64" if dom == 1 else "f32"),
                                          "dram_bytes_per_launch")
        if out["traffic"] is not None:
            out["traffic_launch"] = ("the captured launch: n = 500,000, p = 55 basis columns, q = 8, "
                                     "Gsub and Gout (profiles/)")
    if dom == 6:
        if prof.get("spmm_schedule_f32") == 2:
            out["traffic"] = measured_traffic("k_sparse.cu", SPMM_FUNCS, "spmm_csr_rows_c3_f32.txt",
                                              "dram_bytes_per_launch")
            label = "both phases of the two-phase schedule at b = 8"
        else:
            out["traffic"] = measured_traffic("k_sparse.cu", SPMM_FUSED_FUNCS, "spmm_ata_fused_c3_f32.txt",
                                              "dram_bytes_per_launch")
            label = "the fused single-pass schedule at b = 8"
        if out["traffic"] is not None:
            out["traffic_launch"] = f"the captured product: {label} (profiles/)"
    if dom < 6:
        ach = fl / (t_ms * 1e-3) / 1e12 if t_ms else None
        out.update(bound="alu", achieved=ach, peak=FP64_PEAK_GFLOPS / 1e3, unit="TFLOP/s",
                   frac=(ach * 1e3 / FP64_PEAK_GFLOPS) if ach else None,
                   peak_source="nominal FP64 rate of the GPU (152 SMs x 2 FMA/clk x 2.06 GHz)")
    else:
        ach = by / (t_ms * 1e-3) / 1e9 if t_ms else None
        out.update(bound="hbm", achieved=ach, peak=hbm, unit="GB/s", frac=(ach / hbm) if ach else None,
                   peak_source=peak_kind)
    return out



def run_batched(a):
    """Batched workload: the solves of --batch-count uneven random sparse
    matrices (n ~ U[nlo, nhi], m ~ U[1.2n, 2n], Poisson(8) per row, N(0,1),
    +1e-2 diagonal, seed 5), k smallest and k largest each, as two batched
    mixed-precision calls, against the same solves one after another in FP64.
    Wall-clock of each whole set (host buffers, the call blocks)."""
    import numpy as np
    import torch
    from paper_1408_5535_gb300 import native, synth
    mats = synth.batched_set(a.batch_count, seed=5, n_lo=a.batch_nlo, n_hi=a.batch_nhi)
    tup = [(A.m, A.n, A.row_ptr, A.col, A.val) for A in mats]
    h = native.Handle(0)
    k = a.batch_k
    om = native.default_opts(precision=native.MIXED)
    of = native.default_opts(precision=native.FP64)
    # warm-up: one small batched call (module load, pools)
    native.phsvds_solve_batched(h, tup[:2], k, native.SMALLEST, TOL, native.PREC_NONE, om, concurrency=2)
    res = {}
    t0 = time.perf_counter()
    for tgt in (native.SMALLEST, native.LARGEST):
        res[tgt] = native.phsvds_solve_batched(h, tup, k, tgt, TOL, native.PREC_NONE, om,
                                               concurrency=a.batch_concurrency)[0]
    t_b = time.perf_counter() - t0
    worst = max(max(o[3]) / o[4]["norm_A_est"] for tgt in res for o in res[tgt])
    out = {"metric": "triplets/s over the batched set (k smallest + k largest per matrix)",
           "count": len(mats), "k": k, "n_range": [a.batch_nlo, a.batch_nhi],
           "nnz_total": int(sum(A.nnz for A in mats)), "batched_mixed_s": t_b,
           "batched_triplets_per_s": 2 * k * len(mats) / t_b, "max_resid_over_normA": worst,
           "concurrency": a.batch_concurrency or min(len(mats), 4),
           "iters_total": int(sum(o[4]["iters_stage1"] + o[4]["iters_stage2"] for t in res for o in res[t]))}
    if not a.batch_no_seq:
        t0 = time.perf_counter()
        diff = 0.0
        for tgt in (native.SMALLEST, native.LARGEST):
            for i, (m, n, rp, ci, va) in enumerate(tup):
                sig = native.phsvds_solve(h, m, n, rp, ci, va, k, tgt, TOL, native.PREC_NONE, of,
                                          want_vectors=False)[0]
                diff = max(diff, float(np.max(np.abs(res[tgt][i][0] - sig) / sig)))
        t_s = time.perf_counter() - t0
        out.update(sequential_fp64_s=t_s, sequential_triplets_per_s=2 * k * len(mats) / t_s,
                   speedup_batched_mixed_over_sequential_fp64=t_s / t_b, max_sigma_rel_diff_vs_sequential=diff)
    h.close()
    return out


def run_learned(a):
    """Learned-preconditioner workload: convection-diffusion operators on an
    N x N grid (seeds 1000.. for training, 1200.. held out), k = 5 smallest at
    tol 1e-14 ||A||; training data from the plain method's recorded residuals
    and device-CG inner solves; time to solution per correction operator."""
    import numpy as np
    import torch
    from paper_1408_5535_gb300 import learned, native, synth
    h = native.Handle(0)
    N = a.learned_grid
    t0 = time.perf_counter()
    train_ops = [synth.convdiff_stencil(N, 1000 + i) for i in range(a.learned_train)]
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    data = learned.record_samples(h, train_ops, k=5, per_op=8, every=15, cg_steps=a.learned_cg_steps)
    t_rec = time.perf_counter() - t0
    t0 = time.perf_counter()
    tr = learned.train(h, data, epochs=a.learned_epochs, batch=32, lr=2e-3)
    t_train = time.perf_counter() - t0
    modes = {"none": native.PREC_NONE, "jacobi": native.PREC_JACOBI, "learned": native.PREC_LEARNED}
    res = {m: {"iters": [], "seconds": [], "resid": [], "fell_back": 0} for m in modes}
    sig_ref = {}
    for i in range(a.learned_test):
        A = synth.convdiff_stencil(N, 1200 + i)
        for name, pc in modes.items():
            if pc == native.PREC_LEARNED:
                o, keep = learned.solve_opts(A, tr.params_bf16, stall_window=a.learned_stall)
            else:
                o = native.default_opts()
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            sig, _, _, rs, st, status = native.phsvds_solve(h, A.m, A.n, A.row_ptr, A.col, A.val, 5,
                                                            native.SMALLEST, TOL, pc, o, want_vectors=False,
                                                            raise_on_error=False)
            el = time.perf_counter() - t1
            r = res[name]
            r["iters"].append(int(st["iters_stage1"] + st["iters_stage2"]))
            r["seconds"].append(el)
            r["resid"].append(float(max(rs) / st["norm_A_est"]) if status == 0 else float("nan"))
            r["fell_back"] += int(st["fell_back"])
            if name == "none":
                sig_ref[i] = sig
            elif status == 0:
                r.setdefault("max_sigma_rel_diff_vs_none", 0.0)
                r["max_sigma_rel_diff_vs_none"] = max(r["max_sigma_rel_diff_vs_none"],
                                                       float(np.max(np.abs(sig - sig_ref[i]) / sig_ref[i])))
    summ = {}
    for m, r in res.items():
        summ[m] = {"mean_iters": float(np.mean(r["iters"])), "mean_seconds": float(np.mean(r["seconds"])),
                   "max_resid_over_normA": float(np.nanmax(r["resid"])), "all_converged": bool(
                       np.all(np.isfinite(r["resid"]))), "fell_back": r["fell_back"],
                   "max_sigma_rel_diff_vs_none": r.get("max_sigma_rel_diff_vs_none")}
    h.close()
    return {"workload": f"convection-diffusion {N}x{N}, GRF diffusion, |beta| <= 20; k=5 smallest, tol 1e-14",
            "train_ops": a.learned_train, "test_ops": a.learned_test, "samples": int(data.x.shape[0]),
            "cg_iters_mean": float(np.mean(data.cg_iters)) if data.cg_iters else None,
            "seconds_generate": t_gen, "seconds_record_and_inner_solves": t_rec, "seconds_train": t_train,
            "target": f"{a.learned_cg_steps} CG steps" if a.learned_cg_steps else "converged CG (rtol 1e-6)",
            "stall_window": a.learned_stall,
            "train_steps": tr.steps, "loss_first_epoch": tr.loss_history[0], "loss_last_epoch": tr.loss_history[-1],
            "modes": summ,
            "speedup_learned_over_none": summ["none"]["mean_seconds"] / summ["learned"]["mean_seconds"],
            "speedup_learned_over_jacobi": summ["jacobi"]["mean_seconds"] / summ["learned"]["mean_seconds"]}


def smallest_pair(a, A, k, block, steps, workload):
    """The k smallest triplets of A at tol 1e-14 ||A||, mixed precision
    against FP64 with the same algorithm: the Jacobi preconditioner with the
    scaled Jacobi-Davidson inner solves in stage 1 (FP32 MINRES in the mixed
    form, FP64 MINRES with opts.stage1_inner in the FP64 form), JDQMR in
    stage 2, and ||A|| estimated before stage 1 (opts.norm_A = -1).  Per
    precision one untimed solve (autotuner, graphs), then timed solves with
    CUDA events on the library's stream (`steps` for mixed, one for FP64).
    The residuals of the returned triplets are recomputed here on the host
    against the estimate of ||A||, a lower bound, so the check is at least as
    strict as 1e-14 ||A||; the two precisions' values are compared."""
    import numpy as np
    import scipy.sparse as sp
    import torch
    from paper_1408_5535_gb300 import native
    stream = torch.cuda.Stream()
    h = native.Handle(0, stream.cuda_stream)
    rp, ci, va = (torch.from_numpy(x).cuda() for x in (A.row_ptr, A.col, A.val))
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")
    S = sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.m, A.n))
    legs = {"mixed": (native.default_opts(block_size=block, precision=native.MIXED, mixed_inner=a.c3s_mixed_inner,
                                          stage2_inner=1, norm_A=-1.0, time_limit_s=300.0), max(1, steps)),
            "fp64": (native.default_opts(block_size=block, precision=native.FP64, stage1_inner=1, stage2_inner=1,
                                         norm_A=-1.0, time_limit_s=300.0), 1)}
    out = {}
    for name, (o, nsteps) in legs.items():
        def solve(vectors):
            return native.phsvds_solve(h, A.m, A.n, rp, ci, va, k, native.SMALLEST, TOL, native.PREC_JACOBI, o,
                                       on_device=True, want_vectors=vectors)
        solve(False)
        times, res = [], None
        for i in range(nsteps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = solve(i == nsteps - 1)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        sig, U, V, _, st, _ = res
        rv = np.linalg.norm(S @ V - U * sig, axis=0)
        ru = np.linalg.norm(S.T @ U - V * sig, axis=0)
        nA = st["norm_A_est"]
        ms = float(np.median(times))
        out[name] = {"ms": ms, "ms_all": times, "triplets_per_s": k / (ms / 1e3), "sigma": [float(x) for x in sig],
                     "norm_A_est": nA,
                     "max_resid_over_normA_recomputed": float(np.max(np.sqrt(rv ** 2 + ru ** 2)) / nA),
                     "iters_stage1": st["iters_stage1"], "iters_stage1_fp32": st["iters_stage1_fp32"],
                     "iters_stage2": st["iters_stage2"], "inner_steps_stage1": st["inner_steps"],
                     "inner_steps_stage2": st["inner2_steps"], "t_stage1_ms": st["t_stage1_ms"],
                     "t_stage2_ms": st["t_stage2_ms"]}
    h.close()
    sm, sf = np.array(out["mixed"]["sigma"]), np.array(out["fp64"]["sigma"])
    return {"workload": workload + "; Jacobi preconditioner with scaled Jacobi-Davidson inner solves in stage 1, "
                                   "JDQMR in stage 2, ||A|| estimated by 30 Lanczos steps on C (opts.norm_A = -1); "
                                   f"mixed (FP32 inner solves, opts.mixed_inner = {a.c3s_mixed_inner}) against FP64 "
                                   "(opts.stage1_inner = 1, FP64 inner solves), both with at most 60 inner steps "
                                   "and a 1e-3 residual reduction per solve",
            "mixed": out["mixed"], "fp64": out["fp64"],
            "speedup_mixed_over_fp64": out["fp64"]["ms"] / out["mixed"]["ms"],
            "max_sigma_rel_diff_mixed_vs_fp64": float(np.max(np.abs(sm - sf) / sf))}


def run_c3_smallest(a):
    """C3's k = 20 smallest triplets at full size (the headline's matrix)."""
    from paper_1408_5535_gb300 import synth
    A = synth.random_sparse(1000000, 500000, 12.0, 3)
    r = smallest_pair(a, A, 20, 8, a.c3s_steps,
                      "the headline matrix (random sparse 1000000x500000, seed 3), k=20 smallest, block 8, "
                      "tol 1e-14*||A||")
    r["plain_fp64"] = ("the plain FP64 method (GD+k with the Olsen-Jacobi correction, no inner solves) reaches its "
                       "restart limit on this family already at 100000 x 50000")
    return r


def run_c2(a):
    """The weighted 512 x 512 grid gradient (m = 525,312, n = 262,144,
    log-normal sigma_log = 1.0, seed 2), k = 10 smallest, block 4."""
    from paper_1408_5535_gb300 import synth
    A = synth.grid_gradient(512, 1.0, 2)
    r = smallest_pair(a, A, 10, 4, a.c3s_steps,
                      f"weighted Dirichlet grid gradient 512x512 (log-normal sigma_log=1.0, seed 2), m={A.m}, "
                      f"n={A.n}, nnz={A.nnz}; k=10 smallest, block 4, tol 1e-14*||A||")
    r["plain_fp64"] = ("the plain FP64 method (unpreconditioned GD+k) needs about 5x more outer iterations per "
                       "doubling of the grid: 18,511 at 64 x 64, and does not finish at 128 x 128 in minutes")
    return r


def main():
    a = parse()
    if a.oracle_sample:
        return oracle_sample(a)
    rank, world = dist_init(a)
    if a.impl == "reference":
        return run_reference(a, rank, world)
    import torch
    from paper_1408_5535_gb300 import native
    if a.learned:
        if rank == 0:
            print(json.dumps({"learned": run_learned(a)}), flush=True)
        return
    if a.batched:
        if rank == 0:
            print(json.dumps({"batched": run_batched(a)}), flush=True)
        return
    if a.kernel:
        if rank == 0:
            print(json.dumps({"kernel_only": kernel_only(a)}), flush=True)
        return
    if a.spmm_only:
        r = spmm_full(a)
        if rank == 0:
            print(json.dumps({"spmm": r}), flush=True)
        return
    A, cfg, res = run_ours(a, rank, world)
    head = native.MIXED if native.MIXED in res else native.FP64
    r = res[head]
    st, prof = r["stats"], r["prof"]
    hbm, peak_kind = peaks()
    cls = prof["t_class_ms"]
    dom = int(max(range(len(cls)), key=lambda i: cls[i]))
    roof = roofline_for(A, prof, dom, hbm, peak_kind)
    per_class = {}
    for c in range(len(cls)):
        if cls[c] > 0 and prof["n_class"][c]:
            rc = roofline_for(A, prof, c, hbm, peak_kind)
            per_class[CLASS_NAMES[c]] = {"ms": cls[c], "launches": prof["n_class"][c], "bound": rc["bound"],
                                         "achieved": rc["achieved"], "unit": rc["unit"], "frac": rc["frac"]}
    roof.update(dominant_class=CLASS_NAMES[dom], classes=per_class)
    line = {
        "metric": METRIC,
        "value": world * cfg["k"] / (r["ms"] / 1e3),
        "unit": "triplets/s",
        "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": r["ms"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64" if head == native.MIXED else "f64",
        "data": "synthetic",
        "config": dict({k: v for k, v in cfg.items() if k != "golden"},
                       precision="mixed" if head == native.MIXED else "fp64", parallelism=f"replicas{world}"),
        "roofline": roof,
        "gpu_launches": r["launches"],
        "gpu_launches_per_step": r["launches"] // max(r["steps"], 1),
        "clocks": r["clocks"],
        "e2e": r["e2e"],
        "solve": {"iters_stage1": st["iters_stage1"], "iters_stage1_fp32": st["iters_stage1_fp32"],
                  "iters_stage2": st["iters_stage2"], "matvecs_A": st["matvecs_A"], "switched": st["switched"],
                  "max_resid_over_normA": max(r["resid_rel"]), "spmm_schedule": st["spmm_schedule"],
                  "spmm_plan_cached": st["spmm_plan_cached"], "jacobi_sweeps": st["jacobi_sweeps"],
                  "jacobi_rotations": st["jacobi_rotations"], "restarts": st["restarts"],
                  "inner_solves": st["inner_solves"], "inner_steps": st["inner_steps"],
                  "ms_min": min(r["times"]), "ms_max": max(r["times"])},
    }
    g = golden(a)
    if g:
        par = {"oracle": f"tests/golden/oracle_counts.json[{cfg['golden']}] (FP64 oracle, {g['iters_stage1']} + "
                         f"{g['iters_stage2']} outer iterations)",
               "sigma_oracle": g["sigma"]}
        for p_, nm in ((native.MIXED, "mixed"), (native.FP64, "fp64")):
            if p_ in res and res[p_]["err_vs_oracle"] is not None:
                e = res[p_]["err_vs_oracle"]
                par[f"sigma_rel_err_{nm}"] = e
                par[f"max_sigma_rel_err_{nm}"] = max(e)
                par[f"max_resid_over_normA_{nm}"] = max(res[p_]["resid_rel"])
        line["parity"] = par
    if native.FP64 in res and head != native.FP64:
        f = res[native.FP64]
        line["fp64"] = {"value": world * cfg["k"] / (f["ms"] / 1e3), "ms_per_step": f["ms"], "steps": f["steps"],
                        "iters_stage1": f["stats"]["iters_stage1"], "iters_stage2": f["stats"]["iters_stage2"],
                        "speedup_mixed_over_fp64": f["ms"] / r["ms"],
                        "max_sigma_rel_diff_vs_mixed": max(abs(x - y) / y for x, y in zip(r["sigma"], f["sigma"])),
                        "class_ms": {CLASS_NAMES[i]: v for i, v in enumerate(f["prof"]["t_class_ms"]) if v > 0},
                        "e2e": f["e2e"]}
    if a.spmm_cases and a.spmm_cases != "none":
        sp = spmm_full(a)
        line["spmm"] = sp
        best = max((x for x in sp if x["case"] == "c3" and x["dtype"] == "f32"), key=lambda x: x["GBps"], default=None)
        if best is None and sp:
            best = max(sp, key=lambda x: x["GBps"])
        if best:
            line["spmm_roofline"] = {"bound": "hbm", "kernel": f"fused A^T A SpMM, {best['schedule']}, {best['dtype']}",
                                     "workload": best["workload"], "achieved": best["GBps"], "peak": hbm,
                                     "unit": "GB/s", "frac": best["GBps"] / hbm, "traffic": None,
                                     "bytes_per_launch": best["alg_bytes"], "avg_launch_ms": best["avg_launch_ms"]}
    if rank == 0 and not a.no_forms:
        line["forms"] = run_forms()
    if rank == 0 and a.workload == "c3" and a.c3s_steps > 0:
        line["c3_smallest"] = run_c3_smallest(a)
        line["c2_grid512_smallest"] = run_c2(a)
    if rank == 0 and not a.no_cpu:
        line["cpu_baseline"] = cpu_baseline(a, cfg["k"], st["iters_stage1"] + st["iters_stage2"])
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_reference(a, rank, world):
    """The oracle (plain CPU FP64 PHSVDS, as it stands) on the host cores, on the
    same workload; rank 0 only, the other ranks exit without work.  Each step
    is a bounded sample: the first --ref-iters outer iterations of the solve,
    with every host core as a BLAS thread; its triplets/s is the sample's time
    per iteration scaled to the oracle's own recorded iteration count for the
    workload (labelled extrapolated), its ms_per_step the sample's real time."""
    if rank != 0:
        return
    ncpu = os.cpu_count() or 1
    if "numpy" not in sys.modules:      # the BLAS pool size is fixed when numpy loads
        for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
            os.environ.setdefault(v, str(ncpu))
    threads = int(os.environ.get("OPENBLAS_NUM_THREADS", ncpu))
    from oracle import phsvds_ref as R
    A, cfg = workload(a)
    k = cfg["k"]
    gi = golden_iters(a)
    total = gi if gi else 4000

    class Stop(Exception):
        pass

    vals, secs, its = [], [], []
    for i in range(a.warmup + a.steps):
        state = {"it": 0}

        def tr(stage, it, d):
            state["it"] += 1
            if state["it"] >= a.ref_iters:
                raise Stop()

        t0 = time.perf_counter()
        try:
            R.phsvds(A, k, largest=cfg["target"] == "largest", delta=TOL, o=R.Opts(block=a.block,
                                                                                  precond=a.precond, trace=tr))
            done = True
        except Stop:
            done = False
        el = time.perf_counter() - t0
        if i >= a.warmup:
            n_it = max(state["it"], 1)
            est = el if done else el / n_it * total
            vals.append(k / est)
            secs.append(el)
            its.append(n_it)
    v = sum(vals) / len(vals)
    ms = 1e3 * sum(secs) / len(secs)
    sample = (f"EXTRAPOLATED: each step runs the first {its[-1]} of the oracle's {total} outer iterations "
              f"({ms / 1e3:.1f} s), scaled to a whole solve ({k / v:.0f} s); {threads} BLAS threads "
              f"(scipy sparse products single-threaded)")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "triplets/s", "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict({kk: vv for kk, vv in cfg.items() if kk != "golden"}, precision="fp64",
                           parallelism="host cores"),
            "cpu_baseline": {"value": v, "unit": "triplets/s", "cores": threads, "kind": "oracle",
                             "sample": sample, "extrapolated": True},
            "e2e": {"value": v, "unit": "triplets/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
