"""Benchmark of the PHSVDS hot path on one GB300 (or N replicas).

One step = one complete PHSVDS solve (stage 1 GD+k on A^T A, switch test,
Rayleigh-Ritz post-process, stage 2 refined projection on the augmented matrix,
final residuals) of the synthetic workload, through the C ABI.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--grid G] [--precision mixed|fp64|both]

Prints one JSON line (rank 0).  ``value`` = whole-job triplets/s with the CSR
already resident in device memory; ``e2e`` = the same solve through the same
call with host buffers (host->device copy of A and device->host copy of the
singular triplets inside the timed region).
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
    p.add_argument("--grid", type=int, default=64, help="grid side of the weighted gradient workload")
    p.add_argument("--sigma-log", type=float, default=1.0)
    p.add_argument("--k", type=int, default=10)
    p.add_argument("--block", type=int, default=4)
    p.add_argument("--precision", default="both", choices=["mixed", "fp64", "both"])
    p.add_argument("--precond", default="none", choices=["none", "jacobi"])
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--spmm-only", action="store_true", help="only the full-size fused A^T A SpMM timings")
    p.add_argument("--spmm-cases", default="c2,c3", help="full-size SpMM workloads: c2 (512^2 grid), c3 (1e6 x 5e5)")
    p.add_argument("--spmm-reps", type=int, default=10)
    p.add_argument("--spmm-sweep", action="store_true", help="time every group width around the automatic one")
    p.add_argument("--batched", action="store_true",
                   help="batched workload: many uneven random sparse matrices, batched mixed vs sequential FP64")
    p.add_argument("--batch-count", type=int, default=64)
    p.add_argument("--batch-nlo", type=int, default=2000)
    p.add_argument("--batch-nhi", type=int, default=60000)
    p.add_argument("--batch-k", type=int, default=5)
    p.add_argument("--batch-concurrency", type=int, default=0)
    p.add_argument("--batch-no-seq", action="store_true", help="skip the sequential FP64 reference solves")
    p.add_argument("--learned", action="store_true",
                   help="learned-preconditioner workload: train, then none / Jacobi / network on held-out operators")
    p.add_argument("--learned-grid", type=int, default=32)
    p.add_argument("--learned-train", type=int, default=200)
    p.add_argument("--learned-test", type=int, default=10)
    p.add_argument("--learned-epochs", type=int, default=100)
    p.add_argument("--learned-cg-steps", type=int, default=3)
    p.add_argument("--learned-stall", type=int, default=200, help="stall window of the learned correction")
    return p.parse_args()


def workload(a):
    from paper_1408_5535_gb300 import synth
    A = synth.grid_gradient(a.grid, a.sigma_log, 2)
    cfg = {"workload": f"weighted Dirichlet grid gradient {a.grid}x{a.grid} (log-normal sigma_log={a.sigma_log}, "
                       f"seed 2), m={A.m}, n={A.n}, nnz={A.nnz}; k={a.k} smallest, block {a.block}, "
                       f"tol 1e-14*||A||, precond {a.precond}",
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
        for key in [c for c in a.spmm_cases.split(",") if c]:
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


def golden_iters(a):
    """The oracle's own outer-iteration count (stage 1 + stage 2) on this
    workload, recorded by tests/golden/make_oracle_counts.py, or None."""
    try:
        with open(os.path.join(ROOT, "tests", "golden", "oracle_counts.json")) as f:
            g = json.load(f).get(f"grid{a.grid}")
    except Exception:
        return None
    if not g or g["k"] != a.k or g["block"] != a.block or abs(a.sigma_log - 1.0) > 0 or a.precond != "none":
        return None
    return g["iters_stage1"] + g["iters_stage2"]


def cpu_baseline(A, a, k, fallback_iters):
    """The oracle (plain CPU FP64 PHSVDS, as it stands) on the host cores, on a
    bounded sample of the same solve: it runs for at most --cpu-seconds; if it
    has not finished, its time per outer iteration is scaled by the oracle's
    own recorded iteration count for the workload (else by fallback_iters)."""
    from oracle import phsvds_ref as R
    threads = os.environ.get("OMP_NUM_THREADS") or str(os.cpu_count() or 1)

    class Stop(Exception):
        pass

    state = {"it": 0, "t0": None}

    def tr(stage, it, d):
        state["it"] += 1
        if time.perf_counter() - state["t0"] > a.cpu_seconds:
            raise Stop()

    o = R.Opts(block=a.block, precond=a.precond, trace=tr)
    state["t0"] = time.perf_counter()
    try:
        R.phsvds(A, k, delta=TOL, o=o)
        done = True
    except Stop:
        done = False
    el = time.perf_counter() - state["t0"]
    iters = max(state["it"], 1)
    gi = golden_iters(a)
    total = gi if gi else fallback_iters
    est = el if done else el / iters * total
    return {"value": k / est, "unit": "triplets/s", "cores": int(threads), "kind": "oracle",
            "sample": (f"the whole oracle solve of the workload ({iters} outer iterations) in {el:.1f} s" if done
                       else f"{iters} oracle outer iterations in {el:.1f} s, scaled to "
                            f"{'the oracle' if gi else 'the GPU solve'}'s {total} iterations ({est:.0f} s estimated)"),
            "seconds": el, "iterations_sampled": iters, "finished": done}


def run_ours(a, rank, world):
    import numpy as np
    import torch
    from paper_1408_5535_gb300 import native
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    A, cfg = workload(a)
    stream = torch.cuda.Stream(device=dev)
    h = native.Handle(dev, stream.cuda_stream)
    rp = torch.from_numpy(A.row_ptr).cuda()
    ci = torch.from_numpy(A.col).cuda()
    va = torch.from_numpy(A.val).cuda()
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")
    precs = {"mixed": [native.MIXED], "fp64": [native.FP64], "both": [native.MIXED, native.FP64]}[a.precision]
    prec_id = native.PREC_JACOBI if a.precond == "jacobi" else native.PREC_NONE
    results = {}
    for pi, prec in enumerate(precs):
        head = pi == 0                 # the headline precision; the second is the comparison leg
        steps = a.steps if head else max(1, min(a.steps, 2))
        o = native.default_opts(block_size=a.block, precision=prec, profile=0)
        op = native.default_opts(block_size=a.block, precision=prec, profile=1)

        def solve(opts, on_device=True, vectors=False):
            return native.phsvds_solve(h, A.m, A.n, rp if on_device else A.row_ptr, ci if on_device else A.col,
                                       va if on_device else A.val, a.k, native.SMALLEST, TOL, prec_id, opts,
                                       on_device=on_device, want_vectors=vectors)

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
        # end to end: host CSR in, host triplets out, through the same call
        e2e = None
        if not a.no_e2e:
            ee = []
            for _ in range(1):
                flush.fill_(1.0)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                solve(o, on_device=False, vectors=True)
                ee.append((time.perf_counter() - t0) * 1e3)
            e_ms = max_over_ranks(float(np.mean(ee)), world)
            h2d = 8 * (A.m + 1) + 4 * A.nnz + 8 * A.nnz
            d2h = 8 * a.k * (2 + A.m + A.n)
            e2e = {"value": world * a.k / (e_ms / 1e3), "unit": "triplets/s", "h2d_bytes_per_step": h2d,
                   "d2h_bytes_per_step": d2h, "ms_per_step": e_ms}
        results[prec] = dict(ms=ms, sigma=sig.tolist(), resid_rel=(resid / st["norm_A_est"]).tolist(), stats=st,
                             prof=prof, e2e=e2e, clocks=clk.summary(), launches=launches, steps=steps)
    h.close()
    return A, cfg, results


# FP64 peak of one GB300 (nominal 1.25 TFLOP/s: 152 SMs x 2 FP64 FMA per clock
# per SM x 2 flop x ~2.06 GHz); the cluster Jacobi occupies 8 of the 152 SMs.
FP64_PEAK_GFLOPS = 1250.0
JACOBI_CTAS = 8


# the stage-1 projected eigensolve of a call: the FP32 pass and the FP64
# clean-up of the target pairs, with the device helpers they call
JACOBI_FUNCS = ["rr_pair", "rot_params", "rot_params_small", "k_jacobi_eig", "k_jacobi_targets"]


def kernel_source_sha256(kernel_file, names):
    """sha256 of the source text of the named functions of a .cu file (each
    from the line that declares it to its closing brace in column 0), so that
    edits elsewhere in the file do not invalidate a capture."""
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
        if len(starts) != 1:
            return None
        i = starts[0]
        while i < len(lines) and lines[i] != "}":
            h.update(lines[i].encode() + b"\n")
            i += 1
    return h.hexdigest()


def measured_traffic(kernel_file, names, summary, key):
    """DRAM bytes from a committed ncu summary, if the captured kernels' source
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
    Stage-1 projected eigensolve (class 5: the FP32 Jacobi pass with its FP64
    clean-up of the target pairs, or the FP64 cluster Jacobi): algorithmic
    flops per call = 18 j per rotation (rows and columns of H and the columns
    of S, 6 j each) x rotations per call, against the GPU's FP64 peak.
    Otherwise the fused SpMM against the measured HBM copy rate with the
    one-read-of-A byte count."""
    if dom == 5 and prof["n_class"][5] and prof["jacobi_calls"]:
        # whole-solve algorithmic flops of the stage-1 projected solves over
        # the class's whole device time (a solve is one or two launches)
        calls = prof["jacobi_calls"]
        j_avg = prof["jacobi_dim_sum"] / calls
        rot = prof["jacobi_rotations"] / calls
        flops = 18.0 * j_avg * rot
        per_call_ms = prof["t_class_ms"][5] / calls
        ach = flops / (per_call_ms * 1e-3) / 1e9
        tr = measured_traffic("k_small.cu", JACOBI_FUNCS, "jacobi_fp32_targets_grid32.txt", "dram_bytes_per_call")
        return {"bound": "alu", "kernel": "stage-1 projected eigensolve (Jacobi kernels of k_small.cu)",
                "achieved": ach / 1e3, "peak": FP64_PEAK_GFLOPS / 1e3, "unit": "TFLOP/s",
                "frac": ach / FP64_PEAK_GFLOPS, "traffic": tr,
                "peak_source": "nominal FP64 rate of the GPU (152 SMs x 2 FMA/clk)",
                "flops_per_solve_call": flops, "ms_per_solve_call": per_call_ms,
                "launches_per_call": prof["n_class"][5] / calls, "j_avg": j_avg, "rotations_per_call": rot}
    calls = prof["n_class"][0]
    avg_ms = prof["t_class_ms"][0] / calls if calls else None
    width = prof["spmm_c_width"]
    p_bytes = 4 if prof["iters_stage1_fp32"] > 0 else 8
    bytes_per = spmm_bytes(A.m, A.n, A.nnz, width, p_bytes)
    ach = bytes_per / (avg_ms * 1e-3) / 1e9 if avg_ms else None
    return {"bound": "hbm", "kernel": "fused A^T A SpMM (products with C)", "achieved": ach, "peak": hbm,
            "unit": "GB/s", "frac": (ach / hbm) if ach else None, "traffic": None, "peak_source": peak_kind,
            "bytes_per_launch": bytes_per, "avg_launch_ms": avg_ms}


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
           "concurrency": a.batch_concurrency or min(len(mats), 16),
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


def main():
    a = parse()
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
    names = ["fused A^T A SpMM", "Gram / CGS2 passes", "basis transforms / Ritz",
             "refined vector of stage 2 (inverse iteration on R)", "A / A^T products (stage 2)",
             "projected eigensolvers (Jacobi: FP32 pass + FP64 clean-up, or FP64 cluster)"]
    cls = prof["t_class_ms"]
    dom = int(max(range(len(cls)), key=lambda i: cls[i]))
    roof = roofline_for(A, prof, dom, hbm, peak_kind)
    roof.update(dominant_class=names[dom], class_ms=dict(zip(names, cls)),
                class_calls=dict(zip(names, prof["n_class"])))
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
        "config": dict(cfg, precision="mixed" if head == native.MIXED else "fp64",
                       parallelism=f"replicas{world}"),
        "roofline": roof,
        "gpu_launches": r["launches"],
        "gpu_launches_per_step": r["launches"] // max(r["steps"], 1),
        "clocks": r["clocks"],
        "e2e": r["e2e"],
        "solve": {"iters_stage1": st["iters_stage1"], "iters_stage1_fp32": st["iters_stage1_fp32"],
                  "iters_stage2": st["iters_stage2"], "matvecs_A": st["matvecs_A"], "switched": st["switched"],
                  "max_resid_over_normA": max(r["resid_rel"]), "spmm_schedule": st["spmm_schedule"],
                  "jacobi_sweeps": st["jacobi_sweeps"], "jacobi_rotations": st["jacobi_rotations"],
                  "restarts": st["restarts"]},
    }
    if native.FP64 in res and head != native.FP64:
        f = res[native.FP64]
        line["fp64"] = {"value": world * cfg["k"] / (f["ms"] / 1e3), "ms_per_step": f["ms"], "steps": f["steps"],
                        "iters_stage1": f["stats"]["iters_stage1"], "iters_stage2": f["stats"]["iters_stage2"],
                        "speedup_mixed_over_fp64": f["ms"] / r["ms"],
                        "max_sigma_rel_diff_vs_mixed": max(abs(x - y) / y for x, y in zip(r["sigma"], f["sigma"])),
                        "class_ms": dict(zip(names, f["prof"]["t_class_ms"]))}
    if a.spmm_cases:
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
    if rank == 0 and not a.no_cpu:
        line["cpu_baseline"] = cpu_baseline(A, a, cfg["k"], st["iters_stage1"] + st["iters_stage2"])
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_reference(a, rank, world):
    """The oracle (plain CPU FP64 PHSVDS, as it stands) on the host cores, on the
    same workload; rank 0 only, the other ranks exit without work."""
    if rank != 0:
        return
    A, cfg = workload(a)
    steps = []
    for i in range(a.warmup + a.steps):
        cb = cpu_baseline(A, a, cfg["k"], fallback_iters=golden_iters(a) or 4000)
        if i >= a.warmup:
            steps.append(cb)
    v = sum(x["value"] for x in steps) / len(steps)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "triplets/s", "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * cfg["k"] / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(cfg, precision="fp64", parallelism="host cores"),
            "cpu_baseline": dict(steps[-1], value=v),
            "e2e": {"value": v, "unit": "triplets/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
