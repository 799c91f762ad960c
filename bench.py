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

    def lanes_for(avg):
        return 1 if avg <= 2.5 else 2 if avg <= 6 else 4 if avg <= 16 else 8

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
            la0, lt0 = lanes_for(A.nnz / A.m), lanes_for(A.nnz / A.n)
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


def cpu_baseline(A, a, gpu_stats, k):
    """Oracle (plain CPU FP64) on a bounded sample of the same solve: its stage-1
    iterations are timed for about --cpu-seconds, and the per-iteration time is
    scaled by the outer iterations the GPU solve needed."""
    import numpy as np
    from oracle import phsvds_ref as R
    threads = os.environ.get("OMP_NUM_THREADS") or str(os.cpu_count() or 1)

    class Stop(Exception):
        pass

    state = {"it": 0, "t0": None}

    def tr(stage, it, d):
        state["it"] = it
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
    total_iters = gpu_stats["iters_stage1"] + gpu_stats["iters_stage2"]
    est = el if done else el / iters * total_iters
    return {"value": k / est, "unit": "triplets/s", "cores": int(threads), "kind": "oracle",
            "sample": (f"oracle solved the workload in {el:.1f} s" if done else
                       f"{iters} oracle stage-1 iterations in {el:.1f} s, scaled to the "
                       f"{total_iters} outer iterations of the GPU solve ({est:.0f} s estimated)"),
            "seconds": el}


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
    for prec in precs:
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
            for _ in range(a.steps):
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
            for _ in range(max(1, min(a.steps, 2))):
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
                             prof=prof, e2e=e2e, clocks=clk.summary(), launches=launches // max(a.steps, 1))
    h.close()
    return A, cfg, results


def main():
    a = parse()
    rank, world = dist_init(a)
    if a.impl == "reference":
        return run_reference(a, rank, world)
    import torch
    from paper_1408_5535_gb300 import native
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
    # dominant kernel class of the profiled solve and the fused SpMM roofline
    names = ["fused A^T A SpMM", "Gram / CGS2 passes", "basis transforms / Ritz", "one-CTA Jacobi eig/SVD",
             "A / A^T products (stage 2)"]
    cls = prof["t_class_ms"]
    dom = int(max(range(5), key=lambda i: cls[i]))
    p_bytes = 4 if head == native.MIXED and prof["iters_stage1_fp32"] > 0 else 8
    calls = prof["n_class"][0]
    avg_ms = prof["t_class_ms"][0] / calls if calls else None
    bytes_per = spmm_bytes(A.m, A.n, A.nnz, prof["spmm_c_width"], 8)
    achieved = bytes_per / (avg_ms * 1e-3) / 1e9 if avg_ms else None
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
        "roofline": {"bound": "hbm", "kernel": "fused A^T A SpMM (products with C)",
                     "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": (achieved / hbm) if achieved else None, "traffic": None,
                     "peak_source": peak_kind, "bytes_per_launch": bytes_per, "avg_launch_ms": avg_ms,
                     "dominant_class": names[dom],
                     "class_ms": dict(zip(names, cls)), "class_calls": dict(zip(names, prof["n_class"]))},
        "gpu_launches": r["launches"],
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
        line["fp64"] = {"value": world * cfg["k"] / (f["ms"] / 1e3), "ms_per_step": f["ms"],
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
        line["cpu_baseline"] = cpu_baseline(A, a, st, cfg["k"])
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_reference(a, rank, world):
    """The oracle (plain CPU FP64 PHSVDS) on the host cores; rank 0 only."""
    if rank != 0:
        return
    A, cfg = workload(a)
    from oracle import phsvds_ref as R
    # each step: a bounded sample of the solve (see cpu_baseline), scaled to one solve
    est = None
    steps = []
    for i in range(a.warmup + a.steps):
        cb = cpu_baseline(A, a, {"iters_stage1": a.ref_iters, "iters_stage2": 0} if hasattr(a, "ref_iters")
                          else {"iters_stage1": 20000, "iters_stage2": 2000}, cfg["k"])
        if i >= a.warmup:
            steps.append(cb)
    v = sum(s["value"] for s in steps) / len(steps)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "triplets/s", "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * cfg["k"] / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
            "cpu_baseline": dict(steps[-1], value=v),
            "e2e": {"value": v, "unit": "triplets/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
