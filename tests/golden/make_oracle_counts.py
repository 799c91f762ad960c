"""Writes oracle_counts.json: what the oracle (plain CPU FP64 PHSVDS) does on the
weighted Dirichlet grid-gradient workloads of the benchmark and the tests --
outer iterations per stage, products with A, singular values and residuals.

The benchmark's reference arm uses the recorded iteration counts to scale a
bounded sample of oracle iterations to a whole solve; the tests re-run the
smallest case and compare.  Calls only oracle/ (and the seeded generator).

    python tests/golden/make_oracle_counts.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from paper_1408_5535_gb300 import synth  # noqa: E402
from oracle import phsvds_ref as R  # noqa: E402

# (grid side, sigma_log, seed, k, block): the benchmark solve is grid 64
CASES = [(16, 1.0, 2, 10, 4), (32, 1.0, 2, 10, 4), (64, 1.0, 2, 10, 4)]


def run(N, sl, seed, k, b):
    A = synth.grid_gradient(N, sl, seed)
    t0 = time.perf_counter()
    res = R.phsvds(A, k, largest=False, delta=1e-14, o=R.Opts(block=b))
    el = time.perf_counter() - t0
    st = res.stats
    return {"workload": f"grid_gradient({N}, {sl}, {seed})", "m": A.m, "n": A.n, "nnz": A.nnz, "k": k, "block": b,
            "delta": 1e-14, "iters_stage1": int(st["iters"]), "iters_stage2": int(st.get("iters2", 0)),
            "restarts_stage1": int(st["restarts"]), "mv_A": int(st["mv_A"]), "switched": bool(st["switched"]),
            "sigma": [float(x) for x in res.sigma], "resid_over_normA": [float(x / res.normA) for x in res.resid],
            "oracle_seconds": el}


if __name__ == "__main__":
    out = {f"grid{N}": run(N, sl, seed, k, b) for N, sl, seed, k, b in CASES}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_counts.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({k: (v["iters_stage1"], v["iters_stage2"], round(v["oracle_seconds"], 1)) for k, v in out.items()}))
