"""Writes oracle_counts.json: what the oracle (plain CPU FP64 PHSVDS) does on the
workloads of the benchmark and the tests -- outer iterations per stage, products
with A, singular values and residuals:

* the weighted Dirichlet grid gradients (16^2, 32^2, 64^2; k = 10 smallest);
* the random sparse 1,000,000 x 500,000 matrix (Poisson(12) entries per row,
  log-normal(2) values with random signs, + 1e-3 [I; 0], seed 3), k = 20
  largest, block 8.

The benchmark's CPU baseline and reference arm use the recorded iteration
counts to scale a bounded sample of oracle iterations to a whole solve, and
the benchmark states every triplet's error against the recorded singular
values; the tests re-run the small cases and compare.  Calls only oracle/ (and
the seeded generator).

    python tests/golden/make_oracle_counts.py [case ...]     (default: all)
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from paper_1408_5535_gb300 import synth  # noqa: E402
from oracle import phsvds_ref as R  # noqa: E402

# name -> (generator call as text, generator, k, largest, block)
CASES = {
    "grid16": ("grid_gradient(16, 1.0, 2)", lambda: synth.grid_gradient(16, 1.0, 2), 10, False, 4),
    "grid32": ("grid_gradient(32, 1.0, 2)", lambda: synth.grid_gradient(32, 1.0, 2), 10, False, 4),
    "grid64": ("grid_gradient(64, 1.0, 2)", lambda: synth.grid_gradient(64, 1.0, 2), 10, False, 4),
    "c3_largest": ("random_sparse(1000000, 500000, 12.0, 3)",
                   lambda: synth.random_sparse(1000000, 500000, 12.0, 3), 20, True, 8),
}
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_counts.json")


def run(name):
    text, gen, k, largest, b = CASES[name]
    A = gen()
    t0 = time.perf_counter()
    res = R.phsvds(A, k, largest=largest, delta=1e-14, o=R.Opts(block=b))
    el = time.perf_counter() - t0
    st = res.stats
    return {"workload": text, "m": A.m, "n": A.n, "nnz": A.nnz, "k": k, "block": b,
            "target": "largest" if largest else "smallest",
            "delta": 1e-14, "iters_stage1": int(st["iters"]), "iters_stage2": int(st.get("iters2", 0)),
            "restarts_stage1": int(st["restarts"]), "mv_A": int(st["mv_A"]), "switched": bool(st["switched"]),
            "sigma": [float(x) for x in res.sigma], "resid_over_normA": [float(x / res.normA) for x in res.resid],
            "normA": float(res.normA), "oracle_seconds": el}


if __name__ == "__main__":
    names = sys.argv[1:] or list(CASES)
    try:
        with open(OUT) as f:
            out = json.load(f)
    except OSError:
        out = {}
    for nm in names:
        out[nm] = run(nm)
        print(nm, out[nm]["iters_stage1"], out[nm]["iters_stage2"], round(out[nm]["oracle_seconds"], 1), flush=True)
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
