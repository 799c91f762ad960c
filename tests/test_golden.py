"""Stored values: the paper's printed worked example (Table 1) and the oracle's
own recorded behaviour on the benchmark workloads (tests/golden/)."""
import json
import math
import os

import numpy as np
import pytest

from paper_1408_5535_gb300 import synth
from oracle import phsvds_ref as R

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _table1():
    rows = [l.split() for l in open(os.path.join(GOLD, "table1_clustered_tiny.txt")) if l.strip() and l[0] != "#"]
    return np.array([[float(x) for x in r] for r in rows])


def test_table1_spectrum_is_the_generators():
    """The exact column of Table 1 is the ten smallest values of the generator's
    diag(1e-14, 1e-12, 1e-8:1e-8:4e-8, 1e-3:1e-3:1)."""
    t = _table1()
    sig = np.sort(synth.table1_sigma())
    assert sig.size == 1006
    assert np.allclose(t[:, 0], sig[:10], rtol=1e-15, atol=0)


def test_table1_printed_errors_obey_the_residual_bound():
    """For the symmetric B, an approximate eigenpair with residual ||r_B|| has an
    eigenvalue within ||r_B|| (Weyl / Bauer-Fike): every printed sigma~ is within
    its printed ||r_B|| of the exact value -- the accuracy is absolute (about
    delta ||A||), not relative, which is how the tests read the tolerance."""
    t = _table1()
    err = np.abs(t[:, 1] - t[:, 0])
    assert np.all(err <= t[:, 2])
    assert np.all(t[:, 2] <= 1e-15)       # the user tolerance delta ||A||, ||A|| = 1
    assert err[0] / t[0, 0] > 1e-3        # the smallest is only absolutely accurate


def test_oracle_counts_rerun_smallest_case():
    """The recorded oracle run on the 16 x 16 grid reproduces: same iteration
    counts, same singular values to 1e-12, every residual <= 1e-14 ||A||."""
    g = json.load(open(os.path.join(GOLD, "oracle_counts.json")))["grid16"]
    A = synth.grid_gradient(16, 1.0, 2)
    res = R.phsvds(A, g["k"], largest=False, delta=g["delta"], o=R.Opts(block=g["block"]))
    assert int(res.stats["iters"]) == g["iters_stage1"]
    assert int(res.stats.get("iters2", 0)) == g["iters_stage2"]
    assert np.allclose(res.sigma, g["sigma"], rtol=1e-12, atol=0)
    assert max(g["resid_over_normA"]) <= 1e-14


def test_oracle_counts_cover_the_benchmark_workload():
    g = json.load(open(os.path.join(GOLD, "oracle_counts.json")))
    assert {"grid16", "grid32", "c3_largest"} <= set(g)
    for name, v in g.items():
        assert v["iters_stage1"] > 0 and max(v["resid_over_normA"]) <= 1e-14
        if name.startswith("grid"):
            assert v["switched"]        # smallest triplets of a grid need stage 2
    c3 = g["c3_largest"]
    assert c3["target"] == "largest" and c3["k"] == 20 and c3["n"] == 500000 and c3["nnz"] == 12495439
    sig = np.asarray(c3["sigma"])
    assert np.all(np.diff(sig) < 0) and abs(c3["normA"] - sig[0]) <= 1e-12 * sig[0]


def test_oracle_jdqmr_form_reproduces_table1():
    """The paper's worked example (Sec. 5.1, Table 1) run by the oracle's
    JDQMR form of stage 2 at the printed settings (block 2 in stage 1,
    identity preconditioner, delta = 1e-15): all ten clustered tiny values,
    each within the printed ||r_B|| of the exact one (the accuracy Weyl's
    bound gives the printed run) and with a triplet residual <= 1e-15 ||A||."""
    t = _table1()
    A = synth.diag_matrix(synth.table1_sigma())
    res = R.phsvds(A, 10, largest=False, delta=1e-15, o=R.Opts(block=2, stage2_inner="qmr"))
    assert np.all(np.abs(res.sigma - t[:, 0]) <= t[:, 2])
    assert np.all(res.resid <= 1e-15 * res.normA)
    assert res.stats["switched"]
