"""The weighted grid gradients (C2's family) through the Jacobi-Davidson path
on the GPU: the Jacobi preconditioner with the scaled Jacobi-Davidson inner
solves of stage 1, JDQMR in stage 2, ||A|| estimated before stage 1.

* 64 x 64, both precisions (FP32 MINRES in the mixed form, in its FP64
  continuation or, with opts.mixed_inner = 2, in its FP32 stage as well;
  FP64 MINRES with opts.stage1_inner): the oracle's recorded 10 smallest values
  (tests/golden/oracle_counts.json, the plain method run to completion) to
  1e-10 relative, residuals recomputed here <= 1e-14 ||A||.
* 512 x 512 (C2 at full size, m = 525,312, n = 262,144), mixed precision
  (both opts.mixed_inner forms):
  the 10 smallest values of a shift-invert Lanczos run on C = A^T A (scipy's
  eigsh about 0, a library routine independent of this code) to 1e-10
  relative, residuals recomputed here <= 1e-14 ||A|| with ||A|| from scipy's
  svds; the plain method does not finish at this size.
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse.linalg as sla

from paper_1408_5535_gb300 import native, synth
from oracle import phsvds_ref as R
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu
DELTA = 1e-14
GOLD = os.path.join(os.path.dirname(__file__), "golden", "oracle_counts.json")


@pytest.fixture(scope="module")
def h():
    need_gpu()
    with native.Handle(0) as hh:
        yield hh


def _resid(S, sig, U, V):
    rv = np.linalg.norm(S @ V - U * sig, axis=0)
    ru = np.linalg.norm(S.T @ U - V * sig, axis=0)
    return np.sqrt(rv ** 2 + ru ** 2)


def _opts(prec, k_block=4, mixed_inner=1):
    if prec == native.MIXED:
        return native.default_opts(block_size=k_block, precision=native.MIXED, mixed_inner=mixed_inner,
                                   stage2_inner=1, norm_A=-1.0, time_limit_s=120.0)
    return native.default_opts(block_size=k_block, precision=native.FP64, stage1_inner=1, stage2_inner=1,
                               norm_A=-1.0, time_limit_s=120.0)


@pytest.mark.parametrize("prec,mixed_inner", [(native.MIXED, 1), (native.MIXED, 2), (native.FP64, 1)],
                         ids=["mixed", "mixed-fp32-stage-jd", "fp64"])
def test_grid64_matches_the_oracle(h, prec, mixed_inner):
    g = json.load(open(GOLD))["grid64"]
    A = synth.grid_gradient(64, 1.0, 2)
    S = R.as_scipy(A)
    nA = sla.svds(S, k=1, return_singular_vectors=False)[0]
    sig, U, V, res, st, _ = native.phsvds_solve(h, A.m, A.n, A.row_ptr, A.col, A.val, 10, native.SMALLEST, DELTA,
                                                native.PREC_JACOBI, _opts(prec, mixed_inner=mixed_inner))
    ref = np.array(g["sigma"])
    assert np.all(np.abs(sig - ref) <= 1e-10 * ref), np.max(np.abs(sig - ref) / ref)
    assert np.all(_resid(S, sig, U, V) <= DELTA * nA)
    assert st["inner_solves"] > 0
    assert st["iters_stage1"] < g["iters_stage1"] / 10


@pytest.mark.parametrize("mixed_inner", [1, 2], ids=["mixed", "mixed-fp32-stage-jd"])
def test_grid512_full_size_matches_shift_invert_lanczos(h, mixed_inner):
    A = synth.grid_gradient(512, 1.0, 2)
    S = R.as_scipy(A)
    C = (S.T @ S).tocsc()
    w = sla.eigsh(C, k=10, sigma=0.0, which="LM", tol=0, return_eigenvectors=False)
    ref = np.sort(np.sqrt(w))
    nA = sla.svds(S, k=1, return_singular_vectors=False)[0]
    sig, U, V, res, st, _ = native.phsvds_solve(h, A.m, A.n, A.row_ptr, A.col, A.val, 10, native.SMALLEST, DELTA,
                                                native.PREC_JACOBI, _opts(native.MIXED, mixed_inner=mixed_inner))
    assert np.all(np.abs(sig - ref) <= 1e-10 * ref), np.max(np.abs(sig - ref) / ref)
    assert np.all(_resid(S, sig, U, V) <= DELTA * nA), np.max(_resid(S, sig, U, V)) / nA
    assert abs(st["norm_A_est"] - nA) <= 1e-6 * nA
