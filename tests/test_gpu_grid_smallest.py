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


def _scaled_columns_300():
    import scipy.sparse as sp
    A0 = synth.random_sparse(300, 150, 6.0, 21, values="gaussian", shift=0.05)
    S = R.as_scipy(A0)
    S = (S @ sp.diags(10.0 ** (-2.0 * synth.uniform(31, 1, 150)))).tocsr()
    S.sort_indices()
    return synth.Csr(S.shape[0], S.shape[1], S.indptr.astype(np.int64), S.indices.astype(np.int32), S.data)


@pytest.mark.parametrize("case", ["grid16-unscaled", "scaled-columns-jacobi"])
def test_fp64_jacobi_davidson_stage1_against_the_oracles_form(h, case):
    """The FP64 Jacobi-Davidson stage 1 (opts.stage1_inner) against the
    oracle's form of it (Opts.stage1_inner = "minres", jd1_correction): the
    same values to 1e-10 relative, residuals recomputed here <= 1e-14 ||A||,
    and outer iteration counts of the same order (the oracle's inner solver
    reorthogonalises its Lanczos vectors, the GPU's runs the three-term
    recurrence, so the counts are not equal)."""
    if case == "grid16-unscaled":
        A, k, b, prec, oprec = synth.grid_gradient(16, 1.0, 2), 10, 4, native.PREC_NONE, "none"
    else:
        A, k, b, prec, oprec = _scaled_columns_300(), 4, 2, native.PREC_JACOBI, "jacobi"
    S = R.as_scipy(A)
    nA = float(np.linalg.norm(S.toarray(), 2))
    o = native.default_opts(block_size=b, precision=native.FP64, stage1_inner=1, stage2=0, time_limit_s=60.0)
    sig, U, V, res, st, _ = native.phsvds_solve(h, A.m, A.n, A.row_ptr, A.col, A.val, k, native.SMALLEST, DELTA,
                                                prec, o)
    ref = R.phsvds(A, k, largest=False, delta=DELTA, o=R.Opts(block=b, precond=oprec, stage1_inner="minres",
                                                               stage2=False))
    assert np.all(np.abs(sig - ref.sigma) <= 1e-10 * ref.sigma), (sig, ref.sigma)
    assert np.all(_resid(S, sig, U, V) <= 1e-12 * nA)
    assert st["inner_solves"] > 0 and ref.stats["inner1"] > 0
    it_gpu, it_ref = st["iters_stage1"], ref.stats["iters"]
    assert it_gpu <= 3 * it_ref + 20 and it_ref <= 3 * it_gpu + 20, (it_gpu, it_ref)
