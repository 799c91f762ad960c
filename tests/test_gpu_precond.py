"""The preconditioned forms of Sec. 4 on the GPU, against the oracle.

* The stage-2 preconditioner built from stage 1's M ~ C^{-1}: [0 A M; M A^T 0]
  with M = diag(C)^{-1} (opts.stage2_precond), in the Olsen form, on a matrix
  whose columns are scaled over two decades: the same smallest triplets as
  the oracle's form and the dense SVD (1e-10 relative, residuals recomputed
  here <= 1e-14 ||A||) in fewer stage-2 iterations than plain GD.
* A preconditioner M ~ A given by the caller (PHSVDS_PREC_GIVEN): M^{-1} M^{-T}
  for C in stage 1 and [0 M^{-1}; M^{-T} 0] for B in stage 2, on the
  demonstration of Sec. 5.1 (A = diag([1:10, 1000:100:1e6]),
  M = A + diag(1e4 rand)): stage 1 alone stops near its attainable
  eps ||A|| / sigma; the two stages find sigma_min = 1 at 1e-14 ||A||, as the
  oracle does.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_1408_5535_gb300 import native, synth
from oracle import phsvds_ref as R
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu
DELTA = 1e-14
EPS64 = 2.0 ** -52


@pytest.fixture(scope="module")
def h():
    need_gpu()
    with native.Handle(0) as hh:
        yield hh


def _scaled_columns():
    A0 = synth.random_sparse(300, 150, 6.0, 21, values="gaussian", shift=0.05)
    S = R.as_scipy(A0)
    S = (S @ sp.diags(10.0 ** (-2.0 * synth.uniform(31, 1, 150)))).tocsr()
    S.sort_indices()
    return synth.Csr(S.shape[0], S.shape[1], S.indptr.astype(np.int64), S.indices.astype(np.int32), S.data), S


def _resid(S, sig, U, V):
    rv = np.linalg.norm(S @ V - U * sig, axis=0)
    ru = np.linalg.norm(S.T @ U - V * sig, axis=0)
    return np.sqrt(rv ** 2 + ru ** 2)


def test_stage2_preconditioner_same_triplets_fewer_iterations(h):
    A, S = _scaled_columns()
    k = 4
    runs = {}
    for sp2 in (0, 1):
        o = native.default_opts(block_size=2, stage2_precond=sp2)
        runs[sp2] = native.phsvds_solve(h, A.m, A.n, A.row_ptr, A.col, A.val, k, native.SMALLEST, DELTA,
                                        native.PREC_JACOBI, o)
    sv = np.sort(np.linalg.svd(S.toarray(), compute_uv=False))[:k]
    nA = float(np.linalg.norm(S.toarray(), 2))
    ref = R.phsvds(A, k, largest=False, delta=DELTA, o=R.Opts(block=2, precond="jacobi", stage2_precond=True))
    for sp2, (sig, U, V, res, st, _) in runs.items():
        assert st["switched"]
        assert np.max(np.abs(sig - sv) / sv) <= 1e-10
        assert np.max(np.abs(sig - ref.sigma) / ref.sigma) <= 1e-10
        assert np.all(_resid(S, sig, U, V) <= DELTA * nA)
    assert runs[1][4]["iters_stage2"] < runs[0][4]["iters_stage2"], (runs[1][4]["iters_stage2"],
                                                                     runs[0][4]["iters_stage2"])


def test_given_preconditioner_on_the_two_stage_demonstration(h):
    A, M = synth.e3_diag()
    S = R.as_scipy(A)
    nA = 1e6
    o1 = native.default_opts(stage2=0)
    one = native.phsvds_solve(h, A.m, A.n, A.row_ptr, A.col, A.val, 1, native.SMALLEST, DELTA,
                              native.PREC_GIVEN, o1, precond_M=M)
    two = native.phsvds_solve(h, A.m, A.n, A.row_ptr, A.col, A.val, 1, native.SMALLEST, DELTA,
                              native.PREC_GIVEN, native.default_opts(), precond_M=M)
    ref = R.phsvds(A, 1, largest=False, delta=DELTA, o=R.Opts(precond="given", precond_M=M))
    # stage 1 alone: near its attainable eps ||A|| / sigma, above the tolerance
    r1 = float(_resid(S, one[0], one[1], one[2])[0]) / nA
    assert r1 > DELTA and r1 < 10 * EPS64 * nA / 1.0
    # both stages: sigma_min = 1, like the oracle, at 1e-14 ||A||
    sig, U, V, res, st, _ = two
    assert st["switched"] and st["iters_stage2"] >= 1
    assert abs(sig[0] - 1.0) <= 1e-10 and abs(sig[0] - ref.sigma[0]) <= 1e-10
    assert float(_resid(S, sig, U, V)[0]) <= DELTA * nA
    assert abs(abs(V[:, 0] @ ref.V[:, 0]) - 1) <= 1e-10


def test_given_preconditioner_needs_a_square_matrix_and_a_diagonal(h):
    A = synth.random_sparse(60, 30, 5.0, 2, values="gaussian")
    o = native.default_opts(max_basis=14, min_restart=8)
    *_, status = native.phsvds_solve(h, A.m, A.n, A.row_ptr, A.col, A.val, 2, native.SMALLEST, DELTA,
                                     native.PREC_GIVEN, o, precond_M=np.ones(30), raise_on_error=False)
    assert status == native.PHSVDS_ERR_INVALID                  # m != n
    D = synth.diag_matrix(np.arange(1.0, 31.0))
    *_, status = native.phsvds_solve(h, D.m, D.n, D.row_ptr, D.col, D.val, 2, native.SMALLEST, DELTA,
                                     native.PREC_GIVEN, o, raise_on_error=False)
    assert status == native.PHSVDS_ERR_INVALID                  # no M
    Mz = np.ones(30)
    Mz[3] = 0.0
    *_, status = native.phsvds_solve(h, D.m, D.n, D.row_ptr, D.col, D.val, 2, native.SMALLEST, DELTA,
                                     native.PREC_GIVEN, o, precond_M=Mz, raise_on_error=False)
    assert status == native.PHSVDS_ERR_INVALID                  # a zero entry


def test_scaled_jd_inner_solve_with_jacobi(h):
    """The Jacobi-preconditioned correction equation of the FP64 continuation
    (mixed precision, PHSVDS_PREC_JACOBI, opts.mixed_inner = 1: MINRES on
    D^{-1/2} P (C - theta I) P D^{-1/2}, D = diag(C)) on a matrix whose columns
    are scaled over three decades: the dense SVD's smallest triplets
    (1e-10 relative, residuals <= 1e-14 ||A||), as with the Olsen-Jacobi
    correction (mixed_inner = 0), in fewer FP64 outer iterations."""
    A0 = synth.random_sparse(3000, 1500, 8.0, 41, values="gaussian", shift=0.05)
    S = R.as_scipy(A0)
    S = (S @ sp.diags(10.0 ** (-3.0 * synth.uniform(43, 1, 1500)))).tocsr()
    S.sort_indices()
    A = synth.Csr(S.shape[0], S.shape[1], S.indptr.astype(np.int64), S.indices.astype(np.int32), S.data)
    k = 5
    dense = S.toarray()
    sv = np.sort(np.linalg.svd(dense, compute_uv=False))[:k]
    nA = float(np.linalg.norm(dense, 2))
    runs = {}
    for inner in (0, 1):
        o = native.default_opts(block_size=4, precision=native.MIXED, mixed_inner=inner)
        runs[inner] = native.phsvds_solve(h, A.m, A.n, A.row_ptr, A.col, A.val, k, native.SMALLEST, DELTA,
                                          native.PREC_JACOBI, o)
    for inner, (sig, U, V, res, st, _) in runs.items():
        assert np.all(np.abs(sig - sv) <= 1e-10 * sv), (inner, sig, sv)
        assert np.all(_resid(S, sig, U, V) <= DELTA * nA), (inner, _resid(S, sig, U, V) / nA)
    st0, st1 = runs[0][4], runs[1][4]
    assert st1["inner_solves"] > 0 and st0["inner_solves"] == 0
    fp64_its = {i: r[4]["iters_stage1"] - r[4]["iters_stage1_fp32"] for i, r in runs.items()}
    print("FP64 outer iterations (Olsen-Jacobi, scaled JD):", fp64_its[0], fp64_its[1], "inner steps",
          st1["inner_steps"])
    assert fp64_its[1] < fp64_its[0], fp64_its
