"""Algorithm 3 (Sec. 4, dynamic switching between GD+k on C and on B under
preconditioning; opts.dynamic = 1) on the GPU, against the oracle's form
(`dynamic_phsvds`) and the dense SVD.

* The two-stage demonstration of Sec. 5.1 (A = diag([1:10, 1000:100:1e6]),
  the caller's M = A + diag(1e4 rand)): sigma_min = 1 at 1e-14 ||A||, as the
  oracle's dynamic form finds it.
* A 300 x 150 random matrix with columns scaled over two decades and the
  Jacobi family of preconditioners: the 4 smallest triplets of the dense SVD.
* The unpreconditioned form on a small random matrix.
Every residual is recomputed here in FP64; the runs and switches follow the
algorithm's maxIter rule (at least the two initial tests).
"""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_1408_5535_gb300 import native, synth
from oracle import phsvds_ref as R
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu
DELTA = 1e-14


@pytest.fixture(scope="module")
def h():
    need_gpu()
    with native.Handle(0) as hh:
        yield hh


def _resid(S, sig, U, V):
    rv = np.linalg.norm(S @ V - U * sig, axis=0)
    ru = np.linalg.norm(S.T @ U - V * sig, axis=0)
    return np.sqrt(rv ** 2 + ru ** 2)


def test_dynamic_on_the_two_stage_demonstration(h):
    A, M = synth.e3_diag()
    S = R.as_scipy(A)
    o = native.default_opts(dynamic=1)
    sig, U, V, res, st, _ = native.phsvds_solve(h, A.m, A.n, A.row_ptr, A.col, A.val, 1, native.SMALLEST, DELTA,
                                                native.PREC_GIVEN, o, precond_M=M)
    ref = R.dynamic_phsvds(A, 1, delta=DELTA, o=R.Opts(precond="given", precond_M=M))
    assert abs(sig[0] - 1.0) <= 1e-10 and abs(sig[0] - ref.sigma[0]) <= 1e-10
    assert _resid(S, sig, U, V)[0] <= DELTA * 1e6
    assert st["dynamic_runs"] >= 2 and st["dynamic_route"] in (1, 2, 3, 4)


def test_dynamic_with_the_jacobi_family_matches_the_dense_svd(h):
    A0 = synth.random_sparse(300, 150, 6.0, 21, values="gaussian", shift=0.05)
    S = R.as_scipy(A0)
    S = (S @ sp.diags(10.0 ** (-2.0 * synth.uniform(31, 1, 150)))).tocsr()
    S.sort_indices()
    A = synth.Csr(S.shape[0], S.shape[1], S.indptr.astype(np.int64), S.indices.astype(np.int32), S.data)
    k = 4
    o = native.default_opts(block_size=2, dynamic=1)
    sig, U, V, res, st, _ = native.phsvds_solve(h, A.m, A.n, A.row_ptr, A.col, A.val, k, native.SMALLEST, DELTA,
                                                native.PREC_JACOBI, o)
    sv = np.sort(np.linalg.svd(S.toarray(), compute_uv=False))[:k]
    nA = float(np.linalg.norm(S.toarray(), 2))
    assert np.max(np.abs(sig - sv) / sv) <= 1e-10, (sig, sv)
    assert np.all(_resid(S, sig, U, V) <= DELTA * nA)
    assert st["dynamic_runs"] >= 2


def test_dynamic_unpreconditioned_small(h):
    A = synth.random_sparse(200, 90, 6.0, 7, values="gaussian", shift=0.3)
    S = R.as_scipy(A)
    k = 3
    o = native.default_opts(block_size=1, dynamic=1, dyn_init_iter=30)
    sig, U, V, res, st, _ = native.phsvds_solve(h, A.m, A.n, A.row_ptr, A.col, A.val, k, native.SMALLEST, DELTA,
                                                native.PREC_NONE, o)
    sv = np.sort(np.linalg.svd(S.toarray(), compute_uv=False))[:k]
    nA = float(np.linalg.norm(S.toarray(), 2))
    assert np.max(np.abs(sig - sv) / sv) <= 1e-10
    assert np.all(_resid(S, sig, U, V) <= DELTA * nA)


def test_dynamic_is_for_the_smallest_in_fp64(h):
    A = synth.random_sparse(60, 30, 5.0, 2, values="gaussian")
    for kw, target in ((dict(dynamic=1), native.LARGEST), (dict(dynamic=1, precision=native.MIXED), native.SMALLEST),
                       (dict(dynamic=2), native.SMALLEST)):
        o = native.default_opts(max_basis=14, min_restart=8, **kw)
        *_, status = native.phsvds_solve(h, A.m, A.n, A.row_ptr, A.col, A.val, 2, target, DELTA, native.PREC_NONE,
                                         o, raise_on_error=False)
        assert status == native.PHSVDS_ERR_INVALID
