"""Batched PHSVDS (phsvds_solve_batched) against single solves and the oracle.

The batch is a down-scaled instance of the batched workload: uneven random
sparse matrices, n ~ U[150, 500], m ~ U[1.2n, 2n], Poisson(8) entries per row,
N(0,1) values plus 1e-2 on the diagonal.  Every batched result must meet the
plain definition (residual <= 1e-14 ||A||, recomputed here), equal the single
solve of the same matrix (relative sigma difference <= 1e-10), and for two of
the matrices match the oracle and a dense SVD (same index set).
"""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_1408_5535_gb300 import native, synth
from oracle import phsvds_ref as R
from oracle.dense_jacobi import dense_triplets
from tests.gpu_util import torch, need_gpu

pytestmark = pytest.mark.gpu
DELTA = 1e-14


@pytest.fixture(scope="module")
def h():
    need_gpu()
    with native.Handle(0) as hh:
        yield hh


@pytest.fixture(scope="module")
def batch():
    return synth.batched_set(6, seed=5, n_lo=150, n_hi=500)


def _resid(A, sig, U, V):
    S = sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.m, A.n))
    rv = np.linalg.norm(S @ V - U * sig, axis=0)
    ru = np.linalg.norm(S.T @ U - V * sig, axis=0)
    return np.sqrt(ru ** 2 + rv ** 2)


@pytest.mark.parametrize("largest,precision", [(False, "fp64"), (True, "mixed"), (False, "mixed")])
def test_batched_equals_single_solves(h, batch, largest, precision):
    k = 5
    prec = native.MIXED if precision == "mixed" else native.FP64
    o = native.default_opts(precision=prec)
    tgt = native.LARGEST if largest else native.SMALLEST
    mats = [(A.m, A.n, A.row_ptr, A.col, A.val) for A in batch]
    out, status = native.phsvds_solve_batched(h, mats, k, tgt, DELTA, native.PREC_NONE, o, concurrency=4,
                                              want_vectors=True)
    assert status == native.PHSVDS_OK
    for A, (sig, U, V, res, st, s_i, msg) in zip(batch, out):
        assert s_i == native.PHSVDS_OK, msg
        normA = st["norm_A_est"]
        assert np.all(_resid(A, sig, U, V) <= DELTA * normA)
        assert np.all(np.diff(sig) <= 0) if largest else np.all(np.diff(sig) >= 0)
        s1 = native.phsvds_solve(h, A.m, A.n, A.row_ptr, A.col, A.val, k, tgt, DELTA, native.PREC_NONE, o,
                                 want_vectors=False)[0]
        assert np.max(np.abs(sig - s1) / s1) <= 1e-10


def test_batched_vs_oracle_and_dense(h, batch):
    """Two matrices of the batch: the batched sigma against the oracle's and the
    dense SVD's (relative 1e-10, same index set)."""
    k = 5
    mats = [(A.m, A.n, A.row_ptr, A.col, A.val) for A in batch]
    out, _ = native.phsvds_solve_batched(h, mats, k, native.SMALLEST, DELTA, native.PREC_NONE,
                                         native.default_opts(), concurrency=3)
    for i in (0, 3):
        A = batch[i]
        ref = R.phsvds(A, k, largest=False, delta=DELTA)
        ex = dense_triplets(A.to_dense(), k)[0]
        sig = out[i][0]
        assert np.max(np.abs(sig - ref.sigma) / ref.sigma) <= 1e-10
        assert np.max(np.abs(sig - ex) / ex) <= 1e-10


def test_batched_reports_per_matrix_status(h, batch):
    """A matrix the method rejects (m < n) gets its own INVALID status and
    message; the others of the batch are unaffected."""
    k = 3
    mats = [(A.m, A.n, A.row_ptr, A.col, A.val) for A in batch[:3]]
    tall = synth.random_sparse(300, 100, 4.0, 9)
    W = sp.csr_matrix((tall.val, tall.col, tall.row_ptr), shape=(tall.m, tall.n)).T.tocsr()   # 100 x 300
    W.sort_indices()
    mats.append((W.shape[0], W.shape[1], W.indptr.astype(np.int64), W.indices.astype(np.int32), W.data))
    out, status = native.phsvds_solve_batched(h, mats, k, native.SMALLEST, DELTA, native.PREC_NONE,
                                              native.default_opts(), concurrency=2, raise_on_error=False)
    assert [o[5] for o in out[:3]] == [native.PHSVDS_OK] * 3
    assert out[3][5] == native.PHSVDS_ERR_INVALID and out[3][6]
    assert status == native.PHSVDS_ERR_INVALID


def test_batched_empty_and_invalid(h):
    out, status = native.phsvds_solve_batched(h, [], 3)
    assert out == [] and status == native.PHSVDS_OK


def test_full_size_members_batched_equal_single_solves(h):
    """The four largest members of the full batched workload (64 matrices,
    n ~ U[2000, 60000]; here n ~ 5.4e4-5.9e4), k = 5 smallest and k = 5
    largest, mixed precision, 4 workers: every result meets the plain
    definition (residual <= 1e-14 ||A||, recomputed here with ||A|| = the
    largest sigma found) and equals the single FP64 solve of the same matrix
    to 1e-10 relative."""
    mats = synth.batched_set(64)
    big = sorted(mats, key=lambda A: -A.nnz)[:4]
    tup = [(A.m, A.n, A.row_ptr, A.col, A.val) for A in big]
    om = native.default_opts(precision=native.MIXED, time_limit_s=120.0)
    of = native.default_opts(precision=native.FP64, time_limit_s=120.0)
    res = {}
    for tgt in (native.SMALLEST, native.LARGEST):
        out, status = native.phsvds_solve_batched(h, tup, 5, tgt, DELTA, native.PREC_NONE, om, concurrency=4,
                                                  want_vectors=True)
        assert status == native.PHSVDS_OK
        res[tgt] = out
    for i, A in enumerate(big):
        nA = res[native.LARGEST][i][0][0]
        for tgt in (native.SMALLEST, native.LARGEST):
            sig, U, V = res[tgt][i][0], res[tgt][i][1], res[tgt][i][2]
            assert np.all(_resid(A, sig, U, V) <= DELTA * nA), (i, tgt)
            ref = native.phsvds_solve(h, A.m, A.n, A.row_ptr, A.col, A.val, 5, tgt, DELTA, native.PREC_NONE, of,
                                      want_vectors=False)[0]
            assert np.all(np.abs(sig - ref) <= 1e-10 * ref), (i, tgt, sig, ref)
