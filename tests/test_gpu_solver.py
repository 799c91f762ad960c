"""PHSVDS on the GPU against the CPU oracle and the plain definition."""
import math

import numpy as np
import pytest

from paper_1408_5535_gb300 import native, synth
from oracle import phsvds_ref as R
from oracle.dense_jacobi import dense_triplets
from tests.gpu_util import torch, need_gpu, dev

pytestmark = pytest.mark.gpu
DELTA = 1e-14


def _orth_ok(X, sig, normA):
    """Orthonormal columns up to what the residuals allow: |x_i^T x_j| <=
    4 delta ||A|| / |s_i - s_j| (Davis-Kahan), never looser than 1e-7 and
    never tighter than 1e-12."""
    G = X.T @ X
    k = G.shape[0]
    assert np.max(np.abs(np.diag(G) - 1)) < 1e-12
    for i in range(k):
        for j in range(i + 1, k):
            gap = abs(sig[i] - sig[j])
            tol = 1e-12 if gap == 0 else min(1e-7, max(1e-12, 4 * DELTA * normA / gap))
            assert abs(G[i, j]) <= tol, (i, j, G[i, j], tol)


@pytest.fixture(scope="module")
def h():
    need_gpu()
    with native.Handle(0) as hh:
        yield hh


def _solve(h, A, k, largest=False, **kw):
    prec = kw.pop("precond", native.PREC_NONE)
    o = native.default_opts(**kw)
    return native.phsvds_solve(h, A.m, A.n, A.row_ptr, A.col, A.val, k,
                               native.LARGEST if largest else native.SMALLEST, DELTA, prec, o)


def _check(A, sig, U, V, res, k, sig_ex, normA, rel=1e-10):
    d = A.to_dense() if A.m * A.n < 4e7 else None
    assert np.max(np.abs(sig - sig_ex) / sig_ex) < rel, (sig, sig_ex)
    # residuals recomputed here from A (FP64, CPU)
    import scipy.sparse as sp
    S = sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.m, A.n))
    rv = np.linalg.norm(S @ V - U * sig, axis=0)
    ru = np.linalg.norm(S.T @ U - V * sig, axis=0)
    assert np.all(np.sqrt(ru ** 2 + rv ** 2) <= DELTA * normA), np.sqrt(ru ** 2 + rv ** 2) / normA
    assert np.all(res <= DELTA * normA * (1 + 1e-6))
    _orth_ok(V, sig, normA)
    _orth_ok(U, sig, normA)


@pytest.mark.parametrize("largest", [False, True])
@pytest.mark.parametrize("b", [1, 3])
def test_tiny_vs_dense_jacobi_and_oracle(h, largest, b):
    A = synth.random_sparse(80, 40, 5.0, 11, values="gaussian", shift=0.05)
    sig, U, V, res, st, _ = _solve(h, A, 4, largest, block_size=b, max_basis=14, min_restart=8)
    sd, Ud, Vd = dense_triplets(A.to_dense(), 4, largest)
    _check(A, sig, U, V, res, 4, sd, np.linalg.norm(A.to_dense(), 2))
    ref = R.phsvds(A, 4, largest=largest, delta=DELTA, o=R.Opts(block=b, max_basis=14, min_restart=8))
    assert np.max(np.abs(sig - ref.sigma) / ref.sigma) < 1e-10
    assert np.all(np.abs(np.abs(np.sum(V * ref.V, axis=0)) - 1) < 1e-8)   # simple values: same vectors


def test_exact_spectrum_cluster_c1(h):
    """2000 x 1000 Givens-conjugated spectrum, cluster 1e-4 + {0,1,2}e-7, k=3, b=1, basis 30."""
    sigx = synth.cluster_spectrum_c1()
    A = synth.givens_diag(sigma=sigx)
    sig, U, V, res, st, _ = _solve(h, A, 3, block_size=1, max_basis=30, min_restart=18)
    assert st["switched"] == 1
    _check(A, sig, U, V, res, 3, np.sort(sigx)[:3], 1.0)
    ref = R.phsvds(A, 3, delta=DELTA, o=R.Opts(block=1, max_basis=30, min_restart=18))
    assert np.max(np.abs(sig - ref.sigma) / ref.sigma) < 1e-10


def test_grid_closed_form(h):
    A = synth.grid_gradient(20, 0.0, 2)
    sig, U, V, res, st, _ = _solve(h, A, 6, block_size=2)
    _check(A, sig, U, V, res, 6, A.sigma_exact[:6], A.sigma_exact[-1])


@pytest.mark.parametrize("projected_solver", [0, 1, 2])
def test_weighted_grid_vs_oracle(h, projected_solver):
    """Every projected eigensolver of stage 1 (FP64 cluster Jacobi, one-CTA
    compacted FP64 Jacobi, gated FP32 pass + FP64 clean-up) gives the oracle's
    triplets."""
    A = synth.grid_gradient(24, 1.0, 2)
    sig, U, V, res, st, _ = _solve(h, A, 10, block_size=4, projected_solver=projected_solver)
    ref = R.phsvds(A, 10, delta=DELTA, o=R.Opts(block=4))
    nA = np.linalg.norm(A.to_dense(), 2)
    _check(A, sig, U, V, res, 10, ref.sigma, nA)


def test_mixed_precision_vs_fp64_oracle(h):
    A = synth.grid_gradient(24, 1.0, 2)
    sig, U, V, res, st, _ = _solve(h, A, 10, block_size=4, precision=native.MIXED)
    assert st["iters_stage1_fp32"] > 0
    ref = R.phsvds(A, 10, delta=DELTA, o=R.Opts(block=4))
    nA = np.linalg.norm(A.to_dense(), 2)
    _check(A, sig, U, V, res, 10, ref.sigma, nA)


def test_jacobi_preconditioner_vs_oracle(h):
    A = synth.grid_gradient(20, 1.0, 2)
    sig, U, V, res, st, _ = _solve(h, A, 5, block_size=1, precond=native.PREC_JACOBI)
    ref = R.phsvds(A, 5, delta=DELTA, o=R.Opts(block=1, precond="jacobi"))
    nA = np.linalg.norm(A.to_dense(), 2)
    _check(A, sig, U, V, res, 5, ref.sigma, nA)


@pytest.mark.parametrize("schedule", [1, 2])
def test_spmm_schedules_agree(h, schedule):
    A = synth.random_sparse(600, 300, 8.0, 9, values="gaussian", shift=0.1)
    sig, U, V, res, st, _ = _solve(h, A, 4, block_size=2, spmm=schedule)
    assert st["spmm_schedule"] == schedule
    sd, _, _ = dense_triplets(A.to_dense(), 4)
    _check(A, sig, U, V, res, 4, sd, np.linalg.norm(A.to_dense(), 2))


def test_device_pointer_input(h):
    A = synth.random_sparse(120, 60, 5.0, 17, values="gaussian", shift=0.1)
    rp, ci, va = dev(A.row_ptr), dev(A.col), dev(A.val)
    sig, U, V, res, st, _ = native.phsvds_solve(h, A.m, A.n, rp, ci, va, 3, native.SMALLEST, DELTA,
                                                opts=native.default_opts(max_basis=16, min_restart=8),
                                                on_device=True)
    sd, _, _ = dense_triplets(A.to_dense(), 3)
    _check(A, sig, U, V, res, 3, sd, np.linalg.norm(A.to_dense(), 2))


def test_warm_start_from_an_earlier_solve(h):
    """opts.init_V, the hand-off between runs (Sec. 3.3): the right singular
    vectors of a finished solve, given as the initial guess of stage 1, give
    the same triplets in far fewer stage-1 iterations; a bad init_nv is
    refused before anything runs."""
    A = synth.grid_gradient(20, 1.0, 2)
    sig, U, V, res, st, _ = _solve(h, A, 5, block_size=2)
    o = native.default_opts(block_size=2)
    sig2, U2, V2, res2, st2, _ = native.phsvds_solve(h, A.m, A.n, A.row_ptr, A.col, A.val, 5, native.SMALLEST,
                                                     DELTA, native.PREC_NONE, o, init_V=V)
    ref = R.phsvds(A, 5, delta=DELTA, o=R.Opts(block=2))
    nA = np.linalg.norm(A.to_dense(), 2)
    _check(A, sig2, U2, V2, res2, 5, ref.sigma, nA)
    assert st2["iters_stage1"] * 4 <= st["iters_stage1"], (st2["iters_stage1"], st["iters_stage1"])
    bad = native.default_opts(block_size=2, max_basis=20)
    x0 = np.ascontiguousarray(np.ones((A.n, 1)))
    bad.init_V = x0.ctypes.data
    bad.init_nv = 21
    *_, status = native.phsvds_solve(h, A.m, A.n, A.row_ptr, A.col, A.val, 5, native.SMALLEST, DELTA,
                                     native.PREC_NONE, bad, raise_on_error=False)
    assert status == native.PHSVDS_ERR_INVALID


def test_spmm_plan_is_kept_by_the_handle(h):
    """The autotuned SpMM schedule of a matrix shape is reused by the next
    solve of that shape on the same handle, with the same triplets."""
    A = synth.random_sparse(500, 250, 7.0, 31, values="gaussian", shift=0.1)
    with native.Handle(0) as h2:
        o = native.default_opts(block_size=2)
        r1 = native.phsvds_solve(h2, A.m, A.n, A.row_ptr, A.col, A.val, 3, native.SMALLEST, DELTA, opts=o)
        r2 = native.phsvds_solve(h2, A.m, A.n, A.row_ptr, A.col, A.val, 3, native.SMALLEST, DELTA, opts=o)
    assert r1[4]["spmm_plan_cached"] == 0 and r2[4]["spmm_plan_cached"] == 1
    assert r1[4]["spmm_schedule"] == r2[4]["spmm_schedule"]
    sd, _, _ = dense_triplets(A.to_dense(), 3)
    _check(A, r2[0], r2[1], r2[2], r2[3], 3, sd, np.linalg.norm(A.to_dense(), 2))
    # the work counters of the roofline: products with C counted at 4 nnz b flops each
    st = r2[4]
    assert st["class_flops"][0] > 0 and st["class_bytes"][1] > 0


@pytest.mark.parametrize("kw", [dict(block_size=2), dict(block_size=2, precision=native.MIXED),
                                dict(block_size=2, stage2_inner=1)])
def test_solves_repeat_bit_for_bit(kw):
    """opts.deterministic (the default): every cross-block reduction sums in a
    fixed order and the SpMM plan of the handle is reused, so a second solve
    on the same handle gives the same bits and the same iteration counts."""
    need_gpu()
    A = synth.grid_gradient(20, 1.0, 2)
    with native.Handle(0) as h2:
        o = native.default_opts(**kw)
        r1 = native.phsvds_solve(h2, A.m, A.n, A.row_ptr, A.col, A.val, 4, native.SMALLEST, DELTA, opts=o)
        r2 = native.phsvds_solve(h2, A.m, A.n, A.row_ptr, A.col, A.val, 4, native.SMALLEST, DELTA, opts=o)
    assert r1[4]["spmm_schedule"] == 2
    assert np.array_equal(r1[0], r2[0]) and np.array_equal(r1[1], r2[1]) and np.array_equal(r1[2], r2[2])
    for key in ("iters_stage1", "iters_stage2", "matvecs_A", "inner_steps", "inner2_steps"):
        assert r1[4][key] == r2[4][key], key


# ---- edge cases and failure paths (host-side, no GPU fault)
_OK = dict(max_basis=14, min_restart=8)


def _status(h, A, k, rp=None, col=None, val=None, **kw):
    o = native.default_opts(**dict(_OK, **kw))
    *_, status = native.phsvds_solve(h, A.m, A.n, A.row_ptr if rp is None else rp, A.col if col is None else col,
                                     A.val if val is None else val, k, opts=o, raise_on_error=False)
    return status


def test_valid_baseline_of_the_error_cases(h):
    A = synth.random_sparse(60, 30, 5.0, 2, values="gaussian")
    assert _status(h, A, 2) == native.PHSVDS_OK

def test_invalid_shape(h):
    A = synth.random_sparse(30, 40, 3.0, 1, values="gaussian", shift=0.0)   # m < n
    assert _status(h, A, 2) == native.PHSVDS_ERR_INVALID


def test_invalid_csr_unsorted_columns(h):
    A = synth.random_sparse(60, 30, 5.0, 2, values="gaussian")
    col = A.col.copy()
    r = int(np.argmax(np.diff(A.row_ptr) >= 2))
    e = A.row_ptr[r]
    col[e], col[e + 1] = col[e + 1], col[e]
    assert _status(h, A, 2, col=col) == native.PHSVDS_ERR_INVALID


def test_invalid_row_ptr(h):
    A = synth.random_sparse(60, 30, 5.0, 2, values="gaussian")
    rp = A.row_ptr.copy()
    rp[10] = rp[11] + 5          # decreasing offsets
    assert _status(h, A, 2, rp=rp) == native.PHSVDS_ERR_INVALID


def test_nan_in_values(h):
    A = synth.random_sparse(60, 30, 5.0, 2, values="gaussian")
    val = A.val.copy()
    val[7] = np.nan
    assert _status(h, A, 2, val=val) == native.PHSVDS_ERR_NAN


def test_not_converged_reports_status(h):
    A = synth.givens_diag(sigma=synth.cluster_spectrum_c1())
    o = native.default_opts(max_basis=30, min_restart=18, max_restarts=2)
    *_, status = native.phsvds_solve(h, A.m, A.n, A.row_ptr, A.col, A.val, 3, opts=o, raise_on_error=False)
    assert status == native.PHSVDS_ERR_NOT_CONVERGED


def test_basis_too_small_for_the_block(h):
    """A restart must leave room for a whole block: min_restart + b <=
    max_basis, else INVALID before anything runs."""
    A = synth.random_sparse(60, 30, 5.0, 2, values="gaussian")
    assert _status(h, A, 4, block_size=4, max_basis=14, min_restart=11) == native.PHSVDS_ERR_INVALID
    assert _status(h, A, 4, block_size=4, max_basis=14, min_restart=10) == native.PHSVDS_OK


def test_k_out_of_range(h):
    A = synth.random_sparse(60, 30, 5.0, 2, values="gaussian")
    assert _status(h, A, 8) == native.PHSVDS_ERR_INVALID      # k >= min_restart
    assert _status(h, A, 0) == native.PHSVDS_ERR_INVALID
    assert _status(h, A, 2, block_size=9) == native.PHSVDS_ERR_INVALID
