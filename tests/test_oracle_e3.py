"""The two-stage demonstration of Sec. 5.1 (A = diag([1:10, 1000:100:1e6]),
preconditioner M = A + diag(1e4 * rand)) in the oracle, with the user-given
preconditioner forms of Sec. 4: M^-1 M^-T for C and [0 M^-1; M^-T 0] for B."""
import numpy as np

from oracle import phsvds_ref as R
from paper_1408_5535_gb300 import synth

EPS64 = 2.0 ** -52


def test_e3_workload():
    A, M = synth.e3_diag()
    s = np.sort(A.val)
    assert A.m == A.n == 10001
    assert np.array_equal(s[:10], np.arange(1.0, 11.0)) and s[10] == 1000.0 and s[-1] == 1e6
    d = M - A.val
    assert np.all(d >= 0) and np.all(d < 1e4) and d.std() > 2e3


def test_given_b_preconditioner_is_the_inverse_for_m_equal_a():
    """With M = A (square, diagonal) the stage-2 operator is exactly B^-1."""
    sig = np.array([1.0, 3.0, 7.0, 20.0])
    n = sig.size
    B = np.block([[np.zeros((n, n)), np.diag(sig)], [np.diag(sig), np.zeros((n, n))]])
    P = np.column_stack([R.given_b_precond(sig, n, e) for e in np.eye(2 * n)])
    assert np.allclose(P @ B, np.eye(2 * n), rtol=0, atol=1e-15)


def test_two_stages_reach_full_accuracy_where_stage_one_stalls():
    """Stage 1 alone stalls near its attainable eps ||A|| / sigma relative
    residual (Sec. 3.1; here about 2e-10 ||A||); the two-stage method finds
    sigma_min = 1 with residual <= 1e-14 ||A||."""
    A, M = synth.e3_diag()
    one = R.phsvds(A, 1, largest=False, delta=1e-14, o=R.Opts(precond="given", precond_M=M, stage2=False))
    two = R.phsvds(A, 1, largest=False, delta=1e-14, o=R.Opts(precond="given", precond_M=M))
    limit = EPS64 * two.normA / 1.0
    assert one.resid[0] / one.normA > 1e-14
    assert 0.1 * limit < one.resid[0] / one.normA < 10 * limit
    assert two.stats["switched"] and two.stats["iters2"] >= 1
    assert abs(two.sigma[0] - 1.0) <= 1e-10
    assert two.resid[0] <= 1e-14 * two.normA
