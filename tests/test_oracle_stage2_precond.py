"""Pins of the oracle's stage-2 preconditioner (Sec. 4: from a preconditioner
M ~ C^{-1} of the first stage, [0 A M; M A^T 0] for the augmented matrix):
its block structure against a dense build, the generalised-inverse identity
B P B = B when M = C^{-1} exactly, and a whole solve with the Jacobi M."""
import numpy as np
import scipy.sparse as sp

from oracle import phsvds_ref as R
from paper_1408_5535_gb300 import synth


def _small(m=30, n=12, seed=4):
    A = synth.random_sparse(m, n, 5.0, seed, values="gaussian", shift=0.1)
    return R.as_scipy(A)


def test_block_structure_against_a_dense_build():
    S = _small()
    m, n = S.shape
    ops = R.Ops(S)
    Md = np.diag(1.0 / (1.0 + np.arange(n)))
    Ad = S.toarray()
    P = np.block([[np.zeros((n, n)), Md @ Ad.T], [Ad @ Md, np.zeros((m, m))]])   # [v; u] order
    y = np.random.default_rng(1).standard_normal(m + n)
    got = R.b_precond(ops, lambda z: Md @ z, y)
    assert np.allclose(got, P @ y, rtol=1e-13, atol=1e-13)
    assert np.allclose(P, P.T)          # symmetric, like B


def test_exact_inverse_of_c_gives_a_generalised_inverse_of_b():
    """With M = C^{-1} and A of full column rank, P B = diag(I, A C^{-1} A^T),
    so B P B = B (B P is the orthogonal projector onto range(B))."""
    S = _small()
    m, n = S.shape
    ops = R.Ops(S)
    Ad = S.toarray()
    Cinv = np.linalg.inv(Ad.T @ Ad)
    Bd = np.block([[np.zeros((n, n)), Ad.T], [Ad, np.zeros((m, m))]])
    cols = [R.b_precond(ops, lambda z: Cinv @ z, Bd[:, c]) for c in range(m + n)]
    PB = np.column_stack(cols)
    assert np.allclose(Bd @ PB, Bd, atol=1e-10 * np.linalg.norm(Bd, 2))
    assert np.allclose(PB[:n, :n], np.eye(n), atol=1e-10)


def test_jacobi_stage2_preconditioner_same_triplets_fewer_iterations():
    """Columns scaled over two decades: the Jacobi-built stage-2
    preconditioner reaches the same smallest triplets (1e-14 ||A||) in fewer
    stage-2 iterations than plain GD."""
    A0 = synth.random_sparse(300, 150, 6.0, 21, values="gaussian", shift=0.05)
    S = R.as_scipy(A0)
    S = (S @ sp.diags(10.0 ** (-2.0 * np.random.default_rng(3).random(150)))).tocsr()
    Csr = synth.Csr(S.shape[0], S.shape[1], S.indptr.astype(np.int64), S.indices.astype(np.int32), S.data)
    o0 = R.Opts(block=2, precond="jacobi")
    o1 = R.Opts(block=2, precond="jacobi", stage2_precond=True)
    plain = R.phsvds(Csr, 4, largest=False, delta=1e-14, o=o0)
    pre = R.phsvds(Csr, 4, largest=False, delta=1e-14, o=o1)
    assert np.max(np.abs(pre.sigma - plain.sigma) / plain.sigma) <= 1e-10
    assert np.all(pre.resid <= 1e-14 * pre.normA)
    assert pre.stats["iters2"] < plain.stats["iters2"]
    sv = np.linalg.svd(S.toarray(), compute_uv=False)
    assert np.max(np.abs(pre.sigma - np.sort(sv)[:4]) / np.sort(sv)[:4]) <= 1e-10
