"""Pins of the hand-written dense Jacobi eigensolver / SVD of the oracle.

They are checked against what mathematics fixes (orthogonality, reconstruction
to a few n*eps, closed-form spectra) and against LAPACK as an independent
library routine.
"""
import numpy as np
import pytest

from oracle.dense_jacobi import jacobi_eig, jacobi_svd, dense_triplets

EPS = 2.0 ** -52


@pytest.mark.parametrize("n", [1, 2, 3, 7, 16])
def test_jacobi_eig_random(n):
    rng = np.random.default_rng(n)
    M = rng.standard_normal((n, n))
    H = M + M.T
    th, S = jacobi_eig(H)
    nrm = np.linalg.norm(H, 2)
    assert np.max(np.abs(S.T @ S - np.eye(n))) < 20 * n * EPS
    assert np.linalg.norm(H @ S - S * th) < 20 * n * EPS * nrm
    assert np.all(np.diff(th) >= 0)
    assert np.max(np.abs(th - np.linalg.eigvalsh(H))) < 20 * n * EPS * nrm


def test_jacobi_eig_closed_form_tridiagonal():
    # eigenvalues of tridiag(-1, 2, -1) are 2 - 2 cos(k pi / (n+1))
    n = 9
    H = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    th, _ = jacobi_eig(H)
    ex = 2 - 2 * np.cos(np.arange(1, n + 1) * np.pi / (n + 1))
    assert np.max(np.abs(th - np.sort(ex))) < 1e-14


@pytest.mark.parametrize("m,n", [(1, 1), (5, 3), (12, 12), (30, 9)])
def test_jacobi_svd_random(m, n):
    rng = np.random.default_rng(m * 100 + n)
    A = rng.standard_normal((m, n))
    s, U, V = jacobi_svd(A)
    nrm = np.linalg.norm(A, 2)
    assert np.linalg.norm(A - U @ np.diag(s) @ V.T) < 10 * n * EPS * nrm
    assert np.max(np.abs(U.T @ U - np.eye(n))) < 10 * n * EPS * nrm / s.min()
    assert np.max(np.abs(V.T @ V - np.eye(n))) < 10 * n * EPS
    assert np.max(np.abs(s - np.sort(np.linalg.svd(A, compute_uv=False)))) < 10 * n * EPS * nrm


def test_jacobi_svd_diagonal_and_graded():
    d = np.array([3.0, -1e-6, 2.0, 1e-12, -5.0])
    s, U, V = jacobi_svd(np.vstack([np.diag(d), np.zeros((2, 5))]))
    assert np.allclose(s, np.sort(np.abs(d)), rtol=1e-15, atol=0)


def test_dense_triplets_order_and_definition():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((10, 6))
    s, U, V = dense_triplets(A, 3)
    assert np.all(np.diff(s) > 0)
    assert np.allclose(A @ V, U * s, atol=1e-13)
    sl, Ul, Vl = dense_triplets(A, 2, largest=True)
    assert sl[0] >= sl[1] and abs(sl[0] - np.linalg.norm(A, 2)) < 1e-13
