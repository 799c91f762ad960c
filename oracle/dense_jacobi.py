"""Hand-written dense Jacobi methods (FP64, plain loops) -- oracle code.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this module;
only the tests, the smoke check and the CPU-baseline leg of the benchmark do.

* ``jacobi_eig``  -- cyclic two-sided Jacobi for a symmetric matrix
                     (Golub & Van Loan, Matrix Computations, Sec. 8.5).
* ``jacobi_svd``  -- one-sided (Hestenes) Jacobi SVD of a dense m x n matrix,
                     m >= n.  It is the plain definition of the singular
                     triplets (Section 1, eq. 1.1: A = U Sigma V^T) used to pin
                     the PHSVDS oracle on tiny inputs.
"""
from __future__ import annotations

import math

import numpy as np


def jacobi_eig(H: np.ndarray, tol: float = 1e-15, max_sweeps: int = 60):
    """Eigen-decomposition H = S diag(theta) S^T by cyclic Jacobi rotations.

    Returns (theta ascending, S with orthonormal columns).
    """
    A = np.array(H, dtype=np.float64, copy=True)
    n = A.shape[0]
    S = np.eye(n)
    for _ in range(max_sweeps):
        off = math.sqrt(float(np.sum((A - np.diag(np.diag(A))) ** 2)))
        if off <= tol * max(np.linalg.norm(A), 1e-300):
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                apq = A[p, q]
                if apq == 0.0:
                    continue
                app, aqq = A[p, p], A[q, q]
                tau = (aqq - app) / (2.0 * apq)
                t = (1.0 if tau >= 0 else -1.0) / (abs(tau) + math.sqrt(1.0 + tau * tau))
                c = 1.0 / math.sqrt(1.0 + t * t)
                s = t * c
                # A <- J^T A J with J the rotation in the (p, q) plane
                ap = A[:, p].copy()
                aq = A[:, q].copy()
                A[:, p] = c * ap - s * aq
                A[:, q] = s * ap + c * aq
                ap = A[p, :].copy()
                aq = A[q, :].copy()
                A[p, :] = c * ap - s * aq
                A[q, :] = s * ap + c * aq
                sp_ = S[:, p].copy()
                sq_ = S[:, q].copy()
                S[:, p] = c * sp_ - s * sq_
                S[:, q] = s * sp_ + c * sq_
    theta = np.diag(A).copy()
    order = np.argsort(theta, kind="stable")
    return theta[order], S[:, order]


def jacobi_svd(A: np.ndarray, tol: float = 1e-15, max_sweeps: int = 80):
    """One-sided Jacobi SVD: A (m x n, m >= n) = U diag(sigma) V^T.

    Columns of a working copy G = A V are rotated pairwise until every pair is
    numerically orthogonal; then sigma_j = ||G e_j||, U e_j = G e_j / sigma_j.
    Returns (sigma ascending, U (m x n), V (n x n)).
    """
    G = np.array(A, dtype=np.float64, copy=True)
    m, n = G.shape
    assert m >= n
    V = np.eye(n)
    for _ in range(max_sweeps):
        rotated = False
        for p in range(n - 1):
            for q in range(p + 1, n):
                alpha = float(G[:, p] @ G[:, p])
                beta = float(G[:, q] @ G[:, q])
                gamma = float(G[:, p] @ G[:, q])
                if abs(gamma) <= tol * math.sqrt(alpha * beta) or gamma == 0.0:
                    continue
                rotated = True
                zeta = (beta - alpha) / (2.0 * gamma)
                t = (1.0 if zeta >= 0 else -1.0) / (abs(zeta) + math.sqrt(1.0 + zeta * zeta))
                c = 1.0 / math.sqrt(1.0 + t * t)
                s = c * t
                gp = G[:, p].copy()
                gq = G[:, q].copy()
                G[:, p] = c * gp - s * gq
                G[:, q] = s * gp + c * gq
                vp = V[:, p].copy()
                vq = V[:, q].copy()
                V[:, p] = c * vp - s * vq
                V[:, q] = s * vp + c * vq
        if not rotated:
            break
    sigma = np.sqrt(np.sum(G * G, axis=0))
    U = np.zeros_like(G)
    for j in range(n):
        if sigma[j] > 0:
            U[:, j] = G[:, j] / sigma[j]
    order = np.argsort(sigma, kind="stable")
    return sigma[order], U[:, order], V[:, order]


def dense_triplets(A: np.ndarray, k: int, largest: bool = False):
    """The k smallest (or largest) singular triplets of a dense A by ``jacobi_svd``.

    Returns (sigma, U (m x k), V (n x k)), sigma ascending for smallest and
    descending for largest (Section 1: sigma_1 <= ... <= sigma_n).
    """
    sigma, U, V = jacobi_svd(A)
    idx = np.arange(k) if not largest else np.arange(sigma.size - 1, sigma.size - 1 - k, -1)
    return sigma[idx], U[:, idx], V[:, idx]
