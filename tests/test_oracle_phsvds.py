"""Pins of the PHSVDS oracle against the plain definition of singular triplets.

* tiny inputs: the hand-written dense Jacobi SVD gives the exact triplets;
* exactly known spectra: the Givens-conjugated diagonal (orthogonal factors)
  and the unweighted Dirichlet grid gradient (closed form);
* invariants: ||A v - s u||, ||A^T u - s v|| recomputed independently,
  orthonormal U and V, eigenvalues +-s of B (Section 1), and the residual
  relations ||r_u|| = ||r_C|| / s = sqrt(2) ||r_B|| of Section 3.1;
* planted mistakes: a sign error in B, a transposed product in C and a
  dropped shift in the refined QR each make a pin fail.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from paper_1408_5535_gb300 import synth
from oracle import phsvds_ref as R
from oracle.dense_jacobi import dense_triplets

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


def _check(A, res, k, largest, sig_ex=None, normA=None, rel=1e-10):
    d = A.to_dense()
    if sig_ex is None:
        sig_ex, Uex, Vex = dense_triplets(d, k, largest)
    else:
        sig_ex = np.asarray(sig_ex)
    normA = np.linalg.norm(d, 2) if normA is None else normA
    assert res.sigma.shape == (k,)
    # same index set and relative accuracy
    assert np.max(np.abs(res.sigma - sig_ex) / sig_ex) < rel
    # residual criterion of Section 5, recomputed here from A directly
    rv = np.linalg.norm(d @ res.V - res.U * res.sigma, axis=0)
    ru = np.linalg.norm(d.T @ res.U - res.V * res.sigma, axis=0)
    assert np.all(np.sqrt(ru ** 2 + rv ** 2) <= DELTA * normA)
    _orth_ok(res.V, res.sigma, normA)
    _orth_ok(res.U, res.sigma, normA)
    return sig_ex


@pytest.mark.parametrize("largest", [False, True])
@pytest.mark.parametrize("b", [1, 3])
def test_tiny_random_vs_dense_jacobi(largest, b):
    A = synth.random_sparse(80, 40, 5.0, 11, values="gaussian", shift=0.05)
    o = R.Opts(block=b, max_basis=14, min_restart=8)
    res = R.phsvds(A, 4, largest=largest, delta=DELTA, o=o)
    _check(A, res, 4, largest)


def test_square_tiny_vs_dense_jacobi():
    A = synth.random_sparse(50, 50, 6.0, 12, values="gaussian", shift=0.5)
    res = R.phsvds(A, 3, delta=DELTA, o=R.Opts(block=2, max_basis=12, min_restart=6))
    _check(A, res, 3, False)


def test_vectors_match_dense_jacobi_up_to_sign():
    A = synth.random_sparse(60, 30, 5.0, 13, values="gaussian", shift=0.05)
    res = R.phsvds(A, 3, delta=DELTA, o=R.Opts(block=1, max_basis=12, min_restart=6))
    s, U, V = dense_triplets(A.to_dense(), 3)
    gaps = np.diff(np.linalg.svd(A.to_dense(), compute_uv=False)[::-1])[:3]
    assert np.all(gaps > 1e-3)
    assert np.all(np.abs(np.abs(np.sum(res.V * V, axis=0)) - 1) < 1e-10)
    assert np.all(np.abs(np.abs(np.sum(res.U * U, axis=0)) - 1) < 1e-10)


def test_grid_gradient_closed_form_multiplicity():
    N = 20
    A = synth.grid_gradient(N, 0.0, 2)
    k = 6
    res = R.phsvds(A, k, delta=DELTA, o=R.Opts(block=2))
    ex = A.sigma_exact[:k]
    normA = A.sigma_exact[-1]
    _check(A, res, k, False, sig_ex=ex, normA=normA)
    # sigma_2 = sigma_3 is a double value: compare the spanned subspace
    P = np.linalg.svd(res.V[:, 1:3].T @ np.linalg.svd(A.to_dense())[2][::-1][1:3].T, compute_uv=False)
    assert np.min(P) > 1 - 1e-10


@pytest.mark.slow
def test_givens_cluster_exact_spectrum():
    """The exact-spectrum stress case: a cluster 1e-4 + {0,1,2}e-7 needs stage 2."""
    sig = synth.cluster_spectrum_c1()
    A = synth.givens_diag(sigma=sig)
    res = R.phsvds(A, 3, delta=DELTA, o=R.Opts(block=1, max_basis=30, min_restart=18))
    assert res.stats["switched"]
    _check(A, res, 3, False, sig_ex=np.sort(sig)[:3], normA=1.0)


def test_largest_stage1_only_and_bauer_fike():
    """For the largest triplets delta_C = delta, so stage 1 suffices (Sec. 3.1) and
    |s - s~| <= delta ||A|| / 2 (Bauer-Fike)."""
    A = synth.grid_gradient(12, 1.0, 2)
    res = R.phsvds(A, 3, largest=True, delta=DELTA, o=R.Opts(block=1))
    assert not res.stats["switched"]
    sv = np.sort(np.linalg.svd(A.to_dense(), compute_uv=False))[::-1][:3]
    nA = sv[0]
    assert np.all(np.abs(res.sigma - sv) <= DELTA * nA / 2)
    _check(A, res, 3, True)


def test_residual_relations_section_3_1():
    """||r_u|| = ||r_C|| / s = sqrt(2) ||r_B|| for u = A v / s, ||v|| = 1 (r_v = 0)."""
    A = synth.random_sparse(70, 30, 5.0, 14, values="gaussian", shift=0.1)
    As = R.as_scipy(A)
    rng = np.random.default_rng(0)
    _, _, Vt = np.linalg.svd(A.to_dense())
    v = Vt[-1] + 1e-4 * rng.standard_normal(30)
    v /= np.linalg.norm(v)
    lam = v @ (As.T @ (As @ v))
    s = math.sqrt(lam)
    u = As @ v / s
    rC = As.T @ (As @ v) - lam * v
    ru = As.T @ u - s * v
    rv = As @ v - s * u
    x = np.concatenate([v, u])
    Bx = np.concatenate([As.T @ u, As @ v])
    rB = (Bx - s * x) / np.linalg.norm(x)
    assert np.linalg.norm(rv) < 1e-14
    assert abs(np.linalg.norm(ru) - np.linalg.norm(rC) / s) < 1e-12 * np.linalg.norm(ru)
    assert abs(np.linalg.norm(ru) - math.sqrt(2) * np.linalg.norm(rB)) < 1e-12 * np.linalg.norm(ru)


def test_augmented_operator_spectrum():
    """B = [0 A^T; A 0] has eigenvalues +-sigma_i and m - n zeros (Section 1)."""
    A = synth.random_sparse(9, 5, 3.0, 15, values="gaussian", shift=0.3)
    ops = R.Ops(R.as_scipy(A))
    Bd = ops.B(np.eye(14))
    ev = np.sort(np.linalg.eigvalsh(0.5 * (Bd + Bd.T)))
    sv = np.linalg.svd(A.to_dense(), compute_uv=False)
    ex = np.sort(np.concatenate([sv, -sv, np.zeros(4)]))
    assert np.max(np.abs(ev - ex)) < 1e-13


def test_splitmix_method_stream_matches_published():
    z = R._splitmix(1234567, 0, 2)
    assert [int(x) for x in z] == [6457827717110365317, 3203168211198807973]


# ---------------------------------------------------------------------------
# planted mistakes: each must make a pin fail
# ---------------------------------------------------------------------------

def _tiny_case():
    return synth.random_sparse(60, 30, 5.0, 16, values="gaussian", shift=0.05)


def _stage2_case():
    """Small exact-spectrum case whose smallest pair needs stage 2."""
    sig = np.sort(np.concatenate([[1e-3, 1e-3 + 1e-6, 2e-3], np.logspace(-1, 0, 117)]))
    return synth.givens_diag(200, 120, sigma=sig, n_rot=60, seed=3)


def test_stage2_case_is_sane():
    A = _stage2_case()
    res = R.phsvds(A, 2, delta=DELTA, o=R.Opts(block=1, max_basis=20, min_restart=10, max_restarts=300))
    assert res.stats["switched"]
    _check(A, res, 2, False, sig_ex=np.sort(A.sigma_exact)[:2], normA=1.0)


def test_planted_sign_error_in_B_is_caught(monkeypatch):
    def bad_B(self, X):
        X = X.reshape(self.m + self.n, -1)
        n = self.n
        return np.vstack([self.At @ X[n:], -(self.A @ X[:n])])   # wrong sign
    monkeypatch.setattr(R.Ops, "B", bad_B)
    A = _stage2_case()
    with pytest.raises((AssertionError, RuntimeError, ValueError, np.linalg.LinAlgError)):
        res = R.phsvds(A, 2, delta=DELTA, o=R.Opts(block=1, max_basis=20, min_restart=10, max_restarts=300))
        _check(A, res, 2, False, sig_ex=np.sort(A.sigma_exact)[:2], normA=1.0)


def test_planted_error_in_C_is_caught(monkeypatch):
    """Stage 1 alone (largest triplets, stage 2 off) must expose a wrong C product."""
    def bad_C(self, X):
        X = X.reshape(self.n, -1)
        return self.At @ (self.A @ X) + 1e-3 * X[::-1]          # a stray extra term
    monkeypatch.setattr(R.Ops, "C", bad_C)
    A = _tiny_case()
    with pytest.raises((AssertionError, RuntimeError)):
        res = R.phsvds(A, 2, largest=True, delta=DELTA,
                       o=R.Opts(block=1, max_basis=12, min_restart=6, max_restarts=200, stage2=False))
        _check(A, res, 2, True)


def test_planted_dropped_shift_in_refined_qr_is_caught(monkeypatch):
    orig = R.qr_cgs2

    def bad_qr(Z, seed, counter):
        return orig(Z + 0.37 * np.ones_like(Z) / math.sqrt(Z.shape[0]), seed, counter)
    monkeypatch.setattr(R, "qr_cgs2", bad_qr)
    A = _stage2_case()
    with pytest.raises((AssertionError, RuntimeError)):
        res = R.phsvds(A, 2, delta=DELTA, o=R.Opts(block=1, max_basis=20, min_restart=10, max_restarts=300))
        _check(A, res, 2, False, sig_ex=np.sort(A.sigma_exact)[:2], normA=1.0)
