"""Pins of the oracle's Jacobi-Davidson form of stage 1 and of its Lanczos
estimate of ||A|| (oracle/phsvds_ref.py: jd1_correction, lanczos_norm_c).

* With as many steps as the complement has dimensions and a tiny tolerance,
  the correction solves its equation exactly: (I - QQ^T)(C - theta I)(I -
  QQ^T) t = r, unscaled and Jacobi-scaled; a scaled operator that drops the
  projection of its input (a planted mistake) does not.
* Whole solves with the correction reach the dense SVD's (and the recorded
  oracle's) smallest values in fewer outer iterations than GD+k.
* The Lanczos estimate is a lower bound of ||A||^2 within 1e-10 of it.
"""
import json
import os

import numpy as np
import scipy.sparse as sp

from paper_1408_5535_gb300 import synth
from oracle import phsvds_ref as R

GOLD = os.path.join(os.path.dirname(__file__), "golden", "oracle_counts.json")


def _small_problem(seed=7, m=90, n=40):
    A0 = synth.random_sparse(m, n, 6.0, seed, values="gaussian", shift=0.05)
    S = R.as_scipy(A0)
    S = (S @ sp.diags(10.0 ** (-1.5 * synth.uniform(seed + 100, 1, n)))).tocsr()
    C = (S.T @ S).toarray()
    w, U = np.linalg.eigh(C)
    # approximate eigenvectors, as Ritz vectors are: not invariant under C
    Q = np.linalg.qr(U[:, :3] + 1e-2 * np.column_stack([R.rand_vec(5, 20 + c, n) for c in range(3)]))[0]
    theta = float(w[0]) * 1.01
    r = R.rand_vec(3, 11, n)
    r = r - Q @ (Q.T @ r)
    return C, Q, theta, r


def _projected_residual(C, Q, theta, r, t):
    P = np.eye(C.shape[0]) - Q @ Q.T
    return float(np.linalg.norm(P @ (C - theta * np.eye(C.shape[0])) @ P @ t - r) / np.linalg.norm(r))


def test_correction_solves_its_equation_unscaled_and_scaled():
    C, Q, theta, r = _small_problem()
    apply_C = lambda X: C @ X
    st = {}
    t = R.jd1_correction(apply_C, Q, theta, r, None, C.shape[0], 1e-14, st)
    assert _projected_residual(C, Q, theta, r, t) < 1e-9
    sc = 1.0 / np.sqrt(np.diag(C))
    ts = R.jd1_correction(apply_C, Q, theta, r, sc, 2 * C.shape[0], 1e-14, st)
    assert _projected_residual(C, Q, theta, r, ts) < 1e-9
    assert st["inner1"] > 0


def test_a_dropped_input_projection_is_caught():
    """The planted mistake: the scaled operator of jd1_correction without the
    projection of its input, run through the same symmetric QMR.  It is not
    symmetric on the scaled space, and its iterate misses the equation by far
    more than the pin's 1e-9."""
    C, Q, theta, r = _small_problem()
    n = C.shape[0]
    sc = 1.0 / np.sqrt(np.diag(C))

    def proj(z):
        for _ in range(2):
            z = z - Q @ (Q.T @ z)
        return z

    def wrong_apply(q):
        return sc * proj(C @ (sc * q) - theta * (sc * q)), None   # no P on the input side

    t = None
    for t, g, _, _ in R.symmetric_qmr(wrong_apply, sc * r, np.zeros((n, 0)), 2 * n):
        if g <= 1e-14 * np.linalg.norm(sc * r):
            break
    assert _projected_residual(C, Q, theta, r, sc * t) > 1e-6


def test_stage1_jacobi_davidson_matches_dense_svd_in_fewer_iterations():
    A0 = synth.random_sparse(300, 150, 6.0, 21, values="gaussian", shift=0.05)
    S = R.as_scipy(A0)
    S = (S @ sp.diags(10.0 ** (-2.0 * synth.uniform(31, 1, 150)))).tocsr()
    S.sort_indices()
    A = synth.Csr(S.shape[0], S.shape[1], S.indptr.astype(np.int64), S.indices.astype(np.int32), S.data)
    sv = np.sort(np.linalg.svd(S.toarray(), compute_uv=False))[:4]
    runs = {}
    for inner in ("none", "minres"):
        runs[inner] = R.phsvds(A, 4, largest=False, delta=1e-14,
                               o=R.Opts(block=2, precond="jacobi", stage1_inner=inner))
    for res in runs.values():
        assert np.all(np.abs(res.sigma - sv) <= 1e-10 * sv)
        assert np.all(res.resid <= 1e-14 * res.normA)
    assert runs["minres"].stats["inner1"] > 0
    assert runs["minres"].stats["iters"] < runs["none"].stats["iters"]


def test_unscaled_jacobi_davidson_on_the_grid_matches_the_recorded_run():
    g = json.load(open(GOLD))["grid16"]
    A = synth.grid_gradient(16, 1.0, 2)
    res = R.phsvds(A, 10, largest=False, delta=1e-14, o=R.Opts(block=4, stage1_inner="minres"))
    ref = np.array(g["sigma"])
    assert np.all(np.abs(res.sigma - ref) <= 1e-10 * ref)
    assert res.stats["iters"] < g["iters_stage1"] / 2


def test_lanczos_norm_estimate_is_a_close_lower_bound():
    A0 = synth.random_sparse(400, 200, 8.0, 5)
    S = R.as_scipy(A0)
    nC = float(np.linalg.norm(S.toarray(), 2)) ** 2
    est = R.lanczos_norm_c(lambda X: S.T @ (S @ X), S.shape[1], 0)
    assert est <= nC * (1 + 1e-12)
    assert est >= nC * (1 - 1e-10)
    res = R.phsvds(A0, 3, largest=False, delta=1e-14, o=R.Opts(block=1, norm_A=-1.0, stage2=False))
    assert abs(res.normA - np.sqrt(nC)) <= 1e-9 * np.sqrt(nC)
