"""Pins of the oracle's JDQMR form of stage 2 (CPU only): the symmetric QMR
inner solver against brute force over its Krylov space and against the exact
solve, the Jacobi-Davidson correction against the Rayleigh-quotient-iteration
bound, and whole solves against the dense SVD and the grid closed form."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import dense_jacobi as D
from oracle import phsvds_ref as R
from paper_1408_5535_gb300 import synth


def _sym_indefinite(n, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.concatenate([-np.linspace(0.5, 2.0, n // 2), np.linspace(0.3, 3.0, n - n // 2)])
    return (Q * lam) @ Q.T, rng.standard_normal(n)


def _iterates(M, b, Qd, steps):
    def apply_M(q):
        w = M @ q
        if Qd.shape[1]:
            w = w - Qd @ (Qd.T @ w)
        return w, None
    return [(t, g) for t, g, _, _ in R.symmetric_qmr(apply_M, b, Qd, steps)]


def test_qmr_iterates_minimise_the_residual_over_the_krylov_space():
    """Iterate k is argmin ||b - M t|| over K_k(M, b), checked by brute force
    on an explicitly built (QR-orthonormalised) Krylov basis; the residual
    norms never increase."""
    M, b = _sym_indefinite(12, 1)
    its = _iterates(M, b, np.zeros((12, 0)), 8)
    K = [b]
    for k, (t, g) in enumerate(its, start=1):
        Kb = np.linalg.qr(np.column_stack(K))[0]
        c = np.linalg.lstsq(M @ Kb, b, rcond=None)[0]
        t_bf = Kb @ c
        assert np.linalg.norm(t - t_bf) <= 1e-9 * np.linalg.norm(t_bf)
        assert g == pytest.approx(np.linalg.norm(b - M @ t), rel=1e-9, abs=1e-12)
        K.append(M @ K[-1])
    gs = [g for _, g in its]
    assert all(g2 <= g1 * (1 + 1e-12) for g1, g2 in zip(gs, gs[1:]))


def test_qmr_full_dimension_is_the_exact_solve():
    M, b = _sym_indefinite(10, 2)
    t, g = _iterates(M, b, np.zeros((10, 0)), 10)[-1]
    assert np.allclose(t, np.linalg.solve(M, b), rtol=1e-9, atol=1e-10)
    assert g < 1e-9 * np.linalg.norm(b)


def test_qmr_with_deflation_stays_in_the_complement():
    """With deflation columns Qd the iterates stay orthogonal to Qd and solve
    the projected system on the complement."""
    n = 14
    M, b = _sym_indefinite(n, 3)
    rng = np.random.default_rng(4)
    Qd = np.linalg.qr(rng.standard_normal((n, 3)))[0]
    P = np.eye(n) - Qd @ Qd.T
    bp = P @ b
    t, g = _iterates(P @ M @ P, bp, Qd, n - 3)[-1]
    assert np.linalg.norm(Qd.T @ t) <= 1e-12 * np.linalg.norm(t)
    Z = np.linalg.qr(P @ rng.standard_normal((n, n - 3)))[0]       # basis of the complement
    t_ref = Z @ np.linalg.solve(Z.T @ M @ Z, Z.T @ bp)
    assert np.allclose(t, t_ref, rtol=1e-8, atol=1e-10)


def _jd_setup(n=40, seed=5, pert=1e-5):
    """A small A, its B, an eigenvector of B perturbed by pert, with the
    quantities jd_correction takes."""
    rng = np.random.default_rng(seed)
    m = n + 10
    A = sp.csr_matrix(rng.standard_normal((m, n)))
    ops = R.Ops(A)
    Bd = np.block([[np.zeros((n, n)), A.T.toarray()], [A.toarray(), np.zeros((m, m))]])
    lam, X = np.linalg.eigh(Bd)
    i = int(np.argmin(np.abs(lam - 0.5 * np.max(lam))))        # an interior eigenvalue
    x = X[:, i] + pert * rng.standard_normal(m + n)
    x /= np.linalg.norm(x)
    Bx = Bd @ x
    mu = float(x @ Bx)
    r = Bx - mu * x
    return ops, Bd, x, Bx, mu, r


def _eta(Bd, z):
    z = z / np.linalg.norm(z)
    Bz = Bd @ z
    return float(np.linalg.norm(Bz - (z @ Bz) * z))


def test_jd_correction_is_orthogonal_and_acts_like_rqi():
    """The correction is orthogonal to x (and the locked vectors); solved far
    enough (no dynamic stop) it is a Rayleigh-quotient-iteration step, whose
    eigen-residual is of the order of the old one cubed over the gap squared:
    one step from a 1e-5 perturbation lands far below 1e-6 of the old
    residual."""
    ops, Bd, x, Bx, mu, r = _jd_setup()
    st = {}
    t = R.jd_correction(ops, np.zeros((x.size, 0)), x, Bx, mu, r, 0.0, 90, st, patience=90)
    assert abs(x @ t) <= 1e-12 * np.linalg.norm(t)
    eta0, eta1 = _eta(Bd, x), _eta(Bd, x + t)
    assert eta1 <= 1e-6 * eta0
    assert st["inner2"] >= 1


def test_planted_plain_residual_instead_of_the_correction_is_caught(monkeypatch):
    """Planting the GD expansion (t = r, no inner solve) in place of the
    symmetric QMR makes the RQI pin fail."""
    def no_solve(apply_M, b, Qd, steps):
        yield -b, float(np.linalg.norm(b)), [apply_M(b / np.linalg.norm(b))[1]], np.array([-np.linalg.norm(b)])
    monkeypatch.setattr(R, "symmetric_qmr", no_solve)
    ops, Bd, x, Bx, mu, r = _jd_setup()
    t = R.jd_correction(ops, np.zeros((x.size, 0)), x, Bx, mu, r, 0.0, 90, {}, patience=90)
    assert not _eta(Bd, x + t) <= 1e-6 * _eta(Bd, x)


@pytest.mark.parametrize("largest", [False, True])
def test_jdqmr_stage2_tiny_random_vs_dense_svd(largest):
    A = synth.random_sparse(80, 40, 5.0, 11, values="gaussian", shift=0.05)
    k = 4
    res = R.phsvds(A, k, largest=largest, delta=1e-14,
                   o=R.Opts(max_basis=14, min_restart=8, stage2_inner="qmr"))
    s = D.jacobi_svd(A.to_dense())[0]
    ref = np.sort(s)[::-1][:k] if largest else np.sort(s)[:k]
    assert np.max(np.abs(res.sigma - ref) / ref) <= 1e-10
    assert np.all(res.resid <= 1e-14 * res.normA)


def test_jdqmr_stage2_grid_closed_form():
    """16 x 16 Dirichlet gradient, 10 smallest: the closed-form values."""
    A = synth.grid_gradient(16, 0.0, 2)
    k = 10
    jd = R.phsvds(A, k, largest=False, delta=1e-14, o=R.Opts(block=4, stage2_inner="qmr"))
    exact = np.sort(synth.grid_gradient_sigma(16))[:k]
    assert np.max(np.abs(jd.sigma - exact) / exact) <= 1e-10
    assert np.all(jd.resid <= 1e-14 * jd.normA)


def test_jdqmr_stage2_needs_fewer_outer_iterations_than_gd():
    """Weighted 16 x 16 grid (log-normal weights), 10 smallest: the same
    values as with GD in stage 2, in fewer stage-2 outer iterations (the
    paper's reason to prefer an inner-outer method there, Sec. 4)."""
    A = synth.grid_gradient(16, 1.0, 2)
    k = 10
    gd = R.phsvds(A, k, largest=False, delta=1e-14, o=R.Opts(block=4))
    jd = R.phsvds(A, k, largest=False, delta=1e-14, o=R.Opts(block=4, stage2_inner="qmr"))
    assert np.max(np.abs(jd.sigma - gd.sigma) / gd.sigma) <= 1e-10
    assert np.all(jd.resid <= 1e-14 * jd.normA)
    assert jd.stats["iters2"] < gd.stats["iters2"]
