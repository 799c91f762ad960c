"""Seeded input generators: reproducibility and exactly known spectra."""
import math

import numpy as np

from paper_1408_5535_gb300 import synth


def test_splitmix64_published_vectors():
    # Vigna's splitmix64 from state 0: first output 0xE220A8397B1DCDAF.
    assert int(synth.splitmix64(0, 0, 1)[0]) == 0xE220A8397B1DCDAF
    # Java SplittableRandom(1234567).nextLong() sequence (same mixing function).
    got = [int(x) for x in synth.splitmix64(1234567, 0, 3)]
    assert got == [6457827717110365317, 3203168211198807973, 9817491932198370423]


def test_distributions_sane():
    u = synth.uniform(3, 7, 200000)
    assert 0.0 <= u.min() and u.max() < 1.0 and abs(u.mean() - 0.5) < 5e-3
    z = synth.normal(3, 8, 200000)
    assert abs(z.mean()) < 1e-2 and abs(z.std() - 1.0) < 1e-2
    p = synth.poisson(3, 9, 200000, 12.0)
    assert abs(p.mean() - 12.0) < 0.05 and abs(p.var() - 12.0) < 0.3


def test_givens_diag_exact_spectrum():
    sig = synth.cluster_spectrum(200, lo=1e-2, hi=1.0, n_cluster=3, gap=1e-5)
    A = synth.givens_diag(400, 200, sigma=sig, n_rot=80, seed=4)
    sv = np.sort(np.linalg.svd(A.to_dense(), compute_uv=False))
    assert np.max(np.abs(sv - np.sort(sig))) < 1e-14
    assert A.nnz > 200  # the rotations fill in


def test_grid_gradient_closed_form():
    N = 12
    A = synth.grid_gradient(N, 0.0, 2)
    assert A.m == 2 * N * (N + 1) and A.n == N * N
    sv = np.sort(np.linalg.svd(A.to_dense(), compute_uv=False))
    assert np.max(np.abs(sv - A.sigma_exact)) < 1e-13
    # A^T A is the 5-point Dirichlet Laplacian
    d = A.to_dense()
    L = d.T @ d
    assert np.allclose(np.diag(L), 4.0)


def test_grid_gradient_weighted_structure():
    A = synth.grid_gradient(16, 1.0, 2)
    cnt = np.diff(A.row_ptr)
    assert set(np.unique(cnt)) <= {1, 2}
    assert A.nnz == 2 * 16 * 15 * 2 + 4 * 16  # interior edges 2 nnz, boundary edges 1


def test_random_sparse_shape_and_shift():
    A = synth.random_sparse(3000, 1000, 12.0, 3)
    assert A.m == 3000 and A.n == 1000
    assert abs(A.nnz / A.m - 12.0) < 0.6
    d = A.to_dense()
    assert np.linalg.matrix_rank(d) == 1000
    B = synth.random_sparse(3000, 1000, 12.0, 3, shift=0.0)
    diff = d - B.to_dense()
    assert np.allclose(np.diag(diff[:1000]), 1e-3) and abs(diff).sum() - 1.0 < 1e-9
    # reproducible
    C = synth.random_sparse(3000, 1000, 12.0, 3)
    assert np.array_equal(C.val, A.val) and np.array_equal(C.col, A.col)


def test_batched_set_ranges():
    mats = synth.batched_set(count=6, seed=5, n_lo=200, n_hi=600)
    for A in mats:
        assert 200 <= A.n <= 600 and 1.2 * A.n - 1 <= A.m <= 2 * A.n
