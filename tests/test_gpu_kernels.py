"""GPU kernels against the oracle, element by element (through the C ABI)."""
import numpy as np
import pytest

from paper_1408_5535_gb300 import native, synth
from oracle import phsvds_ref as R
from oracle.dense_jacobi import jacobi_eig, jacobi_svd
from tests.gpu_util import torch, need_gpu, dev, device_csr

pytestmark = pytest.mark.gpu
EPS64, EPS32 = 2.0 ** -52, 2.0 ** -23


@pytest.fixture(scope="module")
def h():
    need_gpu()
    with native.Handle(0) as hh:
        yield hh


def _cases():
    return [synth.givens_diag(400, 200, sigma=synth.cluster_spectrum(200, 1e-3, 1.0, 3, 1e-6), n_rot=80, seed=1),
            synth.random_sparse(3001, 1499, 12.0, 3),          # ragged tails, lognormal, several tiles
            synth.grid_gradient(23, 1.0, 2),                   # 1-2 entries per row
            synth.random_sparse(777, 333, 30.0, 4, values="gaussian", shift=0.0)]   # long rows


@pytest.mark.parametrize("case", range(4))
@pytest.mark.parametrize("b", [1, 2, 4, 8])
@pytest.mark.parametrize("schedule", [1, 2])
@pytest.mark.parametrize("fp32", [False, True])
def test_ata_spmm_vs_oracle(h, case, b, schedule, fp32):
    A = _cases()[case]
    d = device_csr(A, fp32)
    X = (synth.uniform(5, 10 + b, A.n * b) * 2 - 1).reshape(A.n, b)
    ref = R.Ops(d["scipy"]).C(X)                                   # oracle product, FP64
    absA = abs(d["scipy"])
    bound = absA.T @ (absA @ np.abs(X))
    vt = torch.float32 if fp32 else torch.float64
    Xd = dev(X, vt)
    Yd = torch.empty((A.n, b), dtype=vt, device="cuda")
    z = torch.empty((A.m, b), dtype=vt, device="cuda")
    native.phsvds_ata_spmm(h, schedule, A.m, A.n, A.nnz, d["rp"], d["ci"], d["va"], d["cp"], d["ri"], d["cv"], b,
                           Xd, Yd, z, fp32=fp32)
    native.phsvds_sync(h)
    Y = Yd.double().cpu().numpy()
    rowmax = np.diff(A.row_ptr).max() + 2
    eps = EPS32 if fp32 else EPS64
    assert np.all(np.abs(Y - ref) <= 4 * rowmax * eps * bound + 1e-300)


@pytest.mark.parametrize("lanes", [1, 2, 4, 8, 16, -2, -8])
@pytest.mark.parametrize("fp32", [False, True])
@pytest.mark.parametrize("offset", [0, 1])
def test_ata_spmm_lane_widths_and_narrow_gathers(h, lanes, fp32, offset):
    """Every group width, both schedules, and 32-byte rows (b=8 FP32, b=4 FP64)
    gathered wide (X 32-byte aligned) and narrow (X shifted by 16 bytes)."""
    A = synth.random_sparse(3001, 1499, 12.0, 3)
    d = device_csr(A, fp32)
    b = 8 if fp32 else 4
    vt = torch.float32 if fp32 else torch.float64
    X = (synth.uniform(5, 40 + lanes, A.n * b) * 2 - 1).reshape(A.n, b)
    ref = R.Ops(d["scipy"]).C(X)
    absA = abs(d["scipy"])
    bound = 4 * (np.diff(A.row_ptr).max() + 2) * (EPS32 if fp32 else EPS64) * (absA.T @ (absA @ np.abs(X)))
    half = 16 // (4 if fp32 else 8)                    # elements in 16 bytes
    buf = torch.empty(A.n * b + 2 * half, dtype=vt, device="cuda")
    assert buf.data_ptr() % 32 == 0
    Xd = buf[offset * half: offset * half + A.n * b].view(A.n, b)
    Xd.copy_(torch.from_numpy(X).to(vt))
    assert (Xd.data_ptr() % 32 == 0) == (offset == 0)
    for schedule in (1, 2):
        Yd = torch.full((A.n, b), float("nan"), dtype=vt, device="cuda")
        z = torch.empty((A.m, b), dtype=vt, device="cuda")
        native.phsvds_ata_spmm(h, schedule, A.m, A.n, A.nnz, d["rp"], d["ci"], d["va"], d["cp"], d["ri"], d["cv"], b,
                               Xd, Yd, z, fp32=fp32, lanes_a=lanes, lanes_at=lanes)
        native.phsvds_sync(h)
        Y = Yd.double().cpu().numpy()
        assert np.all(np.abs(Y - ref) <= bound + 1e-300), (schedule, lanes)


def test_ata_spmm_rejects_bad_lanes(h):
    A = synth.random_sparse(300, 100, 4.0, 3)
    d = device_csr(A)
    X = torch.zeros((A.n, 2), dtype=torch.float64, device="cuda")
    Y = torch.zeros_like(X)
    with pytest.raises(native.PhsvdsError):
        native.phsvds_ata_spmm(h, 1, A.m, A.n, A.nnz, d["rp"], d["ci"], d["va"], d["cp"], d["ri"], d["cv"], 2, X, Y,
                               lanes_a=3)


def test_csr_to_csc_exact(h):
    A = synth.random_sparse(5003, 2001, 9.0, 6)
    d = device_csr(A)
    cp = torch.empty(A.n + 1, dtype=torch.int32, device="cuda")
    ri = torch.empty(A.nnz, dtype=torch.int32, device="cuda")
    cv = torch.empty(A.nnz, dtype=torch.float64, device="cuda")
    native.phsvds_csr_to_csc(h, A.m, A.n, A.nnz, d["rp"], d["ci"], d["va"], cp, ri, cv)
    native.phsvds_sync(h)
    T = d["scipy"].tocsc()
    T.sort_indices()
    assert np.array_equal(cp.cpu().numpy(), T.indptr)
    assert np.array_equal(ri.cpu().numpy(), T.indices)
    assert np.array_equal(cv.cpu().numpy(), T.data)


@pytest.mark.parametrize("cluster", [False, True])
@pytest.mark.parametrize("j", [1, 2, 7, 20, 35, 64])
def test_jacobi_eig_vs_oracle(h, j, cluster):
    rng = np.random.default_rng(j)
    M = rng.standard_normal((j, j))
    H = M + M.T
    if j > 4:   # a tight cluster and a graded tail
        Q, _ = np.linalg.qr(rng.standard_normal((j, j)))
        ev = np.concatenate([[1e-8, 1e-8 + 1e-14, 2e-8], np.logspace(-6, 1, j - 3)])
        H = Q @ np.diag(ev) @ Q.T
        H = 0.5 * (H + H.T)
    Hd = dev(np.asfortranarray(H).ravel(order="F"))
    Sd = dev(np.eye(j).ravel(order="F"))
    th = torch.empty(j, dtype=torch.float64, device="cuda")
    sw = torch.zeros(1, dtype=torch.int32, device="cuda")
    native.phsvds_jacobi_eig(h, j, Hd, Sd, th, 1e-17, 60, sw, cluster=cluster)
    native.phsvds_sync(h)
    S = Sd.cpu().numpy().reshape(j, j, order="F")
    theta = th.cpu().numpy()
    nrm = np.linalg.norm(H, 2)
    ref, _ = jacobi_eig(H)                    # oracle's hand-written Jacobi
    assert np.max(np.abs(np.sort(theta) - ref)) <= 10 * j * EPS64 * nrm
    assert np.max(np.abs(S.T @ S - np.eye(j))) <= 50 * j * EPS64
    assert np.linalg.norm(H @ S - S * theta) <= 50 * j * EPS64 * nrm
    assert 0 < int(sw.item()) < 60 or j == 1


@pytest.mark.parametrize("j", [1, 3, 21, 35, 64])
def test_jacobi_svd_vs_oracle(h, j):
    rng = np.random.default_rng(100 + j)
    G = np.triu(rng.standard_normal((j, j)))
    if j > 3:
        G[:, -1] *= 1e-12   # one tiny singular value, as in the refined projection
    Gd = dev(G.ravel(order="F"))
    Sd = dev(np.eye(j).ravel(order="F"))
    sig = torch.empty(j, dtype=torch.float64, device="cuda")
    native.phsvds_jacobi_svd(h, j, Gd, Sd, sig, 1e-15, 60)
    native.phsvds_sync(h)
    S = Sd.cpu().numpy().reshape(j, j, order="F")
    Go = Gd.cpu().numpy().reshape(j, j, order="F")
    s = sig.cpu().numpy()
    ref, _, _ = jacobi_svd(G)
    nrm = np.linalg.norm(G, 2)
    assert np.max(np.abs(np.sort(s) - ref)) <= 50 * j * EPS64 * nrm
    assert np.max(np.abs(S.T @ S - np.eye(j))) <= 50 * j * EPS64
    assert np.linalg.norm(G @ S - Go) <= 50 * j * EPS64 * nrm
    # the smallest singular vector is accurate (relative to the gap)
    i = int(np.argmin(s))
    _, _, Vt = np.linalg.svd(G)
    assert abs(abs(S[:, i] @ Vt[-1]) - 1) < 1e-8


@pytest.mark.parametrize("j,warm", [(1, False), (2, False), (21, False), (33, True), (35, False), (64, True)])
def test_refined_vector_vs_oracle(h, j, warm):
    """The stage-2 refined vector kernel (inverse iteration on R) against the
    oracle's dense Jacobi SVD: the smallest singular value of R as ||R s1||,
    the smallest right singular vector, and theta1 = s1^T H s1.  R is graded
    like the refined projection near convergence (one tiny singular value);
    the leading dimension is that of the solver's workspaces (64)."""
    rng = np.random.default_rng(300 + j)
    U = np.linalg.qr(rng.standard_normal((j, j)))[0]
    V = np.linalg.qr(rng.standard_normal((j, j)))[0]
    s = np.logspace(0, -2, j)
    s[-1] = 1e-12
    R = np.linalg.qr(U @ np.diag(s) @ V.T)[1]
    Hs = rng.standard_normal((j, j))
    Hs = Hs + Hs.T
    LDp = 64
    Rp = np.zeros((LDp, LDp))
    Rp[:j, :j] = R
    Rp[j:, :] = np.nan                      # rows past j must not be read
    Hp = np.zeros((LDp, LDp))
    Hp[:j, :j] = Hs
    sig_ref, _, Vref = jacobi_svd(R)        # oracle: ascending singular values
    vmin = Vref[:, 0]
    x0 = None
    if warm:
        x0 = dev(vmin + 1e-3 * rng.standard_normal(j))
    s1 = torch.empty(j, dtype=torch.float64, device="cuda")
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    steps = torch.zeros(1, dtype=torch.int32, device="cuda")
    native.phsvds_refined_vector(h, j, dev(Rp.ravel(order="F")), LDp, x0, dev(Hp.ravel(order="F")), LDp, s1, out,
                                 24, 1e-10, steps)
    native.phsvds_sync(h)
    x = s1.cpu().numpy()
    th, rho = out.cpu().numpy()
    nrm = np.linalg.norm(R, 2)
    assert abs(np.linalg.norm(x) - 1) <= 1e-14
    assert abs(rho - sig_ref[0]) <= 1e-10 * sig_ref[0] + 4 * j * EPS64 * nrm
    assert abs(rho - np.linalg.norm(R @ x)) <= 4 * j * EPS64 * nrm
    if j > 1:
        assert abs(abs(x @ vmin) - 1) <= 1e-12
    assert abs(th - x @ Hs @ x) <= 4 * j * EPS64 * np.linalg.norm(Hs, 2)
    assert 1 <= int(steps.item()) <= 4


def test_refined_vector_rejects_bad_arguments(h):
    R = dev(np.eye(4).ravel())
    s1 = torch.empty(4, dtype=torch.float64, device="cuda")
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    for j, ldr, maxit in [(0, 4, 1), (65, 65, 1), (4, 3, 1), (4, 4, 0)]:
        with pytest.raises(native.PhsvdsError):
            native.phsvds_refined_vector(h, j, R, ldr, None, R, 4, s1, out, maxit)
