"""The learned correction: network kernels against the CPU oracle, the inner
solve (CG), residual recording, training, and solves with the network as the
stage-1 correction (parity with the oracle at 1e-14 ||A||, fallback on stall)."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from paper_1408_5535_gb300 import learned, native, synth
from oracle import cnn_ref as N
from oracle import phsvds_ref as R
from tests.gpu_util import torch, need_gpu

pytestmark = pytest.mark.gpu
DELTA = 1e-14


@pytest.fixture(scope="module")
def h():
    need_gpu()
    with native.Handle(0) as hh:
        yield hh


def _bf16_params(seed=3, scale=1.0):
    w = learned.init_params(seed) * scale
    bits = learned.to_bf16_bits(w)
    return bits, N.bf16_round(w)


@pytest.mark.parametrize("B,nx,ny", [(1, 16, 16), (3, 20, 17), (2, 33, 9)])
def test_forward_and_backward_vs_oracle(h, B, nx, ny):
    """Ragged tiles (20 x 17, 33 x 9): GPU FP32 with BF16 weights against the
    FP64 oracle at the same (BF16-rounded) weights."""
    bits, wref = _bf16_params()
    x = (synth.normal(11, B, B * 4 * ny * nx)).reshape(B, 4, ny, nx).astype(np.float32)
    t = (synth.normal(12, B, B * ny * nx)).reshape(B, 1, ny, nx).astype(np.float32)
    y_ref, _ = N.forward(wref, x.astype(np.float64))
    L_ref, g_ref = N.backward(wref, x.astype(np.float64), t.astype(np.float64))
    dev = "cuda"
    P = torch.from_numpy(bits.view(np.int16)).to(dev)
    X = torch.from_numpy(x).to(dev)
    T = torch.from_numpy(t[:, 0]).contiguous().to(dev)
    Y = torch.empty((B, ny, nx), dtype=torch.float32, device=dev)
    work = torch.empty(native.cnn_work_floats(B, nx * ny), dtype=torch.float32, device=dev)
    grad = torch.zeros(native.CNN_NPARAM, dtype=torch.float32, device=dev)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    native.phsvds_cnn_forward(h, B, nx, ny, P, X, Y, work)
    native.phsvds_cnn_backward(h, B, nx, ny, P, X, Y, T, work, grad, loss)
    native.phsvds_sync(h)
    y = Y.cpu().numpy()
    assert np.max(np.abs(y - y_ref[:, 0])) <= 1e-5 * max(1.0, np.max(np.abs(y_ref)))
    assert float(loss.item()) == pytest.approx(L_ref, rel=1e-5)
    g = grad.cpu().numpy()
    assert np.linalg.norm(g - g_ref) <= 1e-4 * np.linalg.norm(g_ref)


def test_adam_step_and_bf16_rounding(h):
    """One Adam step (Kingma & Ba, bias-corrected) against its definition."""
    rng = np.random.default_rng(1)
    w = rng.standard_normal(native.CNN_NPARAM).astype(np.float32)
    g = rng.standard_normal(native.CNN_NPARAM).astype(np.float32)
    m0 = rng.standard_normal(native.CNN_NPARAM).astype(np.float32) * 0.1
    v0 = np.abs(rng.standard_normal(native.CNN_NPARAM)).astype(np.float32) * 0.1
    lr, b1, b2, eps, step = 1e-2, 0.9, 0.999, 1e-8, 3
    tt = lambda a: torch.from_numpy(a.copy()).cuda()
    W, G, M, V = tt(w), tt(g), tt(m0), tt(v0)
    P = torch.zeros(native.CNN_NPARAM, dtype=torch.int16, device="cuda")
    native.phsvds_cnn_adam(h, W, G, M, V, step, lr, P, b1, b2, eps)
    native.phsvds_sync(h)
    m1 = b1 * m0.astype(np.float64) + (1 - b1) * g
    v1 = b2 * v0.astype(np.float64) + (1 - b2) * g.astype(np.float64) ** 2
    w1 = w - lr * (m1 / (1 - b1 ** step)) / (np.sqrt(v1 / (1 - b2 ** step)) + eps)
    assert np.allclose(W.cpu().numpy(), w1, rtol=1e-5, atol=1e-6)
    assert np.all(G.cpu().numpy() == 0)
    bits = P.cpu().numpy().view(np.uint16)
    assert np.array_equal(bits, learned.to_bf16_bits(W.cpu().numpy()))


@pytest.mark.parametrize("count", [1, 3, 8, 11])
def test_normal_cg_solves_the_shifted_normal_equations(h, count):
    A = synth.convdiff_stencil(16, 1001)
    S = sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.m, A.n))
    C = (S.T @ S).tocsr()
    lam_min = np.linalg.eigvalsh(C.toarray())[0]
    shift = 0.5 * lam_min
    Rhs = synth.normal(5, count, A.n * count).reshape(count, A.n).T.copy()
    X, its, st = native.phsvds_normal_cg(h, A.m, A.n, A.row_ptr, A.col, A.val, Rhs, shift=shift, rtol=1e-8)
    assert st == native.PHSVDS_OK and np.all(its > 0)
    res = (C @ X - shift * X) - Rhs
    assert np.all(np.linalg.norm(res, axis=0) <= 1e-7 * np.linalg.norm(Rhs, axis=0))


def test_normal_cg_rejects_indefinite_shift(h):
    A = synth.convdiff_stencil(8, 1002)
    with pytest.raises(native.PhsvdsError):
        native.phsvds_normal_cg(h, A.m, A.n, A.row_ptr, A.col, A.val, np.ones((A.n, 1)), shift=1e6)


def test_recording_counts_and_shapes(h):
    A = synth.convdiff_stencil(16, 1003)
    rec = np.full((5, A.n), np.nan)
    o = native.default_opts(record_r=rec.ctypes.data, record_max=5, record_every=7)
    sig, _, _, res, st, status = native.phsvds_solve(h, A.m, A.n, A.row_ptr, A.col, A.val, 3, native.SMALLEST,
                                                     DELTA, native.PREC_NONE, o, want_vectors=False)
    assert status == native.PHSVDS_OK
    assert st["recorded"] == min(5, st["iters_stage1"] // 7 + 1)
    assert np.all(np.isfinite(rec[: st["recorded"]]))
    assert np.all(np.linalg.norm(rec[: st["recorded"]], axis=1) > 0)


@pytest.fixture(scope="module")
def trained(h):
    ops = [synth.convdiff_stencil(16, 1000 + i) for i in range(12)]
    data = learned.record_samples(h, ops, k=3, per_op=6, every=10)
    tr = learned.train(h, data, epochs=40, batch=16, lr=3e-3)
    return data, tr


def test_training_lowers_the_loss(trained):
    data, tr = trained
    assert data.x.shape[1:] == (4, 16, 16) and data.x.shape[0] >= 48
    assert tr.loss_history[-1] < 0.7 * tr.loss_history[0]


@pytest.mark.parametrize("seed", [1100, 1101])
def test_learned_solve_matches_oracle(h, trained, seed):
    """A held-out operator solved with the trained network as the stage-1
    correction: same triplets as the oracle (plain GD+k) to 1e-10, residuals
    <= 1e-14 ||A|| recomputed here; the plain GPU solve is reported beside it."""
    _, tr = trained
    A = synth.convdiff_stencil(16, seed)
    k = 5
    o, keep = learned.solve_opts(A, tr.params_bf16)
    sig, U, V, res, st, status = native.phsvds_solve(h, A.m, A.n, A.row_ptr, A.col, A.val, k, native.SMALLEST,
                                                     DELTA, native.PREC_LEARNED, o)
    assert status == native.PHSVDS_OK
    ref = R.phsvds(A, k, largest=False, delta=DELTA)
    assert np.max(np.abs(sig - ref.sigma) / ref.sigma) <= 1e-10
    S = sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.m, A.n))
    r = np.sqrt(np.linalg.norm(S @ V - U * sig, axis=0) ** 2 + np.linalg.norm(S.T @ U - V * sig, axis=0) ** 2)
    assert np.all(r <= DELTA * st["norm_A_est"])
    plain = native.phsvds_solve(h, A.m, A.n, A.row_ptr, A.col, A.val, k, native.SMALLEST, DELTA,
                                native.PREC_NONE, native.default_opts(), want_vectors=False)[4]
    print(f"\nseed {seed}: stage-1 iterations plain {plain['iters_stage1']}, learned {st['iters_stage1']}"
          f" (fell back: {st['fell_back']})")


def test_fallback_on_stall(h):
    """A network that outputs nothing useful (all-zero weights) stalls: the
    solver falls back to Jacobi and still converges to the same triplets."""
    A = synth.convdiff_stencil(16, 1102)
    k = 3
    zero = np.zeros(native.CNN_NPARAM, dtype=np.uint16)
    o, keep = learned.solve_opts(A, zero, stall_window=30)
    sig, _, _, res, st, status = native.phsvds_solve(h, A.m, A.n, A.row_ptr, A.col, A.val, k, native.SMALLEST,
                                                     DELTA, native.PREC_LEARNED, o, want_vectors=False)
    assert status == native.PHSVDS_OK and st["fell_back"] == 1 and st["fell_back_at"] >= 30
    ref = R.phsvds(A, k, largest=False, delta=DELTA)
    assert np.max(np.abs(sig - ref.sigma) / ref.sigma) <= 1e-10


def test_learned_rejects_bad_grid(h):
    A = synth.convdiff_stencil(8, 1003)
    o, keep = learned.solve_opts(A, np.zeros(native.CNN_NPARAM, dtype=np.uint16))
    o.grid_nx = 7
    with pytest.raises(native.PhsvdsError):
        native.phsvds_solve(h, A.m, A.n, A.row_ptr, A.col, A.val, 2, native.SMALLEST, DELTA, native.PREC_LEARNED, o)
