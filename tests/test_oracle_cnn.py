"""Pins of the CPU reference of the correction network (oracle/cnn_ref.py)."""
import numpy as np
import pytest

from oracle import cnn_ref as N


def _brute_conv(a, W):
    B, C, ny, nx = a.shape
    O = W.shape[0]
    out = np.zeros((B, O, ny, nx))
    for b in range(B):
        for o in range(O):
            for i in range(ny):
                for j in range(nx):
                    s = 0.0
                    for c in range(C):
                        for p in (-1, 0, 1):
                            for q in (-1, 0, 1):
                                if 0 <= i + p < ny and 0 <= j + q < nx:
                                    s += W[o, c, p + 1, q + 1] * a[b, c, i + p, j + q]
                    out[b, o, i, j] = s
    return out


def test_conv_equals_brute_force():
    rng = np.random.default_rng(1)
    a = rng.standard_normal((2, 3, 5, 7))
    W = rng.standard_normal((4, 3, 3, 3))
    assert np.allclose(N.conv(a, W), _brute_conv(a, W), rtol=1e-13, atol=1e-13)


def test_conv_identity_and_shift_kernels():
    rng = np.random.default_rng(2)
    a = rng.standard_normal((1, 2, 6, 5))
    W = np.zeros((2, 2, 3, 3))
    W[0, 0, 1, 1] = W[1, 1, 1, 1] = 1.0
    assert np.array_equal(N.conv(a, W), a)
    W = np.zeros((1, 2, 3, 3))
    W[0, 1, 0, 1] = 1.0                       # reads a[c=1, i-1, j]
    ref = np.zeros((1, 1, 6, 5))
    ref[0, 0, 1:, :] = a[0, 1, :-1, :]
    assert np.array_equal(N.conv(a, W), ref)


def test_input_and_weight_gradients_are_adjoints():
    rng = np.random.default_rng(3)
    a = rng.standard_normal((2, 4, 6, 5))
    W = rng.standard_normal((3, 4, 3, 3))
    g = rng.standard_normal((2, 3, 6, 5))
    lhs = np.sum(g * N.conv(a, W))
    assert np.isclose(lhs, np.sum(N.conv_input_grad(g, W) * a), rtol=1e-12)
    assert np.isclose(lhs, np.sum(N.conv_weight_grad(a, g) * W), rtol=1e-12)


def test_backward_matches_central_differences():
    rng = np.random.default_rng(4)
    x = rng.standard_normal((2, 4, 5, 6))
    t = rng.standard_normal((2, 1, 5, 6))
    th = rng.standard_normal(N.NPARAM) * 0.3
    L, g = N.backward(th, x, t)
    assert L == pytest.approx(N.loss(N.forward(th, x)[0], t))
    idx = rng.choice(N.NPARAM, 60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros(N.NPARAM)
        e[i] = h
        fd = (N.loss(N.forward(th + e, x)[0], t) - N.loss(N.forward(th - e, x)[0], t)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_positive_homogeneity():
    rng = np.random.default_rng(5)
    x = rng.standard_normal((1, 4, 6, 6))
    th = rng.standard_normal(N.NPARAM)
    y1 = N.forward(th, x)[0]
    assert np.allclose(N.forward(th, 3.5 * x)[0], 3.5 * y1, rtol=1e-12, atol=1e-12)


def test_bf16_rounding():
    v = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -2.5, 0.0, 3.0e-39])
    r = N.bf16_round(v)
    assert r[0] == 1.0 and r[1] == 1.0                  # tie -> even
    assert r[2] == 1.0 + 2.0 ** -6                       # 1 + 3*2^-8 rounds up to 1 + 4*2^-8
    assert r[3] == -2.5 and r[4] == 0.0
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(6).standard_normal(1000).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(N.bf16_round(x), ref)
