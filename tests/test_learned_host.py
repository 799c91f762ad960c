"""Host-side helpers of the learned correction (no GPU): BF16 rounding of the
parameters, the initialisation, the feature planes of an operator."""
import math

import numpy as np

from paper_1408_5535_gb300 import learned, synth
from oracle import cnn_ref as N


def test_bf16_bits_round_like_the_oracle():
    x = np.random.default_rng(3).standard_normal(5000).astype(np.float32) * 10.0 ** np.random.default_rng(4).integers(
        -6, 6, 5000)
    bits = learned.to_bf16_bits(x)
    back = (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    assert np.array_equal(back, N.bf16_round(x))


def test_init_params_layout_and_scale():
    w = learned.init_params(7)
    assert w.shape == (N.NPARAM,) and w.dtype == np.float32
    W1, W2, W3 = N.unpack(w.astype(np.float64))
    # He-normal spreads, the output layer scaled by 0.1
    assert abs(W1.std() - math.sqrt(2 / 36)) < 0.25 * math.sqrt(2 / 36)
    assert abs(W2.std() - math.sqrt(2 / 144)) < 0.15 * math.sqrt(2 / 144)
    assert abs(W3.std() - 0.1 * math.sqrt(2 / 144)) < 0.35 * 0.1 * math.sqrt(2 / 144)
    assert np.array_equal(w, learned.init_params(7))


def test_feature_planes_of_an_operator():
    A = synth.convdiff_stencil(16, 1005)
    f = learned.features(A)
    assert f.shape == (3, A.n) and f.dtype == np.float32
    bx, by = A.meta["beta"]
    assert np.allclose(f[0], A.meta["log_diffusion"], rtol=1e-6)
    assert np.all(f[1] == np.float32(bx / 20.0)) and np.all(f[2] == np.float32(by / 20.0))
    assert abs(bx) <= 20 and abs(by) <= 20
