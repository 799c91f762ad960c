"""Plain CPU FP64 reference of the learned correction network -- oracle code.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline
leg of the benchmark may import this module.  It shares no code with the GPU
kernels.

The network (the learned-preconditioner form of the spec description;
the paper's own preconditioners are Sec. 4) maps a residual image plus feature
channels to a correction image on the operator's grid:

    a0 = x                                   (B, 4, ny, nx): [r, log kappa, beta_x, beta_y]
    z1 = conv(a0, W1), a1 = relu(z1)         W1: (16, 4, 3, 3)
    z2 = conv(a1, W2), a2 = relu(z2)         W2: (16, 16, 3, 3)
    y  = conv(a2, W3)                        W3: (1, 16, 3, 3)

conv is the 3 x 3 cross-correlation with zero padding and no bias:
    conv(a, W)[b, o, i, j] = sum_c sum_{p,q in -1..1} W[o, c, p+1, q+1] a[b, c, i+p, j+q].
Without biases the network is positively homogeneous: scaling all input
channels by s > 0 scales y by s.

Loss (relative L2 per sample, mean over the batch):
    L = (1/B) sum_b ||y_b - t_b||^2 / ||t_b||^2.
"""
from __future__ import annotations

import numpy as np

SHAPES = [(16, 4, 3, 3), (16, 16, 3, 3), (1, 16, 3, 3)]
NPARAM = sum(int(np.prod(s)) for s in SHAPES)   # 3024


def unpack(theta: np.ndarray):
    """Flat parameter vector -> [W1, W2, W3] (layer-major, then o, c, p, q)."""
    out, o = [], 0
    for s in SHAPES:
        k = int(np.prod(s))
        out.append(np.asarray(theta[o:o + k], dtype=np.float64).reshape(s))
        o += k
    return out


def conv(a: np.ndarray, W: np.ndarray) -> np.ndarray:
    """3 x 3 cross-correlation, zero padding, written out over the nine taps."""
    B, C, ny, nx = a.shape
    O = W.shape[0]
    ap = np.zeros((B, C, ny + 2, nx + 2))
    ap[:, :, 1:-1, 1:-1] = a
    out = np.zeros((B, O, ny, nx))
    for p in range(3):
        for q in range(3):
            win = ap[:, :, p:p + ny, q:q + nx]                     # a[b, c, i+p-1, j+q-1]
            out += np.einsum("oc,bcij->boij", W[:, :, p, q], win)
    return out


def conv_input_grad(g: np.ndarray, W: np.ndarray) -> np.ndarray:
    """d/da of sum(g * conv(a, W)): each output tap sends g back to the input
    pixel it read."""
    B, O, ny, nx = g.shape
    C = W.shape[1]
    dap = np.zeros((B, C, ny + 2, nx + 2))
    for p in range(3):
        for q in range(3):
            dap[:, :, p:p + ny, q:q + nx] += np.einsum("oc,boij->bcij", W[:, :, p, q], g)
    return dap[:, :, 1:-1, 1:-1]


def conv_weight_grad(a: np.ndarray, g: np.ndarray) -> np.ndarray:
    """d/dW of sum(g * conv(a, W))."""
    B, C, ny, nx = a.shape
    O = g.shape[1]
    ap = np.zeros((B, C, ny + 2, nx + 2))
    ap[:, :, 1:-1, 1:-1] = a
    dW = np.zeros((O, C, 3, 3))
    for p in range(3):
        for q in range(3):
            dW[:, :, p, q] = np.einsum("boij,bcij->oc", g, ap[:, :, p:p + ny, q:q + nx])
    return dW


def forward(theta: np.ndarray, x: np.ndarray):
    W1, W2, W3 = unpack(theta)
    z1 = conv(x, W1)
    a1 = np.maximum(z1, 0.0)
    z2 = conv(a1, W2)
    a2 = np.maximum(z2, 0.0)
    y = conv(a2, W3)
    return y, (x, a1, a2)


def loss(y: np.ndarray, t: np.ndarray) -> float:
    B = y.shape[0]
    num = np.sum((y - t) ** 2, axis=(1, 2, 3))
    den = np.sum(t ** 2, axis=(1, 2, 3))
    return float(np.sum(num / den) / B)


def loss_grad(y: np.ndarray, t: np.ndarray) -> np.ndarray:
    B = y.shape[0]
    den = np.sum(t ** 2, axis=(1, 2, 3))
    return 2.0 * (y - t) / (B * den[:, None, None, None])


def backward(theta: np.ndarray, x: np.ndarray, t: np.ndarray):
    """Loss and its gradient with respect to the flat parameters (chain rule
    through the three layers, the ReLU derivative 1[z > 0])."""
    W1, W2, W3 = unpack(theta)
    y, (a0, a1, a2) = forward(theta, x)
    L = loss(y, t)
    g3 = loss_grad(y, t)
    dW3 = conv_weight_grad(a2, g3)
    g2 = conv_input_grad(g3, W3) * (a2 > 0)
    dW2 = conv_weight_grad(a1, g2)
    g1 = conv_input_grad(g2, W2) * (a1 > 0)
    dW1 = conv_weight_grad(a0, g1)
    return L, np.concatenate([dW1.ravel(), dW2.ravel(), dW3.ravel()])


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round FP32 values to the nearest bfloat16 (ties to even), returned as FP64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return r.astype(np.uint32).view(np.float32).astype(np.float64)
