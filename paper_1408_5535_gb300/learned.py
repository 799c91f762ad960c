"""Training of the learned correction network (PHSVDS_PREC_LEARNED).

Data: for each training operator, the plain method (GD+k, no preconditioner,
FP64) runs through phsvds_solve with residual recording on; each recorded
residual r gets its inner-solve target from the library's device CG on
(A^T A - shift I) t = r (phsvds_normal_cg): a few CG steps by default, a
polynomial in A^T A of low degree that the network's 7 x 7 receptive field
can represent, or the converged solve.  Both are normalised to norm sqrt(n)
(the subspace method only uses the correction's direction, and the solver
feeds the network r * sqrt(n) / ||r||).  Inputs are the four planes
[r, log diffusion, beta_x / 20, beta_y / 20] on the operator's grid.

Training: relative-L2 loss, Adam, with the library's forward / backward /
Adam kernels (phsvds_cnn_*); PyTorch only allocates device memory and copies
arrays.  Everything here is argument marshalling around those calls.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import native, synth

BETA_SCALE = 20.0


def features(A: synth.Csr) -> np.ndarray:
    """Feature planes (3 x n float32) of a convection-diffusion operator from
    synth.convdiff_stencil: log diffusion per cell, beta_x / 20, beta_y / 20."""
    meta = A.meta
    n = A.n
    bx, by = meta["beta"]
    return np.stack([np.asarray(meta["log_diffusion"], dtype=np.float32),
                     np.full(n, bx / BETA_SCALE, dtype=np.float32),
                     np.full(n, by / BETA_SCALE, dtype=np.float32)])


def init_params(seed: int = 7, last_scale: float = 0.1) -> np.ndarray:
    """He-normal initial weights (FP32, 3024) from the seeded generator; the
    output layer is scaled by last_scale so the first outputs are small next
    to the unit-RMS targets (relative loss near 1 rather than far above)."""
    shapes = [(16, 4), (16, 16), (1, 16)]
    out = []
    for li, (o, c) in enumerate(shapes):
        std = math.sqrt(2.0 / (9 * c)) * (last_scale if li == 2 else 1.0)
        out.append(synth.normal(seed, 700 + li, o * c * 9) * std)
    return np.concatenate(out).astype(np.float32)


def to_bf16_bits(w: np.ndarray) -> np.ndarray:
    """FP32 -> BF16 bit patterns (round to nearest even), as uint16."""
    u = np.asarray(w, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return r.astype(np.uint16)


@dataclass
class Samples:
    x: np.ndarray        # (S, 4, ny, nx) float32
    t: np.ndarray        # (S, ny, nx) float32
    nx: int
    ny: int
    cg_iters: list = field(default_factory=list)


def record_samples(h: native.Handle, ops: list, k: int = 5, per_op: int = 8, every: int = 15,
                   shift: float = 0.0, cg_rtol: float = 1e-6, cg_steps: int = 3) -> Samples:
    """Residuals of the plain method on each operator, and their inner-solve
    corrections, as normalised network inputs / targets.  cg_steps > 0: the
    target is the cg_steps-th CG iterate from zero (a degree cg_steps - 1
    polynomial in A^T A applied to r, which a 3-layer 3 x 3 network can
    represent); 0: CG to relative residual cg_rtol."""
    xs, ts, its = [], [], []
    N = None
    for A in ops:
        n = A.n
        N = int(round(math.sqrt(n)))
        assert N * N == n
        rec = np.zeros((per_op, n))
        # stop the plain run once enough residuals are recorded
        o = native.default_opts(record_r=rec.ctypes.data, record_max=per_op, record_every=every,
                                max_restarts=max(2, per_op * every // 10 + 2), stage2=0)
        res = native.phsvds_solve(h, A.m, A.n, A.row_ptr, A.col, A.val, k, native.SMALLEST, 1e-14,
                                  native.PREC_NONE, o, want_vectors=False, raise_on_error=False)
        cnt = int(res[4]["recorded"])
        if cnt == 0:
            continue
        R = rec[:cnt].T.copy()
        X, it, _ = native.phsvds_normal_cg(h, A.m, A.n, A.row_ptr, A.col, A.val, R, shift=shift,
                                           rtol=1e-30 if cg_steps > 0 else cg_rtol,
                                           maxit=cg_steps if cg_steps > 0 else 10000, raise_on_error=False)
        its.extend(int(v) for v in it)
        f = features(A)
        for c in range(cnt):
            r, t = R[:, c], X[:, c]
            nr, nt = np.linalg.norm(r), np.linalg.norm(t)
            if not (nr > 0 and nt > 0):
                continue
            x = np.empty((4, n), dtype=np.float32)
            x[0] = r * (math.sqrt(n) / nr)
            x[1:] = f
            xs.append(x.reshape(4, N, N))
            ts.append((t * (math.sqrt(n) / nt)).astype(np.float32).reshape(N, N))
    return Samples(np.stack(xs), np.stack(ts), N, N, its)


@dataclass
class TrainResult:
    params_bf16: np.ndarray      # uint16 bit patterns, 3024
    master: np.ndarray           # float32
    loss_history: list
    steps: int


def train(h: native.Handle, data: Samples, epochs: int = 60, batch: int = 32, lr: float = 3e-3, seed: int = 7,
          init: np.ndarray | None = None) -> TrainResult:
    """Adam on the relative-L2 loss over the samples, on the device."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    S = data.x.shape[0]
    npix = data.nx * data.ny
    w0 = init if init is not None else init_params(seed)
    master = torch.from_numpy(w0.copy()).to(dev)
    params = torch.from_numpy(to_bf16_bits(w0).view(np.int16)).to(dev)
    grad = torch.zeros(native.CNN_NPARAM, dtype=torch.float32, device=dev)
    m = torch.zeros_like(grad)
    v = torch.zeros_like(grad)
    X = torch.from_numpy(data.x).to(dev)
    T = torch.from_numpy(data.t).to(dev)
    work = torch.empty(native.cnn_work_floats(batch, npix), dtype=torch.float32, device=dev)
    y = torch.empty((batch, data.ny, data.nx), dtype=torch.float32, device=dev)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    order_rng = synth.uniform(seed, 800, epochs * S)
    hist, step = [], 0
    for ep in range(epochs):
        perm = np.argsort(order_rng[ep * S:(ep + 1) * S], kind="stable")
        loss.zero_()
        nb = 0
        for b0 in range(0, S - batch + 1, batch):
            idx = torch.from_numpy(perm[b0:b0 + batch]).to(dev)
            xb = X.index_select(0, idx).contiguous()
            tb = T.index_select(0, idx).contiguous()
            native.phsvds_cnn_forward(h, batch, data.nx, data.ny, params, xb, y, work)
            native.phsvds_cnn_backward(h, batch, data.nx, data.ny, params, xb, y, tb, work, grad, loss)
            step += 1
            native.phsvds_cnn_adam(h, master, grad, m, v, step, lr, params)
            nb += 1
        native.phsvds_sync(h)
        hist.append(float(loss.item()) / max(nb, 1))
    return TrainResult(params.cpu().numpy().view(np.uint16).copy(), master.cpu().numpy(), hist, step)


def solve_opts(A: synth.Csr, params_bf16: np.ndarray, **kw):
    """Options for a PHSVDS_PREC_LEARNED solve of operator A (the returned
    holder keeps the host arrays alive while the options are used)."""
    f = np.ascontiguousarray(features(A))
    p = np.ascontiguousarray(params_bf16.astype(np.uint16))
    N = int(round(math.sqrt(A.n)))
    o = native.default_opts(learned_params=p.ctypes.data, learned_features=f.ctypes.data, grid_nx=N, grid_ny=N, **kw)
    return o, (f, p)
