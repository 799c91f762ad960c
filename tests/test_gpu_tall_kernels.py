"""The tall-skinny kernels at the solver's full sizes, through the C ABI,
against numpy FP64.

* One pass of block classical Gram-Schmidt (phsvds_block_cgs_*): the
  subtraction T - P Gsub, the projection P^T T and the Gram T^T T, on a
  two-piece basis [P1 | P2] (locked vectors and basis), as stage 1 runs it
  at n = 500,000 (55 columns against a block of 8) and stage 2 at
  N = m + n = 1,500,000 (35 columns against one).
* Out = P Y - Xs diag(theta) with column norms (phsvds_tall_small_*): the
  Ritz vectors, residuals and restart transforms, in place and out of place.

The sizes put several row chunks on every thread block (the grids are capped
at a few blocks per SM), plus a ragged last chunk.  The bounds are the
rounding bounds of the summations: products accumulate per thread in the
storage precision over at most a few hundred terms and across thread blocks
in FP64, so |error| <= c eps_T (|P|^T |T|) elementwise with c a few hundred.
The inputs of the FP32 cases are FP32 values, so the reference sees exactly
what the kernel sees.
"""
import numpy as np
import pytest

from paper_1408_5535_gb300 import native, synth
from tests.gpu_util import torch, need_gpu

pytestmark = pytest.mark.gpu
EPS = {np.float64: 2.0 ** -52, np.float32: 2.0 ** -23}


@pytest.fixture(scope="module")
def h():
    need_gpu()
    with native.Handle(0) as hh:
        yield hh


def _mat(seed, n, c, dt):
    return ((synth.uniform(seed, 1, n * c) * 2 - 1).reshape(c, n).T).astype(dt)   # column-major n x c


def _cm(x, dt):
    """Device tensor holding the column-major data of x (n x c)."""
    return torch.from_numpy(np.ascontiguousarray(x.T)).to({np.float64: torch.float64, np.float32: torch.float32}[dt]).cuda()


def _host(t, n, c):
    return t.cpu().numpy().reshape(c, n).T.astype(np.float64)


@pytest.mark.parametrize("n,p1,p2,q,dt", [(500000, 20, 35, 8, np.float64), (500000, 20, 35, 8, np.float32),
                                          (1500000, 0, 35, 1, np.float64), (1500001, 6, 29, 1, np.float64),
                                          (77825, 3, 4, 3, np.float64), (300007, 12, 9, 4, np.float32)])
def test_block_cgs_pass_full_size(h, n, p1, p2, q, dt):
    eps = EPS[dt]
    p = p1 + p2
    P = _mat(11, n, p, dt)
    T = _mat(12, n, q, dt)
    Gs = (synth.uniform(13, 1, p * q).reshape(q, p).T * 2 - 1) / n     # p x q, column-major
    P_d = _cm(P, dt)
    T_d = _cm(T, dt)
    Gs_d = torch.from_numpy(np.ascontiguousarray(Gs.T)).cuda()
    Gout = torch.zeros(p * q, dtype=torch.float64, device="cuda")
    Tout = torch.zeros(q * q, dtype=torch.float64, device="cuda")
    P1 = P_d[: p1] if p1 else None
    P2 = P_d[p1:]
    # pass 1: subtraction and projection; pass 2 (same block): Gram only
    native.phsvds_block_cgs(h, n, P1, n, p1, T_d, n, q, Gsub=Gs_d, Gout=Gout, P2=P2, ld2=n, p2=p2,
                            fp32=dt == np.float32)
    native.phsvds_block_cgs(h, n, None, n, 0, T_d, n, q, Tout=Tout, fp32=dt == np.float32)
    native.phsvds_sync(h)
    Pd = P.astype(np.float64)
    Tnew_ref = T.astype(np.float64) - Pd @ Gs.astype(dt).astype(np.float64)
    Tn = _host(T_d, n, q)
    bt = (p + 4) * eps * (np.abs(T.astype(np.float64)) + np.abs(Pd) @ np.abs(Gs))
    assert np.all(np.abs(Tn - Tnew_ref) <= bt)
    # projection and Gram of the updated block as the kernel stored it
    G_ref = Pd.T @ Tn
    bG = 600 * eps * (np.abs(Pd).T @ np.abs(Tn))
    G = Gout.cpu().numpy().reshape(q, p).T
    assert np.all(np.abs(G - G_ref) <= bG)
    Tt = Tout.cpu().numpy().reshape(q, q).T
    assert np.all(np.abs(Tt - Tn.T @ Tn) <= 600 * eps * (np.abs(Tn).T @ np.abs(Tn)))


@pytest.mark.parametrize("n,p,r,dt,inplace", [(500000, 35, 8, np.float64, False), (500000, 35, 8, np.float32, False),
                                              (500000, 35, 21, np.float64, True), (1500000, 35, 1, np.float64, False),
                                              (155649, 30, 21, np.float32, True)])
def test_tall_times_small_full_size(h, n, p, r, dt, inplace):
    eps = EPS[dt]
    P = _mat(21, n, p, dt)
    Y = synth.uniform(22, 1, p * r).reshape(r, p).T * 2 - 1          # p x r FP64
    Xs = _mat(23, n, r, dt)
    th = synth.uniform(24, 1, r) * 3
    P_d = _cm(P, dt)
    Y_d = torch.from_numpy(np.ascontiguousarray(Y.T)).cuda()
    Xs_d = _cm(Xs, dt)
    th_d = torch.from_numpy(th).cuda()
    nrm = torch.zeros(r, dtype=torch.float64, device="cuda")
    Yt = Y.astype(dt).astype(np.float64)                                # the kernel rounds Y to the storage type
    Pd = P.astype(np.float64)
    if inplace:
        native.phsvds_tall_small(h, n, P_d, n, p, Y_d, p, r, P_d, n, norms2=nrm, fp32=dt == np.float32)
        native.phsvds_sync(h)
        Out = _host(P_d, n, p)[:, :r]
        ref = Pd @ Yt
        bound = (p + 2) * eps * (np.abs(Pd) @ np.abs(Yt))
    else:
        O_d = torch.zeros_like(Xs_d)
        thd = th.astype(dt).astype(np.float64)
        native.phsvds_tall_small(h, n, P_d, n, p, Y_d, p, r, O_d, n, Xs=Xs_d, ldx=n, theta=th_d, norms2=nrm,
                                 fp32=dt == np.float32)
        native.phsvds_sync(h)
        Out = _host(O_d, n, r)
        Xd = Xs.astype(np.float64)
        ref = Pd @ Yt - Xd * thd
        bound = (p + 4) * eps * (np.abs(Pd) @ np.abs(Yt) + np.abs(Xd) * thd)
    assert np.all(np.abs(Out - ref) <= bound)
    nr = nrm.cpu().numpy()
    n2 = np.sum(Out * Out, axis=0)
    assert np.all(np.abs(nr - n2) <= 400 * 2.0 ** -52 * n2)
