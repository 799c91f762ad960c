"""S1 at the benchmark's full sizes, in the launch configurations the
benchmark times by default: the 512 x 512 weighted grid at b = 4 and the
1e6 x 5e5 random matrix at b = 8, both schedules at the default group widths,
FP64 and FP32, with the CSC built by the library.  Every output row is
compared with the oracle's product (FP64 on the host) within the rounding
bound of the longest accumulation (row or column)."""
import numpy as np
import pytest

import bench
from oracle import phsvds_ref as R
from paper_1408_5535_gb300 import native, synth
from tests.gpu_util import torch, need_gpu, dev

pytestmark = pytest.mark.gpu
EPS64, EPS32 = 2.0 ** -52, 2.0 ** -23

CASES = {"grid512": (lambda: synth.grid_gradient(512, 1.0, 2), 4),
         "random1e6": (lambda: synth.random_sparse(1000000, 500000, 12.0, 3), 8)}


@pytest.fixture(scope="module")
def h():
    need_gpu()
    with native.Handle(0) as hh:
        yield hh


@pytest.fixture(scope="module", params=list(CASES))
def full(request, h):
    gen, b = CASES[request.param]
    A = gen()
    rp = torch.from_numpy(A.row_ptr.astype(np.int32)).cuda()
    ci = torch.from_numpy(A.col).cuda()
    va = torch.from_numpy(A.val).cuda()
    cp = torch.empty(A.n + 1, dtype=torch.int32, device="cuda")
    ri = torch.empty(A.nnz, dtype=torch.int32, device="cuda")
    cv = torch.empty(A.nnz, dtype=torch.float64, device="cuda")
    native.phsvds_csr_to_csc(h, A.m, A.n, A.nnz, rp, ci, va, cp, ri, cv)
    native.phsvds_sync(h)
    S = R.as_scipy(A)
    X = (synth.uniform(7, 20 + b, A.n * b) * 2 - 1).reshape(A.n, b)
    ref = R.Ops(S).C(X)
    absS = abs(S)
    bound = absS.T @ (absS @ np.abs(X))
    acc = max(int(np.diff(A.row_ptr).max()), int(np.bincount(A.col, minlength=A.n).max())) + 2
    yield dict(A=A, b=b, rp=rp, ci=ci, va=va, cp=cp, ri=ri, cv=cv, X=X, ref=ref, bound=bound, acc=acc)


@pytest.mark.parametrize("schedule", [1, 2])
@pytest.mark.parametrize("fp32", [False, True])
def test_full_size_product_vs_oracle(h, full, schedule, fp32):
    A, b = full["A"], full["b"]
    la = bench.spmm_lanes(A.nnz / A.m)
    lt = bench.spmm_lanes(A.nnz / A.n) if schedule == 2 else 0
    vt = torch.float32 if fp32 else torch.float64
    v1, v2 = (full["va"].float(), full["cv"].float()) if fp32 else (full["va"], full["cv"])
    X = dev(full["X"], vt)
    Y = torch.empty((A.n, b), dtype=vt, device="cuda")
    Z = torch.empty((A.m, b), dtype=vt, device="cuda")
    native.phsvds_ata_spmm(h, schedule, A.m, A.n, A.nnz, full["rp"], full["ci"], v1, full["cp"], full["ri"], v2,
                           b, X, Y, Z, fp32=fp32, lanes_a=la, lanes_at=lt)
    native.phsvds_sync(h)
    got = Y.double().cpu().numpy()
    lim = 4 * full["acc"] * (EPS32 if fp32 else EPS64) * full["bound"] + 1e-300
    err = np.abs(got - full["ref"])
    assert np.all(err <= lim), float(np.max(err / lim))
