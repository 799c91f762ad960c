"""The allocation-free A^T (A X) entry point (phsvds_ata_spmm_static_f64).

It is meant for callers that cannot allocate device memory while it runs (all
memory handed to their own pool, or a loop where a cudaMalloc is not
acceptable), so it keeps the intermediate A X in a fixed device array of the
library.  These tests call it through the C ABI twice in a row and compare
each result with the existing two-phase entry point (which takes a caller
buffer) and with the CPU product A^T (A X) of the oracle's sparse operator,
both within the rounding bound of the SpMM parity tests; they also check that
oversized inputs and NULL arrays are refused before anything runs, and that
the calls take no device memory beyond the fixed array itself (which the
driver may place at the process's first call).
The file name keeps it last in collection, so it runs both after the other GPU
tests and alone.  (The header constant is checked against the binding on the
CPU, in test_abi.py.)
"""
import numpy as np
import pytest

from paper_1408_5535_gb300 import native, synth
from oracle import phsvds_ref as R
from tests.gpu_util import torch, need_gpu, dev, device_csr

pytestmark = pytest.mark.gpu
EPS64 = 2.0 ** -52
STATIC_BYTES = 8 * native.STATIC_Z_MAX          # the fixed array: 2 MiB


@pytest.fixture(scope="module")
def h():
    need_gpu()
    with native.Handle(0) as hh:
        yield hh


def _bound(A, S, X):
    absA = abs(S)
    rowmax = max(np.diff(A.row_ptr).max(), 1) + 2
    return 4 * rowmax * EPS64 * (absA.T @ (absA @ np.abs(X)))


def _existing(h, A, d, b, X):
    """The same product through phsvds_ata_spmm_f64, two-phase, caller scratch."""
    Yd = torch.empty((A.n, b), dtype=torch.float64, device="cuda")
    z = torch.empty((A.m, b), dtype=torch.float64, device="cuda")
    native.phsvds_ata_spmm(h, 2, A.m, A.n, A.nnz, d["rp"], d["ci"], d["va"], d["cp"], d["ri"], d["cv"], b, dev(X),
                           Yd, z)
    native.phsvds_sync(h)
    return Yd.cpu().numpy()


@pytest.mark.parametrize("case,b", [(0, 8), (1, 4), (2, 1), (3, 8)])
def test_two_calls_in_a_row_match_existing_entry_point(h, case, b):
    cases = [lambda: synth.random_sparse(3001, 1499, 12.0, 3),            # ragged tails, several tiles
             lambda: synth.grid_gradient(23, 1.0, 2),                      # 1-2 entries per row
             lambda: synth.random_sparse(777, 333, 30.0, 4, values="gaussian", shift=0.0),
             lambda: synth.random_sparse(native.STATIC_Z_MAX // 8, 16000, 6.0, 5)]   # m * b at the limit
    A = cases[case]()
    assert A.m * b <= native.STATIC_Z_MAX
    d = device_csr(A)
    nnz = int(A.row_ptr[-1])
    Xs = [(synth.uniform(7, 30 + t, A.n * b) * 2 - 1).reshape(A.n, b) for t in range(2)]
    refs = [_existing(h, A, d, b, X) for X in Xs]
    ops = R.Ops(R.as_scipy(A))
    cpu = [ops.C(X) for X in Xs]                      # the oracle's A^T (A X), FP64 on the CPU
    Xd = [dev(X) for X in Xs]
    Yd = [torch.full((A.n, b), float("nan"), dtype=torch.float64, device="cuda") for _ in Xs]
    torch.cuda.synchronize()
    free = [torch.cuda.mem_get_info()[0]]              # library loaded, before the first static call
    for t in range(2):
        native.phsvds_ata_spmm_static(h, A.m, A.n, nnz, d["rp"], d["ci"], d["va"], d["cp"], d["ri"], d["cv"], b,
                                      Xd[t], Yd[t])
        native.phsvds_sync(h)
        free.append(torch.cuda.mem_get_info()[0])
    # The first call of a process looks the fixed array up, and with lazy
    # module loading that is when the driver places it: free memory may drop
    # by the array itself (2 MiB) then, and by nothing more; later calls do
    # not change it at all.
    assert 0 <= free[0] - free[1] <= STATIC_BYTES, free
    assert free[2] == free[1], free
    for t in range(2):
        Y = Yd[t].cpu().numpy()
        bound = _bound(A, d["scipy"], Xs[t]) + 1e-300
        assert np.all(np.isfinite(Y))
        assert np.all(np.abs(Y - refs[t]) <= bound)
        assert np.all(np.abs(Y - cpu[t]) <= bound)


def test_null_arrays_are_refused_before_launch(h):
    A = synth.random_sparse(300, 120, 5.0, 8)
    d = device_csr(A)
    b = 2
    X = dev(np.ones((A.n, b)))
    Y = torch.full((A.n, b), 7.0, dtype=torch.float64, device="cuda")
    nnz = int(A.row_ptr[-1])
    for drop in ("ci", "va", "ri", "cv"):
        args = {k: d[k] for k in ("rp", "ci", "va", "cp", "ri", "cv")}
        args[drop] = None
        with pytest.raises(native.PhsvdsError) as ei:
            native.phsvds_ata_spmm_static(h, A.m, A.n, nnz, args["rp"], args["ci"], args["va"], args["cp"],
                                          args["ri"], args["cv"], b, X, Y)
        assert ei.value.status == 1
    native.phsvds_sync(h)
    assert bool(torch.all(Y == 7.0))


def test_oversized_input_is_refused_before_launch(h):
    A = synth.random_sparse(native.STATIC_Z_MAX // 4 + 1, 2000, 3.0, 6)
    d = device_csr(A)
    b = 4
    X = dev(np.ones((A.n, b)))
    Y = torch.full((A.n, b), 7.0, dtype=torch.float64, device="cuda")
    with pytest.raises(native.PhsvdsError) as ei:
        native.phsvds_ata_spmm_static(h, A.m, A.n, int(A.row_ptr[-1]), d["rp"], d["ci"], d["va"], d["cp"], d["ri"],
                                      d["cv"], b, X, Y)
    assert ei.value.status == 1 and "exceeds the fixed scratch" in str(ei.value)
    native.phsvds_sync(h)
    assert bool(torch.all(Y == 7.0))
