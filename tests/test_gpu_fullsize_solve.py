"""The whole solve at the benchmark's full size, against the CPU oracle.

The random sparse 1,000,000 x 500,000 matrix (Poisson(12) entries per row,
log-normal(2) values with random signs, + 1e-3 [I; 0], seed 3), k = 20 largest
triplets to 1e-14 ||A||, block 8 -- the benchmark's workload and launch
configuration -- in FP64 and in mixed precision.  The oracle (plain CPU FP64
PHSVDS) runs the same solve here; the GPU triplets must give:

* the same index set and singular values within 1e-10 relative (also against
  the oracle's recorded values in tests/golden/oracle_counts.json);
* residuals sqrt(||A v - s u||^2 + ||A^T u - s v||^2) <= 1e-14 ||A||,
  recomputed here in FP64 on the CPU (Sec. 5's criterion);
* the oracle's singular vectors up to sign (each value is simple and far
  from its neighbours, so each vector is determined to the residual over the
  gap), and orthonormal U and V.

At n = 500,000 the tall-skinny kernels (block Gram-Schmidt, basis
transforms, Ritz vectors) run their grid-stride loops over several row
chunks per thread block, which the smaller parity cases do not reach.
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

from paper_1408_5535_gb300 import native, synth
from oracle import phsvds_ref as R
from tests.gpu_util import torch, need_gpu

pytestmark = pytest.mark.gpu
DELTA = 1e-14
K = 20
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_counts.json")


@pytest.fixture(scope="module")
def c3():
    need_gpu()
    A = synth.random_sparse(1000000, 500000, 12.0, 3)
    ref = R.phsvds(A, K, largest=True, delta=DELTA, o=R.Opts(block=8))
    S = sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.m, A.n))
    return A, S, ref


@pytest.fixture(scope="module")
def h():
    need_gpu()
    stream = torch.cuda.Stream()
    with native.Handle(0, stream.cuda_stream) as hh:
        yield hh


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_full_size_largest_matches_oracle(h, c3, precision):
    A, S, ref = c3
    prec = native.MIXED if precision == "mixed" else native.FP64
    rp = torch.from_numpy(A.row_ptr).cuda()
    ci = torch.from_numpy(A.col).cuda()
    va = torch.from_numpy(A.val).cuda()
    o = native.default_opts(block_size=8, precision=prec)
    sig, U, V, res, st, _ = native.phsvds_solve(h, A.m, A.n, rp, ci, va, K, native.LARGEST, DELTA,
                                                native.PREC_NONE, o, on_device=True)
    normA = float(ref.sigma[0])            # the largest singular value, FP64 oracle
    # values: same index set (the 20 largest, in order) and 1e-10 relative
    assert np.all(np.diff(sig) <= 0)
    assert np.max(np.abs(sig - ref.sigma) / ref.sigma) <= 1e-10, np.abs(sig - ref.sigma) / ref.sigma
    gold = np.asarray(json.load(open(GOLD))["c3_largest"]["sigma"])
    assert np.max(np.abs(sig - gold) / gold) <= 1e-10
    # residuals recomputed on the CPU in FP64
    rv = np.linalg.norm(S @ V - U * sig, axis=0)
    ru = np.linalg.norm(S.T @ U - V * sig, axis=0)
    r = np.sqrt(rv ** 2 + ru ** 2)
    assert np.all(r <= DELTA * normA), r / normA
    assert np.all(res <= DELTA * normA * (1 + 1e-6))
    # vectors: the oracle's up to sign
    cv = np.abs(np.sum(V * ref.V, axis=0))
    cu = np.abs(np.sum(U * ref.U, axis=0))
    assert np.all(cv >= 1 - 1e-9) and np.all(cu >= 1 - 1e-9), (cv.min(), cu.min())
    assert np.max(np.abs(V.T @ V - np.eye(K))) <= 1e-12
    assert np.max(np.abs(U.T @ U - np.eye(K))) <= 1e-12
    if precision == "mixed":
        assert st["iters_stage1_fp32"] > 0
