"""Helpers shared by the GPU tests (device staging of seeded inputs)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def device_csr(A, fp32=False):
    """Device CSR (int32 offsets) plus CSC of A, values float64 (or float32)."""
    import scipy.sparse as sp
    S = sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.m, A.n))
    T = S.tocsc()
    T.sort_indices()
    vt = torch.float32 if fp32 else torch.float64
    return dict(rp=dev(A.row_ptr.astype(np.int32)), ci=dev(A.col.astype(np.int32)), va=dev(A.val, vt),
                cp=dev(T.indptr.astype(np.int32)), ri=dev(T.indices.astype(np.int32)), cv=dev(T.data, vt),
                scipy=S)
