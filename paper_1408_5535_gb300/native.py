"""ctypes binding of libphsvds.so (include/phsvds.h): argument marshalling only.

Every step of the method runs in the library's CUDA kernels; this module never
computes anything itself.  Importing it without the built library raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libphsvds.so")

PHSVDS_OK, PHSVDS_ERR_INVALID, PHSVDS_ERR_NOT_CONVERGED, PHSVDS_ERR_BREAKDOWN = 0, 1, 2, 3
PHSVDS_ERR_NAN, PHSVDS_ERR_TIMEOUT, PHSVDS_ERR_CUDA, PHSVDS_ERR_OOM = 4, 5, 6, 7
SMALLEST, LARGEST = 0, 1
PREC_NONE, PREC_JACOBI, PREC_LEARNED, PREC_GIVEN = 0, 1, 2, 3
CNN_NPARAM = 3024


def cnn_work_floats(batch: int, npix: int) -> int:
    """Floats of the phsvds_cnn_forward / _backward workspace."""
    return 65 * batch * npix + 2 * CNN_NPARAM + 2 * batch
FP64, MIXED = 0, 1
SPMM_AUTO, SPMM_FUSED_ATOMIC, SPMM_TWO_PHASE = 0, 1, 2


class Opts(C.Structure):
    _fields_ = [("block_size", C.c_int), ("max_basis", C.c_int), ("min_restart", C.c_int),
                ("max_restarts", C.c_int), ("eps_factor", C.c_double), ("precision", C.c_int),
                ("spmm", C.c_int), ("stage2", C.c_int), ("rayleigh_ritz", C.c_int),
                ("seed", C.c_uint64), ("time_limit_s", C.c_double), ("profile", C.c_int),
                ("learned_params", C.c_void_p), ("learned_features", C.c_void_p), ("grid_nx", C.c_int),
                ("grid_ny", C.c_int), ("stall_window", C.c_int), ("record_r", C.c_void_p), ("record_max", C.c_int),
                ("record_every", C.c_int), ("projected_solver", C.c_int), ("init_V", C.c_void_p),
                ("init_nv", C.c_int), ("mixed_inner", C.c_int), ("inner_maxit", C.c_int), ("inner_tol", C.c_double),
                ("stage2_precond", C.c_int), ("precond_M", C.c_void_p), ("stage2_inner", C.c_int),
                ("inner2_maxit", C.c_int), ("inner2_patience", C.c_int), ("dynamic", C.c_int),
                ("dyn_init_iter", C.c_int), ("dyn_max_switch", C.c_int), ("deterministic", C.c_int),
                ("norm_A", C.c_double), ("stage1_inner", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("matvecs_A", C.c_int64), ("matvecs_At", C.c_int64), ("iters_stage1", C.c_int64),
                ("iters_stage1_fp32", C.c_int64), ("iters_stage2", C.c_int64), ("restarts", C.c_int64),
                ("switched", C.c_int), ("norm_A_est", C.c_double), ("t_stage1_ms", C.c_double),
                ("t_stage2_ms", C.c_double), ("t_total_ms", C.c_double), ("spmm_schedule", C.c_int),
                ("kernel_launches", C.c_int64), ("t_class_ms", C.c_double * 12), ("n_class", C.c_int64 * 12),
                ("spmm_c_calls", C.c_int64), ("spmm_c_ms", C.c_double), ("spmm_c_width", C.c_int),
                ("jacobi_sweeps", C.c_int64), ("jacobi_rotations", C.c_int64), ("jacobi_calls", C.c_int64),
                ("jacobi_dim_sum", C.c_int64), ("fell_back", C.c_int), ("fell_back_at", C.c_int64),
                ("recorded", C.c_int64), ("stage1_stagnation_locks", C.c_int64), ("spmm_plan_cached", C.c_int),
                ("class_flops", C.c_double * 12), ("class_bytes", C.c_double * 12), ("inner_solves", C.c_int64),
                ("inner_steps", C.c_int64), ("inner2_solves", C.c_int64), ("inner2_steps", C.c_int64),
                ("spmm_schedule_f32", C.c_int), ("dynamic_route", C.c_int), ("dynamic_runs", C.c_int),
                ("dynamic_switches", C.c_int)]

    def as_dict(self) -> dict:
        d = {}
        for f, _ in self._fields_:
            v = getattr(self, f)
            d[f] = list(v) if hasattr(v, "__len__") else v
        return d


class Csr(C.Structure):
    _fields_ = [("m", C.c_int64), ("n", C.c_int64), ("nnz", C.c_int64), ("row_ptr", C.c_void_p),
                ("col_idx", C.c_void_p), ("val", C.c_void_p)]


class Result(C.Structure):
    _fields_ = [("sigma", C.c_void_p), ("U", C.c_void_p), ("V", C.c_void_p), ("resid", C.c_void_p),
                ("status", C.c_int), ("message", C.c_char * 160), ("stats", Stats)]


class PhsvdsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"phsvds status {status}: {msg}")
        self.status = status


def _load() -> C.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libphsvds.so is not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = C.CDLL(LIB_PATH)
    P, I64, I, D = C.c_void_p, C.c_int64, C.c_int, C.c_double
    sig = {
        "phsvds_create": ([C.POINTER(C.c_void_p), I, P], I),
        "phsvds_default_opts": ([C.POINTER(Opts)], I),
        "phsvds_solve": ([P, I64, I64, I64, P, P, P, I, I, I, D, I, C.POINTER(Opts), P, P, P, P,
                          C.POINTER(Stats)], I),
        "phsvds_normal_cg": ([P, I64, I64, I64, P, P, P, I, D, I, P, P, D, I, P], I),
        "phsvds_cnn_forward": ([P, I, I, I, P, P, P, P], I),
        "phsvds_cnn_backward": ([P, I, I, I, P, P, P, P, P, P, P], I),
        "phsvds_cnn_adam": ([P, P, P, P, P, I, C.c_float, C.c_float, C.c_float, C.c_float, P], I),
        "phsvds_solve_batched": ([P, I, C.POINTER(Csr), I, I, I, D, I, C.POINTER(Opts), I, C.POINTER(Result)], I),
        "phsvds_ata_spmm_f64": ([P, I, I, I, I64, I64, I64, P, P, P, P, P, P, I, P, P, P], I),
        "phsvds_ata_spmm_f32": ([P, I, I, I, I64, I64, I64, P, P, P, P, P, P, I, P, P, P], I),
        "phsvds_ata_spmm_static_f64": ([P, I64, I64, I64, P, P, P, P, P, P, I, P, P], I),
        "phsvds_csr_to_csc_f64": ([P, I64, I64, I64, P, P, P, P, P, P], I),
        "phsvds_jacobi_eig_f64": ([P, I, P, P, P, D, I, P], I),
        "phsvds_jacobi_eig_cluster_f64": ([P, I, P, P, P, D, I, P], I),
        "phsvds_jacobi_svd_f64": ([P, I, P, P, P, D, I, P], I),
        "phsvds_refined_vector_f64": ([P, I, P, I, P, P, I, I, D, P, P, P], I),
        "phsvds_block_cgs_f64": ([P, I64, P, I, I, P, I, I, P, I, I, P, P, P], I),
        "phsvds_block_cgs_f32": ([P, I64, P, I, I, P, I, I, P, I, I, P, P, P], I),
        "phsvds_tall_small_f64": ([P, I64, P, I, I, P, I, I, P, I, P, I, P, P], I),
        "phsvds_tall_small_f32": ([P, I64, P, I, I, P, I, I, P, I, P, I, P, P], I),
        "phsvds_sync": ([P], I),
        "phsvds_last_error": ([P], C.c_char_p),
        "phsvds_status_string": ([I], C.c_char_p),
        "phsvds_destroy": ([P], None),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


_lib = None


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        _lib = _load()
    return _lib


EXPORTED = ["phsvds_create", "phsvds_default_opts", "phsvds_solve", "phsvds_solve_batched", "phsvds_normal_cg",
            "phsvds_cnn_forward", "phsvds_cnn_backward", "phsvds_cnn_adam", "phsvds_ata_spmm_f64",
            "phsvds_ata_spmm_f32", "phsvds_ata_spmm_static_f64", "phsvds_csr_to_csc_f64", "phsvds_jacobi_eig_f64", "phsvds_jacobi_eig_cluster_f64",
            "phsvds_jacobi_svd_f64", "phsvds_refined_vector_f64", "phsvds_block_cgs_f64", "phsvds_block_cgs_f32",
            "phsvds_tall_small_f64", "phsvds_tall_small_f32", "phsvds_sync", "phsvds_last_error",
            "phsvds_status_string", "phsvds_destroy"]


def _ptr(x) -> int | None:
    """Address of a numpy array or of a torch tensor (device or host); None for None."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    raise TypeError(type(x))


class Handle:
    """A library context on one CUDA device (phsvds_create / phsvds_destroy)."""

    def __init__(self, device: int = 0, stream: int | None = None):
        self.h = C.c_void_p()
        st = lib().phsvds_create(C.byref(self.h), device, C.c_void_p(stream) if stream else None)
        if st != PHSVDS_OK:
            raise PhsvdsError(st, "phsvds_create failed")

    def check(self, st: int):
        if st != PHSVDS_OK:
            raise PhsvdsError(st, lib().phsvds_last_error(self.h).decode())

    def close(self):
        if self.h:
            lib().phsvds_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def default_opts(**kw) -> Opts:
    o = Opts()
    lib().phsvds_default_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def phsvds_solve(h: Handle, m, n, row_ptr, col_idx, val, k, target=SMALLEST, tol=1e-14,
                 precond=PREC_NONE, opts: Opts | None = None, on_device=False, want_vectors=True,
                 raise_on_error=True, init_V=None, precond_M=None):
    """phsvds_solve: k smallest / largest triplets of the m x n CSR matrix.

    row_ptr int64 (m+1), col_idx int32, val float64, as numpy arrays (host) or
    torch CUDA tensors (on_device=True).  init_V: optional n x c host array,
    the initial guess of stage 1 (opts.init_V / init_nv); precond_M: the
    diagonal of a given M ~ A for precond=PREC_GIVEN (opts.precond_M).
    Returns (sigma, U, V, resid, stats, status).
    """
    nnz = int(row_ptr[-1]) if isinstance(row_ptr, np.ndarray) else int(row_ptr[-1].item())
    sigma = np.zeros(k)
    U = np.zeros((k, m)) if want_vectors else None     # row i = u_i (column-major m x k)
    V = np.zeros((k, n)) if want_vectors else None
    resid = np.zeros(k)
    st = Stats()
    o = opts if opts is not None else default_opts()
    x0 = None
    if precond_M is not None:
        pm = np.ascontiguousarray(np.asarray(precond_M, dtype=np.float64))
        o = Opts.from_buffer_copy(o)
        o.precond_M = pm.ctypes.data
    if init_V is not None:
        x0 = np.asfortranarray(np.asarray(init_V, dtype=np.float64).reshape(n, -1))
        o2 = Opts.from_buffer_copy(o)
        o2.init_V = x0.ctypes.data
        o2.init_nv = x0.shape[1]
        o = o2
    status = lib().phsvds_solve(h.h, m, n, nnz, _ptr(row_ptr), _ptr(col_idx), _ptr(val), 1 if on_device else 0,
                                k, target, tol, precond, C.byref(o), _ptr(sigma), _ptr(U), _ptr(V),
                                _ptr(resid), C.byref(st))
    if raise_on_error:
        h.check(status)
    return sigma, (U.T if U is not None else None), (V.T if V is not None else None), resid, st.as_dict(), status


def phsvds_solve_batched(h: Handle, mats, k, target=SMALLEST, tol=1e-14, precond=PREC_NONE,
                         opts: Opts | None = None, concurrency=0, on_device=False, want_vectors=False,
                         raise_on_error=True):
    """phsvds_solve_batched over a list of (m, n, row_ptr, col_idx, val) CSR
    matrices (numpy host arrays, or torch CUDA tensors with on_device=True).
    Returns (list of per-matrix (sigma, U, V, resid, stats, status, message),
    overall status)."""
    cnt = len(mats)
    arr = (Csr * cnt)()
    res = (Result * cnt)()
    keep = []
    for i, (m, n, rp, ci, va) in enumerate(mats):
        nnz = int(rp[-1]) if isinstance(rp, np.ndarray) else int(rp[-1].item())
        arr[i] = Csr(m, n, nnz, _ptr(rp), _ptr(ci), _ptr(va))
        sig, rs = np.zeros(k), np.zeros(k)
        U = np.zeros((k, m)) if want_vectors else None
        V = np.zeros((k, n)) if want_vectors else None
        keep.append((sig, U, V, rs))
        res[i].sigma, res[i].resid = _ptr(sig), _ptr(rs)
        res[i].U, res[i].V = _ptr(U), _ptr(V)
    o = opts if opts is not None else default_opts()
    status = lib().phsvds_solve_batched(h.h, cnt, arr, 1 if on_device else 0, k, target, tol, precond, C.byref(o),
                                        concurrency, res)
    if raise_on_error and status != PHSVDS_OK:
        bad = [(i, res[i].status, res[i].message.decode()) for i in range(cnt) if res[i].status != PHSVDS_OK]
        raise PhsvdsError(status, f"batched solve: {len(bad)} failed, first {bad[:1]}")
    out = []
    for i in range(cnt):
        sig, U, V, rs = keep[i]
        out.append((sig, U.T if U is not None else None, V.T if V is not None else None, rs,
                    res[i].stats.as_dict(), res[i].status, res[i].message.decode()))
    return out, status


def phsvds_normal_cg(h: Handle, m, n, row_ptr, col_idx, val, R, shift=0.0, rtol=1e-6, maxit=10000,
                     on_device=False, raise_on_error=True):
    """x_i = (A^T A - shift I)^{-1} r_i for the columns of R (host n x count)
    by device CG; returns (X, iterations, status)."""
    R = np.asfortranarray(np.asarray(R, dtype=np.float64).reshape(n, -1))
    cnt = R.shape[1]
    X = np.zeros((n, cnt), order="F")
    its = np.zeros(cnt, dtype=np.int32)
    nnz = int(row_ptr[-1]) if isinstance(row_ptr, np.ndarray) else int(row_ptr[-1].item())
    st = lib().phsvds_normal_cg(h.h, m, n, nnz, _ptr(row_ptr), _ptr(col_idx), _ptr(val), 1 if on_device else 0,
                                shift, cnt, _ptr(R), _ptr(X), rtol, maxit, _ptr(its))
    if raise_on_error:
        h.check(st)
    return X, its, st


def phsvds_cnn_forward(h: Handle, batch, nx, ny, params, x, y, work):
    """Network forward on device tensors (x: batch x 4 x ny x nx float32, y:
    batch x ny x nx, params: 3024 bf16, work: cnn_work_floats floats)."""
    h.check(lib().phsvds_cnn_forward(h.h, batch, nx, ny, _ptr(params), _ptr(x), _ptr(y), _ptr(work)))


def phsvds_cnn_backward(h: Handle, batch, nx, ny, params, x, y, t, work, grad, loss):
    h.check(lib().phsvds_cnn_backward(h.h, batch, nx, ny, _ptr(params), _ptr(x), _ptr(y), _ptr(t), _ptr(work),
                                      _ptr(grad), _ptr(loss)))


def phsvds_cnn_adam(h: Handle, w, grad, m, v, step, lr, params, beta1=0.9, beta2=0.999, eps=1e-8):
    h.check(lib().phsvds_cnn_adam(h.h, _ptr(w), _ptr(grad), _ptr(m), _ptr(v), step, lr, beta1, beta2, eps,
                                  _ptr(params)))


def phsvds_ata_spmm(h: Handle, schedule, m, n, nnz, rp32, ci, va, cp, ri, cv, b, X, Y, z=None, fp32=False,
                    lanes_a=0, lanes_at=0):
    """Kernel-level Y = A^T (A X) on device tensors (row-major n x b blocks)."""
    f = lib().phsvds_ata_spmm_f32 if fp32 else lib().phsvds_ata_spmm_f64
    h.check(f(h.h, schedule, lanes_a, lanes_at, m, n, nnz, _ptr(rp32), _ptr(ci), _ptr(va), _ptr(cp), _ptr(ri),
              _ptr(cv), b, _ptr(X), _ptr(Y), _ptr(z)))


# Capacity (doubles) of the fixed scratch of phsvds_ata_spmm_static_f64: m * b <= this.
STATIC_Z_MAX = 262144


def phsvds_ata_spmm_static(h: Handle, m, n, nnz, rp32, ci, va, cp, ri, cv, b, X, Y):
    """Y = A^T (A X) in FP64 without any device allocation (two-phase schedule,
    intermediate A X in the library's fixed scratch; needs m * b <= STATIC_Z_MAX).
    Calls that can overlap in time race on that one scratch per device."""
    h.check(lib().phsvds_ata_spmm_static_f64(h.h, m, n, nnz, _ptr(rp32), _ptr(ci), _ptr(va), _ptr(cp), _ptr(ri),
                                             _ptr(cv), b, _ptr(X), _ptr(Y)))


def phsvds_csr_to_csc(h: Handle, m, n, nnz, rp32, ci, va, cp, ri, cv):
    h.check(lib().phsvds_csr_to_csc_f64(h.h, m, n, nnz, _ptr(rp32), _ptr(ci), _ptr(va), _ptr(cp), _ptr(ri),
                                        _ptr(cv)))


def phsvds_jacobi_eig(h: Handle, j, H, S, theta, tol=1e-17, max_sweeps=60, sweeps=None, cluster=False):
    f = lib().phsvds_jacobi_eig_cluster_f64 if cluster else lib().phsvds_jacobi_eig_f64
    h.check(f(h.h, j, _ptr(H), _ptr(S), _ptr(theta), tol, max_sweeps, _ptr(sweeps)))


def phsvds_jacobi_svd(h: Handle, j, G, S, sig, tol=1e-15, max_sweeps=60, sweeps=None):
    h.check(lib().phsvds_jacobi_svd_f64(h.h, j, _ptr(G), _ptr(S), _ptr(sig), tol, max_sweeps, _ptr(sweeps)))


def phsvds_refined_vector(h: Handle, j, R, ldr, x0, H, ldh, s1, out, maxit=24, tau=1e-10, steps=None):
    """Refined vector of R (device tensors): s1, out = (theta1, ||R s1||)."""
    h.check(lib().phsvds_refined_vector_f64(h.h, j, _ptr(R), ldr, _ptr(x0), _ptr(H), ldh, maxit, tau, _ptr(s1),
                                            _ptr(out), _ptr(steps)))


def phsvds_block_cgs(h: Handle, n, P1, ld1, p1, T, ldt, q, Gsub=None, Gout=None, Tout=None, P2=None, ld2=0, p2=0,
                     fp32=False):
    """One block CGS pass on device tensors (column-major blocks given by
    pointer, leading dimension and column count; Gsub/Gout/Tout FP64)."""
    f = lib().phsvds_block_cgs_f32 if fp32 else lib().phsvds_block_cgs_f64
    h.check(f(h.h, n, _ptr(P1), ld1, p1, _ptr(P2), ld2, p2, _ptr(T), ldt, q, _ptr(Gsub), _ptr(Gout), _ptr(Tout)))


def phsvds_tall_small(h: Handle, n, P, ldp, p, Y, ldy, r, Out, ldo, Xs=None, ldx=0, theta=None, norms2=None,
                      fp32=False):
    """Out = P Y - Xs diag(theta) (+ column norms^2) on device tensors."""
    f = lib().phsvds_tall_small_f32 if fp32 else lib().phsvds_tall_small_f64
    h.check(f(h.h, n, _ptr(P), ldp, p, _ptr(Y), ldy, r, _ptr(Out), ldo, _ptr(Xs), ldx, _ptr(theta),
              _ptr(norms2)))


def phsvds_sync(h: Handle):
    h.check(lib().phsvds_sync(h.h))
