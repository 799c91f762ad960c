"""Plain CPU FP64 restatement of the PHSVDS method -- oracle code.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline
leg of the benchmark may import this module.  It shares no code with the GPU
path; sparse products (scipy CSR @ dense) and the symmetric eigensolver and SVD
of the small projected matrices (numpy/LAPACK) serve as library primitives.

Paper: L. Wu and A. Stathopoulos, "A preconditioned hybrid SVD method for
computing accurately singular triplets of large matrices" (arXiv 1408.5535).

Steps, in the paper's order:
* stage 1 (Algorithm 1): block GD+k on C = A^T A, convergence test with the
  dynamic tolerance delta_C = max(delta * s_i / s_n, eps) (Sec. 3.1, eq. for
  delta_C, Algorithm 1 step 2), then an optional Rayleigh-Ritz on the returned
  basis (Algorithm 1 step 3, Sec. 3.1);
* switch test delta < eps ||A|| / s_i (Sec. 3.1);
* stage 2 (Algorithm 2): GD on B = [0 A^T; A 0] with the refined projection
  min ||(B - s I) V y|| through an incrementally updated QR of W - s V, one
  target at a time, locking and re-introduction of the next initial guess;
  the basis grows by the residual (GD) or, in the JDQMR form of Sec. 4, by
  an inexact solution of the Jacobi-Davidson correction equation (symmetric
  QMR with a dynamic stop: a READING);
* stage 1 may also grow its basis by the Jacobi-Davidson correction of Sec.
  4 (jd1_correction: symmetric QMR on the projected, shifted C, Jacobi-scaled
  when preconditioned; READINGs), and ||A|| of the user requirement may come
  from a Lanczos estimate (lanczos_norm_c, a READING);
* preconditioning (Sec. 4): Jacobi on C with the Olsen correction; from a
  given M ~ A, M^-1 M^-T for C and [0 M^-1; M^-T 0] for B; from C's Jacobi
  M ~ C^-1, [0 A M; M A^T 0] for B in stage 2;
* Algorithm 3 (Sec. 4): dynamic switching between GD+k on C and on B under
  preconditioning (dynamic_phsvds);
* final triplet test sqrt(||r_u||^2 + ||r_v||^2) < ||A|| delta (Sec. 5).

GD+k itself is named but not defined in the paper (Sec. 2.2, Sec. 5: "GD+k",
"GD_Olsen_PlusK"); the restart with k previous Ritz vectors and the Olsen form
of the correction follow the method as its authors published it
(Stathopoulos, SIAM J. Sci. Comput. 29(2), 2007).

Readings where the paper is silent are marked READING and listed with the
design notes of the repository.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np
import scipy.sparse as sp

EPS64 = 2.0 ** -52
EPS32 = 2.0 ** -23

# SplitMix64 streams for the random vectors the method itself draws.
RS_INIT = 0x1000    # columns 2..b of the initial block
RS_BREAK = 0x2000   # replacement of a numerically dependent new basis vector
RS_U = 0x3000       # random left vector for an (extremely) small sigma
RS_NORM = 0x4000    # start vector of the Lanczos estimate of ||C|| (Opts.norm_A < 0)


# ---------------------------------------------------------------------------
# random vectors the method draws (counter-based SplitMix64, Vigna's constants)
# ---------------------------------------------------------------------------

def _splitmix(seed: int, stream: int, count: int) -> np.ndarray:
    mask = (1 << 64) - 1
    with np.errstate(over="ignore"):
        key = np.uint64(seed & mask) ^ (np.uint64(stream & mask) * np.uint64(0xD1B54A32D192ED03))
        z = np.arange(1, count + 1, dtype=np.uint64) * np.uint64(0x9E3779B97F4A7C15) + key
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def rand_vec(seed: int, stream: int, n: int) -> np.ndarray:
    """Uniform entries in [-1, 1): 2 * (top 53 bits * 2^-53) - 1."""
    z = _splitmix(seed, stream, n)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 / 9007199254740992.0) - 1.0


# ---------------------------------------------------------------------------
# operators
# ---------------------------------------------------------------------------

def as_scipy(csr) -> sp.csr_matrix:
    return sp.csr_matrix((np.asarray(csr.val, dtype=np.float64), np.asarray(csr.col),
                          np.asarray(csr.row_ptr)), shape=(csr.m, csr.n))


class Ops:
    """Products with C = A^T A and B = [0 A^T; A 0] (Section 1), counting matvecs.

    ``mv_A`` / ``mv_At`` count products of one vector with A and with A^T.
    """

    def __init__(self, A: sp.csr_matrix):
        self.A = A
        self.At = A.T.tocsr()
        self.m, self.n = A.shape
        self.mv_A = 0
        self.mv_At = 0

    def C(self, X: np.ndarray) -> np.ndarray:
        X = X.reshape(self.n, -1)
        self.mv_A += X.shape[1]
        self.mv_At += X.shape[1]
        return self.At @ (self.A @ X)

    def B(self, X: np.ndarray) -> np.ndarray:
        X = X.reshape(self.m + self.n, -1)
        n = self.n
        self.mv_A += X.shape[1]
        self.mv_At += X.shape[1]
        return np.vstack([self.At @ X[n:], self.A @ X[:n]])

    def Av(self, v):
        self.mv_A += 1 if v.ndim == 1 else v.shape[1]
        return self.A @ v

    def Atu(self, u):
        self.mv_At += 1 if u.ndim == 1 else u.shape[1]
        return self.At @ u


# ---------------------------------------------------------------------------
# orthogonalisation (classical Gram-Schmidt applied twice)
# ---------------------------------------------------------------------------

def orth_append(Q: np.ndarray, T: np.ndarray, seed: int, counter: list, drop_tol: float = 1e-10):
    """Orthonormalise the columns of T, one at a time, against Q and each other.

    Each column gets two passes of classical Gram-Schmidt against all previous
    columns, then is normalised.  A column whose remaining norm is below
    drop_tol times its input norm is numerically dependent; it is replaced by a
    random vector (stream RS_BREAK + counter) and orthogonalised again.
    """
    basis = Q
    out = []
    for c in range(T.shape[1]):
        t = T[:, c].copy()
        for attempt in range(4):
            nin = np.linalg.norm(t)
            for _ in range(2):
                if basis.shape[1]:
                    t = t - basis @ (basis.T @ t)
            nout = np.linalg.norm(t)
            if nin > 0 and nout > drop_tol * nin:
                break
            t = rand_vec(seed, RS_BREAK + counter[0], T.shape[0])
            counter[0] += 1
        t = t / np.linalg.norm(t)
        out.append(t)
        basis = np.column_stack([basis, t]) if basis.shape[1] else t[:, None]
    return np.column_stack(out) if out else np.zeros((T.shape[0], 0))


def qr_cgs2(Z: np.ndarray, seed: int, counter: list):
    """Z = Q R, column by column with classical Gram-Schmidt applied twice.

    A column that is numerically in the span of the previous ones keeps its
    (tiny) R diagonal and gets a random orthonormal completion for q.
    """
    N, j = Z.shape
    Q = np.zeros((N, j))
    R = np.zeros((j, j))
    for c in range(j):
        Q[:, c], R[:c + 1, c] = qr_add_column(Q[:, :c], Z[:, c], seed, counter)
    return Q, R


def qr_add_column(Q: np.ndarray, z: np.ndarray, seed: int, counter: list):
    """One-column update of a QR factorisation (Algorithm 2, step 8)."""
    c = Q.shape[1]
    r = np.zeros(c + 1)
    q = z.copy()
    for _ in range(2):
        if c:
            h = Q.T @ q
            q = q - Q @ h
            r[:c] += h
    rho = np.linalg.norm(q)
    r[c] = rho
    if rho > 1e-300 and rho > 1e-14 * np.linalg.norm(z):
        q = q / rho
    else:
        # numerically dependent column: keep R, complete Q with a random direction
        q = orth_append(Q, rand_vec(seed, RS_BREAK + counter[0], z.size)[:, None], seed, counter)[:, 0]
        counter[0] += 1
    return q, r


# ---------------------------------------------------------------------------
# options / results
# ---------------------------------------------------------------------------

@dataclass
class Opts:
    block: int = 1              # block size of stage 1
    max_basis: int = 35         # maxBasisSize (Sec. 5)
    min_restart: int = 21       # minRestartSize (Sec. 5)
    max_restarts: int = 10000   # per stage (Sec. 5)
    eps_factor: float = 4.0     # READING: delta_C floor is eps_factor * eps (O(||C|| eps), Sec. 3.1)
    stage1_eps: float = EPS64   # unit roundoff of stage 1 (EPS32 for the mixed form)
    rr: bool = True             # Algorithm 1 step 3
    stage2: bool = True         # False: stage 1 only
    precond: str = "none"       # "none", "jacobi" (diag(C) - theta)^-1, or "given" (below); Olsen form
    precond_M: object = None    # "given": diagonal of M ~ A (square A); C gets M^-1 M^-T, B gets [0 M^-1; M^-T 0]
    seed: int = 0
    max_iters: int = 10 ** 7
    trace: object = None        # optional callable(stage, iteration, info dict)
    stage2_inner: str = "none"  # "none": GD, t = r; "qmr": JDQMR, t from the correction equation (Sec. 4)
    inner_maxit: int = 300      # READING: inner QMR steps per outer iteration, at most
    stage2_precond: bool = False  # smallest targets: GD stage 2 preconditioned by [0 M A^T; A M 0], M = diag(C)^-1 (Sec. 4)
    stage1_inner: str = "none"  # "minres": stage 1 expands by the Jacobi-Davidson correction (Sec. 4), jd1_correction
    inner1_maxit: int = 60      # READING: inner steps per stage-1 correction, at most
    inner1_tol: float = 1e-3    # READING: ... or until the inner residual has fallen by this factor
    norm_A: float = 0.0         # ||A|| of the user requirement: 0 the largest Ritz value of stage 1, > 0 given,
                                # < 0 also the Lanczos estimate lanczos_norm_c (READING, Sec. 3.1)


@dataclass
class Result:
    sigma: np.ndarray
    U: np.ndarray
    V: np.ndarray
    resid: np.ndarray                 # sqrt(||r_u||^2 + ||r_v||^2) per triplet
    normA: float
    stats: dict = field(default_factory=dict)


# ---------------------------------------------------------------------------
# stage 1: block GD+k on a symmetric operator
# ---------------------------------------------------------------------------

def gdk(apply_op, n: int, k: int, largest: bool, tol_fn, o: Opts, diagC=None, X0=None,
        stats=None, order_key=None, apply_prec=None, stop_after=None, history=None):
    """Block GD+k for the k extreme eigenpairs of a symmetric operator.

    Per iteration: Rayleigh-Ritz on the basis V (H = V^T W, W = op(V)); the
    first b unconverged Ritz pairs in target order are the block; residuals
    r = W s - theta V s; converged pairs are locked (moved out of the basis);
    when the basis would exceed max_basis it is restarted with the
    min_restart - b best Ritz vectors plus the b Ritz vectors of the previous
    iteration (the "+k" of GD+k); the correction is t = r (no preconditioner)
    or the Olsen form t = M r - e M x, e = x^T M r / x^T M x, with
    M = (diag(C) - theta I)^-1.  New vectors are orthonormalised against the
    locked vectors and the basis (classical Gram-Schmidt twice).

    tol_fn(theta_i, theta_max) gives the residual threshold of Ritz value
    theta_i, theta_max being the largest Ritz value seen (the ||C|| estimate).
    Returns (lam (k,), X (n x k), state) with the final basis in ``state``.

    Hooks for the dynamic method (Algorithm 3; all default to the plain
    behaviour): order_key(theta) -> sort keys replaces the smallest/largest
    target order (interior targets of B); apply_prec(r, x) -> t replaces the
    correction; stop_after = N ends the run after N iterations and returns
    the k best current approximations (locked ones first) with
    state["nconv"] = the number locked; history collects the residual norm
    of the first unconverged target at every iteration.
    """
    stats = {} if stats is None else stats
    b = max(1, min(o.block, k))
    maxb, mins, kp = o.max_basis, o.min_restart, max(1, min(o.block, k))
    counter = [0]
    Xl = np.zeros((n, 0))
    lam_l = []
    V = np.zeros((n, 0))
    W = np.zeros((n, 0))
    H = np.zeros((0, 0))
    if X0 is not None:
        T = np.array(X0, dtype=np.float64).reshape(n, -1)
    else:
        T = np.empty((n, b))
        T[:, 0] = 1.0 / math.sqrt(n)           # ones(n,1) start (Sec. 5), normalised
        for c in range(1, b):
            T[:, c] = rand_vec(o.seed, RS_INIT + c, n)
    s_prev = np.zeros((0, 0))
    theta_max = 0.0
    it = restarts = 0
    theta = np.zeros(0)
    S = np.zeros((0, 0))
    while True:
        # ---- expand the basis with the new block
        if T.shape[1]:
            Tn = orth_append(np.hstack([Xl, V]), T, o.seed, counter)
            Wn = apply_op(Tn)
            Hvw = V.T @ Wn
            Htt = Tn.T @ Wn
            Htt = 0.5 * (Htt + Htt.T)
            j0 = V.shape[1]
            H = np.block([[H, Hvw], [Hvw.T, Htt]]) if j0 else Htt
            V = np.hstack([V, Tn])
            W = np.hstack([W, Wn])
            if s_prev.shape[1]:
                s_prev = np.vstack([s_prev, np.zeros((Tn.shape[1], s_prev.shape[1]))])
        j = V.shape[1]
        # ---- Rayleigh-Ritz
        theta, S = np.linalg.eigh(H)
        if order_key is not None:
            o_ = np.argsort(order_key(theta), kind="stable")
            theta, S = theta[o_], S[:, o_]
        elif largest:
            theta, S = theta[::-1], S[:, ::-1]
        theta_max = max(theta_max, float(np.max(np.abs(theta))))
        it += 1
        nt = min(b, k - len(lam_l), j)
        X = V @ S[:, :nt]
        R = W @ S[:, :nt] - X * theta[:nt]
        rn = np.linalg.norm(R, axis=0)
        conv = [i for i in range(nt) if rn[i] < tol_fn(theta[i], theta_max)]
        unconv = [i for i in range(nt) if i not in conv]
        if history is not None and unconv:
            history.append(float(rn[unconv[0]]))
        if o.trace is not None:
            o.trace(1, it, dict(j=j, nlock=len(lam_l), theta0=float(theta[0]), rnorm0=float(rn[0]),
                                theta_max=theta_max, nconv=len(conv)))
        for i in conv:
            Xl = np.column_stack([Xl, X[:, i]])
            lam_l.append(float(theta[i]))
        if len(lam_l) >= k:
            stats.update(iters=it, restarts=restarts, theta_max=theta_max)
            order = np.argsort(lam_l)
            if largest:
                order = order[::-1]
            state = dict(V=V, W=W, theta=theta, S=S, conv=conv)
            return np.array(lam_l)[order], Xl[:, order], state
        if stop_after is not None and it >= stop_after:
            nfree = k - len(lam_l)
            cand = [c for c in range(j) if c not in conv][:nfree]
            Xk = np.column_stack([Xl, V @ S[:, cand]]) if Xl.shape[1] else V @ S[:, cand]
            lk = np.concatenate([np.array(lam_l), theta[cand]])
            stats.update(iters=it, restarts=restarts, theta_max=theta_max)
            return lk, Xk, dict(V=V, W=W, theta=theta, S=S, conv=conv, nconv=len(lam_l), partial=True)
        if it >= o.max_iters:
            raise RuntimeError("stage 1: iteration limit")
        keep_all = [c for c in range(j) if c not in conv]
        Y = None
        if len(keep_all) + len(unconv) > maxb:
            # ---- thick restart with +k previous Ritz vectors
            restarts += 1
            if restarts > o.max_restarts:
                raise RuntimeError("stage 1: restart limit")
            nkeep = min(mins - kp, len(keep_all))
            Yk = S[:, keep_all[:nkeep]]
            cols = [Yk]
            if s_prev.shape[1]:
                P = s_prev.copy()
                Sc = S[:, conv]
                basis = np.hstack([Sc, Yk])
                for c in range(P.shape[1]):
                    p = P[:, c]
                    for _ in range(2):
                        p = p - basis @ (basis.T @ p)
                    nrm = np.linalg.norm(p)
                    if nrm > 1e-8:
                        p = p / nrm
                        basis = np.column_stack([basis, p])
                        cols.append(p[:, None])
            Y = np.hstack(cols)
        elif conv:
            Y = S[:, keep_all]
        if Y is not None:
            V = V @ Y
            W = W @ Y
            H = Y.T @ H @ Y
            H = 0.5 * (H + H.T)
            s_prev = Y.T @ S[:, unconv]
        else:
            s_prev = S[:, unconv].copy()
        # ---- corrections for the unconverged targets
        if unconv:
            Ru = R[:, unconv]
            Xu = X[:, unconv]
            if apply_prec is not None:
                T = np.column_stack([apply_prec(Ru[:, c], Xu[:, c]) for c in range(len(unconv))])
            elif o.stage1_inner == "minres" and o.precond in ("none", "jacobi"):
                # the Jacobi-Davidson correction of each target (Sec. 4), with
                # the Jacobi scaling when preconditioned (jd1_correction)
                sc = None
                if o.precond == "jacobi" and diagC is not None:
                    guard = EPS64 * max(theta_max, 1e-300)
                    sc = 1.0 / np.sqrt(np.maximum(diagC, guard))
                T = np.empty_like(Ru)
                for c, i in enumerate(unconv):
                    Q = np.column_stack([Xl, Xu]) if sc is not None else np.column_stack([Xl, Xu[:, c]])
                    T[:, c] = jd1_correction(apply_op, Q, float(theta[i]), Ru[:, c], sc, o.inner1_maxit,
                                             o.inner1_tol, stats)
            elif o.precond == "given" and o.precond_M is not None:
                # M^-1 M^-T for C (Sec. 4), shift-free, Olsen form
                m2 = np.asarray(o.precond_M, dtype=np.float64) ** 2
                T = np.empty_like(Ru)
                for c in range(len(unconv)):
                    Mr = Ru[:, c] / m2
                    Mx = Xu[:, c] / m2
                    T[:, c] = Mr - (float(Xu[:, c] @ Mr) / float(Xu[:, c] @ Mx)) * Mx
            elif o.precond == "jacobi" and diagC is not None:
                T = np.empty_like(Ru)
                for c, i in enumerate(unconv):
                    d = diagC - theta[i]
                    guard = EPS64 * max(theta_max, 1e-300)
                    d = np.where(np.abs(d) < guard, np.where(d < 0, -guard, guard), d)
                    Mr = Ru[:, c] / d
                    Mx = Xu[:, c] / d
                    e = float(Xu[:, c] @ Mr) / float(Xu[:, c] @ Mx)
                    T[:, c] = Mr - e * Mx
            else:
                T = Ru.copy()
        else:
            T = np.zeros((n, 0))


def stage1_tol(delta: float, o: Opts):
    """Algorithm 1 step 2: ||r_C|| < delta_C ||C||, delta_C = max(delta s_i/s_n, eps).

    With ||C|| ~ s_n^2 = theta_max this is ||r_C|| < max(delta s_i s_n, eps theta_max).
    READING: the floor is eps_factor * eps (the attainable O(||C|| eps) of Sec. 3.1).
    """
    floor = o.eps_factor * o.stage1_eps

    def tol(theta_i, theta_max):
        s_i = math.sqrt(max(theta_i, 0.0))
        s_n = math.sqrt(max(theta_max, 0.0))
        return max(delta * s_i * s_n, floor * theta_max)

    return tol


def rayleigh_ritz_post(ops: Ops, Xl: np.ndarray, state: dict, k: int, largest: bool, o: Opts):
    """Algorithm 1 step 3: Rayleigh-Ritz of C on the returned basis.

    READING: the basis is the k locked vectors plus the min_restart - k best
    remaining Ritz vectors of the final basis (min_restart vectors in all, the
    "21 extra matrix-vector operations" of Sec. 5.3), with fresh products.
    """
    V, S = state["V"], state["S"]
    conv = set(state["conv"])
    extra = max(0, min(o.min_restart - k, V.shape[1] - len(conv)))
    cols = [c for c in range(S.shape[1]) if c not in conv][:extra]
    Z = np.hstack([Xl, V @ S[:, cols]]) if cols else Xl
    Q = orth_append(np.zeros((Z.shape[0], 0)), Z, o.seed, [10 ** 6])
    WQ = ops.C(Q)
    Hq = Q.T @ WQ
    Hq = 0.5 * (Hq + Hq.T)
    th, Sq = np.linalg.eigh(Hq)
    if largest:
        th, Sq = th[::-1], Sq[:, ::-1]
    return th[:k], Q @ Sq[:, :k]


# ---------------------------------------------------------------------------
# stage 2: refined projection on B (Algorithm 2)
# ---------------------------------------------------------------------------

def symmetric_qmr(apply_M, b: np.ndarray, Qd: np.ndarray, steps: int):
    """Symmetric QMR iterates for M t = b, M symmetric on the complement of
    Qd (orthonormal columns), b orthogonal to Qd; a generator yielding, after
    step k, (t_k, ||b - M t_k||, the Lanczos basis, the coefficients y_k).

    Lanczos on M from b / ||b|| (each new vector orthogonalised twice against
    Qd and every earlier Lanczos vector), T_k the (k+1) x k tridiagonal, and
    y_k = argmin ||beta e_1 - T_k y||.  With a symmetric M and no
    preconditioner the Lanczos vectors are orthonormal, so the quasi-residual
    that QMR minimises is the true residual (the iterates are MINRES's).
    apply_M(q) returns (M q, extra) and the extras are handed back per step.
    """
    beta0 = float(np.linalg.norm(b))
    if not beta0 > 0:
        return
    Qs = [b / beta0]
    extras = []
    T = np.zeros((steps + 1, steps))
    for k in range(steps):
        w, extra = apply_M(Qs[k])
        extras.append(extra)
        T[k, k] = float(Qs[k] @ w)
        basis = np.column_stack([Qd] + Qs) if Qd.shape[1] else np.column_stack(Qs)
        for _ in range(2):
            w = w - basis @ (basis.T @ w)
        T[k + 1, k] = float(np.linalg.norm(w))
        if k + 1 < steps:
            T[k, k + 1] = T[k + 1, k]
        rhs = np.zeros(k + 2)
        rhs[0] = beta0
        y = np.linalg.lstsq(T[:k + 2, :k + 1], rhs, rcond=None)[0]
        g = float(np.linalg.norm(rhs - T[:k + 2, :k + 1] @ y))
        t = np.column_stack(Qs) @ y
        yield t, g, extras, y
        if not T[k + 1, k] > 1e-300:
            return
        Qs.append(w / T[k + 1, k])


def jd1_correction(apply_C, Q: np.ndarray, theta: float, r: np.ndarray, sc, maxit: int, tol: float,
                   stats: dict) -> np.ndarray:
    """Correction of stage 1 in its Jacobi-Davidson form (Sec. 4's JDQMR idea
    applied to C): an approximate solution t of the correction equation
        (I - QQ^T)(C - theta I)(I - QQ^T) t = r,
    r the residual of the Ritz pair (theta, x), Q orthonormal and containing
    x and the locked vectors, by symmetric QMR (MINRES's iterates here).
    READING (the paper names the inner solver and its inexact stopping but not
    the rule; these are the GPU library's): at most maxit steps, stopping once
    the inner residual has fallen to tol times its start.
    READING (the Jacobi preconditioner D = diag(C), sc = D^{-1/2}): the system
    is solved symmetrically in y = D^{1/2} t,
        D^{-1/2} P (C - theta I) P D^{-1/2} y = D^{-1/2} r,   P = I - QQ^T,
    and t = D^{-1/2} y; the scaled Lanczos vectors leave the complement of Q,
    so P acts on the operator's input as well as on its output, and Q holds
    the locked vectors and every Ritz vector of the block.  Returns t."""
    def proj(z):
        if Q.shape[1]:
            for _ in range(2):
                z = z - Q @ (Q.T @ z)
        return z

    def op(u):
        return apply_C(u[:, None])[:, 0] - theta * u

    if sc is None:
        def apply_M(q):
            return proj(op(proj(q))), None
        b = proj(r)
        Qd = Q
    else:
        def apply_M(q):
            return sc * proj(op(proj(sc * q))), None
        b = sc * r
        Qd = np.zeros((r.size, 0))
    beta0 = float(np.linalg.norm(b))
    t, k = None, 0
    for t_k, g, _, _ in symmetric_qmr(apply_M, b, Qd, maxit):
        k += 1
        t = t_k
        if g <= tol * beta0:
            break
    stats["inner1"] = stats.get("inner1", 0) + k
    if t is None:
        return r.copy()
    return t if sc is None else sc * t


def lanczos_norm_c(apply_C, n: int, seed: int, steps: int = 30) -> float:
    """An estimate of ||C|| = ||A||^2: the largest eigenvalue of the
    tridiagonal matrix of `steps` Lanczos steps on C from the seeded start
    rand_vec(seed, RS_NORM, n) (no reorthogonalisation, which the extreme
    Ritz value does not need).  A lower bound of ||C||.
    READING: the paper's stopping criterion ||r|| < delta ||A|| (Sec. 3.1,
    Sec. 5) needs ||A||; Algorithm 1 estimates it by its current largest Ritz
    value, which for the smallest triplets can sit far below ||A||; this
    estimate is the Opts.norm_A < 0 alternative."""
    v = rand_vec(seed, RS_NORM, n)
    v = v / np.linalg.norm(v)
    v0 = np.zeros(n)
    al, be = [], []
    beta = 0.0
    for i in range(max(1, min(steps, n))):
        w = apply_C(v[:, None])[:, 0]
        a = float(v @ w)
        w = w - a * v - beta * v0
        al.append(a)
        beta = float(np.linalg.norm(w))
        if i + 1 == steps or not beta > 1e-14 * abs(a):
            break
        be.append(beta)
        v0, v = v, w / beta
    T = np.diag(al) + np.diag(be, 1) + np.diag(be, -1)
    return float(np.max(np.linalg.eigvalsh(T)))


def jd_correction(ops: "Ops", Xl: np.ndarray, x: np.ndarray, Bx: np.ndarray, mu: float, r: np.ndarray,
                  tol: float, maxit: int, stats: dict, patience: int = 25) -> np.ndarray:
    """Correction of the Jacobi-Davidson method on B (Sec. 4, the correction
    equation (I - w w^T)(B - mu I)(I - w w^T) t = sigma~ w - B w with w the
    refined vector x, here also deflating the locked vectors Xl), solved
    inexactly by symmetric QMR with a dynamic stop.
    READING (the paper names JDQMR and its near-optimal inner stopping but
    states neither): after each inner step the updated vector
    z = (x + t_k) / ||x + t_k|| is scored by its eigen-residual
    eta_k = ||B z - (z^T B z) z|| (B t_k from the products the Lanczos steps
    already made); the steps stop once eta_k < tol, or once eta has not
    fallen below 0.9 times its best value for `patience` (25) steps in a
    row, or after maxit steps; the iterate with the smallest eta is
    returned.  A short patience cuts the solve off before it resolves a
    cluster near mu (the corrections then act like GD's)."""
    Qd = np.column_stack([Xl, x]) if Xl.shape[1] else x[:, None]

    def apply_M(q):
        bq = ops.B(q)[:, 0]
        w = bq - mu * q
        w = w - Qd @ (Qd.T @ w)
        return w, bq

    b = -(r - Qd @ (Qd.T @ r))
    best_t, best_eta, since = None, math.inf, 0
    k = 0
    for t, g, extras, y in symmetric_qmr(apply_M, b, Qd, maxit):
        k += 1
        z = x + t
        Bz = Bx + np.column_stack(extras) @ y
        nz = float(np.linalg.norm(z))
        z, Bz = z / nz, Bz / nz
        rho = float(z @ Bz)
        eta = float(np.linalg.norm(Bz - rho * z))
        if eta < 0.9 * best_eta:
            since = 0
        else:
            since += 1
        if eta < best_eta:
            best_t, best_eta = t, eta
        if best_eta < tol or since >= patience:
            break
    stats["inner2"] = stats.get("inner2", 0) + k
    return best_t if best_t is not None else r


def b_precond(ops: Ops, apply_M, y: np.ndarray) -> np.ndarray:
    """The stage-2 preconditioner built from a preconditioner M ~ C^{-1} of
    the first stage (Sec. 4): [0 A M; M A^T 0] in the paper's [u; v] order,
    i.e. y = [y_v; y_u] -> [M A^T y_u; A M y_v] in the [v; u] order used
    here.  With M = C^{-1} exactly it is a generalised inverse of B
    (B P B = B for A of full column rank)."""
    n = ops.n
    return np.concatenate([apply_M(ops.Atu(y[n:])), ops.Av(apply_M(y[:n]))])


def given_b_precond(Mdiag, n: int, y: np.ndarray) -> np.ndarray:
    """Stage-2 preconditioner from a given M ~ A (square A, diagonal M here):
    [0 M^-1; M^-T 0] (Sec. 4), which is B^-1 when M = A; in the [v; u] order,
    y = [y_v; y_u] -> [M^-1 y_u; M^-T y_v]."""
    mv = np.asarray(Mdiag, dtype=np.float64)
    return np.concatenate([y[n:] / mv, y[:n] / mv])


def stage2(ops: Ops, sig: np.ndarray, Vt: np.ndarray, normA: float, delta: float, o: Opts,
           stats: dict, diagC=None):
    """Algorithm 2 with a GD outer loop (the PHSVDS(GD+k) variant of Sec. 5).

    Targets are the k stage-1 values in the given order, one at a time, with
    shift s = the stage-1 value.  Per iteration: QR of W - s V (full at start,
    restart and new target; one-column update otherwise); eig of H ordered by
    closeness to s; smallest right singular vector s1 of R gives the refined
    vector x = V s1 and its Rayleigh quotient theta1 = s1^T H s1; the residual
    r = W s1 - theta1 V s1 decides locking (||r_B|| < delta ||A|| / sqrt(2),
    Sec. 3.1).  On locking the next initial guess is re-introduced.  The new
    direction is t = r.
    READINGS: restart keeps [s1, Ritz vectors closest to s, previous s1];
    the shift becomes theta1 at a restart once the residual is below that of
    the initial guess; b = 1.
    """
    m, n = ops.m, ops.n
    N = m + n
    k = sig.size
    mins, maxb = o.min_restart, o.max_basis
    counter = [2 * 10 ** 6]
    # ---- initial guesses [v; A v / s] / sqrt(2) (Algorithm 2 step 1, Sec. 3.3)
    x0 = np.zeros((N, k))
    for i in range(k):
        v = Vt[:, i] / np.linalg.norm(Vt[:, i])
        if sig[i] > math.sqrt(EPS64) * normA:
            u = ops.Av(v) / sig[i]
        else:
            u = rand_vec(o.seed, RS_U + i, m)   # Sec. 3.3: tiny sigma, random left vector
        u = u / np.linalg.norm(u)
        x0[:n, i] = v / math.sqrt(2.0)
        x0[n:, i] = u / math.sqrt(2.0)
    # ---- initial basis: K_{s-k}(B, x0_1) and the guesses (Algorithm 2 step 2)
    q = max(1, mins - k)
    V = orth_append(np.zeros((N, 0)), x0[:, :1], o.seed, counter)
    for _ in range(q - 1):
        V = np.hstack([V, orth_append(V, ops.B(V[:, -1]), o.seed, counter)])
    nguess = min(k - 1, maxb - 1 - V.shape[1])
    if nguess > 0:
        V = np.hstack([V, orth_append(V, x0[:, 1:1 + nguess], o.seed, counter)])
    W = ops.B(V)
    H = V.T @ W
    H = 0.5 * (H + H.T)
    Xl = np.zeros((N, 0))
    Xd = []            # JDQMR form: mirrors [v; -u] of locked tiny pairs, deflated too
    th_l = []
    target = 0
    shift = float(sig[0])
    qr_full = True
    Q = R = None
    s_prev = None
    r0 = None
    it = restarts = 0
    normA_est = normA
    while True:
        it += 1
        if it > o.max_iters:
            raise RuntimeError("stage 2: iteration limit")
        j = V.shape[1]
        if qr_full:
            Q, R = qr_cgs2(W - shift * V, o.seed, counter)
            qr_full = False
        theta, S = np.linalg.eigh(H)
        normA_est = max(normA_est, float(np.max(np.abs(theta))))
        order = np.argsort(np.abs(theta - shift), kind="stable")
        theta, S = theta[order], S[:, order]
        _, _, SRt = np.linalg.svd(R)
        s1 = SRt[-1]
        th1 = float(s1 @ H @ s1)
        x = V @ s1
        r = W @ s1 - th1 * x
        rn = float(np.linalg.norm(r))
        if r0 is None:
            r0 = rn
        if o.trace is not None:
            o.trace(2, it, dict(target=target, shift=shift, theta1=th1, rnorm=rn, j=j, restarts=restarts))
        if rn < delta * normA / math.sqrt(2.0):
            Xl = np.column_stack([Xl, x])
            th_l.append(th1)
            target += 1
            if target >= k:
                break
            Y = SRt[:-1].T                     # orthonormal complement of s1
            if o.stage2_inner == "qmr" and abs(th1) <= math.sqrt(EPS64) * normA:
                # READING (JDQMR form): for a tiny sigma the pair +-sigma of B
                # is not separable at the tolerance, and both eigenvectors
                # [v; +-u] belong to the same triplet: the mirror [v; -u] is
                # deflated as well, from the basis and from later directions
                mir = np.concatenate([x[:n], -x[n:]])
                Xd.append((mir / np.linalg.norm(mir))[:, None])
                D = np.column_stack([Xl] + Xd)
                V = V @ Y
                for _ in range(2):
                    V = V - D @ (D.T @ V)
                V = np.linalg.qr(V)[0]
                W = ops.B(V)
                H = V.T @ W
            else:
                V, W = V @ Y, W @ Y
                H = Y.T @ H @ Y
            H = 0.5 * (H + H.T)
            # re-introduce the next initial guess (Algorithm 2 step 9)
            t = orth_append(np.hstack([Xl] + Xd + [V]), x0[:, target:target + 1], o.seed, counter)
            wt = ops.B(t)
            H = np.block([[H, V.T @ wt], [wt.T @ V, t.T @ wt]])
            H = 0.5 * (H + H.T)
            V, W = np.hstack([V, t]), np.hstack([W, wt])
            shift = float(sig[target])
            qr_full = True
            s_prev = None
            r0 = None
            continue
        if j >= maxb:
            restarts += 1
            if restarts > o.max_restarts:
                raise RuntimeError("stage 2: restart limit")
            cand = [s1] + [S[:, c] for c in range(S.shape[1])]
            if s_prev is not None:
                cand_prev = s_prev
            else:
                cand_prev = None
            cols = []
            for c in cand:
                if len(cols) >= mins - 1:
                    break
                p = c.copy()
                for _ in range(2):
                    for qv in cols:
                        p = p - qv * (qv @ p)
                nrm = np.linalg.norm(p)
                if nrm > 1e-8:
                    cols.append(p / nrm)
            if cand_prev is not None:
                p = cand_prev.copy()
                for _ in range(2):
                    for qv in cols:
                        p = p - qv * (qv @ p)
                nrm = np.linalg.norm(p)
                if nrm > 1e-8:
                    cols.append(p / nrm)
            Y = np.column_stack(cols)
            V, W = V @ Y, W @ Y
            H = Y.T @ H @ Y
            H = 0.5 * (H + H.T)
            s1 = Y.T @ s1
            if rn < r0:
                shift = th1
            qr_full = True
        s_prev = s1.copy()
        # ---- expand with t = r (Algorithm 2 step 4), or with the JD correction
        if o.stage2_inner == "qmr":
            corr = jd_correction(ops, np.column_stack([Xl] + Xd) if Xd else Xl, x, W @ s1, th1, r,
                                 delta * normA / math.sqrt(2.0),
                                 o.inner_maxit, stats)
        elif o.precond == "given" and o.precond_M is not None:
            # [0 M^-1; M^-T 0] for B (Sec. 4), in the [v; u] order, Olsen form
            Pr = given_b_precond(o.precond_M, ops.n, r)
            Px = given_b_precond(o.precond_M, ops.n, x)
            den = float(x @ Px)
            corr = Pr - (float(x @ Pr) / den) * Px if den != 0.0 else Pr
        elif o.stage2_precond and diagC is not None:
            # READING: M = diag(C)^{-1}, the unshifted Jacobi preconditioner of
            # C, so that P = [0 M A^T; A M 0] approximates B^{-1} (the targets
            # are the smallest singular values; a shifted (diag(C) - shift^2)
            # is indefinite across the spectrum and slowed stage 2 down), in
            # the Olsen form t = P r - e P x, e = x^T P r / x^T P x
            d = diagC.copy()
            guard = EPS64 * normA * normA
            d = np.where(np.abs(d) < guard, np.where(d < 0, -guard, guard), d)
            Pr = b_precond(ops, lambda z: z / d, r)
            Px = b_precond(ops, lambda z: z / d, x)
            den = float(x @ Px)
            corr = Pr - (float(x @ Pr) / den) * Px if den != 0.0 else Pr
        else:
            corr = r
        t = orth_append(np.hstack([Xl] + Xd + [V]), corr[:, None], o.seed, counter)
        wt = ops.B(t)
        H = np.block([[H, V.T @ wt], [wt.T @ V, t.T @ wt]])
        H = 0.5 * (H + H.T)
        V, W = np.hstack([V, t]), np.hstack([W, wt])
        s_prev = np.concatenate([s_prev, [0.0]])
        if not qr_full:
            qn, rcol = qr_add_column(Q, (wt - shift * t)[:, 0], o.seed, counter)
            Q = np.column_stack([Q, qn])
            R = np.block([[R, rcol[:-1, None]], [np.zeros((1, R.shape[1])), rcol[-1:, None]]])
    stats.update(iters2=it, restarts2=restarts)
    return np.array(th_l), Xl, normA_est


# ---------------------------------------------------------------------------
# driver
# ---------------------------------------------------------------------------

def next_max_iter(init_iter: int, j: int, same: bool) -> tuple:
    """Algorithm 3 steps 9-13: the same approach again doubles maxIter
    (j <- j + 1), a switch cuts it back (j <- floor(j / 2));
    maxIter = initIter * 2^j.  Returns (j, maxIter)."""
    j = j + 1 if same else j // 2
    return j, init_iter * 2 ** j


def convergence_rate(history: list) -> float:
    """Average reduction per iteration of the residual norm (Sec. 4), as the
    mean slope of log ||r|| over a run; more negative is faster."""
    h = [x for x in history if x > 0]
    if len(h) < 2:
        return 0.0
    return (math.log(h[-1]) - math.log(h[0])) / (len(h) - 1)


def dynamic_phsvds(csr, k: int, delta: float = 1e-14, o: Opts | None = None, init_iter: int = 50,
                   max_switch: int = 8, log: list | None = None) -> Result:
    """Algorithm 3 (Sec. 4): dynamic switching between C and B under
    preconditioning, GD+k on both, for the k smallest triplets.

    The runs alternate between GD+k on C (the stage-1 operator with its
    preconditioner) and GD+k on B (targets: the positive eigenvalues
    nearest zero, with the B preconditioner of the same family), each
    starting from the other's approximations; the convergence rate of each
    is the mean log-reduction of the residual per iteration.  The loop and
    its maxIter rule follow the algorithm's steps; the end follows its
    final branches (all found on B / all found on C / faster C: the
    two-stage method / faster B: B to the end).
    READINGS: the initial tests run C then B, so the first choice compares
    against B; numConverged is the number locked in the latest run; the
    preconditioners are the shift-free forms of Sec. 4 (given M ~ A:
    M^-1 M^-T and [0 M^-1; M^-T 0]; Jacobi: diag(C)^-1 and [0 M A^T; A M 0]),
    in the Olsen form; a B run locks at ||r_B|| < delta ||A|| / sqrt 2; B's
    targets are its eigenvalues above 1e-12 of the largest, so that the
    m - n zero eigenvalues of a rectangular A are not taken for singular
    values.
    """
    o = Opts() if o is None else o
    A = as_scipy(csr)
    m, n = A.shape
    if m < n:
        raise ValueError("PHSVDS needs m >= n")
    ops = Ops(A)
    diagC = np.asarray(A.multiply(A).sum(axis=0)).ravel()
    guard = EPS64 * float(np.max(diagC))
    dC = np.where(diagC < guard, guard, diagC)

    def olsen(Pr, Px, x):
        den = float(x @ Px)
        return Pr - (float(x @ Pr) / den) * Px if den != 0.0 else Pr

    if o.precond == "given" and o.precond_M is not None:
        m2 = np.asarray(o.precond_M, dtype=np.float64) ** 2
        prec_C = lambda r, x: olsen(r / m2, x / m2, x)
        prec_B = lambda r, x: olsen(given_b_precond(o.precond_M, n, r), given_b_precond(o.precond_M, n, x), x)
    elif o.precond == "jacobi":
        prec_C = lambda r, x: olsen(r / dC, x / dC, x)
        prec_B = lambda r, x: olsen(b_precond(ops, lambda z: z / dC, r), b_precond(ops, lambda z: z / dC, x), x)
    else:
        prec_C = prec_B = None
    tolC = stage1_tol(delta, o)
    tolB = lambda th, thmax: delta * thmax / math.sqrt(2.0)
    # the zero eigenvalues of B (m > n) are not singular values: only
    # eigenvalues above 1e-12 max |theta| are targets (READING)
    keyB = lambda th: np.where(th > 1e-12 * np.max(np.abs(th)), th, np.inf)
    log = [] if log is None else log
    cur = {"X": None, "normA": 0.0}

    def run(approach: str, iters):
        h: list = []
        st: dict = {}
        if approach == "C":
            lam, X, state = gdk(ops.C, n, k, False, tolC, o, X0=cur["X"], stats=st, apply_prec=prec_C,
                                stop_after=iters, history=h)
            cur["normA"] = max(cur["normA"], math.sqrt(st["theta_max"]))
            Xv = X
        else:
            X0 = None
            if cur["X"] is not None:
                AV = A @ cur["X"]
                AV = AV / np.maximum(np.linalg.norm(AV, axis=0), 1e-300)
                X0 = np.vstack([cur["X"], AV]) / math.sqrt(2.0)
            lam, X, state = gdk(ops.B, m + n, k, False, tolB, o, X0=X0, stats=st, order_key=keyB,
                                apply_prec=prec_B, stop_after=iters, history=h)
            cur["normA"] = max(cur["normA"], st["theta_max"])
            Xv = X[:n] / np.maximum(np.linalg.norm(X[:n], axis=0), 1e-300)
        cur["X"] = Xv
        done = not state.get("partial", False)
        nconv = k if done else int(state["nconv"])
        rate = convergence_rate(h)
        log.append(dict(approach=approach, max_iter=iters, iters=st["iters"], rate=rate, nconv=nconv))
        return dict(lam=lam, X=X, state=state, stats=st, done=done, nconv=nconv, rate=rate)

    # step 3: initial tests on C and on B
    last = {"C": run("C", init_iter), "B": run("B", init_iter)}
    num_conv = max(last["C"]["nconv"], last["B"]["nconv"])
    prev, num_switch, j, max_iter, undecided = "B", 0, 0, init_iter, True
    while num_switch < max_switch and undecided:
        choice = "C" if last["C"]["rate"] < last["B"]["rate"] else "B"
        if (num_switch == 0 and num_conv > 0) or num_conv > 1:
            undecided = False
        else:
            j, max_iter = next_max_iter(init_iter, j, choice == prev)
        num_switch += 1
        last[choice] = run(choice, max_iter)
        num_conv = last[choice]["nconv"]
        prev = choice
        if last[choice]["done"]:
            break
    faster = "C" if last["C"]["rate"] < last["B"]["rate"] else "B"
    stats = dict(dynamic=log, switches=num_switch, faster=faster)
    if last[prev]["done"] and prev == "B":
        res = last["B"]
        X = res["X"]
        route = "B"
    elif last[prev]["done"] and prev == "C":
        st = dict(last["C"]["stats"])
        st.update(stats)
        out = _after_stage1(A, ops, k, False, delta, o, last["C"]["lam"], last["C"]["X"], last["C"]["state"], st)
        out.stats["route"] = "C then B"
        return out
    elif faster == "C":
        st: dict = {}
        lam, Xv, state = gdk(ops.C, n, k, False, tolC, o, X0=cur["X"], stats=st, apply_prec=prec_C)
        st.update(stats)
        out = _after_stage1(A, ops, k, False, delta, o, lam, Xv, state, st)
        out.stats["route"] = "two-stage"
        return out
    else:
        AV = A @ cur["X"]
        AV = AV / np.maximum(np.linalg.norm(AV, axis=0), 1e-300)
        X0 = np.vstack([cur["X"], AV]) / math.sqrt(2.0)
        st = {}
        lam, X, state = gdk(ops.B, m + n, k, False, tolB, o, X0=X0, stats=st, order_key=keyB, apply_prec=prec_B)
        route = "B to the end"
    Vv = X[:n] / np.linalg.norm(X[:n], axis=0)
    Uu = X[n:] / np.linalg.norm(X[n:], axis=0)
    sig = np.einsum("ij,ij->j", Uu, A @ Vv)
    Uu[:, sig < 0] *= -1.0
    sig = np.abs(sig)
    ru, rv, res_ = triplet_residuals(A, sig, Uu, Vv)
    order = np.argsort(sig)
    stats.update(route=route, mv_A=ops.mv_A, mv_At=ops.mv_At)
    return Result(sig[order], Uu[:, order], Vv[:, order], res_[order], max(cur["normA"], float(np.max(sig))), stats)


def triplet_residuals(A: sp.csr_matrix, sigma, U, V):
    """||A v - s u||, ||A^T u - s v|| and their root-sum-square (Sec. 5 criterion)."""
    rv = np.linalg.norm(A @ V - U * sigma, axis=0)
    ru = np.linalg.norm(A.T @ U - V * sigma, axis=0)
    return ru, rv, np.sqrt(ru * ru + rv * rv)


def phsvds(csr, k: int, largest: bool = False, delta: float = 1e-14, o: Opts | None = None) -> Result:
    """PHSVDS (Sections 3-5) for the k smallest or largest singular triplets of A."""
    o = Opts() if o is None else o
    A = as_scipy(csr)
    m, n = A.shape
    if m < n:
        raise ValueError("PHSVDS needs m >= n")
    ops = Ops(A)
    stats: dict = {}
    if o.norm_A < 0:
        stats["norm_c_est"] = lanczos_norm_c(ops.C, n, o.seed)
    diagC = np.asarray(A.multiply(A).sum(axis=0)).ravel() if o.precond == "jacobi" else None
    lam, Xv, state = gdk(ops.C, n, k, largest, stage1_tol(delta, o), o, diagC=diagC, stats=stats)
    return _after_stage1(A, ops, k, largest, delta, o, lam, Xv, state, stats)


def _after_stage1(A, ops: Ops, k: int, largest: bool, delta: float, o: Opts, lam, Xv, state, stats) -> Result:
    """Switch test (Sec. 3.1), optional Rayleigh-Ritz (Algorithm 1 step 3) and
    stage 2 (Algorithm 2) after a converged stage 1; the final triplets."""
    m, n = A.shape
    theta_max = stats["theta_max"]
    normA = math.sqrt(theta_max)
    # ||A|| of the user requirement (Opts.norm_A): the switch test and stage 2
    if o.norm_A > 0:
        normA = max(normA, float(o.norm_A))
    elif o.norm_A < 0:
        normA = max(normA, math.sqrt(max(stats.get("norm_c_est", 0.0), 0.0)))
    # stage-1 triplets: s = ||A v||, u = A v / s (r_v = 0)
    AV = ops.Av(Xv)
    sig1 = np.linalg.norm(AV, axis=0)
    U1 = AV / np.where(sig1 > 0, sig1, 1.0)
    ru, rv, res = triplet_residuals(A, sig1, U1, Xv)
    ops.mv_At += k
    floor = o.eps_factor * o.stage1_eps
    need2 = bool(np.any(delta < floor * normA / np.maximum(sig1, 1e-300)) or np.any(res >= delta * normA))
    stats.update(stage1_mv_A=ops.mv_A, stage1_mv_At=ops.mv_At, switched=need2)
    if not need2 or not o.stage2:
        order = np.argsort(sig1)[::-1] if largest else np.argsort(sig1)
        return Result(sig1[order], U1[:, order], Xv[:, order], res[order], normA,
                      dict(stats, mv_A=ops.mv_A, mv_At=ops.mv_At))
    if o.rr:
        lam, Xv = rayleigh_ritz_post(ops, Xv, state, k, largest, o)
    sig_s = np.sqrt(np.maximum(lam, 0.0))
    if o.stage2_inner == "qmr":
        # READING (JDQMR form): the targets that stage 1 resolved go first and
        # the tiny ones (sigma~ <= sqrt(eps) ||A||, Sec. 4's "extremely small"
        # values, whose u~ is random) last, each group in the given order, so
        # that the accurate guesses are locked before the ambiguous shifts
        # near zero are worked on
        tiny = sig_s <= math.sqrt(EPS64) * normA
        order2 = np.concatenate([np.where(~tiny)[0], np.where(tiny)[0]])
        sig_s, Xv = sig_s[order2], Xv[:, order2]
    # stage 2 in ascending (smallest) or descending (largest) order of the shifts
    th, X2, normA2 = stage2(ops, sig_s, Xv, normA, delta, o, stats,
                            diagC=np.asarray(A.multiply(A).sum(axis=0)).ravel()
                            if o.stage2_precond and not largest else None)
    Vv = X2[:n]
    Uu = X2[n:]
    Vv = Vv / np.linalg.norm(Vv, axis=0)
    Uu = Uu / np.linalg.norm(Uu, axis=0)
    sig = np.einsum("ij,ij->j", Uu, A @ Vv)
    neg = sig < 0
    Uu[:, neg] *= -1.0
    sig = np.abs(sig)
    ru, rv, res = triplet_residuals(A, sig, Uu, Vv)
    order = np.argsort(sig)[::-1] if largest else np.argsort(sig)
    return Result(sig[order], Uu[:, order], Vv[:, order], res[order], normA,
                  dict(stats, mv_A=ops.mv_A, mv_At=ops.mv_At))
