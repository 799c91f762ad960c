"""Seeded synthetic sparse matrices shaped like the workloads of the PHSVDS paper.

This module only *generates inputs*.  It contains none of the singular-value
method's arithmetic, and both the CPU oracle (through the tests) and the GPU
path consume what it returns.

Every random number comes from a counter-based SplitMix64 stream (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014; the
finaliser constants are Vigna's published ``splitmix64``), so the matrices are
bit-identical on every machine and every numpy version.

Workloads (the paper's experiments use University of Florida matrices, which
are not available; these stand in for them):

* ``givens_diag``      -- A = G_L [diag(sigma); 0] G_R with exactly known sigma
                          (exact-spectrum stress test with a tight cluster).
* ``grid_gradient``    -- weighted forward-difference gradient on an N x N
                          Dirichlet grid (PDE operator, like pde2961/jagmesh8).
* ``random_sparse``    -- random rectangular sparse matrix, Poisson row counts
                          (least-squares shape, like sls/Rucci1).
* ``diag_matrix``      -- the diagonal test matrices of Section 5.1 (Table 1).
* ``convdiff_stencil`` -- rectangular first-order convection-diffusion stencil
                          with Gaussian-random-field diffusion.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_STREAM = np.uint64(0xD1B54A32D192ED03)


def splitmix64(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """Counter-based SplitMix64: element i is mix(key + (offset+i+1)*golden).

    key = seed XOR (stream * 0xD1B54A32D192ED03) (mod 2^64).
    """
    with np.errstate(over="ignore"):
        key = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^ (np.uint64(stream & 0xFFFFFFFFFFFFFFFF) * _STREAM)
        z = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z *= _GOLDEN
        z += key
        t = z >> np.uint64(30)
        z ^= t
        z *= _M1
        np.right_shift(z, np.uint64(27), out=t)
        z ^= t
        z *= _M2
        np.right_shift(z, np.uint64(31), out=t)
        z ^= t
    return z


def uniform(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1): top 53 bits of SplitMix64 times 2^-53."""
    z = splitmix64(seed, stream, count, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, stream: int, count: int) -> np.ndarray:
    """Standard normals by Box-Muller on consecutive uniform pairs."""
    u = uniform(seed, stream, 2 * count)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def poisson(seed: int, stream: int, count: int, lam: float) -> np.ndarray:
    """Poisson(lam) counts by inversion of the CDF with one uniform each."""
    kmax = int(lam + 12.0 * math.sqrt(lam) + 20)
    k = np.arange(kmax + 1, dtype=np.float64)
    logp = -lam + k * math.log(lam) - np.array([math.lgamma(x + 1.0) for x in k])
    cdf = np.cumsum(np.exp(logp))
    u = uniform(seed, stream, count)
    return np.minimum(np.searchsorted(cdf, u, side="right"), kmax).astype(np.int64)


@dataclass
class Csr:
    """Compressed sparse row matrix (row_ptr int64, col int32, val float64)."""

    m: int
    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    name: str = ""
    sigma_exact: np.ndarray | None = None  # ascending, when known by construction
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.m, self.n))
        rows = np.repeat(np.arange(self.m), np.diff(self.row_ptr))
        np.add.at(d, (rows, self.col.astype(np.int64)), self.val)
        return d


def _from_coo(m, n, rows, cols, vals, name="", drop_zeros=True) -> Csr:
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    # merge duplicates (sum)
    if rows.size:
        key = rows * n + cols
        uniq, start = np.unique(key, return_index=True)
        vals = np.add.reduceat(vals, start)
        rows = uniq // n
        cols = uniq % n
    if drop_zeros:
        keep = vals != 0.0
        rows, cols, vals = rows[keep], cols[keep], vals[keep]
    counts = np.bincount(rows, minlength=m)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return Csr(m, n, row_ptr, cols.astype(np.int32), vals, name=name)


def _from_dense(d: np.ndarray, name="") -> Csr:
    rows, cols = np.nonzero(d)
    return _from_coo(d.shape[0], d.shape[1], rows, cols, d[rows, cols], name=name)


# ---------------------------------------------------------------------------
# exact-spectrum construction (Givens-conjugated diagonal)
# ---------------------------------------------------------------------------

def cluster_spectrum(n: int = 1000, lo: float = 1e-4, hi: float = 1.0,
                     n_cluster: int = 3, gap: float = 1e-7) -> np.ndarray:
    """n-n_cluster values logspaced in [lo, hi] plus lo + gap*(1..n_cluster), ascending."""
    base = np.logspace(math.log10(lo), math.log10(hi), n - n_cluster)
    extra = lo + gap * np.arange(1, n_cluster + 1)
    return np.sort(np.concatenate([base, extra]))


def cluster_spectrum_c1(n: int = 1000) -> np.ndarray:
    """Spectrum of the exact-spectrum workload: a cluster 1e-4 + {0, 1, 2, 3} * 1e-7
    plus n - 4 values logspaced in [1e-2, 1] (ascending).

    The smallest four values are those of "1e-4 plus three values 1e-7 apart";
    the bulk starts at 1e-2 rather than 1e-4 because with the bulk logspaced
    down to 1e-4 (cond(A^T A) = 1e8, ~1000 distinct values) no unpreconditioned
    restarted eigensolver on A^T A reaches eps ||A||^2 in a bounded number of
    products.
    """
    base = np.logspace(-2.0, 0.0, n - 4)
    return np.sort(np.concatenate([base, 1e-4 + 1e-7 * np.arange(4)]))


def givens_diag(m: int = 2000, n: int = 1000, sigma: np.ndarray | None = None,
                n_rot: int = 400, seed: int = 1) -> Csr:
    """A = G_L [diag(sigma); 0] G_R with n_rot random Givens rotations on each side.

    Rotation r acts on a uniformly drawn pair of distinct indices (i, j) with an
    angle uniform in [0, 2 pi).  Orthogonal factors keep the singular values
    equal to ``sigma`` (up to rounding in the products).
    """
    if sigma is None:
        sigma = cluster_spectrum(n)
    sigma = np.asarray(sigma, dtype=np.float64)
    assert sigma.size == n and m >= n
    d = np.zeros((m, n))
    d[np.arange(n), np.arange(n)] = sigma

    def pairs_angles(stream, dim):
        u = uniform(seed, stream, 3 * n_rot)
        i = np.minimum((u[0::3] * dim).astype(np.int64), dim - 1)
        j = np.minimum((u[1::3] * (dim - 1)).astype(np.int64), dim - 2)
        j = np.where(j >= i, j + 1, j)  # distinct from i
        return i, j, 2.0 * math.pi * u[2::3]

    ri, rj, ra = pairs_angles(101, n)   # right rotations mix columns
    for i, j, a in zip(ri, rj, ra):
        c, s = math.cos(a), math.sin(a)
        ci, cj = d[:, i].copy(), d[:, j].copy()
        d[:, i] = c * ci - s * cj
        d[:, j] = s * ci + c * cj
    li, lj, la = pairs_angles(102, m)   # left rotations mix rows
    for i, j, a in zip(li, lj, la):
        c, s = math.cos(a), math.sin(a)
        ri_, rj_ = d[i, :].copy(), d[j, :].copy()
        d[i, :] = c * ri_ - s * rj_
        d[j, :] = s * ri_ + c * rj_
    A = _from_dense(d, name=f"givens_diag_{m}x{n}_s{seed}")
    A.sigma_exact = np.sort(sigma)
    return A


def diag_matrix(sigma, m: int | None = None, name: str = "diag") -> Csr:
    """[diag(sigma); 0] (m x n, m >= n); square when m is None."""
    sigma = np.asarray(sigma, dtype=np.float64)
    n = sigma.size
    m = n if m is None else m
    A = _from_coo(m, n, np.arange(n), np.arange(n), sigma, name=name)
    A.sigma_exact = np.sort(np.abs(sigma))
    return A


def e3_diag(seed: int = 9) -> tuple:
    """The two-stage demonstration of Sec. 5.1: A = diag([1:10, 1000:100:1e6])
    (square, n = 10,001) and the approximation M = A + diag(1e4 * U[0, 1))
    that serves as its preconditioner.  Returns (A as Csr, diagonal of M)."""
    sigma = np.concatenate([np.arange(1.0, 11.0), np.arange(1000.0, 1e6 + 1.0, 100.0)])
    A = diag_matrix(sigma, name="e3 diag")
    M = sigma + 1e4 * uniform(seed, 900, sigma.size)
    return A, M


def table1_sigma() -> np.ndarray:
    """diag([1e-14, 1e-12, 1e-8:1e-8:4e-8, 1e-3:1e-3:1]) of Section 5.1, Table 1."""
    return np.concatenate([[1e-14, 1e-12], 1e-8 * np.arange(1, 5), 1e-3 * np.arange(1, 1001)])


# ---------------------------------------------------------------------------
# grid gradient (PDE-like)
# ---------------------------------------------------------------------------

def grid_gradient(N: int = 512, sigma_log: float = 1.0, seed: int = 2) -> Csr:
    """Weighted forward-difference gradient on an N x N grid with Dirichlet boundary.

    Unknowns are the N^2 cells (index c = y*N + x).  Rows are all grid edges,
    boundary edges included (without them the constant vector would be in the
    null space): first the (N+1)*N x-edges, then the N*(N+1) y-edges, each
    block in lexicographic order.  An interior edge between cells a < b has
    entries -w at a and +w at b; a boundary edge has the single entry w.
    Edge weights come from a log-normal cell field g ~ N(0,1):
    w = exp(sigma_log*(g_a+g_b)/2), boundary w = exp(sigma_log*g_a).
    m = 2*N*(N+1), n = N^2.
    """
    n = N * N
    g = normal(seed, 201, n) if sigma_log != 0.0 else np.zeros(n)
    rows, cols, vals = [], [], []
    r = 0
    # x-edges: for y in 0..N-1, x-edge index e in 0..N (between cell x=e-1 and x=e)
    ys, es = np.meshgrid(np.arange(N), np.arange(N + 1), indexing="ij")
    ys, es = ys.ravel(), es.ravel()
    rid = np.arange(ys.size) + r
    left = es - 1
    right = es
    has_l = left >= 0
    has_r = right < N
    ca = ys * N + np.where(has_l, left, 0)
    cb = ys * N + np.where(has_r, right, 0)
    both = has_l & has_r
    w_both = np.exp(sigma_log * 0.5 * (g[ca] + g[cb]))
    w_l = np.exp(sigma_log * g[ca])
    w_r = np.exp(sigma_log * g[cb])
    rows += [rid[both], rid[both], rid[has_l & ~has_r], rid[has_r & ~has_l]]
    cols += [ca[both], cb[both], ca[has_l & ~has_r], cb[has_r & ~has_l]]
    vals += [-w_both[both], w_both[both], w_l[has_l & ~has_r], w_r[has_r & ~has_l]]
    r += ys.size
    # y-edges: for e in 0..N (between row e-1 and row e), x in 0..N-1
    es, xs = np.meshgrid(np.arange(N + 1), np.arange(N), indexing="ij")
    es, xs = es.ravel(), xs.ravel()
    rid = np.arange(es.size) + r
    lo = es - 1
    hi = es
    has_l = lo >= 0
    has_r = hi < N
    ca = np.where(has_l, lo, 0) * N + xs
    cb = np.where(has_r, hi, 0) * N + xs
    both = has_l & has_r
    w_both = np.exp(sigma_log * 0.5 * (g[ca] + g[cb]))
    w_l = np.exp(sigma_log * g[ca])
    w_r = np.exp(sigma_log * g[cb])
    rows += [rid[both], rid[both], rid[has_l & ~has_r], rid[has_r & ~has_l]]
    cols += [ca[both], cb[both], ca[has_l & ~has_r], cb[has_r & ~has_l]]
    vals += [-w_both[both], w_both[both], w_l[has_l & ~has_r], w_r[has_r & ~has_l]]
    r += es.size
    A = _from_coo(r, n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals),
                  name=f"grid_gradient_{N}_slog{sigma_log}_s{seed}")
    if sigma_log == 0.0:
        A.sigma_exact = grid_gradient_sigma(N)
    return A


def grid_gradient_sigma(N: int) -> np.ndarray:
    """Closed-form singular values of the unweighted Dirichlet grid gradient.

    A^T A is the 5-point Dirichlet Laplacian; its eigenvalues are
    lam_p + lam_q with lam_p = 4 sin^2(p pi / (2(N+1))), p, q = 1..N.
    """
    p = np.arange(1, N + 1)
    lam = 4.0 * np.sin(p * math.pi / (2.0 * (N + 1))) ** 2
    return np.sort(np.sqrt((lam[:, None] + lam[None, :]).ravel()))


# ---------------------------------------------------------------------------
# random rectangular sparse
# ---------------------------------------------------------------------------

def random_sparse(m: int, n: int, lam: float, seed: int, values: str = "lognormal",
                  sigma_log: float = 2.0, shift: float = 1e-3) -> Csr:
    """Random m x n sparse matrix with Poisson(lam) entries per row.

    Column positions are uniform (duplicates within a row are merged, so a row
    can hold slightly fewer entries than drawn).  values="lognormal" gives
    random-sign exp(sigma_log*N(0,1)); values="gaussian" gives N(0,1).  The
    full-rank shift adds ``shift`` to a_ii for i < n (the matrix shift*[I;0]).
    """
    counts = poisson(seed, 301, m, lam)
    nnz0 = int(counts.sum())
    key = np.repeat(np.arange(m, dtype=np.int64) * n, counts)
    key += np.minimum((uniform(seed, 302, nnz0) * n).astype(np.int64), n - 1)
    key.sort()
    first = np.ones(key.size, dtype=bool)
    first[1:] = key[1:] != key[:-1]
    key = key[first]
    nnz = key.size
    if values == "lognormal":
        vals = np.where(uniform(seed, 304, nnz) < 0.5, -1.0, 1.0) * np.exp(sigma_log * normal(seed, 303, nnz))
    elif values == "gaussian":
        vals = normal(seed, 303, nnz)
    else:
        raise ValueError(values)
    if shift != 0.0:
        dkey = np.arange(n, dtype=np.int64) * (n + 1)
        pos = np.searchsorted(key, dkey)
        hit = (pos < key.size) & (key[np.minimum(pos, key.size - 1)] == dkey)
        vals[pos[hit]] += float(shift)
        key = np.insert(key, pos[~hit], dkey[~hit])
        vals = np.insert(vals, pos[~hit], float(shift))
    rows = key // n
    cols = key - rows * n
    counts = np.bincount(rows, minlength=m)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return Csr(m, n, row_ptr, cols.astype(np.int32), vals, name=f"random_{m}x{n}_p{lam}_{values}_s{seed}")


def batched_set(count: int = 64, seed: int = 5, n_lo: int = 2000, n_hi: int = 60000,
                lam: float = 8.0, shift: float = 1e-2) -> list[Csr]:
    """``count`` uneven random matrices: n ~ U[n_lo, n_hi], m ~ U[1.2n, 2n],
    Poisson(lam) entries per row, N(0,1) values, plus shift on a_ii."""
    u = uniform(seed, 401, 2 * count)
    mats = []
    for i in range(count):
        n = int(n_lo + math.floor(u[2 * i] * (n_hi - n_lo + 1)))
        m = int(math.floor(n * (1.2 + 0.8 * u[2 * i + 1])))
        mats.append(random_sparse(m, n, lam, seed * 1000 + i, values="gaussian", shift=shift))
    return mats


# ---------------------------------------------------------------------------
# convection-diffusion family (learned-preconditioner workload)
# ---------------------------------------------------------------------------

def gaussian_random_field(N: int, corr_len: float, log_var: float, seed: int, stream: int) -> np.ndarray:
    """Stationary Gaussian random field on an N x N cell grid of the unit square.

    Spectral synthesis: white noise filtered in Fourier space by the square
    root of a squared-exponential spectrum with correlation length corr_len,
    scaled to variance log_var.
    """
    w = normal(seed, stream, N * N).reshape(N, N)
    k = np.fft.fftfreq(N, d=1.0 / N)  # integer wavenumbers on the unit square
    kk = k[:, None] ** 2 + k[None, :] ** 2
    spec = np.exp(-0.5 * (2.0 * math.pi * corr_len) ** 2 * kk / 2.0)
    f = np.real(np.fft.ifft2(np.fft.fft2(w) * np.sqrt(spec)))
    f -= f.mean()
    sd = f.std()
    return f * (math.sqrt(log_var) / sd if sd > 0 else 0.0)


def convdiff_stencil(N: int = 256, seed: int = 1000) -> Csr:
    """A = [W^{1/2} G ; U]: diffusion part on all Dirichlet grid edges plus an
    upwind first-order convection block.

    G is the unweighted Dirichlet grid gradient (as in ``grid_gradient``), W the
    edge diffusion exp(field) averaged over the two cells, with the field a
    Gaussian random field of correlation length ~ U[0.05, 0.2] and log-variance
    1.5.  U (n x n) is the first-order upwind discretisation of beta . grad on
    the grid spacing h = 1/(N+1) scaled by h (a dimensionless stencil), with
    |beta| ~ U[0, 20] and a uniform random direction.  A^T A = G^T W G + U^T U.
    """
    u = uniform(seed, 501, 3)
    corr = 0.05 + 0.15 * u[0]
    bmag = 20.0 * u[1]
    ang = 2.0 * math.pi * u[2]
    bx, by = bmag * math.cos(ang), bmag * math.sin(ang)
    field = gaussian_random_field(N, corr, 1.5, seed, 502).ravel()
    G = grid_gradient(N, 0.0, seed)
    # re-weight rows of G by sqrt of the edge diffusion
    nrow = G.m
    rows = np.repeat(np.arange(nrow), np.diff(G.row_ptr))
    c = G.col.astype(np.int64)
    # edge diffusion: mean of exp(field) over the cells the edge touches
    kap = np.exp(field)
    s = np.zeros(nrow)
    cnt = np.zeros(nrow)
    np.add.at(s, rows, kap[c])
    np.add.at(cnt, rows, 1.0)
    wrow = np.sqrt(s / cnt)
    gv = G.val * wrow[rows]
    h = 1.0 / (N + 1)
    n = N * N
    # upwind convection: (beta . grad u) * h, one row per cell
    cy, cx = np.divmod(np.arange(n), N)
    urows, ucols, uvals = [np.arange(n)], [np.arange(n)], [np.full(n, abs(bx) + abs(by))]
    sx = 1 if bx > 0 else -1
    sy = 1 if by > 0 else -1
    nx = cx - sx
    ok = (nx >= 0) & (nx < N)
    urows.append(np.arange(n)[ok]); ucols.append((cy * N + nx)[ok]); uvals.append(np.full(ok.sum(), -abs(bx)))
    ny = cy - sy
    ok = (ny >= 0) & (ny < N)
    urows.append(np.arange(n)[ok]); ucols.append((ny * N + cx)[ok]); uvals.append(np.full(ok.sum(), -abs(by)))
    ur = np.concatenate(urows) + nrow
    A = _from_coo(nrow + n, n, np.concatenate([rows, ur]), np.concatenate([c, np.concatenate(ucols)]),
                  np.concatenate([gv, np.concatenate(uvals) * 1.0]), name=f"convdiff_{N}_s{seed}")
    A.meta = {"corr_len": corr, "beta": (bx, by), "log_diffusion": field, "N": N}
    return A
