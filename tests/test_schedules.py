"""CPU replays of the index arithmetic of the small-matrix kernels (no GPU):
the round-robin pairing of the cyclic Jacobi kernels, the bipartite schedule
of the FP64 target clean-up, the butterfly reduce-scatter of the CGS pass,
and the lane layout of the stage-2 refined-vector kernel (inverse iteration
on R).  Each replay restates the kernel's rule in Python and checks the
property the kernel relies on (disjoint pairs within a round, every pair
exactly once per sweep, every warp sum landing on exactly one lane, the
smallest right singular vector of R)."""
import itertools

import numpy as np
import pytest

JT_MAXT = 8


def rr_pair(jj, r, k):
    """Circle method: round r, pair k of jj (even) indices."""
    m = jj - 1
    if k == 0:
        a, b = r % m, m
    else:
        a, b = (r + k) % m, (r - k + m) % m
    return min(a, b), max(a, b)


@pytest.mark.parametrize("jj", list(range(2, 66, 2)))
def test_round_robin_pairs_cover_each_pair_once(jj):
    seen = set()
    for r in range(jj - 1):
        idx = [i for k in range(jj // 2) for i in rr_pair(jj, r, k)]
        assert len(idx) == len(set(idx)) == jj          # disjoint within the round
        seen.update(rr_pair(jj, r, k) for k in range(jj // 2))
    assert seen == set(itertools.combinations(range(jj), 2))


def target_rounds(tgt, non):
    """Pairs of each round of one sweep of the target clean-up: first every
    target x non-target pair (the smaller side by lane, the larger shifted
    each round), then the target x target round robin."""
    nt, nn = len(tgt), len(non)
    ntt = nt + (nt & 1)
    na = max(nt, nn) if nt > 0 else 0
    rounds = []
    for rnd in range(na + (ntt - 1 if nt > 1 else 0)):
        pairs = []
        for lane in range(JT_MAXT):
            p = q = -1
            if rnd < na:
                if nt <= nn:
                    if lane < nt:
                        p, q = tgt[lane], non[(rnd + lane) % nn]
                elif lane < nn:
                    p, q = tgt[(rnd + lane) % nt], non[lane]
            elif lane < ntt // 2:
                a, b = rr_pair(ntt, rnd - na, lane)
                if b < nt:
                    p, q = tgt[a], tgt[b]
            if p >= 0:
                pairs.append((min(p, q), max(p, q)))
        rounds.append(pairs)
    return rounds


@pytest.mark.parametrize("j", [2, 3, 5, 8, 9, 17, 27, 35, 64])
def test_target_schedule_is_disjoint_and_complete(j):
    rng = np.random.default_rng(j)
    for nt in range(1, min(JT_MAXT, j - 1) + 1):
        tgt = [int(t) for t in rng.permutation(j)[:nt]]
        non = [i for i in range(j) if i not in tgt]
        want = {(min(t, x), max(t, x)) for t in tgt for x in range(j) if x != t}
        got = []
        for pairs in target_rounds(tgt, non):
            idx = [i for pq in pairs for i in pq]
            assert len(idx) == len(set(idx))             # disjoint within the round
            got.extend(pairs)
        assert len(got) == len(set(got))                 # no pair twice
        assert set(got) == want                          # every pair touching a target


def reduce_scatter(vals):
    """Butterfly reduce-scatter of the N values of each of 32 lanes."""
    v = vals.copy()
    lanes = np.arange(32)
    cur, o = v.shape[1], 16
    while o > 0:
        if cur > 1:
            h = cur // 2
            up = (lanes & o) != 0
            nv = np.empty((32, h))
            for i in range(h):
                send = np.where(up, v[:, i], v[:, i + h])
                keep = np.where(up, v[:, i + h], v[:, i])
                nv[:, i] = keep + send[lanes ^ o]
            v, cur = nv, h
        else:
            v = v.copy()
            v[:, 0] = v[:, 0] + v[lanes ^ o, 0]
        o //= 2
    return v


@pytest.mark.parametrize("nv", [8, 16, 32, 64])
def test_reduce_scatter_lands_each_sum_on_one_lane(nv):
    x = np.random.default_rng(nv).standard_normal((32, nv))
    tot = x.sum(axis=0)
    v = reduce_scatter(x)
    per = nv // 32 if nv >= 32 else 1
    rep = 1 if nv >= 32 else 32 // nv
    owned = []
    for lane in range(32):
        for u in range(per):
            idx = lane * per + u if nv >= 32 else lane // rep
            assert v[lane, u] == pytest.approx(tot[idx], rel=1e-12, abs=1e-12)
            if lane % rep == 0:
                owned.append(idx)
    assert sorted(owned) == list(range(nv))             # one atomic per sum


def refined_inverse_replay(R, x0=None, maxit=24, tau=1e-10):
    """The lane layout of the stage-2 refined-vector kernel (one warp, lane l
    holding rows l and l + 32): guarded pivots, forward solve with R^T and
    back solve with R per step, stop once ||R x|| stops falling."""
    j = R.shape[0]
    rmax = np.max(np.abs(np.triu(R)))
    tiny = rmax * 2.0 ** -52 if rmax > 0 else 1.0
    d = np.diag(R).copy()
    d = np.where(np.abs(d) >= tiny, d, np.where(d < 0, -tiny, tiny))
    invd = 1.0 / d
    rows = np.concatenate([np.arange(32), np.arange(32) + 32])   # lane l: rows l, l + 32
    live = rows < j
    x = np.zeros(64)
    if x0 is not None:
        x[live] = x0[rows[live]]
    if not np.linalg.norm(x) > 0:
        g = 0.6180339887498949
        x[live] = 1.0 + (rows[live] * g - np.floor(rows[live] * g))
    x /= np.linalg.norm(x)
    Rp = np.zeros((64, 64))
    Rp[:j, :j] = np.triu(R)
    rho = np.linalg.norm(Rp @ x)
    steps = 0
    while steps < maxit:
        steps += 1
        b = x.copy()
        for k in range(j):                     # R^T y = x
            b[k] = b[k] * invd[k]
            m = live & (rows > k)
            b[rows[m]] -= Rp[k, rows[m]] * b[k]
        b /= np.linalg.norm(b)
        for k in range(j - 1, -1, -1):         # R z = y
            b[k] = b[k] * invd[k]
            m = rows < k
            b[rows[m]] -= Rp[rows[m], k] * b[k]
        b /= np.linalg.norm(b)
        rn = np.linalg.norm(Rp @ b)
        stalled = not rn < rho * (1 - tau)
        if rn < rho:
            x, rho = b, rn
        if stalled:
            break
    return x[:j], rho, steps


@pytest.mark.parametrize("j", [1, 2, 31, 32, 33, 47, 64])
def test_refined_inverse_replay_finds_the_smallest_singular_vector(j):
    rng = np.random.default_rng(100 + j)
    U, _ = np.linalg.qr(rng.standard_normal((j, j)))
    V, _ = np.linalg.qr(rng.standard_normal((j, j)))
    s = np.logspace(0, -3, j)
    s[-1] = 1e-13                              # the refined residual near convergence
    R = np.linalg.qr(U @ np.diag(s) @ V.T)[1]
    x, rho, steps = refined_inverse_replay(R)
    smin = np.linalg.svd(R, compute_uv=False)[-1]
    assert rho <= smin * (1 + 1e-8) + 64 * 2.0 ** -52 * np.max(np.abs(R))
    assert steps <= 4
    if j > 1:
        vmin = np.linalg.svd(R)[2][-1]
        assert abs(abs(vmin @ x) - 1.0) < 1e-12


def test_refined_inverse_replay_singular_pivot():
    """A zero pivot is raised to 2^-52 max|r|: the guarded solve returns the
    exact null direction of R."""
    rng = np.random.default_rng(7)
    R = np.triu(rng.standard_normal((10, 10)))
    R[:, 4] = 0.0
    x, rho, _ = refined_inverse_replay(R, x0=np.ones(10))
    assert rho < 1e-14 and np.linalg.norm(R @ x) < 1e-14
