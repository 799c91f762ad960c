"""Pins of the oracle's Algorithm 3 (Sec. 4, dynamic switching between C and
B under preconditioning): its maxIter rule and rate estimate, its control
flow on scripted runs, and a whole solve of the E3 demonstration."""
import math

import numpy as np
import pytest

from oracle import phsvds_ref as R
from paper_1408_5535_gb300 import synth


def test_max_iter_rule():
    """Same approach again: j + 1 and maxIter doubles; a switch: floor(j/2)."""
    j, mi = 0, 50
    seq = []
    for same in (True, True, True, False, True, False, False):
        j, mi = R.next_max_iter(50, j, same)
        seq.append(mi)
    assert seq == [100, 200, 400, 100, 200, 100, 50]


def test_convergence_rate_of_a_geometric_history():
    h = [3.0 * 0.8 ** i for i in range(12)]
    assert R.convergence_rate(h) == pytest.approx(math.log(0.8), rel=1e-12)
    assert R.convergence_rate([1.0]) == 0.0


def _scripted(monkeypatch, rates, A):
    """Replace GD+k by scripted runs: each bounded run reports the next rate
    of its approach and converges nothing; an unbounded run converges to the
    exact answer of the diagonal A."""
    m, n = A.shape
    calls = []
    it = {"C": iter(rates["C"]), "B": iter(rates["B"])}

    def fake(apply_op, N, k, largest, tol_fn, o, X0=None, stats=None, order_key=None, apply_prec=None,
             stop_after=None, history=None, diagC=None):
        ap = "C" if N == n else "B"
        calls.append((ap, stop_after))
        sig = np.sort(np.abs(A.diagonal()))[:k]
        if ap == "C":
            X = np.eye(n)[:, :k]
            lam = sig ** 2
        else:
            X = np.vstack([np.eye(n)[:, :k], np.eye(m, n)[:, :k]]) / math.sqrt(2.0)
            lam = sig
        stats.update(iters=stop_after or 1, restarts=0, theta_max=float(np.max(A.diagonal()) ** 2))
        if stop_after is None:
            S = np.eye(k)
            return lam, X, dict(V=X, W=X, theta=lam, S=S, conv=list(range(k)))
        r = next(it[ap])
        history.extend([1.0, math.exp(r * (stop_after - 1))])
        return lam, X, dict(V=X, W=X, theta=lam, S=np.eye(k), conv=[], nconv=0, partial=True)

    monkeypatch.setattr(R, "gdk", fake)
    return calls


def test_control_flow_when_c_is_faster(monkeypatch):
    """C keeps winning: maxIter doubles on each repeat, the switches run out,
    and the faster C continues as the two-stage method."""
    import scipy.sparse as sp
    A = sp.diags(np.arange(1.0, 9.0)).tocsr()
    calls = _scripted(monkeypatch, {"C": [-0.5] * 20, "B": [-0.1] * 20}, A)
    log = []
    res = R.dynamic_phsvds(synth.diag_matrix(np.arange(1.0, 9.0)), 2, o=R.Opts(max_basis=6, min_restart=4),
                           init_iter=10, max_switch=4, log=log)
    bounded = [c for c in calls if c[1] is not None]
    assert bounded[:2] == [("C", 10), ("B", 10)]                 # the initial tests
    assert bounded[2:] == [("C", 10), ("C", 20), ("C", 40), ("C", 80)]
    assert calls[-1] == ("C", None)                             # two-stage continuation
    assert res.stats["route"] == "two-stage" and res.stats["switches"] == 4
    assert np.allclose(res.sigma, [1.0, 2.0])


def test_control_flow_when_b_is_faster(monkeypatch):
    """B wins after the initial tests: it runs with growing maxIter, and the
    faster B continues to the end on the augmented matrix."""
    import scipy.sparse as sp
    A = sp.diags(np.arange(1.0, 9.0)).tocsr()
    calls = _scripted(monkeypatch, {"C": [-0.1] * 20, "B": [-0.5] * 20}, A)
    res = R.dynamic_phsvds(synth.diag_matrix(np.arange(1.0, 9.0)), 2, o=R.Opts(max_basis=6, min_restart=4),
                           init_iter=10, max_switch=3)
    bounded = [c for c in calls if c[1] is not None]
    assert bounded == [("C", 10), ("B", 10), ("B", 20), ("B", 40), ("B", 80)]
    assert calls[-1] == ("B", None)
    assert res.stats["route"] == "B to the end"
    assert np.allclose(res.sigma, [1.0, 2.0]) and np.all(res.resid < 1e-14)


def test_dynamic_switching_on_the_e3_demonstration():
    """The preconditioned two-stage demonstration: the dynamic method settles
    on C, finishes it, and stage 2 reaches sigma_min = 1 at 1e-14 ||A||; the
    logged maxIter values follow the rule."""
    A, M = synth.e3_diag()
    log = []
    res = R.dynamic_phsvds(A, 1, delta=1e-14, o=R.Opts(precond="given", precond_M=M), log=log)
    assert abs(res.sigma[0] - 1.0) <= 1e-10
    assert res.resid[0] <= 1e-14 * res.normA
    assert res.stats["faster"] == "C"
    assert [e["approach"] for e in log[:2]] == ["C", "B"]
    j, prev = 0, "B"
    for e in log[2:]:                      # no run converged a pair before the last one
        j, mi = R.next_max_iter(50, j, e["approach"] == prev)
        assert e["max_iter"] == mi
        prev = e["approach"]


@pytest.mark.parametrize("precond", ["jacobi", "none"])
def test_dynamic_switching_on_a_rectangular_matrix(precond):
    """120 x 60 random sparse A (B has 60 zero eigenvalues, which must not be
    taken for singular values): the three smallest triplets match the dense
    SVD whichever route the switching takes."""
    from oracle.dense_jacobi import jacobi_svd
    A = synth.random_sparse(120, 60, 5.0, 11, values="gaussian", shift=0.05)
    res = R.dynamic_phsvds(A, 3, delta=1e-14, o=R.Opts(precond=precond, max_basis=20, min_restart=10),
                           init_iter=20)
    s = np.sort(jacobi_svd(A.to_dense())[0])[:3]
    assert np.max(np.abs(res.sigma - s) / s) <= 1e-10
    assert np.all(res.resid <= 1e-14 * res.normA)
    assert res.stats["route"] in ("B to the end", "two-stage", "C then B")
