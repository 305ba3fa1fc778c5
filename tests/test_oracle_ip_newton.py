"""The Newton step of the interior-point loop for box-bounded MHE, pinned on the
CPU (Section II: an interior-point method for MHE with inequality constraints
spends its time in Newton steps of the UFTOC form the tree solves).

mhe_ip_solve hands the tree, at every stage t >= 1, the UFTOC problem with
    Q_w + Sigma  and  l_w - c_l/s_l + c_h/s_h - Sigma w,   Sigma = zl/s_l + zh/s_h,
and takes the bounds' new multipliers as
    zl' = c_l/s_l - (zl/s_l) dw,   zh' = c_h/s_h + (zh/s_h) dw
(s_l = w - lo, s_h = hi - w; c_l, c_h the complementarity targets of the
method: mu for path following, the corrector's targets for the
predictor-corrector).  Here that reading, solved by the oracle's Riccati
recursion, is checked against its definition: Newton's method on the full
primal-dual system
    K z' + E^T (zh' - zl') = b                     (the KKT rows, bound multipliers in the w rows)
    zl E (z' - z) + s_l zl' = c_l                  (s_l zl = c_l, linearised)
    -zh E (z' - z) + s_h zh' = c_h                 (s_h zh = c_h, linearised)
formed densely from the C-oracle-independent dense KKT matrix and solved by
LAPACK, at interior iterates with arbitrary positive multipliers and targets.
The new states, inputs, costates and bound multipliers must agree."""
import copy

import numpy as np
import pytest

import oracle
from oracle import dense
from paper_1510_03110_gb300 import synth


def _w_rows(prob, o):
    """Packed input index -> its stationarity row in dense.kkt_matrix."""
    rows = {}
    row = prob.n
    for t in range(prob.N):
        row += prob.n
        for j in range(prob.m[t]):
            rows[o["ow"] + o["wo"][t] + j] = row + j
        row += prob.m[t] + prob.n
    return rows


def _interior_iterate(prob, lo, hi, rng):
    """A dynamically feasible z with every bounded input strictly inside its box,
    and arbitrary costates."""
    n, N, m = prob.n, prob.N, prob.m[1]
    W = lo + (hi - lo) * rng.uniform(0.1, 0.9, (N - 1, m))
    w0 = rng.normal(size=prob.m[0])
    x = np.zeros((N + 1, n))
    x[0] = prob.x0
    x[1] = prob.A[0] @ x[0] + prob.B[0] @ w0 + prob.a[0]
    for t in range(1, N):
        x[t + 1] = prob.A[t] @ x[t] + prob.B[t] @ W[t - 1] + prob.a[t]
    lam = rng.normal(size=(N + 1, n))
    return x, w0, W, lam


@pytest.mark.parametrize("n,m,N,seed", [(3, 2, 6, 0), (4, 2, 9, 1), (2, 1, 12, 2), (6, 3, 5, 3)])
def test_uftoc_newton_model_is_the_primal_dual_newton_step(n, m, N, seed):
    rng = np.random.default_rng(100 + seed)
    prob = oracle.mhe_to_uftoc(synth.mhe_instance(4100 + seed, n, m, m, N))
    c = rng.uniform(0.5, 2.0, m)
    lo, hi = -c, c + rng.uniform(0.1, 0.5, m)
    x, w0, W, lam = _interior_iterate(prob, lo, hi, rng)
    sl, sh = W - lo, hi - W
    zl = rng.uniform(0.05, 3.0, W.shape)
    zh = rng.uniform(0.05, 3.0, W.shape)
    cl = rng.uniform(1e-3, 1.0, W.shape)
    ch = rng.uniform(1e-3, 1.0, W.shape)

    # the reading: the UFTOC problem the loop hands the tree, solved by the oracle
    q = copy.deepcopy(prob)
    sig = zl / sl + zh / sh
    for t in range(1, N):
        Qt = np.array(q.Q[t], dtype=float)
        Qt[n:, n:] += np.diag(sig[t - 1])
        q.Q[t] = Qt
        lt = np.array(q.l[t], dtype=float)
        lt[n:] += -cl[t - 1] / sl[t - 1] + ch[t - 1] / sh[t - 1] - sig[t - 1] * W[t - 1]
        q.l[t] = lt
    r = oracle.riccati(q)
    assert r["status"] == 0
    dW = r["w"][prob.m[0]:].reshape(N - 1, m) - W
    zl_new = cl / sl - zl / sl * dW
    zh_new = ch / sh + zh / sh * dW

    # the definition: the full primal-dual Newton system, dense
    K, b, o = dense.kkt_matrix(prob)
    rows = _w_rows(prob, o)
    dim = K.shape[0]
    bnd = [o["ow"] + o["wo"][t] + j for t in range(1, N) for j in range(m)]
    nb = len(bnd)
    z = np.concatenate([x.ravel(), w0, W.ravel(), lam.ravel()])
    M = np.zeros((dim + 2 * nb, dim + 2 * nb))
    rhs = np.zeros(dim + 2 * nb)
    M[:dim, :dim] = K
    rhs[:dim] = b
    for k, zi in enumerate(bnd):
        M[rows[zi], dim + k] = -1.0
        M[rows[zi], dim + nb + k] = 1.0
        M[dim + k, zi] = zl.ravel()[k]
        M[dim + k, dim + k] = sl.ravel()[k]
        rhs[dim + k] = cl.ravel()[k] + zl.ravel()[k] * z[zi]
        M[dim + nb + k, zi] = -zh.ravel()[k]
        M[dim + nb + k, dim + nb + k] = sh.ravel()[k]
        rhs[dim + nb + k] = ch.ravel()[k] - zh.ravel()[k] * z[zi]
    sol = np.linalg.solve(M, rhs)

    scale = 1.0 + np.abs(sol).max()
    assert np.abs(r["x"].ravel() - sol[o["ox"]:o["ow"]]).max() <= 1e-9 * scale
    assert np.abs(r["w"] - sol[o["ow"]:o["ol"]]).max() <= 1e-9 * scale
    assert np.abs(r["lam"].ravel() - sol[o["ol"]:dim]).max() <= 1e-9 * scale
    assert np.abs(zl_new.ravel() - sol[dim:dim + nb]).max() <= 1e-9 * scale
    assert np.abs(zh_new.ravel() - sol[dim + nb:]).max() <= 1e-9 * scale


def test_a_wrong_sign_in_the_model_is_caught():
    """The same comparison with the upper bound's term of the right-hand side
    negated (a plausible slip) disagrees with the dense Newton step."""
    rng = np.random.default_rng(7)
    n, m, N = 3, 2, 6
    prob = oracle.mhe_to_uftoc(synth.mhe_instance(4200, n, m, m, N))
    lo, hi = -np.ones(m), np.ones(m)
    x, w0, W, lam = _interior_iterate(prob, lo, hi, rng)
    sl, sh = W - lo, hi - W
    zl = rng.uniform(0.05, 3.0, W.shape)
    zh = rng.uniform(0.05, 3.0, W.shape)
    cl = ch = np.full(W.shape, 0.3)
    sols = []
    for sign in (1.0, -1.0):
        q = copy.deepcopy(prob)
        sig = zl / sl + zh / sh
        for t in range(1, N):
            Qt = np.array(q.Q[t], dtype=float)
            Qt[n:, n:] += np.diag(sig[t - 1])
            q.Q[t] = Qt
            lt = np.array(q.l[t], dtype=float)
            lt[n:] += -cl[t - 1] / sl[t - 1] + sign * ch[t - 1] / sh[t - 1] - sig[t - 1] * W[t - 1]
            q.l[t] = lt
        sols.append(oracle.riccati(q)["w"])
    assert np.abs(sols[0] - sols[1]).max() > 1e-3
