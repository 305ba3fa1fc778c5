"""MHE with box-bounded process noise, solved exactly by a primal active-set method.

TEST INFRASTRUCTURE ONLY.  Section II states MHE with inequality constraints on
the noise and notes that an interior-point method spends its time in Newton
steps of the UFTOC form; the constraint sets themselves are not in the paper.
The bounded problem checked here is Eq. org_eqc_problem plus the box
lo <= w_t <= hi on the input of every measured stage t = 1 .. N-1 (the arrival
input w_0 and the states are free).  It is a strictly convex QP, so its solution
is unique and is the point where the KKT conditions hold:
  * the equality rows of the dense KKT system (oracle.dense) hold, with a
    multiplier nu_i added to the stationarity row of every bounded input fixed
    at a bound (the Lagrangian gains nu_i (w_i - bound_i)),
  * every input lies in its box,
  * a fixed input's gradient points into the box: nu_i <= 0 at a lower bound,
    nu_i >= 0 at an upper bound.
The method is the textbook primal active-set iteration for convex QPs (Nocedal
and Wright, Numerical Optimization, 2nd ed., Algorithm 16.3): from a feasible
point, solve the equality-constrained problem on the current working set; move
towards its solution as far as the box allows and add the blocking bound; when
the step is zero, stop if every multiplier has the right sign, else release the
bound whose multiplier is most wrong.  Each equality-constrained problem is the
dense KKT system, solved by LAPACK.  Only for small problems.
"""
from __future__ import annotations

import numpy as np

from . import dense


def _layout(prob):
    n, N = prob.n, prob.N
    m = prob.m
    ow = (N + 1) * n
    wo = np.concatenate([[0], np.cumsum(m)]).astype(int)
    return n, N, m, ow, wo


def bounded_indices(prob, lo, hi):
    """(position in z, lower bound, upper bound) of every bounded input entry:
    w_t[j] for t = 1 .. N-1, j < m_t, with the bounds lo[j], hi[j]."""
    n, N, m, ow, wo = _layout(prob)
    out = []
    for t in range(1, N):
        for j in range(m[t]):
            out.append((ow + wo[t] + j, float(lo[j]), float(hi[j])))
    return out


def _eqp(prob, K, b, rows_w, fixed):
    """Solve the KKT system with the inputs in `fixed` ({z index: value}) held at
    their values; returns (z without the bound multipliers, {index: nu})."""
    dim = K.shape[0]
    k = len(fixed)
    Kf = np.zeros((dim + k, dim + k))
    bf = np.zeros(dim + k)
    Kf[:dim, :dim] = K
    bf[:dim] = b
    for r, (zi, val) in enumerate(sorted(fixed.items())):
        # the stationarity row of input zi gains + nu; a new row pins zi
        Kf[rows_w[zi], dim + r] = 1.0
        Kf[dim + r, zi] = 1.0
        bf[dim + r] = val
    sol = np.linalg.solve(Kf, bf)
    nu = {zi: sol[dim + r] for r, zi in enumerate(sorted(fixed))}
    return sol[:dim], nu


def _stationarity_rows(prob):
    """Row of the dense KKT matrix that is the stationarity condition in each
    input entry (the row order of oracle.dense.kkt_matrix)."""
    n, N, m, ow, wo = _layout(prob)
    rows = {}
    row = n                                   # after the initial condition
    for t in range(N):
        row += n                              # stationarity in x_t
        for j in range(m[t]):
            rows[ow + wo[t] + j] = row + j
        row += m[t] + n                       # stationarity in w_t, dynamics
    return rows


def feasible_start(prob, lo, hi):
    """x_0 = x0, w_0 = 0, w_t = the middle of the box, x by the dynamics."""
    n, N, m, ow, wo = _layout(prob)
    x = np.zeros((N + 1, n))
    w = np.zeros(int(np.sum(m)))
    x[0] = prob.x0
    for t in range(N):
        wt = np.zeros(m[t]) if t == 0 else 0.5 * (np.asarray(lo[:m[t]]) + np.asarray(hi[:m[t]]))
        w[wo[t]:wo[t + 1]] = wt
        x[t + 1] = prob.A[t] @ x[t] + prob.B[t] @ wt + prob.a[t]
    return x, w


def solve(prob, lo, hi, max_iter: int = 10000, tol: float = 1e-12):
    """Exact solution of the box-bounded problem.  Returns dict(x, w, lam, active
    = {z index: 'lo' | 'hi'}, nu = {z index: multiplier}, iters)."""
    n, N, m, ow, wo = _layout(prob)
    K, b, _ = dense.kkt_matrix(prob)
    rows_w = _stationarity_rows(prob)
    bnd = bounded_indices(prob, lo, hi)
    box = {zi: (lb, ub) for zi, lb, ub in bnd}
    x, w = feasible_start(prob, lo, hi)
    nxw = ow + int(np.sum(m))
    z = np.concatenate([x.ravel(), w])
    scale = 1.0 + max(abs(v) for _, l_, h_ in bnd for v in (l_, h_)) if bnd else 1.0
    work = {}                                 # z index -> 'lo' | 'hi'
    for it in range(max_iter):
        fixed = {zi: (lb if work[zi] == "lo" else ub) for zi, lb, ub in bnd if zi in work}
        full, nu = _eqp(prob, K, b, rows_w, fixed)
        p = full[:nxw] - z
        if np.abs(p).max() <= tol * scale * (1.0 + np.abs(z).max()):
            # multipliers of the working set: nu <= 0 at a lower bound, >= 0 at an upper bound
            wrong = {zi: (v if work[zi] == "lo" else -v) for zi, v in nu.items()}
            worst = max(wrong, key=wrong.get) if wrong else None
            if worst is None or wrong[worst] <= 0.0:
                for zi, v in fixed.items():
                    full[zi] = v                  # held inputs exactly on their bound
                lam = full[nxw:].reshape(N + 1, n)
                return dict(x=full[:ow].reshape(N + 1, n), w=full[ow:nxw], lam=lam,
                            active=dict(work), nu=nu, iters=it + 1)
            del work[worst]
            continue
        # the longest step towards the working-set solution that stays in the box
        alpha, block = 1.0, None
        for zi, lb, ub in bnd:
            if zi in work:
                continue
            if p[zi] < 0 and z[zi] + p[zi] < lb:
                a_i = (lb - z[zi]) / p[zi]
                if a_i < alpha:
                    alpha, block = a_i, (zi, "lo")
            elif p[zi] > 0 and z[zi] + p[zi] > ub:
                a_i = (ub - z[zi]) / p[zi]
                if a_i < alpha:
                    alpha, block = a_i, (zi, "hi")
        z = z + alpha * p
        if block is not None:
            zi, side = block
            z[zi] = box[zi][0] if side == "lo" else box[zi][1]   # exactly on the bound
            work[zi] = side
    raise RuntimeError("active-set iteration did not finish")


def objective_of(prob, x, w):
    """Value of the objective of Eq. org_eqc_problem (quadratic and linear terms,
    the constants included) at (x, w), written out stage by stage."""
    n, N, m, ow, wo = _layout(prob)
    f = 0.0
    for t in range(N):
        v = np.concatenate([x[t], w[wo[t]:wo[t + 1]]])
        f += 0.5 * v @ prob.Q[t] @ v + prob.l[t] @ v + prob.c[t]
    f += 0.5 * x[N] @ prob.QN @ x[N] + prob.lN @ x[N] + prob.cN
    return float(f)
