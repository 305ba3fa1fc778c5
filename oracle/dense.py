"""Dense KKT system of Eq. org_eqc_problem, solved by LAPACK LU.

TEST INFRASTRUCTURE ONLY.  This is the Newton step by its plain definition:
the unique solution z = (x_0..x_N, w_0..w_{N-1}, lambda_0..lambda_N) of the
KKT system of the equality-constrained QP (Section III).  Rows, with the
Lagrangian  cost + sum_t lambda_{t+1}^T (A_t x_t + B_t w_t + a_t - x_{t+1})
+ lambda_0^T (x0 - x_0):
    x_0 = x0
    Q_x,t x_t + Q_xw,t w_t + A_t^T lambda_{t+1} - lambda_t = -l_x,t
    Q_xw,t^T x_t + Q_w,t w_t + B_t^T lambda_{t+1}          = -l_w,t
    A_t x_t + B_t w_t - x_{t+1}                            = -a_t
    Q_x,N x_N - lambda_N                                   = -l_N
Only for small problems (the matrix is formed densely).
"""
from __future__ import annotations

import numpy as np


def kkt_matrix(prob):
    n, N, m = prob.n, prob.N, prob.m
    nw = int(sum(m))
    ox = 0
    ow = (N + 1) * n
    ol = ow + nw
    dim = ol + (N + 1) * n
    K = np.zeros((dim, dim))
    b = np.zeros(dim)
    wo = np.concatenate([[0], np.cumsum(m)]).astype(int)
    row = 0
    # initial condition
    for i in range(n):
        K[row + i, ox + i] = 1.0
        b[row + i] = prob.x0[i]
    row += n
    for t in range(N):
        mt = m[t]
        xs = slice(ox + t * n, ox + (t + 1) * n)
        xn = slice(ox + (t + 1) * n, ox + (t + 2) * n)
        ws = slice(ow + wo[t], ow + wo[t + 1])
        lt = slice(ol + t * n, ol + (t + 1) * n)
        ln = slice(ol + (t + 1) * n, ol + (t + 2) * n)
        Q = prob.Q[t]
        # stationarity in x_t
        rs = slice(row, row + n)
        K[rs, xs] = Q[:n, :n]
        K[rs, ws] = Q[:n, n:]
        K[rs, ln] = prob.A[t].T
        K[rs, lt] = -np.eye(n)
        b[rs] = -prob.l[t][:n]
        row += n
        # stationarity in w_t
        rs = slice(row, row + mt)
        K[rs, xs] = Q[n:, :n]
        K[rs, ws] = Q[n:, n:]
        K[rs, ln] = prob.B[t].T
        b[rs] = -prob.l[t][n:]
        row += mt
        # dynamics
        rs = slice(row, row + n)
        K[rs, xs] = prob.A[t]
        K[rs, ws] = prob.B[t]
        K[rs, xn] = -np.eye(n)
        b[rs] = -prob.a[t]
        row += n
    rs = slice(row, row + n)
    K[rs, ox + N * n: ox + (N + 1) * n] = prob.QN
    K[rs, ol + N * n: ol + (N + 1) * n] = -np.eye(n)
    b[rs] = -prob.lN
    row += n
    assert row == dim
    return K, b, dict(ox=ox, ow=ow, ol=ol, wo=wo)


def solve(prob):
    """x (N+1, n), w (packed), lambda (N+1, n) by numpy.linalg.solve (LU)."""
    K, b, o = kkt_matrix(prob)
    z = np.linalg.solve(K, b)
    n, N = prob.n, prob.N
    x = z[o["ox"]:o["ox"] + (N + 1) * n].reshape(N + 1, n)
    w = z[o["ow"]:o["ol"]]
    lam = z[o["ol"]:].reshape(N + 1, n)
    return dict(x=x, w=w, lam=lam, K=K, b=b, z=z)
