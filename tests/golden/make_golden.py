"""Write the exact golden fixtures of tests/golden/ (run: python tests/golden/make_golden.py).

Each fixture is a small MHE problem of Eq. org_mhe (Section II) with rational
data, and its Newton step (the minimiser, which for this equality-constrained
QP is the unique KKT point of Eq. org_eqc_problem) in EXACT rational
arithmetic: no floating point, no call into the oracle or the CUDA library.

How the exact solution is found (independent of the Riccati recursion):
  * the free variables are the first MHE state X_0 and the process noises
    w_0..w_{K-1}; the later states follow from the dynamics
    X_{k+1} = A_k X_k + B_k w_k + a_k;
  * the MHE cost f (arrival cost + sum over k of 1/2 e_k^T R_k e_k with
    e_k = [w_k - w~_k; y~_k - C_k X_k]) is a convex quadratic in them, so its
    gradient and Hessian are read off exactly from values of f (central
    differences are exact for a quadratic);
  * the normal equations H z = -g are solved by Gauss-Jordan elimination in
    fractions.Fraction.
The UFTOC form of Section II puts an arrival stage in front (x_0 = x~0,
A_0 = B_0 = I, input w_0 = X_0 - x~0 weighted by P~0^{-1}) and shifts the MHE
stage k to stage t = k + 1; the multipliers follow from the KKT rows of the
Lagrangian  cost + sum_t lam_{t+1}^T (A_t x_t + B_t w_t + a_t - x_{t+1})
+ lam_0^T (x~0 - x_0):  lam_N = 0 (no terminal cost) and
lam_t = d(stage-t cost)/d x_t + A_t^T lam_{t+1}.
"""
from __future__ import annotations

import os
from fractions import Fraction as F

HERE = os.path.dirname(os.path.abspath(__file__))


# --- small exact linear algebra on lists of Fractions -------------------------

def matvec(M, v):
    return [sum((M[i][j] * v[j] for j in range(len(v))), F(0)) for i in range(len(M))]


def tmatvec(M, v):
    return [sum((M[i][j] * v[i] for i in range(len(M))), F(0)) for j in range(len(M[0]))]


def add(*vs):
    return [sum(c, F(0)) for c in zip(*vs)]


def sub(u, v):
    return [a - b for a, b in zip(u, v)]


def quad(M, v):
    return sum((v[i] * M[i][j] * v[j] for i in range(len(v)) for j in range(len(v))), F(0))


def gauss_jordan(H, rhs):
    """Solve H z = rhs exactly (H nonsingular); partial pivoting on nonzeros."""
    n = len(H)
    M = [list(H[i]) + [rhs[i]] for i in range(n)]
    for c in range(n):
        p = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[p] = M[p], M[c]
        piv = M[c][c]
        M[c] = [v / piv for v in M[c]]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c]
                M[r] = [a - f * b for a, b in zip(M[r], M[c])]
    return [M[i][n] for i in range(n)]


# --- the problem of Eq. org_mhe -------------------------------------------------

def problem_2x1x1():
    """n = 2, nw = 1, ny = 1, five measured stages (UFTOC horizon N = 6);
    non-symmetric A_k, time-varying data, S != 0 except at stage 2, P~0^{-1} not
    the identity."""
    K = 5
    A, B, C, R, a, yt, wt = [], [], [], [], [], [], []
    for k in range(K):
        A.append([[F(9, 10) + F(k, 20), F(1, k + 2)], [F(-1, 4), F(4, 5)]])
        B.append([[F(1, 2)], [F(1) - F(k, 10)]])
        C.append([[F(1), F(k - 1, 3)]])
        s = F(0) if k == 2 else F((-1) ** k, 2)
        R.append([[F(2) + F(k, 2), s], [s, F(3, 2)]])
        a.append([F(k, 4) - F(1, 2), F(1, 8)])
        yt.append([F((-1) ** k * (k + 1), 3)])
        wt.append([F(1, 5) - F(k, 10)])
    return dict(n=2, m=1, q=1, N=K + 1, x0=[F(1), F(-1, 2)], P0inv=[[F(2), F(1, 2)], [F(1, 2), F(1)]],
                A=A, B=B, C=C, R=R, a=a, yt=yt, wt=wt)


def problem_1x1x1():
    """n = nw = ny = 1, three measured stages (UFTOC horizon N = 4)."""
    K = 3
    return dict(n=1, m=1, q=1, N=K + 1, x0=[F(3, 2)], P0inv=[[F(4)]],
                A=[[[F(1, 2) + F(k, 4)]] for k in range(K)],
                B=[[[F(1) + F(k, 3)]] for k in range(K)],
                C=[[[F(2) - F(k, 2)]] for k in range(K)],
                R=[[[F(3), F(1, 2) * (k - 1)], [F(1, 2) * (k - 1), F(2)]] for k in range(K)],
                a=[[F(k, 5)] for k in range(K)],
                yt=[[F(1) - F(k, 3)] for k in range(K)],
                wt=[[F(-1, 4) * k] for k in range(K)])


def problem_4x2x2():
    """n = 4, nw = ny = 2, four measured stages (UFTOC horizon N = 5); the
    cross-weight S of R = [[W, S], [S^T, V]] is a non-symmetric 2 x 2 block, so
    S and S^T cannot be confused without changing the answer."""
    K = 4
    A, B, C, R, a, yt, wt = [], [], [], [], [], [], []
    for k in range(K):
        A.append([[F(4, 5), F(1, 3), F(0), F(k, 10)],
                  [F(-1, 4), F(7, 10), F(1, 5), F(0)],
                  [F(0), F(1, 6), F(9, 10), F(-1, 3)],
                  [F(1, 8), F(0), F(1, 4), F(3, 5) + F(k, 20)]])
        B.append([[F(1, 2), F(0)], [F(1), F(1, 3)], [F(0), F(1, 2)], [F(-1, 4), F(1)]])
        C.append([[F(1), F(0), F(1, 2), F(0)], [F(0), F(1), F(0), F(-1, 3) * (k + 1)]])
        # R = M M^T + I with M lower triangular and rational: symmetric positive definite
        M = [[F(1), F(0), F(0), F(0)],
             [F(1, 2), F(1), F(0), F(0)],
             [F(-1, 3), F(1, 4) * (k + 1), F(1), F(0)],
             [F(1, 5), F(-1, 2), F(1, 3), F(1)]]
        R.append([[sum((M[i][t] * M[j][t] for t in range(4)), F(0)) + (F(1) if i == j else F(0))
                   for j in range(4)] for i in range(4)])
        a.append([F(k, 7), F(-1, 9), F(1, 11), F(0)])
        yt.append([F(1, 2) - F(k, 5), F((-1) ** k, 4)])
        wt.append([F(1, 10) * k, F(-1, 6)])
    return dict(n=4, m=2, q=2, N=K + 1, x0=[F(1, 2), F(-1), F(0), F(2)],
                P0inv=[[F(3), F(1, 2), F(0), F(0)], [F(1, 2), F(2), F(1, 4), F(0)],
                       [F(0), F(1, 4), F(1), F(0)], [F(0), F(0), F(0), F(3, 2)]],
                A=A, B=B, C=C, R=R, a=a, yt=yt, wt=wt)


def states(p, X0, ws):
    """X_0 .. X_K from the dynamics of Eq. org_mhe."""
    X = [X0]
    for k in range(p["N"] - 1):
        X.append(add(matvec(p["A"][k], X[k]), matvec(p["B"][k], ws[k]), p["a"][k]))
    return X


def stage_cost(p, k, x, w):
    """1/2 e^T R_k e, e = [w - w~_k; y~_k - C_k x] (the weighted process and
    measurement noise of MHE stage k)."""
    e = sub(w, p["wt"][k]) + sub(p["yt"][k], matvec(p["C"][k], x))
    return quad(p["R"][k], e) / 2


def arrival_cost(p, X0):
    d = sub(X0, p["x0"])
    return quad(p["P0inv"], d) / 2


def mhe_cost(p, z):
    n, m, K = p["n"], p["m"], p["N"] - 1
    X0 = z[:n]
    ws = [z[n + k * m:n + (k + 1) * m] for k in range(K)]
    X = states(p, X0, ws)
    return arrival_cost(p, X0) + sum((stage_cost(p, k, X[k], ws[k]) for k in range(K)), F(0))


def unit(d, i, s=F(1)):
    v = [F(0)] * d
    v[i] = s
    return v


def minimiser(p):
    """Exact minimiser z = (X_0, w_0, .., w_{K-1}) of the MHE cost."""
    d = p["n"] + (p["N"] - 1) * p["m"]
    f0 = mhe_cost(p, [F(0)] * d)
    fp = [mhe_cost(p, unit(d, i)) for i in range(d)]
    fm = [mhe_cost(p, unit(d, i, F(-1))) for i in range(d)]
    g = [(fp[i] - fm[i]) / 2 for i in range(d)]
    H = [[F(0)] * d for _ in range(d)]
    for i in range(d):
        H[i][i] = fp[i] + fm[i] - 2 * f0
        for j in range(i + 1, d):
            H[i][j] = H[j][i] = mhe_cost(p, add(unit(d, i), unit(d, j))) - fp[i] - fp[j] + f0
    return gauss_jordan(H, [-v for v in g])


def grad(fun, v):
    """Exact gradient of a quadratic function of the vector v."""
    return [(fun(add(v, unit(len(v), i))) - fun(sub(v, unit(len(v), i)))) / 2 for i in range(len(v))]


def uftoc_solution(p, z):
    """(x_0..x_N, w_0..w_{N-1}, lam_0..lam_N) of the UFTOC form, and the cost."""
    n, m, N = p["n"], p["m"], p["N"]
    K = N - 1
    X0 = z[:n]
    ws = [z[n + k * m:n + (k + 1) * m] for k in range(K)]
    X = states(p, X0, ws)
    x = [list(p["x0"])] + X                        # x_0 = x~0, x_{k+1} = X_k
    w = [sub(X0, p["x0"])] + ws                    # arrival input, then w_k
    lam = [None] * (N + 1)
    lam[N] = [F(0)] * n
    for t in range(N - 1, 0, -1):
        k = t - 1
        gx = grad(lambda xv: stage_cost(p, k, xv, ws[k]), x[t])
        lam[t] = add(gx, tmatvec(p["A"][k], lam[t + 1]))
    lam[0] = list(lam[1])                          # A_0 = I and no x-cost at stage 0
    return dict(x=x, w=w, lam=lam, f=mhe_cost(p, z))


# --- fixture text ---------------------------------------------------------------

def fmt(v):
    return " ".join(str(e) for e in v)


def flat(M):
    return [e for row in M for e in row]


def fixture_text(name, p):
    z = minimiser(p)
    s = uftoc_solution(p, z)
    n, m, q, N = p["n"], p["m"], p["q"], p["N"]
    out = [f"# {name}: exact Newton step of an MHE problem (Eq. org_mhe, Section II) in the UFTOC form of",
           "# Eq. org_eqc_problem, written by tests/golden/make_golden.py in rational arithmetic.",
           "# Matrices row-major; stage lines 'key k: ...' are MHE stage k = UFTOC stage k + 1.",
           "# Solution lines are UFTOC stages t = 0..N (x, lam) and t = 0..N-1 (w; w_0 has n entries).",
           f"dims: {n} {m} {q} {N}",
           f"x0: {fmt(p['x0'])}",
           f"P0inv: {fmt(flat(p['P0inv']))}"]
    for key in ("A", "B", "C", "R"):
        for k in range(N - 1):
            out.append(f"{key} {k}: {fmt(flat(p[key][k]))}")
    for key in ("a", "yt", "wt"):
        for k in range(N - 1):
            out.append(f"{key} {k}: {fmt(p[key][k])}")
    for key in ("x", "w", "lam"):
        for t, v in enumerate(s[key]):
            out.append(f"sol_{key} {t}: {fmt(v)}")
    out.append(f"cost: {s['f']}")
    return "\n".join(out) + "\n"


FIXTURES = {"mhe_2x1x1_N6_exact.txt": problem_2x1x1, "mhe_1x1x1_N4_exact.txt": problem_1x1x1,
            "mhe_4x2x2_N5_exact.txt": problem_4x2x2}


def main():
    for fname, make in FIXTURES.items():
        with open(os.path.join(HERE, fname), "w") as fh:
            fh.write(fixture_text(fname[:-4], make()))


if __name__ == "__main__":
    main()
