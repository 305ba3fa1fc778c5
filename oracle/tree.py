"""The paper's parallel scheme, executed serially in FP64 (test helper).

TEST INFRASTRUCTURE ONLY.  Each step follows the paper in order and notation:
  reduce_chunk     Algorithm 4 (reduction using Riccati factorization) for a
                   subproblem with unknown terminal data (P^, Psi^, c^)
  reduce_last      the last subproblem (Section IV-B, last paragraph): its
                   terminal is known, so Algorithms 1-2 factor it fully and
                   only the initial state remains
  master_problem   Eq. red_mpc_problem (Section IV-C)
  tree_solve       Algorithm 5 (reduce level by level) + Algorithm 6 (solve the
                   top, then propagate the solution down), with the down pass
                   either literal ('alg6': re-solve every subproblem with
                   Algorithms 1-3 from its parent's P^, Psi^, x^) or as the
                   back-substitution w_t = k_{0,t+1} + K_{0,t+1} x_t + wbar_t,
                   wbar_t = -L_{t+1} w^_i (Eq. control_signal_def with the
                   T-form of Eq. parric:Qh_Bh_alternative_def), followed by the
                   costate sweep of the KKT rows.
Two forms of the reduced input (Theorem 1):
  'T'   the T-form of Eq. parric:Qh_Bh_alternative_def, Q^_w = B^ = S Qbar^{-1} S^T
        (input width n; singular G^ when S^T is rank deficient, the remark after it);
  'U1'  the form of Eq. Bh_def, with U_1 an orthonormal basis of range(S^T):
        Q^_w = U_1^T Qbar^{-1} U_1, B^ = S Qbar^{-1} U_1 (input width n_uo = rank S^T <= n),
        and the chunk's inputs wbar = Qbar^{-1} U_1 w^ (the parametrisation of Kbar
        and kbar that precedes Eq. reducedGK_S).  It stays well posed for chunks with
        N_s nw < nx, where S^T has fewer than nx independent columns.
Chunking (the paper leaves batch lengths to the user, Section VI remark):
all chunks of a level have length L except the last, which takes the
remainder (1..L stages).
"""
from __future__ import annotations

import numpy as np

from .core import Uftoc, riccati


def _cho(G):
    return np.linalg.cholesky(G)


def _cho_solve(Lg, Y):
    z = np.linalg.solve(Lg, Y)
    return np.linalg.solve(Lg.T, z)


def reduce_chunk(prob: Uftoc, t0: int, t1: int) -> dict:
    """Algorithm 4 on stages t0..t1-1 of prob (terminal unknown).

    Returns A^ = V_0^T, B^ = Q^_w, a^ = v_0, Q^_x = P_0, l^_x = -Psi_0,
    c^ = cbar_0 and, per stage, the preliminary feedback K_{0,t+1}, k_{0,t+1},
    L_{t+1} and G_{t+1} (in stage order t0..t1-1).
    """
    n = prob.n
    P = np.zeros((n, n))
    Psi = np.zeros(n)
    cbar = 0.0
    Qw_hat = np.zeros((n, n))
    V = np.eye(n)
    v = np.zeros(n)
    K_l, k_l, L_l, G_l = [None] * (t1 - t0), [None] * (t1 - t0), [None] * (t1 - t0), [None] * (t1 - t0)
    for t in range(t1 - 1, t0 - 1, -1):
        A, B, a, Q, l = prob.A[t], prob.B[t], prob.a[t], prob.Q[t], prob.l[t]
        Qx, Qxw, Qw = Q[:n, :n], Q[:n, n:], Q[n:, n:]
        lx, lw = l[:n], l[n:]
        F = Qx + A.T @ P @ A
        G = Qw + B.T @ P @ B
        H = Qxw + A.T @ P @ B
        Lg = _cho(G)
        K = _cho_solve(Lg, -H.T)
        k = _cho_solve(Lg, B.T @ Psi - lw - B.T @ P @ a)
        Psi_new = A.T @ Psi - H @ k - lx - A.T @ P @ a
        cbar = cbar + 0.5 * a @ P @ a - Psi @ a - 0.5 * k @ G @ k + prob.c[t]
        P_new = F - K.T @ G @ K
        P_new = 0.5 * (P_new + P_new.T)      # P_t is symmetric (Section III)
        L = _cho_solve(Lg, -B.T @ V)
        V_new = (A.T + K.T @ B.T) @ V
        v = v + V.T @ (a + B @ k)
        Qw_hat = Qw_hat + L.T @ G @ L
        Qw_hat = 0.5 * (Qw_hat + Qw_hat.T)   # Q^_w is symmetric (Eq. Qh_Bh_alternative_def)
        P, Psi, V = P_new, Psi_new, V_new
        i = t - t0
        K_l[i], k_l[i], L_l[i], G_l[i] = K, k, L, G
    return dict(Ahat=V.T, Bhat=Qw_hat, ahat=v, Qxhat=P, lxhat=-Psi, chat=cbar,
                K=K_l, k=k_l, L=L_l, G=G_l)


def s_hat(prob: Uftoc, t0: int, t1: int, red: dict) -> np.ndarray:
    """S of Eq. B for stages t0..t1-1: column block tau is
    (A_{t1-1} + B_{t1-1} K_{0,t1}) ... (A_{tau+1} + B_{tau+1} K_{0,tau+2}) B_tau."""
    n = prob.n
    blocks = []
    Phi = np.eye(n)                      # product of the closed-loop matrices after tau
    for t in range(t1 - 1, t0 - 1, -1):
        blocks.append(Phi @ prob.B[t])
        Phi = Phi @ (prob.A[t] + prob.B[t] @ red["K"][t - t0])
    return np.hstack(blocks[::-1])


def qbar_inv(red: dict) -> np.ndarray:
    """Qbar^{-1}, Qbar = blkdiag(G_{0,t+1}) over the chunk's stages (Eq. QuA)."""
    Gs = red["G"]
    dims = [G.shape[0] for G in Gs]
    Qi = np.zeros((sum(dims), sum(dims)))
    o = 0
    for G, d in zip(Gs, dims):
        Qi[o:o + d, o:o + d] = np.linalg.inv(G)
        o += d
    return Qi


def reduce_u1(prob: Uftoc, t0: int, t1: int, red: dict) -> dict:
    """The U_1 form of Theorem 1 (Eq. Bh_def): U_1 = orthonormal basis of range(S^T)
    from the SVD of S^T (numerical rank with the usual threshold
    sigma_max * max(shape) * eps), Q^_w = U_1^T Qbar^{-1} U_1, B^ = S Qbar^{-1} U_1."""
    S = s_hat(prob, t0, t1, red)
    U, sig, _ = np.linalg.svd(S.T, full_matrices=False)
    tol = (sig[0] if sig.size else 0.0) * max(S.shape) * np.finfo(float).eps
    U1 = U[:, :int(np.sum(sig > tol))]
    Qi = qbar_inv(red)
    Qw = U1.T @ Qi @ U1
    return dict(S=S, U1=U1, Qbar_inv=Qi, Qw=0.5 * (Qw + Qw.T), Bhat=S @ Qi @ U1)


def sub_problem(prob: Uftoc, t0: int, t1: int, QN=None, lN=None, cN=0.0, x0=None) -> Uftoc:
    """Stages t0..t1-1 of prob as a UFTOC problem (Eq. sub_problem_dscr)."""
    n = prob.n
    return Uftoc(n, prob.A[t0:t1], prob.B[t0:t1], prob.a[t0:t1], prob.Q[t0:t1],
                 prob.l[t0:t1], prob.c[t0:t1],
                 np.zeros((n, n)) if QN is None else QN,
                 np.zeros(n) if lN is None else lN, cN,
                 np.zeros(n) if x0 is None else x0)


def reduce_last(prob: Uftoc, t0: int) -> dict:
    """Last subproblem: terminal known, Algorithms 1-2 give P_0, Psi_0, cbar_0."""
    sp = sub_problem(prob, t0, prob.N, prob.QN, prob.lN, prob.cN)
    r = riccati(sp)
    assert r["status"] == 0
    return dict(Qxhat=r["P0"], lxhat=-r["Psi0"], chat=r["cbar0"])


def master_problem(prob: Uftoc, reds: list, last: dict, u1s: list = None) -> Uftoc:
    """Eq. red_mpc_problem: stage i has A^_i, B^_i, a^_i, Q^_i = blkdiag(Q^_x,i, Q^_w,i),
    l = (l^_x,i, 0), c^_i; terminal (Q^_x,p, l^_x,p, c^_p).  T-form: Q^_w,i = B^_i
    (n x n); with u1s (reduce_u1 per chunk): B^_i = S Qbar^{-1} U_1 (n x n_uo,i) and
    Q^_w,i = U_1^T Qbar^{-1} U_1."""
    n = prob.n
    A, B, a, Q, l, c = [], [], [], [], [], []
    for i, r in enumerate(reds):
        Bi, Qw = (r["Bhat"], r["Bhat"]) if u1s is None else (u1s[i]["Bhat"], u1s[i]["Qw"])
        mi = Bi.shape[1]
        A.append(r["Ahat"])
        B.append(Bi)
        a.append(r["ahat"])
        Qi = np.zeros((n + mi, n + mi))
        Qi[:n, :n] = r["Qxhat"]
        Qi[n:, n:] = Qw
        Q.append(Qi)
        l.append(np.concatenate([r["lxhat"], np.zeros(mi)]))
        c.append(r["chat"])
    return Uftoc(n, A, B, a, Q, l, c, last["Qxhat"], last["lxhat"], last["chat"],
                 np.asarray(prob.x0, float).copy())


def chunk_bounds(N: int, L: int) -> list:
    """Chunks of length L, the last one taking the remainder (>= 2 chunks)."""
    if N <= L:
        L = (N + 1) // 2
    c = -(-N // L)
    b = [i * L for i in range(c)] + [N]
    return b


def tree_solve(prob: Uftoc, leaf_len: int = 4, branching: int = 2, top_len: int = 4,
               down: str = "backsub", _level: int = 0, _trace=None, form: str = "T") -> dict:
    """Algorithms 5 + 6.  Returns x (N+1, n), w (list per stage), lam (N+1, n)
    and, for down='alg6', P and Psi at every stage (from the bottom subproblems).
    form: 'T' or 'U1', the reduced input of every master stage (module docstring)."""
    n, N = prob.n, prob.N
    if N <= top_len or N < 2:
        r = riccati(prob, want_all=True)
        assert r["status"] == 0
        w, o = [], 0
        for mt in prob.m:
            w.append(r["w"][o:o + mt])
            o += mt
        if _trace is not None:
            _trace.append(("top", _level, N))
        return dict(x=r["x"], w=w, lam=r["lam"], P=r["P"], Psi=r["Psi"], levels=_level)
    L = leaf_len if _level == 0 else branching
    bnd = chunk_bounds(N, L)
    p = len(bnd) - 2                      # chunks 0..p, chunk p is the last one
    reds = [reduce_chunk(prob, bnd[i], bnd[i + 1]) for i in range(p)]
    last = reduce_last(prob, bnd[p])
    u1s = [reduce_u1(prob, bnd[i], bnd[i + 1], reds[i]) for i in range(p)] if form == "U1" else None
    master = master_problem(prob, reds, last, u1s)
    if _trace is not None:
        _trace.append(("level", _level, N, bnd))
    top = tree_solve(master, leaf_len, branching, top_len, down, _level + 1, _trace, form)
    xh, wh, lh = top["x"], top["w"], top["lam"]
    x = np.zeros((N + 1, n))
    lam = np.zeros((N + 1, n))
    w = [None] * N
    Pout = [None] * (N + 1)
    Psiout = [None] * (N + 1)
    for i in range(p + 1):
        t0, t1 = bnd[i], bnd[i + 1]
        if down == "alg6":
            # Algorithm 6: solve subproblem i with Algorithms 1-3 using the
            # parent's x^_i, P^_{i+1}, Psi^_{i+1}, c^_{i+1}.
            if i < p:
                sp = sub_problem(prob, t0, t1, top["P"][i + 1], -top["Psi"][i + 1], 0.0, xh[i])
            else:
                sp = sub_problem(prob, t0, t1, prob.QN, prob.lN, prob.cN, xh[i])
            r = riccati(sp, want_all=True)
            assert r["status"] == 0
            x[t0:t1 + 1] = r["x"]
            lam[t0:t1 + 1] = r["lam"]
            o = 0
            for t in range(t0, t1):
                mt = prob.B[t].shape[1]
                w[t] = r["w"][o:o + mt]
                o += mt
            for j in range(t1 - t0 + 1):
                Pout[t0 + j] = r["P"][j]
                Psiout[t0 + j] = r["Psi"][j]
        else:
            # back-substitution with the stored preliminary feedback
            xt = np.asarray(xh[i], float).copy()
            x[t0] = xt
            if i < p and u1s is not None:
                # U_1 form: the chunk's inputs wbar = Qbar^{-1} U_1 w^_i, split per stage
                wbar = u1s[i]["Qbar_inv"] @ (u1s[i]["U1"] @ wh[i])
                wofs = np.concatenate([[0], np.cumsum([prob.B[t].shape[1] for t in range(t0, t1)])])
            for t in range(t0, t1):
                A, B, a = prob.A[t], prob.B[t], prob.a[t]
                if i < p:
                    j = t - t0
                    if u1s is None:
                        wt = reds[i]["k"][j] + reds[i]["K"][j] @ xt - reds[i]["L"][j] @ wh[i]
                    else:
                        wt = reds[i]["k"][j] + reds[i]["K"][j] @ xt + wbar[wofs[j]:wofs[j + 1]]
                else:
                    wt = None
                if wt is None:
                    break
                w[t] = wt
                xt = A @ xt + B @ wt + a
                x[t + 1] = xt
            if i == p:
                # last chunk: its own full Riccati solve with the known terminal
                sp = sub_problem(prob, t0, t1, prob.QN, prob.lN, prob.cN, xh[i])
                r = riccati(sp)
                assert r["status"] == 0
                x[t0:t1 + 1] = r["x"]
                o = 0
                for t in range(t0, t1):
                    mt = prob.B[t].shape[1]
                    w[t] = r["w"][o:o + mt]
                    o += mt
                lam[t1] = prob.QN @ x[t1] + prob.lN
            else:
                lam[t1] = lh[i + 1]
            # costate sweep: lambda_t = Q_x x_t + Q_xw w_t + l_x + A^T lambda_{t+1}
            for t in range(t1 - 1, t0 - 1, -1):
                Q, l, A = prob.Q[t], prob.l[t], prob.A[t]
                lam[t] = Q[:n, :n] @ x[t] + Q[:n, n:] @ w[t] + l[:n] + A.T @ lam[t + 1]
    out = dict(x=x, w=w, lam=lam, levels=top["levels"])
    if down == "alg6":
        out["P"], out["Psi"] = Pout, Psiout
    return out
