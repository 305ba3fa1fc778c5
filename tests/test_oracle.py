"""Pins for the oracle (CPU only).

Each test ties the oracle to something other than itself: the dense KKT LU
solve (the Newton step by definition), a hand-derived closed form, the
textbook Kalman/RTS smoother, direct expansion of the MHE cost, the closed
forms of Section IV (Eqs. QuA, B, a, Qxh_lxh_def, Qh_Bh_alternative_def),
Theorem 1, and invariance of the solution to how the tree is cut.
"""
import numpy as np
import pytest

import oracle
from oracle import dense, rts, tree
from oracle.core import Uftoc
from paper_1510_03110_gb300 import synth


def random_uftoc(seed, n, N, widths, terminal=True):
    """A generic UFTOC with SPD stage Hessians and a PSD terminal cost."""
    rng = np.random.default_rng(seed)
    A, B, a, Q, l, c = [], [], [], [], [], []
    for t in range(N):
        mt = widths[t % len(widths)]
        A.append(rng.standard_normal((n, n)) * 0.6)
        B.append(rng.standard_normal((n, mt)))
        a.append(rng.standard_normal(n))
        M = rng.standard_normal((n + mt, n + mt))
        Q.append(M @ M.T + 0.2 * np.eye(n + mt))
        l.append(rng.standard_normal(n + mt))
        c.append(float(rng.standard_normal()))
    if terminal:
        M = rng.standard_normal((n, n))
        QN, lN, cN = M @ M.T, rng.standard_normal(n), 0.7
    else:
        QN, lN, cN = np.zeros((n, n)), np.zeros(n), 0.0
    return Uftoc(n, A, B, a, Q, l, c, QN, lN, cN, rng.standard_normal(n))


def rel(a, b):
    a, b = np.asarray(a, float).ravel(), np.asarray(b, float).ravel()
    return np.abs(a - b).max() / max(1e-300, np.abs(b).max())


CASES = [(1, 1, [1]), (1, 3, [1]), (2, 5, [1, 2]), (3, 7, [2, 3, 1]), (4, 16, [2]),
         (6, 9, [3, 6]), (5, 2, [5])]


@pytest.mark.parametrize("n,N,widths", CASES)
def test_riccati_equals_dense_lu(n, N, widths):
    p = random_uftoc(10 * n + N, n, N, widths)
    r = oracle.riccati(p)
    d = dense.solve(p)
    assert r["status"] == 0
    assert rel(r["x"], d["x"]) < 1e-10
    assert rel(r["w"], d["w"]) < 1e-10
    assert rel(r["lam"], d["lam"]) < 1e-10


def test_riccati_equals_dense_lu_mhe_config1():
    """nx=4, nw=2, ny=2, N=64, seed 0 (the small FP64 case)."""
    p = synth.mhe_instance(0, 4, 2, 2, 64)
    u = oracle.mhe_to_uftoc(p)
    r = oracle.riccati(u)
    d = dense.solve(u)
    for k in ("x", "w", "lam"):
        assert rel(r[k], d[k]) < 1e-10, k


@pytest.mark.parametrize("n,N,widths", CASES)
def test_kkt_residual_of_oracle(n, N, widths):
    p = random_uftoc(7 + n * N, n, N, widths)
    r = oracle.riccati(p)
    res = oracle.kkt_residual(p, r["x"], r["w"], r["lam"])
    assert res["relres"] <= 1e-12
    # the residual routine agrees with b - K z from the dense matrix
    d = dense.solve(p)
    z = np.concatenate([r["x"].ravel(), r["w"], r["lam"].ravel()])
    rd = d["b"] - d["K"] @ z
    assert abs(res["r_inf"] - np.abs(rd).max()) <= 1e-14 + 1e-10 * np.abs(rd).max()
    assert res["K_inf"] == pytest.approx(np.abs(d["K"]).sum(axis=1).max(), rel=1e-14)
    assert res["b_inf"] == pytest.approx(np.abs(d["b"]).max(), rel=1e-14)


def test_kkt_residual_correction_rhs_solves_the_defect():
    """The returned correction right-hand side, solved as a UFTOC, gives dz with
    z + dz = the exact solution (it is r of K dz = r written in UFTOC form)."""
    p = random_uftoc(3, 3, 6, [2, 3])
    r = oracle.riccati(p)
    rng = np.random.default_rng(1)
    x = r["x"] + 1e-3 * rng.standard_normal(r["x"].shape)
    w = r["w"] + 1e-3 * rng.standard_normal(r["w"].shape)
    lam = r["lam"] + 1e-3 * rng.standard_normal(r["lam"].shape)
    res = oracle.kkt_residual(p, x, w, lam)
    assert res["r_inf"] > 1e-5
    wl = oracle.split_solution(p, res["rl"])
    l_list, o = [], 0
    for t in range(p.N):
        nq = p.n + p.m[t]
        l_list.append(res["rl"][o:o + nq])
        o += nq
    corr = p.with_rhs(l=l_list, a=list(res["ra"].reshape(p.N, p.n)), lN=res["rlN"], x0=res["rx0"])
    corr.c = [0.0] * p.N
    dz = oracle.riccati(corr)
    assert rel(x + dz["x"], r["x"]) < 1e-10
    assert rel(w + dz["w"], r["w"]) < 1e-10
    assert rel(lam + dz["lam"], r["lam"]) < 1e-10
    del wl


@pytest.mark.parametrize("n,N,widths", CASES)
def test_objective_two_ways(n, N, widths):
    """Alg 2's cbar recursion: the optimal value equals
    1/2 x0^T P_0 x0 - Psi_0^T x0 + cbar_0 (the cost-to-go at t = 0)."""
    p = random_uftoc(100 + n, n, N, widths)
    r = oracle.riccati(p)
    x0 = p.x0
    v1 = 0.5 * x0 @ r["P0"] @ x0 - r["Psi0"] @ x0 + r["cbar0"]
    v2 = oracle.objective(p, r["x"], r["w"])
    assert v1 == pytest.approx(v2, rel=1e-10, abs=1e-10)


def test_scalar_closed_form():
    """n = m = 1, N = 1, worked by hand from the KKT rows:
    w (q_w + b^2 q_N) = -(q_xw x0 + l_w + b q_N (a x0 + a0) + b l_N),
    x1 = a x0 + b w + a0,  lam1 = q_N x1 + l_N,
    lam0 = q_x x0 + q_xw w + l_x + a lam1."""
    qx, qxw, qw, lx, lw, A, b, a0, qN, lN, x0 = 2.0, 0.3, 1.5, -0.4, 0.9, 0.8, 1.7, 0.25, 3.0, -1.1, 0.6
    p = Uftoc(1, [np.array([[A]])], [np.array([[b]])], [np.array([a0])],
              [np.array([[qx, qxw], [qxw, qw]])], [np.array([lx, lw])], [0.0],
              np.array([[qN]]), np.array([lN]), 0.0, np.array([x0]))
    w = -(qxw * x0 + lw + b * qN * (A * x0 + a0) + b * lN) / (qw + b * b * qN)
    x1 = A * x0 + b * w + a0
    lam1 = qN * x1 + lN
    lam0 = qx * x0 + qxw * w + lx + A * lam1
    r = oracle.riccati(p)
    assert r["w"][0] == pytest.approx(w, rel=1e-14)
    assert r["x"][1, 0] == pytest.approx(x1, rel=1e-14)
    assert r["lam"][1, 0] == pytest.approx(lam1, rel=1e-13)
    assert r["lam"][0, 0] == pytest.approx(lam0, rel=1e-13)


@pytest.mark.parametrize("n,N", [(1, 1), (3, 5), (4, 40)])
def test_integrator_special_case(n, N):
    """A_t = B_t = I, Q_xw = 0, Q_x = q_x I, Q_w = q_w I, Q_x,N = q_N I, no linear
    terms: every P_t of Algorithm 1 is p_t I with the scalar recursion
    p_t = q_x + q_w p_{t+1} / (q_w + p_{t+1}), p_N = q_N (eliminating w_t by hand),
    and the closed-loop state is x_{t+1} = q_w / (q_w + p_{t+1}) x_t.  The tree
    reproduces it."""
    qx, qw, qN = 0.7, 1.9, 2.5
    I = np.eye(n)
    Q = np.block([[qx * I, np.zeros((n, n))], [np.zeros((n, n)), qw * I]])
    x0 = np.linspace(1.0, -1.0, n)
    p = Uftoc(n, [I] * N, [I] * N, [np.zeros(n)] * N, [Q] * N, [np.zeros(2 * n)] * N, [0.0] * N,
              qN * I, np.zeros(n), 0.0, x0)
    r = oracle.riccati(p, want_all=True)
    assert r["status"] == 0
    pt = [0.0] * (N + 1)
    pt[N] = qN
    for t in range(N - 1, -1, -1):
        pt[t] = qx + qw * pt[t + 1] / (qw + pt[t + 1])
    for t in range(N + 1):
        assert np.abs(r["P"][t] - pt[t] * I).max() <= 1e-14 * pt[t]
    x = x0.copy()
    for t in range(N):
        assert rel(r["x"][t], x) < 1e-13
        x = qw / (qw + pt[t + 1]) * x
    assert rel(r["x"][N], x) < 1e-13
    if N >= 4:
        t = tree.tree_solve(p, 2, 2, 2, "backsub")
        assert rel(t["x"], r["x"]) < 1e-12 and rel(t["lam"], r["lam"]) < 1e-12


def _mhe_cost(p, xm, wm):
    """Eq. org_mhe evaluated directly: arrival cost plus the weighted process and
    sensor noise, with v_k eliminated through y~_k = C_k x_k + (v_k - v~_k)."""
    e0 = xm[0] - p["x0"]
    f = 0.5 * e0 @ p["P0inv"] @ e0
    for k in range(p["N"] - 1):
        e = np.concatenate([wm[k] - p["wt"][k], p["yt"][k] - p["C"][k] @ xm[k]])
        f += 0.5 * e @ p["R"][k] @ e
    return f


@pytest.mark.parametrize("n,m,q", [(3, 2, 2), (4, 1, 3), (2, 3, 1), (1, 1, 1)])
def test_mhe_assembly_equals_mhe_cost(n, m, q):
    """The UFTOC stage data of Section II (with S != 0) reproduce the MHE cost of
    Eq. org_mhe at arbitrary feasible points, constants included."""
    p = synth.mhe_instance(5 + n + m, n, m, q, 7)
    u = oracle.mhe_to_uftoc(p)
    rng = np.random.default_rng(2)
    for _ in range(3):
        xm0 = rng.standard_normal(n)
        wm = [rng.standard_normal(m) for _ in range(p["N"] - 1)]
        xm = [xm0]
        for k in range(p["N"] - 1):
            xm.append(p["A"][k] @ xm[k] + p["B"][k] @ wm[k] + p["a"][k])
        # UFTOC variables: x_0 = x~0, w_0 = x_0^mhe - x~0, x_t = x_{t-1}^mhe
        xu = np.vstack([p["x0"]] + xm)
        wu = np.concatenate([xm0 - p["x0"]] + wm)
        assert oracle.objective(u, xu, wu) == pytest.approx(_mhe_cost(p, xm, wm), rel=1e-12)


@pytest.mark.parametrize("n,m,q,N", [(4, 2, 2, 20), (3, 3, 1, 9), (1, 1, 1, 6)])
def test_mhe_solution_equals_rts_smoother(n, m, q, N):
    p = synth.mhe_instance(11 + n, n, m, q, N, s_zero=True)
    u = oracle.mhe_to_uftoc(p)
    r = oracle.riccati(u)
    xs, ws = rts.smooth(p)
    assert rel(r["x"][1:], xs) < 1e-9
    wsol = oracle.split_solution(u, r["w"])
    assert rel(wsol[0], xs[0] - p["x0"]) < 1e-8
    assert rel(np.array(wsol[1:]), ws) < 1e-9


def _feedback_by_probing(sp):
    """Recover the Riccati feedback K_{t+1}, k_{t+1} of a problem from the oracle's
    solutions alone: w_t = k + K x_t is affine in x_t, so n + 1 solves from
    different initial states determine it."""
    n, N = sp.n, sp.N
    rng = np.random.default_rng(9)
    sols = []
    for j in range(n + 1):
        x0 = rng.standard_normal(n) * 3.0
        s = sp.with_rhs(x0=x0)
        r = oracle.riccati(s)
        sols.append((r["x"], oracle.split_solution(s, r["w"])))
    K, k = [], []
    for t in range(N):
        X = np.array([np.concatenate([[1.0], s[0][t]]) for s in sols])
        Wt = np.array([s[1][t] for s in sols])
        coef = np.linalg.solve(X, Wt)
        k.append(coef[0])
        K.append(coef[1:].T)
    return K, k


@pytest.mark.parametrize("n,m,L", [(4, 2, 3), (3, 1, 4), (2, 2, 1)])
def test_alg4_matches_closed_forms(n, m, L):
    """Algorithm 4 output vs the dense definitions of Section IV-B:
    A^ = prod (A_t + B_t K_{0,t+1}) (Eq. QuA), a^ (Eq. a), S = [..] (Eq. B),
    Q^_w = B^ = S Qbar^{-1} S^T (Eq. Qh_Bh_alternative_def), Q^_x = P_{0,0},
    l^_x = -Psi_{0,0} (Eq. Qxh_lxh_def)."""
    p = random_uftoc(21 + n + L, n, L, [m], terminal=False)
    red = tree.reduce_chunk(p, 0, L)
    sp = tree.sub_problem(p, 0, L)
    K0, k0 = _feedback_by_probing(sp)
    full = oracle.riccati(sp, want_all=True)
    G = [p.Q[t][n:, n:] + p.B[t].T @ full["P"][t + 1] @ p.B[t] for t in range(L)]
    Acl = [p.A[t] + p.B[t] @ K0[t] for t in range(L)]

    def prod(t1, t2):          # A_{t2} ... A_{t1} of closed-loop matrices
        M = np.eye(n)
        for t in range(t1, t2 + 1):
            M = Acl[t] @ M
        return M
    Ahat = prod(0, L - 1)
    S = np.hstack([prod(t + 1, L - 1) @ p.B[t] for t in range(L)])
    ahat = sum(prod(t + 1, L - 1) @ (p.a[t] + p.B[t] @ k0[t]) for t in range(L))
    Qbar = np.zeros((L * m, L * m))
    for t in range(L):
        Qbar[t * m:(t + 1) * m, t * m:(t + 1) * m] = G[t]
    Bhat = S @ np.linalg.solve(Qbar, S.T)
    assert rel(red["Ahat"], Ahat) < 1e-10
    assert rel(red["ahat"], ahat) < 1e-10
    assert rel(red["Bhat"], Bhat) < 1e-10
    assert rel(red["Qxhat"], full["P0"]) < 1e-10
    assert rel(red["lxhat"], -full["Psi0"]) < 1e-10
    for t in range(L):
        assert rel(red["K"][t], K0[t]) < 1e-8
        assert rel(red["k"][t], k0[t]) < 1e-8
    # the U_1 form's building blocks: S of Eq. B and Qbar^{-1} from Algorithm 4's stored factors
    assert rel(tree.s_hat(p, 0, L, red), S) < 1e-10
    assert rel(tree.qbar_inv(red), np.linalg.inv(Qbar)) < 1e-10


@pytest.mark.parametrize("n,m,L", [(4, 2, 2), (4, 2, 5), (3, 3, 3), (5, 1, 6)])
def test_theorem1_reduced_problem_is_equivalent(n, m, L):
    """Theorem 1: for any terminal cost (P^, Psi^, c^), the reduced problem
    (horizon 1, input w^ in R^n, T-form) has the same optimal value and the same
    final state as the chunk it replaces."""
    p = random_uftoc(31 + n * L, n, L, [m], terminal=False)
    red = tree.reduce_chunk(p, 0, L)
    rng = np.random.default_rng(n + L)
    for _ in range(3):
        M = rng.standard_normal((n, n))
        Ph, Psih, ch = M @ M.T, rng.standard_normal(n), 0.3
        x0 = rng.standard_normal(n)
        full = oracle.riccati(tree.sub_problem(p, 0, L, Ph, -Psih, ch, x0))
        Qr = np.zeros((2 * n, 2 * n))
        Qr[:n, :n] = red["Qxhat"]
        Qr[n:, n:] = red["Bhat"]
        rp = Uftoc(n, [red["Ahat"]], [red["Bhat"]], [red["ahat"]], [Qr],
                   [np.concatenate([red["lxhat"], np.zeros(n)])], [red["chat"]],
                   Ph, -Psih, ch, x0)
        rr = oracle.riccati(rp)
        vf = oracle.objective(tree.sub_problem(p, 0, L, Ph, -Psih, ch, x0), full["x"], full["w"])
        vr = oracle.objective(rp, rr["x"], rr["w"])
        assert vr == pytest.approx(vf, rel=1e-9)
        assert rel(rr["x"][1], full["x"][L]) < 1e-9
        # and the multiplier of the boundary state is the same
        assert rel(rr["lam"][1], full["lam"][L]) < 1e-8


@pytest.mark.parametrize("n,m,L", [(4, 2, 3), (6, 1, 2), (5, 1, 1), (3, 3, 2), (6, 2, 2)])
def test_theorem1_u1_form(n, m, L):
    """Theorem 1 in the form of Eq. Bh_def: U_1 is an orthonormal basis of range(S^T)
    with n_uo = rank S^T = min(n, L m) columns; the reduced problem (horizon 1,
    input w^ in R^{n_uo}, Q^_w = U_1^T Qbar^{-1} U_1, B^ = S Qbar^{-1} U_1) has, for
    any terminal cost, the chunk's optimal value, final state and boundary
    multiplier, and wbar = Qbar^{-1} U_1 w^ in w_t = k_{0,t+1} + K_{0,t+1} x_t + wbar_t
    (Eq. control_signal_def) gives back the chunk's inputs.  With L m < n the
    T-form's Q^_w = S Qbar^{-1} S^T has rank L m < n (the remark after Eq.
    Qh_Bh_alternative_def: its G^ is singular) while the U_1 form stays well posed."""
    p = random_uftoc(51 + n * L + m, n, L, [m], terminal=False)
    red = tree.reduce_chunk(p, 0, L)
    u1 = tree.reduce_u1(p, 0, L, red)
    U1, S, r = u1["U1"], u1["S"], min(n, L * m)
    assert U1.shape == (L * m, r)
    assert np.abs(U1.T @ U1 - np.eye(r)).max() < 1e-12
    assert rel(U1 @ (U1.T @ S.T), S.T) < 1e-12
    assert np.linalg.matrix_rank(red["Bhat"]) == r
    assert np.linalg.eigvalsh(u1["Qw"]).min() > 0
    rng = np.random.default_rng(n + 7 * L + m)
    for _ in range(3):
        M = rng.standard_normal((n, n))
        Ph, Psih, ch = M @ M.T, rng.standard_normal(n), -0.2
        x0 = rng.standard_normal(n)
        sp = tree.sub_problem(p, 0, L, Ph, -Psih, ch, x0)
        full = oracle.riccati(sp)
        Qr = np.zeros((n + r, n + r))
        Qr[:n, :n] = red["Qxhat"]
        Qr[n:, n:] = u1["Qw"]
        rp = Uftoc(n, [red["Ahat"]], [u1["Bhat"]], [red["ahat"]], [Qr],
                   [np.concatenate([red["lxhat"], np.zeros(r)])], [red["chat"]], Ph, -Psih, ch, x0)
        rr = oracle.riccati(rp)
        assert rr["status"] == 0
        vf = oracle.objective(sp, full["x"], full["w"])
        assert oracle.objective(rp, rr["x"], rr["w"]) == pytest.approx(vf, rel=1e-9)
        assert rel(rr["x"][1], full["x"][L]) < 1e-9
        assert rel(rr["lam"][1], full["lam"][L]) < 1e-8
        wbar = u1["Qbar_inv"] @ (U1 @ rr["w"])
        xt = x0.copy()
        for t in range(L):
            wt = red["k"][t] + red["K"][t] @ xt + wbar[t * m:(t + 1) * m]
            assert rel(wt, full["w"][t * m:(t + 1) * m]) < 1e-8, t
            xt = p.A[t] @ xt + p.B[t] @ wt + p.a[t]


def test_master_problem_boundary_states_by_lu():
    """Section IV-C: the master problem, solved by dense LU, gives the states of
    the original solution at the batch boundaries t_i."""
    p = synth.mhe_instance(3, 4, 2, 2, 40)
    u = oracle.mhe_to_uftoc(p)
    full = oracle.riccati(u)
    bnd = tree.chunk_bounds(u.N, 6)
    pp = len(bnd) - 2
    reds = [tree.reduce_chunk(u, bnd[i], bnd[i + 1]) for i in range(pp)]
    last = tree.reduce_last(u, bnd[pp])
    mp = tree.master_problem(u, reds, last)
    d = dense.solve(mp)
    for i in range(pp + 1):
        assert rel(d["x"][i], full["x"][bnd[i]]) < 1e-9
        assert rel(d["lam"][i], full["lam"][bnd[i]]) < 1e-8


TREES = [(2, 2, 2), (3, 2, 1), (4, 3, 4), (5, 4, 2), (8, 8, 8), (7, 3, 5), (16, 2, 3)]


@pytest.mark.parametrize("leaf,br,top", TREES)
@pytest.mark.parametrize("down", ["backsub", "alg6"])
def test_tree_invariance_mhe(leaf, br, top, down):
    """The solution does not depend on how the horizon is cut (Algorithms 5-6)."""
    p = synth.mhe_instance(0, 4, 2, 2, 64)
    u = oracle.mhe_to_uftoc(p)
    r = oracle.riccati(u)
    t = tree.tree_solve(u, leaf, br, top, down)
    assert t["levels"] >= 1
    assert rel(t["x"], r["x"]) < 1e-9
    assert rel(np.concatenate(t["w"]), r["w"]) < 1e-9
    assert rel(t["lam"], r["lam"]) < 1e-9


@pytest.mark.parametrize("N", [2, 3, 5, 17, 33])
def test_tree_invariance_generic_terminal(N):
    """Generic UFTOC with a nonzero terminal cost, uneven last chunks."""
    p = random_uftoc(40 + N, 3, N, [3, 2])
    r = oracle.riccati(p)
    for leaf, br, top in [(2, 2, 1), (3, 2, 2), (4, 5, 1)]:
        t = tree.tree_solve(p, leaf, br, top, "backsub")
        assert rel(t["x"], r["x"]) < 1e-9
        assert rel(np.concatenate(t["w"]), r["w"]) < 1e-9
        assert rel(t["lam"], r["lam"]) < 1e-9


U1_TREES = [(6, 1, 2, 2, 2), (6, 1, 3, 2, 1), (5, 1, 1, 2, 1), (3, 1, 1, 3, 1), (4, 2, 4, 3, 2), (6, 3, 2, 2, 2)]


@pytest.mark.parametrize("n,m,leaf,br,top", U1_TREES)
@pytest.mark.parametrize("down", ["backsub", "alg6"])
def test_tree_u1_form_solves_short_chunks(n, m, leaf, br, top, down):
    """Algorithms 5-6 with every master stage in the U_1 form equal the serial
    solution, including plans whose leaf chunks are too short for the T-form
    (leaf_len * nw < nx: S^T rank deficient, G^ singular)."""
    p = synth.mhe_instance(7, n, m, m, 40)
    u = oracle.mhe_to_uftoc(p)
    r = oracle.riccati(u)
    t = tree.tree_solve(u, leaf, br, top, down, form="U1")
    assert t["levels"] >= 1
    assert rel(t["x"], r["x"]) < 1e-9
    assert rel(np.concatenate(t["w"]), r["w"]) < 1e-9
    assert rel(t["lam"], r["lam"]) < 1e-9


def _pivoted_cholesky(M, rtol=1e-10):
    """M = Pi R^T R Pi^T with R = [R11 R12] (r x n, R11 upper triangular), r the
    number of pivots above rtol * max diag; returns (perm, R)."""
    M = np.array(M, float)
    n = M.shape[0]
    perm = np.arange(n)
    R = np.zeros((n, n))
    thr = rtol * max(np.max(np.diag(M)), 1e-300)
    r = 0
    for j in range(n):
        i = j + int(np.argmax(np.diag(M)[j:]))
        if M[i, i] <= thr:
            break
        M[[j, i], :] = M[[i, j], :]
        M[:, [j, i]] = M[:, [i, j]]
        R[:, [j, i]] = R[:, [i, j]]
        perm[[j, i]] = perm[[i, j]]
        R[j, j] = np.sqrt(M[j, j])
        R[j, j + 1:] = M[j, j + 1:] / R[j, j]
        M[j + 1:, j + 1:] -= np.outer(R[j, j + 1:], R[j, j + 1:])
        r += 1
    return perm, R[:r]


@pytest.mark.parametrize("n,m,L", [(6, 1, 2), (5, 1, 3), (4, 2, 2), (6, 2, 2)])
def test_pivoted_square_root_basis_gives_the_same_step(n, m, L):
    """Theorem 1 holds for any basis of range(S^T), not only an orthonormal one:
    with the T-form's Q^_w = S Qbar^{-1} S^T factored by a pivoted Cholesky,
    Pi^T Q^_w Pi = R^T R, R = [R11 R12] of rank r = min(n, L nw), the master stage
    B = Pi R^T (n x r), Q_w = I_r and, in the down pass, w^ = Pi [R11^{-1} w^'; 0]
    before wbar_t = -L_{t+1} w^ give the serial solution -- also for
    L nw < n, where the T-form's master G is singular.  (The square-root master
    stage of the CUDA path is the full-rank case, Pi = I.)"""
    q = synth.mhe_instance(11 + n + L, n, m, m, 7 * L + 3)
    u = oracle.mhe_to_uftoc(q)
    ref = oracle.riccati(u)
    bnd = tree.chunk_bounds(u.N, L)
    p = len(bnd) - 2
    reds = [tree.reduce_chunk(u, bnd[i], bnd[i + 1]) for i in range(p)]
    last = tree.reduce_last(u, bnd[p])
    A, B, a, Q, lv, c, facs = [], [], [], [], [], [], []
    for i, r in enumerate(reds):
        perm, R = _pivoted_cholesky(r["Bhat"])
        rank = R.shape[0]
        assert rank == (n if i == 0 else min(n, (bnd[i + 1] - bnd[i]) * m))   # chunk 0 holds the arrival stage
        Pi = np.eye(n)[:, perm]
        assert np.abs(Pi @ R.T @ R @ Pi.T - r["Bhat"]).max() <= 1e-10 * np.abs(r["Bhat"]).max()
        facs.append((Pi, R))
        A.append(r["Ahat"])
        B.append(Pi @ R.T)
        a.append(r["ahat"])
        Qi = np.zeros((n + rank, n + rank))
        Qi[:n, :n] = r["Qxhat"]
        Qi[n:, n:] = np.eye(rank)
        Q.append(Qi)
        lv.append(np.concatenate([r["lxhat"], np.zeros(rank)]))
        c.append(0.0)
    master = Uftoc(n, A, B, a, Q, lv, c, last["Qxhat"], last["lxhat"], 0.0, u.x0)
    mr = oracle.riccati(master)
    assert mr["status"] == 0
    wo = np.concatenate([[0], np.cumsum(master.m)])
    for i in range(p):
        Pi, R = facs[i]
        rank = R.shape[0]
        wp = mr["w"][wo[i]:wo[i + 1]]
        wT = Pi @ np.concatenate([np.linalg.solve(R[:, :rank], wp), np.zeros(n - rank)])
        xt = mr["x"][i].copy()
        assert rel(xt, ref["x"][bnd[i]]) < 1e-9
        for t in range(bnd[i], bnd[i + 1]):
            j = t - bnd[i]
            wt = reds[i]["k"][j] + reds[i]["K"][j] @ xt - reds[i]["L"][j] @ wT
            woff = int(np.sum([u.m[s] for s in range(t)]))
            assert rel(wt, ref["w"][woff:woff + u.m[t]]) < 1e-8, (i, t)
            xt = u.A[t] @ xt + u.B[t] @ wt + u.a[t]
        assert rel(xt, ref["x"][bnd[i + 1]]) < 1e-9


def test_backsubstitution_equals_literal_alg6():
    p = synth.mhe_instance(4, 3, 2, 2, 50)
    u = oracle.mhe_to_uftoc(p)
    a = tree.tree_solve(u, 3, 3, 2, "backsub")
    b = tree.tree_solve(u, 3, 3, 2, "alg6")
    assert rel(a["x"], b["x"]) < 1e-10
    assert rel(a["lam"], b["lam"]) < 1e-10
    assert rel(np.concatenate(a["w"]), np.concatenate(b["w"])) < 1e-10
    # Algorithm 6's bottom-level P, Psi reproduce lambda = P x - Psi (Section V)
    for t in range(u.N + 1):
        assert rel(b["P"][t] @ b["x"][t] - b["Psi"][t], b["lam"][t]) < 1e-9


def test_long_horizon_stays_accurate():
    """Section III: P_t is symmetric positive semidefinite; with it kept symmetric the
    recursion stays backward stable over long horizons (nx=20, N=600)."""
    p = synth.mhe_instance(105, 20, 10, 10, 600)
    u = oracle.mhe_to_uftoc(p)
    r = oracle.riccati(u)
    assert r["status"] == 0
    assert oracle.relres(u, r["x"], r["w"], r["lam"]) <= 1e-13


def test_non_pd_stage_reports_status():
    p = random_uftoc(5, 2, 4, [2], terminal=False)
    p.Q[2] = -np.eye(4)
    r = oracle.riccati(p)
    assert r["status"] == -(2 + 1)
