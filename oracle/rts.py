"""Kalman filter + Rauch-Tung-Striebel smoother for the MHE model of Eq. org_mhe.

TEST INFRASTRUCTURE ONLY.  The paper compares its method with the RTS smoother
(Section VI).  For a linear-Gaussian model with uncorrelated noises (S = 0) the
smoothed means are the minimiser of Eq. org_mhe, so this textbook recursion
pins the MHE -> UFTOC transform of Section II independently of the Riccati
code:
    x_0 ~ N(x~0, P~0),  w_k ~ N(w~_k, W_k^{-1}),  y~_k = C_k x_k + e_k,
    e_k ~ N(0, V_k^{-1}),  x_{k+1} = A_k x_k + B_k w_k + a_k,
for k = 0..N^mhe, with measurements at k = 0..N^mhe.
"""
from __future__ import annotations

import numpy as np


def smooth(p: dict):
    """Smoothed means of x_0..x_{N^mhe+1} and w_0..w_{N^mhe} (requires S = 0)."""
    n, m, N = p["n"], p["m"], p["N"]
    K_steps = N - 1                       # N^mhe + 1 measured stages
    P0 = np.linalg.inv(p["P0inv"])
    xp = [None] * (K_steps + 1)           # predicted x_{k|k-1}
    Pp = [None] * (K_steps + 1)
    xf = [None] * K_steps                 # filtered x_{k|k}
    Pf = [None] * K_steps
    xp[0], Pp[0] = np.asarray(p["x0"], float), P0
    for k in range(K_steps):
        R = p["R"][k]
        W, V = R[:m, :m], R[m:, m:]
        assert np.allclose(R[:m, m:], 0.0), "RTS pin needs S = 0"
        C, A, B = p["C"][k], p["A"][k], p["B"][k]
        S = C @ Pp[k] @ C.T + np.linalg.inv(V)
        Kg = Pp[k] @ C.T @ np.linalg.inv(S)
        xf[k] = xp[k] + Kg @ (p["yt"][k] - C @ xp[k])
        Pf[k] = (np.eye(n) - Kg @ C) @ Pp[k]
        Winv = np.linalg.inv(W)
        xp[k + 1] = A @ xf[k] + B @ p["wt"][k] + p["a"][k]
        Pp[k + 1] = A @ Pf[k] @ A.T + B @ Winv @ B.T
    xs = [None] * (K_steps + 1)
    ws = [None] * K_steps
    xs[K_steps] = xp[K_steps]
    for k in range(K_steps - 1, -1, -1):
        A, B = p["A"][k], p["B"][k]
        W = p["R"][k][:m, :m]
        Ppi = np.linalg.inv(Pp[k + 1])
        J = Pf[k] @ A.T @ Ppi
        d = xs[k + 1] - xp[k + 1]
        xs[k] = xf[k] + J @ d
        ws[k] = p["wt"][k] + np.linalg.inv(W) @ B.T @ Ppi @ d
    return np.array(xs), np.array(ws)
