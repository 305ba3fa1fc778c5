"""ctypes binding of the plain-C serial oracle, plus the generic UFTOC container.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The generic problem is Eq. org_eqc_problem of the paper:
    min  sum_{t<N} 1/2 [x_t; w_t]^T Q_t [x_t; w_t] + l_t^T [x_t; w_t] + c_t
         + 1/2 x_N^T Q_{x,N} x_N + l_N^T x_N + c_N
    s.t. x_0 = x0,  x_{t+1} = A_t x_t + B_t w_t + a_t.
Stage t may have its own input width m_t.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "uftoc_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc into oracle/_liboracle.so (plain -O2)."""
    if force or not os.path.exists(_LIB_PATH) or \
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c99",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def load(path):
    """Load a compiled oracle library from path and declare its signatures."""
    L = ctypes.CDLL(path)
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    c_int, c_double = ctypes.c_int, ctypes.c_double
    L.orc_mhe_stage.argtypes = [c_int, c_int, c_int, dp, dp, dp, dp, dp, dp, dp]
    L.orc_mhe_stage.restype = None
    L.orc_riccati.argtypes = [c_int, c_int, ip, dp, dp, dp, dp, dp, dp, dp, dp,
                              c_double, dp, dp, dp, dp, dp, dp, dp, dp, dp]
    L.orc_riccati.restype = c_int
    L.orc_kkt_residual.argtypes = [c_int, c_int, ip, dp, dp, dp, dp, dp, dp, dp, dp,
                                   dp, dp, dp, dp, dp, dp, dp, dp]
    L.orc_kkt_residual.restype = None
    L.orc_objective.argtypes = [c_int, c_int, ip, dp, dp, dp, dp, dp, c_double, dp, dp]
    L.orc_objective.restype = c_double
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load(build())
    return _lib


def _p(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _cm(M):
    """Column-major flat copy of a 2-D matrix."""
    return np.ascontiguousarray(np.asarray(M, dtype=np.float64).T).reshape(-1)


@dataclass
class Uftoc:
    """One instance of Eq. org_eqc_problem, one numpy array per stage."""
    n: int
    A: list            # N arrays (n, n)
    B: list            # N arrays (n, m_t)
    a: list            # N arrays (n,)
    Q: list            # N arrays (n+m_t, n+m_t)
    l: list            # N arrays (n+m_t,)
    c: list            # N floats
    QN: np.ndarray     # (n, n)
    lN: np.ndarray     # (n,)
    cN: float
    x0: np.ndarray     # (n,)
    meta: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return len(self.A)

    @property
    def m(self) -> list:
        return [B.shape[1] for B in self.B]

    def packed(self):
        mt = np.asarray(self.m, dtype=np.int32)
        A = np.concatenate([_cm(x) for x in self.A]) if self.N else np.zeros(1)
        B = np.concatenate([_cm(x) for x in self.B]) if self.N else np.zeros(1)
        a = np.concatenate([np.asarray(x, np.float64) for x in self.a]) if self.N else np.zeros(1)
        Q = np.concatenate([_cm(x) for x in self.Q]) if self.N else np.zeros(1)
        l = np.concatenate([np.asarray(x, np.float64) for x in self.l]) if self.N else np.zeros(1)
        c = np.asarray(self.c, np.float64) if self.N else np.zeros(1)
        return dict(m=mt, A=A, B=B, a=a, Q=Q, l=l, c=c, QN=_cm(self.QN),
                    lN=np.asarray(self.lN, np.float64).copy(),
                    x0=np.asarray(self.x0, np.float64).copy())

    def with_rhs(self, l=None, a=None, lN=None, x0=None) -> "Uftoc":
        return Uftoc(self.n, self.A, self.B, a if a is not None else self.a, self.Q,
                     l if l is not None else self.l, self.c, self.QN,
                     lN if lN is not None else self.lN, self.cN,
                     x0 if x0 is not None else self.x0, dict(self.meta))


def mhe_stage(C, R, yt, wt, n, m, q):
    """Section II stage data (Q_t, l_t, c_t) from MHE weights; see the C source."""
    L = lib()
    Q = np.zeros((n + m) * (n + m))
    l = np.zeros(n + m)
    c = np.zeros(1)
    Cc, Rc = _cm(C), _cm(R)
    y = np.ascontiguousarray(yt, np.float64)
    w = np.ascontiguousarray(wt, np.float64)
    L.orc_mhe_stage(n, m, q, _p(Cc), _p(Rc), _p(y), _p(w), _p(Q), _p(l), _p(c))
    return Q.reshape(n + m, n + m).T.copy(), l, float(c[0])


def mhe_to_uftoc(p: dict) -> Uftoc:
    """Eq. org_mhe -> Eq. org_eqc_problem (Section II).

    Stage 0 is the arrival stage: A_0 = B_0 = I, Q_0 = diag(0, P~0^{-1}),
    l_0 = 0, c_0 = 0, a_0 = 0 (input width n).  Stages t = 1..N-1 carry the
    MHE stage k = t-1 (dynamics A_k, B_k, a_k; weights from C_k, R_k, y~_k,
    w~_k).  Terminal: Q_{x,N} = 0, l_N = 0, c_N = 0.  The horizon N is the
    UFTOC horizon, N = N^mhe + 2.
    """
    n, m, q, N = p["n"], p["m"], p["q"], p["N"]
    A = [np.eye(n)]
    B = [np.eye(n)]
    a = [np.zeros(n)]
    Q0 = np.zeros((2 * n, 2 * n))
    Q0[n:, n:] = p["P0inv"]
    Q = [Q0]
    l = [np.zeros(2 * n)]
    c = [0.0]
    for s in range(N - 1):
        Qt, lt, ct = mhe_stage(p["C"][s], p["R"][s], p["yt"][s], p["wt"][s], n, m, q)
        A.append(np.asarray(p["A"][s], np.float64))
        B.append(np.asarray(p["B"][s], np.float64))
        a.append(np.asarray(p["a"][s], np.float64))
        Q.append(Qt)
        l.append(lt)
        c.append(ct)
    return Uftoc(n, A, B, a, Q, l, c, np.zeros((n, n)), np.zeros(n), 0.0,
                 np.asarray(p["x0"], np.float64).copy(), dict(kind="mhe"))


def split_solution(prob: Uftoc, w_flat):
    """Packed w -> list of per-stage vectors."""
    out, o = [], 0
    for mt in prob.m:
        out.append(w_flat[o:o + mt])
        o += mt
    return out


def riccati(prob: Uftoc, want_all: bool = False) -> dict:
    """Serial Riccati solve of Eq. org_eqc_problem (Algorithms 1-3)."""
    L = lib()
    n, N = prob.n, prob.N
    d = prob.packed()
    x = np.zeros((N + 1) * n)
    w = np.zeros(max(1, int(np.sum(d["m"]))))
    lam = np.zeros((N + 1) * n)
    P_all = np.zeros((N + 1) * n * n) if want_all else None
    Psi_all = np.zeros((N + 1) * n) if want_all else None
    P0 = np.zeros(n * n)
    Psi0 = np.zeros(n)
    cb = np.zeros(1)
    st = L.orc_riccati(n, N, d["m"].ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                       _p(d["A"]), _p(d["B"]), _p(d["a"]), _p(d["Q"]), _p(d["l"]), _p(d["c"]),
                       _p(d["QN"]), _p(d["lN"]), float(prob.cN), _p(d["x0"]),
                       _p(x), _p(w), _p(lam), _p(P_all), _p(Psi_all), _p(P0), _p(Psi0), _p(cb))
    out = dict(status=st, x=x.reshape(N + 1, n), w=w[:int(np.sum(d["m"]))],
               lam=lam.reshape(N + 1, n), P0=P0.reshape(n, n).T.copy(), Psi0=Psi0,
               cbar0=float(cb[0]))
    if want_all:
        out["P"] = [M.reshape(n, n).T.copy() for M in P_all.reshape(N + 1, n * n)]
        out["Psi"] = [v.copy() for v in Psi_all.reshape(N + 1, n)]
    return out


def kkt_residual(prob: Uftoc, x, w, lam) -> dict:
    """KKT residual r = b - K z (rows as in the C source) and its norms."""
    L = lib()
    n, N = prob.n, prob.N
    d = prob.packed()
    x = np.ascontiguousarray(x, np.float64).reshape(-1)
    w = np.ascontiguousarray(w, np.float64).reshape(-1)
    if w.size == 0:
        w = np.zeros(1)
    lam = np.ascontiguousarray(lam, np.float64).reshape(-1)
    rx0 = np.zeros(n)
    rl = np.zeros(max(1, d["l"].size))
    ra = np.zeros(max(1, N * n))
    rlN = np.zeros(n)
    norms = np.zeros(4)
    L.orc_kkt_residual(n, N, d["m"].ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                       _p(d["A"]), _p(d["B"]), _p(d["a"]), _p(d["Q"]), _p(d["l"]),
                       _p(d["QN"]), _p(d["lN"]), _p(d["x0"]), _p(x), _p(w), _p(lam),
                       _p(rx0), _p(rl), _p(ra), _p(rlN), _p(norms))
    return dict(rx0=rx0, rl=rl, ra=ra, rlN=rlN, r_inf=norms[0], K_inf=norms[1],
                z_inf=norms[2], b_inf=norms[3],
                relres=norms[0] / (norms[1] * norms[2] + norms[3]))


def relres(prob: Uftoc, x, w, lam) -> float:
    """Normwise backward error ||r||_inf / (||K||_inf ||z||_inf + ||b||_inf)."""
    return kkt_residual(prob, x, w, lam)["relres"]


def objective(prob: Uftoc, x, w) -> float:
    """Value of the objective of Eq. org_eqc_problem at (x, w)."""
    L = lib()
    d = prob.packed()
    x = np.ascontiguousarray(x, np.float64).reshape(-1)
    w = np.ascontiguousarray(w, np.float64).reshape(-1)
    if w.size == 0:
        w = np.zeros(1)
    return float(L.orc_objective(prob.n, prob.N,
                                 d["m"].ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                 _p(d["Q"]), _p(d["l"]), _p(d["c"]), _p(d["QN"]), _p(d["lN"]),
                                 float(prob.cN), _p(x), _p(w)))
