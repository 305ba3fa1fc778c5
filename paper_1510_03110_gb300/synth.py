"""Seeded synthetic MHE problems (input generation only; none of the method).

Construction of one MHE stage k (the data of UFTOC stage t = k + 1):
  A_k  = 0.95 * A_raw / rho(A_raw),  A_raw ~ N(0,1)^{n x n}   (spectral radius 0.95)
  B_k  ~ N(0,1)^{n x nw}        process-noise input matrix
  C_k  ~ N(0,1)^{ny x n}        measurement matrix
  R_k  = M M^T + 0.1 I,  M ~ N(0,1)^{(nw+ny) x (nw+ny)}; R_k = [[W, S], [S^T, V]]
         is the inverse joint noise covariance of (w_k, v_k) of Eq. org_mhe
  a_k, y~_k, w~_k ~ N(0,1)     offsets (y~ = y - d - v~ folds d and v~)
and per instance x~0 ~ N(0,1)^n, arrival cost P~0 = I (so P~0^{-1} = I).
Each field of an instance is drawn as one block, in the order
  A_raw (S,n,n), B (S,n,nw), C (S,ny,n), M (S,nw+ny,nw+ny), a (S,n), y~ (S,ny),
  w~ (S,nw), x~0 (n)
from numpy.random.default_rng (PCG64), S = N - 1 stages (N = UFTOC horizon).

Large workloads draw their stages from a seeded pool: `stage_pool` makes P
independent stages of one shape with the construction above, and each
instance picks its stage sequence with a seeded index stream.  Every stage
then has exactly the distribution above; stages in different places of a
very large workload may repeat.

Arrays are returned in math orientation (numpy row/column = matrix row/column).
The CUDA library takes column-major blocks: `colmajor` converts.
"""
from __future__ import annotations

import numpy as np

RHO = 0.95


def _spectral_scale(A_raw: np.ndarray) -> np.ndarray:
    rho = np.max(np.abs(np.linalg.eigvals(A_raw)), axis=-1)
    return RHO * A_raw / rho[..., None, None]


def stage_pool(rng: np.random.Generator, n: int, m: int, q: int, S: int,
               s_zero: bool = False) -> dict:
    """S independent MHE stages of shape (n, m, q) drawn in the documented order."""
    A = _spectral_scale(rng.standard_normal((S, n, n)))
    B = rng.standard_normal((S, n, m))
    C = rng.standard_normal((S, q, n))
    M = rng.standard_normal((S, m + q, m + q))
    R = M @ M.transpose(0, 2, 1) + 0.1 * np.eye(m + q)
    if s_zero:
        R[:, :m, m:] = 0.0
        R[:, m:, :m] = 0.0
    a = rng.standard_normal((S, n))
    yt = rng.standard_normal((S, q))
    wt = rng.standard_normal((S, m))
    return dict(A=A, B=B, C=C, R=R, a=a, yt=yt, wt=wt)


def mhe_instance(seed, n: int, m: int, q: int, N: int, s_zero: bool = False) -> dict:
    """One MHE problem with UFTOC horizon N (N - 1 measured stages)."""
    rng = np.random.default_rng(seed)
    st = stage_pool(rng, n, m, q, N - 1, s_zero=s_zero)
    x0 = rng.standard_normal(n)
    return dict(n=n, m=m, q=q, N=N, x0=x0, P0inv=np.eye(n), **st)


def instance_from_pool(pool: dict, idx: np.ndarray, x0: np.ndarray, n, m, q) -> dict:
    N = len(idx) + 1
    d = {k: pool[k][idx] for k in ("A", "B", "C", "R", "a", "yt", "wt")}
    return dict(n=n, m=m, q=q, N=N, x0=x0, P0inv=np.eye(n), **d)


def colmajor(X: np.ndarray) -> np.ndarray:
    """Stack of matrices (..., r, c) -> contiguous column-major blocks."""
    return np.ascontiguousarray(np.swapaxes(X, -1, -2))


# --- the benchmark workloads -------------------------------------------------

def batch_uneven(seed: int, count: int = 4096, nx_choices=(6, 12, 24),
                 n_lo: int = 32, n_hi: int = 2048, pool_size: int = 1 << 16) -> dict:
    """Batched uneven instances: nx ~ U{nx_choices}, nw = ny = nx/2,
    N ~ U[n_lo, n_hi] (integers), stages drawn from per-shape pools."""
    rng = np.random.default_rng(seed)
    nx = rng.choice(np.asarray(nx_choices), size=count)
    N = rng.integers(n_lo, n_hi + 1, size=count)
    buckets = {}
    for n in sorted(set(int(v) for v in nx)):
        m = q = n // 2
        members = np.nonzero(nx == n)[0]
        total = int(np.sum(N[members] - 1))
        prng = np.random.default_rng([seed, n])
        P = min(pool_size, total)
        pool = stage_pool(prng, n, m, q, P)
        irng = np.random.default_rng([seed, n, 1])
        idx = irng.integers(0, P, size=total) if P < total else np.arange(total)
        x0 = irng.standard_normal((len(members), n))
        buckets[n] = dict(n=n, m=m, q=q, members=members, N=N[members].astype(np.int64),
                          pool=pool, idx=idx, x0=x0)
    return dict(nx=nx, N=N, buckets=buckets)


def bucket_instance(b: dict, j: int) -> dict:
    """Instance j of a bucket from batch_uneven, as an mhe_instance-style dict."""
    off = int(np.sum(b["N"][:j] - 1))
    S = int(b["N"][j] - 1)
    return instance_from_pool(b["pool"], b["idx"][off:off + S], b["x0"][j], b["n"], b["m"], b["q"])


def plant_stream(seed, n: int, m: int, q: int, length: int, meas_var: float = 0.01) -> dict:
    """A receding-horizon MHE stream: `length` stages of a simulated plant.

    A_k, B_k, C_k as in stage_pool; W_k = M M^T + 0.1 I (nw x nw), R_k =
    blkdiag(W_k, (1/meas_var) I) (uncorrelated noises, V = (0.01 I)^{-1});
    the plant x_{k+1} = A_k x_k + B_k w_k + a_k with w_k ~ N(0, W_k^{-1}),
    measured y_k = C_k x_k + v_k with v_k ~ N(0, meas_var I); y~_k = y_k,
    w~_k = 0.  Fields as in stage_pool, plus x_true (length + 1, n)."""
    rng = np.random.default_rng(seed)
    A = _spectral_scale(rng.standard_normal((length, n, n)))
    B = rng.standard_normal((length, n, m))
    C = rng.standard_normal((length, q, n))
    Mw = rng.standard_normal((length, m, m))
    W = Mw @ Mw.transpose(0, 2, 1) + 0.1 * np.eye(m)
    R = np.zeros((length, m + q, m + q))
    R[:, :m, :m] = W
    R[:, m:, m:] = np.eye(q) / meas_var
    a = 0.1 * rng.standard_normal((length, n))
    x = np.zeros((length + 1, n))
    x[0] = rng.standard_normal(n)
    yt = np.zeros((length, q))
    for k in range(length):
        Lw = np.linalg.cholesky(np.linalg.inv(W[k]))
        w = Lw @ rng.standard_normal(m)
        yt[k] = C[k] @ x[k] + np.sqrt(meas_var) * rng.standard_normal(q)
        x[k + 1] = A[k] @ x[k] + B[k] @ w + a[k]
    return dict(A=A, B=B, C=C, R=R, a=a, yt=yt, wt=np.zeros((length, m)), x_true=x)


def window_of(stream: dict, start: int, N: int, x0, n: int, m: int, q: int) -> dict:
    """The MHE problem over stream stages start .. start+N-2 with arrival x~0 (P~0 = I)."""
    sl = slice(start, start + N - 1)
    return dict(n=n, m=m, q=q, N=N, x0=np.asarray(x0, float), P0inv=np.eye(n),
                **{k: stream[k][sl] for k in ("A", "B", "C", "R", "a", "yt", "wt")})


def plant_streams(seed, n: int, m: int, q: int, E: int, length: int, meas_var: float = 0.01,
                  pool_size: int = 1 << 14) -> dict:
    """E simulated plants of one shape, `length` stages each, vectorised over the
    plants; A_k, B_k, C_k, W_k drawn from a seeded pool (construction as in
    plant_stream), the plants' noises and measurements drawn per stage."""
    rng = np.random.default_rng(seed)
    P = pool_size
    A = _spectral_scale(rng.standard_normal((P, n, n)))
    B = rng.standard_normal((P, n, m))
    C = rng.standard_normal((P, q, n))
    Mw = rng.standard_normal((P, m, m))
    W = Mw @ Mw.transpose(0, 2, 1) + 0.1 * np.eye(m)
    Lw = np.linalg.cholesky(np.linalg.inv(W))
    a = 0.1 * rng.standard_normal((P, n))
    idx = rng.integers(0, P, size=(E, length))
    x = rng.standard_normal((E, n))
    yt = np.zeros((E, length, q))
    for k in range(length):
        i = idx[:, k]
        w = np.einsum("eij,ej->ei", Lw[i], rng.standard_normal((E, m)))
        yt[:, k] = np.einsum("eij,ej->ei", C[i], x) + np.sqrt(meas_var) * rng.standard_normal((E, q))
        x = np.einsum("eij,ej->ei", A[i], x) + np.einsum("eij,ej->ei", B[i], w) + a[i]
    R = np.zeros((P, m + q, m + q))
    R[:, :m, :m] = W
    R[:, m:, m:] = np.eye(q) / meas_var
    return dict(pool=dict(A=A, B=B, C=C, R=R, a=a), idx=idx, yt=yt, wt=np.zeros(m))


def stream_of(ps: dict, e: int) -> dict:
    """Plant e of plant_streams as a plant_stream-style dict."""
    i = ps["idx"][e]
    L = len(i)
    return dict(A=ps["pool"]["A"][i], B=ps["pool"]["B"][i], C=ps["pool"]["C"][i], R=ps["pool"]["R"][i],
                a=ps["pool"]["a"][i], yt=ps["yt"][e], wt=np.zeros((L, len(ps["wt"]))))
