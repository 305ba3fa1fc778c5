"""Helpers for the GPU tests: marshal seeded MHE instances into the library's
layout (column-major blocks, instance-major stage arrays) and split its outputs
back per instance.  No arithmetic of the method lives here."""
from __future__ import annotations

import numpy as np

from paper_1510_03110_gb300 import mhe, synth


def device_inputs(insts, device="cuda"):
    """MHE-form data of several instances with equal (n, m, q) -> torch tensors."""
    import torch
    n, m, q = insts[0]["n"], insts[0]["m"], insts[0]["q"]
    cat = lambda key, cm: np.concatenate(  # noqa: E731
        [(synth.colmajor(p[key]) if cm else p[key]).reshape(-1) for p in insts] + [np.zeros(0)])
    t = lambda arr: torch.from_numpy(np.ascontiguousarray(arr, dtype=np.float64)).to(device)  # noqa: E731
    S = int(sum(p["N"] - 1 for p in insts))
    d = dict(n=n, m=m, q=q, S=S, N=[p["N"] for p in insts],
             A=t(cat("A", True)), B=t(cat("B", True)), C=t(cat("C", True)), R=t(cat("R", True)),
             a=t(cat("a", False)), yt=t(cat("yt", False)), wt=t(cat("wt", False)),
             x0=t(np.concatenate([p["x0"] for p in insts])),
             P0inv=t(np.concatenate([synth.colmajor(p["P0inv"]).reshape(-1) for p in insts])))
    nq = n + m
    d["Q"] = torch.empty(max(1, S * nq * nq), dtype=torch.float64, device=device)
    d["l"] = torch.empty(max(1, S * nq), dtype=torch.float64, device=device)
    if S > 0:
        mhe.mhe_assemble(n, m, q, d["C"].view(S, -1), d["R"], d["yt"], d["wt"], d["Q"], d["l"])
    return d


def split(x, w, lam, N, n, m):
    x = x.double().cpu().numpy().reshape(-1, n)
    lam = lam.double().cpu().numpy().reshape(-1, n)
    w = w.double().cpu().numpy().reshape(-1)
    out, xo, wo = [], 0, 0
    for Nb in N:
        nw_b = n + (Nb - 1) * m
        out.append(dict(x=x[xo:xo + Nb + 1], lam=lam[xo:xo + Nb + 1], w=w[wo:wo + nw_b]))
        xo += Nb + 1
        wo += nw_b
    return out


def rel_err(sol, ref) -> float:
    """max over x, w, lambda of ||z - z_ref||_inf / ||z_ref||_inf."""
    e = 0.0
    for k in ("x", "w", "lam"):
        a, b = np.asarray(sol[k]).ravel(), np.asarray(ref[k]).ravel()
        if b.size == 0:
            continue
        den = np.abs(b).max()
        e = max(e, float(np.abs(a - b).max() / den) if den > 0 else float(np.abs(a - b).max()))
    return e


def device_from_pool(n, m, q, pool, idx, x0, device="cuda"):
    """Stages drawn from a seeded pool (synth.batch_uneven / stage_pool) -> device
    arrays in the library's layout, expanded on the device by an index gather."""
    import torch
    ix = torch.from_numpy(np.asarray(idx, dtype=np.int64)).to(device)
    d = {}
    for k in ("A", "B", "C", "R"):
        p = torch.from_numpy(synth.colmajor(pool[k]).reshape(len(pool[k]), -1)).to(device)
        d[k] = p.index_select(0, ix).contiguous().reshape(-1)
    for k in ("a", "yt", "wt"):
        p = torch.from_numpy(np.ascontiguousarray(pool[k])).to(device)
        d[k] = p.index_select(0, ix).contiguous().reshape(-1)
    x0 = np.asarray(x0, dtype=np.float64).reshape(-1, n)
    d["x0"] = torch.from_numpy(np.ascontiguousarray(x0).reshape(-1)).to(device)
    d["P0inv"] = torch.eye(n, dtype=torch.float64, device=device).reshape(1, -1).repeat(len(x0), 1).reshape(-1)
    return d
