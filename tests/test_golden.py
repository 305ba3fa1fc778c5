"""Golden fixtures: small MHE problems (Eq. org_mhe, Section II) with their Newton
step in exact rational arithmetic (tests/golden/*.txt, written by
tests/golden/make_golden.py, which uses neither the oracle nor the CUDA path).

* The stored step is checked by substitution, exactly: x_0 = x~0, the
  dynamics, and every KKT row of Eq. org_eqc_problem (Lagrangian
  cost + sum_t lam_{t+1}^T (A_t x_t + B_t w_t + a_t - x_{t+1}) + lam_0^T (x~0 - x_0)),
  with the stage cost's gradient taken from its definition 1/2 e^T R e,
  e = [w - w~; y~ - C x], by exact central differences; the stored cost is
  the MHE cost at the stored point.
* The oracle (stage assembly + Algorithms 1-3, the dense LU solve, and the
  tree of Algorithms 4-6 over several plans, in the T-form and, with leaf
  chunks shorter than nx / nw, in the U_1 form) reproduces it to rounding.
* On the GPU, the CUDA path through the C-ABI reproduces it.
"""
import importlib.util
import os
from fractions import Fraction as F

import numpy as np
import pytest

import oracle
from oracle import dense, tree

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
NAMES = ["mhe_2x1x1_N6_exact", "mhe_1x1x1_N4_exact", "mhe_4x2x2_N5_exact"]


def load(name):
    """Fixture -> dict of exact data (lists of Fractions) in math orientation."""
    rows = {}
    for line in open(os.path.join(GOLDEN, name + ".txt")):
        if not line.strip() or line.startswith("#"):
            continue
        key, vals = line.split(":", 1)
        rows[key.strip()] = [F(v) for v in vals.split()]
    n, m, q, N = (int(v) for v in rows["dims"])

    def mat(v, r, c):
        return [v[i * c:(i + 1) * c] for i in range(r)]

    p = dict(n=n, m=m, q=q, N=N, x0=rows["x0"], P0inv=mat(rows["P0inv"], n, n), cost=rows["cost"][0])
    shapes = dict(A=(n, n), B=(n, m), C=(q, n), R=(m + q, m + q))
    for key, (r, c) in shapes.items():
        p[key] = [mat(rows[f"{key} {k}"], r, c) for k in range(N - 1)]
    for key in ("a", "yt", "wt"):
        p[key] = [rows[f"{key} {k}"] for k in range(N - 1)]
    p["sol_x"] = [rows[f"sol_x {t}"] for t in range(N + 1)]
    p["sol_w"] = [rows[f"sol_w {t}"] for t in range(N)]
    p["sol_lam"] = [rows[f"sol_lam {t}"] for t in range(N + 1)]
    return p


def as_float(p):
    """The fixture as an mhe_instance-style dict of float64 arrays."""
    fl = lambda v: np.array(v, dtype=np.float64)  # noqa: E731
    out = dict(n=p["n"], m=p["m"], q=p["q"], N=p["N"], x0=fl(p["x0"]), P0inv=fl(p["P0inv"]))
    for k in ("A", "B", "C", "R", "a", "yt", "wt"):
        out[k] = fl(p[k])
    sol = dict(x=fl(p["sol_x"]), w=np.concatenate([fl(v) for v in p["sol_w"]]), lam=fl(p["sol_lam"]))
    return out, sol


def mv(M, v):
    return [sum((M[i][j] * v[j] for j in range(len(v))), F(0)) for i in range(len(M))]


def mtv(M, v):
    return [sum((M[i][j] * v[i] for i in range(len(M))), F(0)) for j in range(len(M[0]))]


def stage_cost(p, k, x, w):
    e = [w[i] - p["wt"][k][i] for i in range(p["m"])] + \
        [p["yt"][k][i] - y for i, y in enumerate(mv(p["C"][k], x))]
    Re = mv(p["R"][k], e)
    return sum((a * b for a, b in zip(e, Re)), F(0)) / 2


def exact_grad(fun, v):
    g = []
    for i in range(len(v)):
        up, dn = list(v), list(v)
        up[i] += 1
        dn[i] -= 1
        g.append((fun(up) - fun(dn)) / 2)
    return g


@pytest.mark.parametrize("name", NAMES)
def test_fixture_is_what_the_generator_writes(name):
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(GOLDEN, "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    make = mg.FIXTURES[name + ".txt"]
    assert mg.fixture_text(name, make()) == open(os.path.join(GOLDEN, name + ".txt")).read()


@pytest.mark.parametrize("name", NAMES)
def test_exact_kkt_rows_hold_by_substitution(name):
    p = load(name)
    n, N = p["n"], p["N"]
    x, w, lam = p["sol_x"], p["sol_w"], p["sol_lam"]
    zero = [F(0)] * n
    assert x[0] == p["x0"]
    # arrival stage: A_0 = B_0 = I, a_0 = 0, cost 1/2 w_0^T P~0^{-1} w_0 (no x_0 term)
    assert [x[0][i] + w[0][i] for i in range(n)] == x[1]
    assert [lam[1][i] - lam[0][i] for i in range(n)] == zero
    assert [a + b for a, b in zip(mv(p["P0inv"], w[0]), lam[1])] == zero
    for t in range(1, N):
        k = t - 1
        xn = [a + b + c for a, b, c in zip(mv(p["A"][k], x[t]), mv(p["B"][k], w[t]), p["a"][k])]
        assert xn == x[t + 1], t
        gx = exact_grad(lambda v: stage_cost(p, k, v, w[t]), x[t])
        gw = exact_grad(lambda v: stage_cost(p, k, x[t], v), w[t])
        assert [a + b - c for a, b, c in zip(gx, mtv(p["A"][k], lam[t + 1]), lam[t])] == zero, t
        assert [a + b for a, b in zip(gw, mtv(p["B"][k], lam[t + 1]))] == [F(0)] * p["m"], t
    assert lam[N] == zero      # no terminal cost: Q_x,N = 0, l_N = 0
    e0 = [x[1][i] - p["x0"][i] for i in range(n)]
    f = sum((a * b for a, b in zip(e0, mv(p["P0inv"], e0))), F(0)) / 2
    f += sum((stage_cost(p, t - 1, x[t], w[t]) for t in range(1, N)), F(0))
    assert f == p["cost"]


def _rel(a, b):
    a, b = np.asarray(a, dtype=np.float64).ravel(), np.asarray(b, dtype=np.float64).ravel()
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("name", NAMES)
def test_oracle_reproduces_the_exact_step(name):
    p = load(name)
    pf, sol = as_float(p)
    u = oracle.mhe_to_uftoc(pf)
    r = oracle.riccati(u)
    assert r["status"] == 0
    for k in ("x", "w", "lam"):
        assert _rel(r[k], sol[k]) <= 1e-13, k
    assert abs(oracle.objective(u, r["x"], r["w"]) - float(p["cost"])) <= 1e-13 * abs(float(p["cost"]))
    assert oracle.relres(u, sol["x"], sol["w"], sol["lam"]) <= 1e-15
    d = dense.solve(u)
    for k in ("x", "w", "lam"):
        assert _rel(d[k], sol[k]) <= 1e-13, k
    plans = [(max(2, p["n"]), 2, 1, "T"), (3, 2, 2, "T"), (4, 3, 2, "T"), (1, 2, 1, "U1"), (2, 3, 1, "U1")]
    for leaf, br, top, form in plans:      # leaf_len 1 with nw = 1 < nx: only the U_1 form
        for down in ("backsub", "alg6"):
            t = tree.tree_solve(u, leaf_len=leaf, branching=br, top_len=top, down=down, form=form)
            assert _rel(t["x"], sol["x"]) <= 1e-12, (leaf, br, top, down, form)
            assert _rel(np.concatenate(t["w"]), sol["w"]) <= 1e-12, (leaf, br, top, down, form)
            assert _rel(t["lam"], sol["lam"]) <= 1e-12, (leaf, br, top, down, form)


@pytest.mark.gpu
@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("plan", [dict(leaf_len=4, branching=3, top_len=2), dict(top_len=1000)])
def test_cuda_path_reproduces_the_exact_step(name, plan):
    import torch

    from gpu_util import device_inputs, split
    from paper_1510_03110_gb300 import mhe

    pf, sol = as_float(load(name))
    d = device_inputs([pf])
    s = mhe.Solver(d["n"], d["m"], d["N"], prec=mhe.MHE_FP64, **plan)
    x, w, lam = s.factor_solve(d["A"], d["B"], d["Q"], d["P0inv"], d["l"], d["a"], d["x0"])
    torch.cuda.synchronize()
    got = split(x, w, lam, d["N"], d["n"], d["m"])[0]
    info = s.infos()
    s.close()
    assert info["status"][0] == 0
    for k in ("x", "w", "lam"):
        assert _rel(got[k], sol[k]) <= 1e-10, k


@pytest.mark.gpu
@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("prec,bound", [(0, 1e-10), (1, 1e-8)])
@pytest.mark.parametrize("plan", [dict(leaf_len=4, branching=3, top_len=2), dict(top_len=1000)])
def test_mhe_form_entry_reproduces_the_exact_step(name, prec, bound, plan):
    """mhe_estimate from the MHE weights (C, R, y~, w~): in MHE_FP32_IR the FP32 preparation pass
    (Q from FP32 products of C and R) and the FP64 residual that applies Q in its factors, which
    the bench times; in MHE_FP64 the FP64 assembly.  Both reproduce the exact rational step."""
    import torch

    from gpu_util import device_inputs, split
    from paper_1510_03110_gb300 import mhe

    pf, sol = as_float(load(name))
    d = device_inputs([pf])
    s = mhe.Solver(d["n"], d["m"], d["N"], prec=prec, **plan)
    x, w, lam = s.estimate(d["q"], d["A"], d["B"], d["C"], d["R"], d["a"], d["yt"], d["wt"], d["x0"],
                           d["P0inv"])
    torch.cuda.synchronize()
    got = split(x, w, lam, d["N"], d["n"], d["m"])[0]
    info = s.infos()
    s.close()
    assert info["status"][0] == 0
    for k in ("x", "w", "lam"):
        assert _rel(got[k], sol[k]) <= bound, k
