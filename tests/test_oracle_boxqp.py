"""Pins of the box-bounded MHE oracle (oracle/boxqp.py), the exact solution the
interior-point outer loop is checked against (Section II: MHE with inequality
constraints, the Newton steps being UFTOC problems).

The pins do not use the active-set method's own reasoning:
  * a box that binds nothing gives the unconstrained Newton step (dense LU);
  * a separable scalar problem (A_t = 0 after the arrival stage, no cross
    terms) has the closed form w_t = clip(unconstrained w_t, lo, hi), derived
    by hand below;
  * on tiny instances, brute force over every face of the box (each input
    free, at its lower or at its upper bound): the solution is the feasible
    face minimiser of least cost;
  * the bound multipliers, recomputed as the KKT residual of the C oracle's
    plain rows at the solution, have the signs of a minimum.
Planted mistakes in a copy of the module must each fail one of these pins."""
import importlib.util
import itertools
import os
import sys
import tempfile

import numpy as np
import pytest

import oracle
from oracle import boxqp, dense
from oracle.core import Uftoc
from paper_1510_03110_gb300 import synth


def _instance(seed, n, m, q, N, frac=0.6):
    p = synth.mhe_instance(seed, n, m, q, N)
    prob = oracle.mhe_to_uftoc(p)
    ref = dense.solve(prob)
    wt = ref["w"][n:].reshape(N - 1, m) if N > 1 else np.zeros((0, m))
    c = frac * (np.abs(wt).max(axis=0) if N > 1 else np.ones(m))
    lo, hi = -c + 0.1 * c, c + 0.1 * c
    return prob, ref, lo, hi


def test_loose_box_is_the_unconstrained_step():
    for seed, (n, m, N) in enumerate([(3, 2, 6), (4, 2, 9), (2, 1, 5)]):
        prob, ref, lo, hi = _instance(40 + seed, n, m, m, N)
        big = 1e3 * (np.abs(hi) + np.abs(lo) + 1.0)
        out = boxqp.solve(prob, -big, big)
        assert not out["active"]
        for k in ("x", "w", "lam"):
            assert np.abs(out[k] - ref[k]).max() <= 1e-11 * (1 + np.abs(ref[k]).max()), k


def _separable(seed, N):
    """n = m = 1; arrival stage 0 (A_0 = B_0 = 1); A_t = 0 for t >= 1, Q_t diagonal."""
    rng = np.random.default_rng(seed)
    A = [np.eye(1)] + [np.zeros((1, 1)) for _ in range(N - 1)]
    B = [np.eye(1)] + [rng.uniform(0.5, 2.0, (1, 1)) * rng.choice([-1, 1]) for _ in range(N - 1)]
    a = [np.zeros(1)] + [rng.normal(size=1) for _ in range(N - 1)]
    Q = [np.diag([rng.uniform(0.5, 2.0), rng.uniform(0.5, 2.0)]) for _ in range(N)]
    l = [rng.normal(size=2) for _ in range(N)]
    c = [0.0] * N
    QN = np.array([[rng.uniform(0.5, 2.0)]])
    lN = rng.normal(size=1)
    return Uftoc(1, A, B, a, Q, l, c, QN, lN, 0.0, rng.normal(size=1))


def test_separable_scalar_problem_is_a_clipped_closed_form():
    """For t >= 1, x_{t+1} = b_t w_t + a_t depends on w_t alone and no cost term
    couples two inputs, so w_t minimises
        1/2 qw_t w^2 + lw_t w + 1/2 qx_{t+1} (b_t w + a_t)^2 + lx_{t+1} (b_t w + a_t)
    over [lo, hi] (qx_N, lx_N the terminal terms): a convex parabola, whose
    minimiser on an interval is its vertex clipped to the interval."""
    for seed in range(5):
        N = 7
        prob = _separable(100 + seed, N)
        lo, hi = np.array([-0.3]), np.array([0.4])
        out = boxqp.solve(prob, lo, hi)
        for t in range(1, N):
            b, at = prob.B[t][0, 0], prob.a[t][0]
            qw, lw = prob.Q[t][1, 1], prob.l[t][1]
            qx = prob.QN[0, 0] if t == N - 1 else prob.Q[t + 1][0, 0]
            lx = prob.lN[0] if t == N - 1 else prob.l[t + 1][0]
            vertex = -(lw + b * (qx * at + lx)) / (qw + b * b * qx)
            want = min(max(vertex, lo[0]), hi[0])
            assert abs(out["w"][t] - want) <= 1e-12, (seed, t)
        # w_0 is free: x_1 = x0 + w_0 and only stage 1's x-terms see it
        qw0, lw0 = prob.Q[0][1, 1], prob.l[0][1]
        qx1, lx1 = prob.Q[1][0, 0], prob.l[1][0]
        x0 = prob.x0[0]
        w0 = -(lw0 + qx1 * x0 + lx1) / (qw0 + qx1)
        assert abs(out["w"][0] - w0) <= 1e-12


def _face_minimiser(prob, lo, hi, pattern):
    """Minimiser of the objective with the bounded inputs of `pattern` held at a
    bound (0 free, -1 lower, +1 upper): the dense KKT system with one extra
    row per held input, by LAPACK."""
    K, b, o = dense.kkt_matrix(prob)
    bnd = boxqp.bounded_indices(prob, lo, hi)
    held = [(zi, lb if s < 0 else ub) for (zi, lb, ub), s in zip(bnd, pattern) if s != 0]
    dim = K.shape[0]
    E = np.zeros((len(held), dim))
    for r, (zi, _) in enumerate(held):
        E[r, zi] = 1.0
    # stationarity rows: K's rows with E^T nu added; the hold rows E z = value
    M = np.block([[K, np.zeros((dim, len(held)))], [E, np.zeros((len(held), len(held)))]])
    # the multiplier of a held input enters the stationarity row of that input,
    # found as the row of K whose w-column pattern is Q's row for that input
    rows = {}
    row = prob.n
    for t in range(prob.N):
        row += prob.n
        for j in range(prob.m[t]):
            rows[o["ow"] + o["wo"][t] + j] = row + j
        row += prob.m[t] + prob.n
    for r, (zi, _) in enumerate(held):
        M[rows[zi], dim + r] = 1.0
    rhs = np.concatenate([b, [v for _, v in held]])
    z = np.linalg.solve(M, rhs)
    return z[:o["ol"]]


def test_brute_force_over_every_face():
    for seed, (n, m, N) in enumerate([(3, 2, 5), (2, 2, 5), (2, 1, 9)]):
        prob, ref, lo, hi = _instance(70 + seed, n, m, m, N)
        bnd = boxqp.bounded_indices(prob, lo, hi)
        assert len(bnd) <= 8
        o = (N + 1) * n
        best, best_z = None, None
        for pattern in itertools.product((-1, 0, 1), repeat=len(bnd)):
            z = _face_minimiser(prob, lo, hi, pattern)
            if any(z[zi] < lb - 1e-12 or z[zi] > ub + 1e-12 for zi, lb, ub in bnd):
                continue
            f = boxqp.objective_of(prob, z[:o].reshape(N + 1, n), z[o:])
            if best is None or f < best - 1e-13:
                best, best_z = f, z
        out = boxqp.solve(prob, lo, hi)
        assert out["active"], "the box should bind somewhere"
        f = boxqp.objective_of(prob, out["x"], out["w"])
        assert abs(f - best) <= 1e-10 * (1 + abs(best))
        assert np.abs(out["w"] - best_z[o:]).max() <= 1e-9 * (1 + np.abs(best_z[o:]).max())
        assert np.abs(out["x"].ravel() - best_z[:o]).max() <= 1e-9 * (1 + np.abs(best_z[:o]).max())


def test_multipliers_from_the_c_residual_have_the_signs_of_a_minimum():
    """r = b - K z of the plain KKT rows (the C oracle) at the bounded solution:
    zero in every row but the stationarity rows of inputs held at a bound, where
    it is the bound's multiplier nu (<= 0 at a lower, >= 0 at an upper bound)."""
    for seed, (n, m, N) in enumerate([(4, 2, 12), (6, 3, 20), (3, 3, 30)]):
        prob, ref, lo, hi = _instance(90 + seed, n, m, m, N)
        out = boxqp.solve(prob, lo, hi)
        assert out["active"]
        r = oracle.kkt_residual(prob, out["x"], out["w"], out["lam"])
        scale = r["K_inf"] * r["z_inf"] + r["b_inf"]
        assert np.abs(r["rx0"]).max() <= 1e-12 * scale
        assert np.abs(r["ra"]).max() <= 1e-12 * scale
        assert np.abs(r["rlN"]).max() <= 1e-12 * scale
        # the packed l rows: stage t has n x-rows then m_t w-rows
        off, ow = 0, (N + 1) * n
        wo = np.concatenate([[0], np.cumsum(prob.m)])
        for t in range(N):
            assert np.abs(r["rl"][off:off + n]).max() <= 1e-12 * scale, t
            for j in range(prob.m[t]):
                zi = ow + wo[t] + j
                rv = -r["rl"][off + n + j]   # the C oracle returns -r as the correction's l
                side = out["active"].get(zi)
                if side is None:
                    assert abs(rv) <= 1e-12 * scale, (t, j)
                else:
                    w_ij = out["w"][wo[t] + j]
                    bound = lo[j] if side == "lo" else hi[j]
                    assert w_ij == bound
                    assert (rv <= 1e-12 * scale) if side == "lo" else (rv >= -1e-12 * scale), (t, j, side, rv)
                    assert abs(rv - out["nu"][zi]) <= 1e-10 * scale
            off += n + prob.m[t]
        # every input inside its box
        for t in range(1, N):
            wt = out["w"][wo[t]:wo[t + 1]]
            assert np.all(wt >= lo) and np.all(wt <= hi)


# planted mistakes: a copy of the module with one slip must fail a pin above
BOX_MUTATIONS = {
    # the multiplier sign test of a lower bound inverted
    "sign_test_swapped": ('(v if work[zi] == "lo" else -v)', '(-v if work[zi] == "lo" else v)'),
    # the full step taken even where a bound blocks it
    "step_not_shortened": ("z = z + alpha * p", "z = z + p"),
    # the bound multiplier entered in the row of the next input
    "multiplier_row_shifted": ("rows[ow + wo[t] + j] = row + j", "rows[ow + wo[t] + j] = row + j + 1"),
    # the arrival input bounded too
    "arrival_input_bounded": ("for t in range(1, N):\n        for j in range(m[t]):\n            out.append",
                              "for t in range(0, N):\n        for j in range(min(m[t], len(lo))):\n            out.append"),
}


def _mutant_module(name, tmp):
    src = open(boxqp.__file__).read()
    old, new = BOX_MUTATIONS[name]
    assert src.count(old) == 1, name
    path = os.path.join(tmp, f"boxqp_{name}.py")
    open(path, "w").write(src.replace(old, new).replace("from . import dense", "from oracle import dense"))
    spec = importlib.util.spec_from_file_location(f"boxqp_{name}", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _all_pins_pass():
    try:
        test_loose_box_is_the_unconstrained_step()
        test_separable_scalar_problem_is_a_clipped_closed_form()
        test_brute_force_over_every_face()
        test_multipliers_from_the_c_residual_have_the_signs_of_a_minimum()
    except (AssertionError, RuntimeError, np.linalg.LinAlgError, IndexError, KeyError):
        return False
    return True


@pytest.mark.parametrize("name", sorted(BOX_MUTATIONS))
def test_planted_boxqp_mistake_is_caught(monkeypatch, name):
    with tempfile.TemporaryDirectory() as tmp:
        mod = _mutant_module(name, tmp)
        monkeypatch.setattr(sys.modules[__name__], "boxqp", mod)
        assert not _all_pins_pass(), name
