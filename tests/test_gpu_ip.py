"""The interior-point outer loop (mhe_ip_solve) for MHE with box-bounded
process noise (Section II: constrained MHE, whose Newton steps are UFTOC
problems solved by the tree), in both of its methods: Mehrotra's
predictor-corrector and barrier path following.

Against the oracle's exact solution of the bounded problem (oracle/boxqp.py,
a primal active-set method on the dense KKT system):
  * every bounded input strictly inside its box;
  * the objective above the exact minimum by no more than the log barrier's
    duality gap (2 log terms per bounded input, each worth mu_final), with a
    factor 10 for the iterate being only near the central path;
  * the inputs close to the exact ones;
and at sizes the oracle's active-set method is too slow for, the optimality
conditions themselves, from the C oracle's KKT rows: the equality rows hold,
and each bounded input's gradient is that of a log barrier of parameter at
most 10 mu_final (so an input far from its bounds has a vanishing gradient,
and one near a bound a gradient pointing into the box)."""
import numpy as np
import pytest

import oracle
from oracle import boxqp, dense
from paper_1510_03110_gb300 import mhe, synth

from gpu_util import device_inputs, rel_err, split

pytestmark = pytest.mark.gpu


def _bounds(insts, frac, seed):
    """Per instance, a box around zero whose half-width is frac times the largest
    |w_t[j]| of the unconstrained step (the oracle's), shifted by 10%."""
    rng = np.random.default_rng(seed)
    los, his, refs = [], [], []
    for p in insts:
        prob = oracle.mhe_to_uftoc(p)
        ref = oracle.riccati(prob)
        n, m, N = p["n"], p["m"], p["N"]
        wt = ref["w"][n:].reshape(N - 1, m) if N > 1 else np.ones((1, m))
        c = frac * np.maximum(np.abs(wt).max(axis=0), 1e-3)
        s = rng.uniform(-0.1, 0.1, m) * c
        los.append(-c + s)
        his.append(c + s)
        refs.append((prob, ref))
    return np.stack(los), np.stack(his), refs


METHODS = [mhe.MHE_IP_PREDICTOR_CORRECTOR, mhe.MHE_IP_PATH_FOLLOWING]


def _run(insts, lo, hi, prec=mhe.MHE_FP64, mu_final=0.0, method=mhe.MHE_IP_PREDICTOR_CORRECTOR, **kw):
    import torch
    n, m = insts[0]["n"], insts[0]["m"]
    Ns = [p["N"] for p in insts]
    d = device_inputs(insts)
    s = mhe.Solver(n, m, Ns, prec=prec, **kw)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float64).reshape(-1)).cuda()  # noqa: E731
    x, w, lam, steps = s.ip_solve(d["A"], d["B"], d["Q"], d["P0inv"], d["l"], d["a"], d["x0"], t(lo), t(hi),
                                  mu_final=mu_final, method=method)
    torch.cuda.synchronize()
    info = s.infos()
    s.close()
    return split(x, w, lam, Ns, n, m), steps, info


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("n,m", [(4, 2), (3, 2), (6, 3)])
def test_ip_matches_the_exact_bounded_solution(n, m, method):
    Ns = [2, 5, 17, 33]
    insts = [synth.mhe_instance(2300 + 7 * i + n, n, m, m, N) for i, N in enumerate(Ns)]
    lo, hi, refs = _bounds(insts, 0.6, 5 + n)
    mu_final = 1e-9
    got, steps, info = _run(insts, lo, hi, mu_final=mu_final, method=method)
    assert 0 < steps <= 200
    assert [int(v) for v in info["status"]] == [0] * len(Ns)
    for b, p in enumerate(insts):
        prob = refs[b][0]
        exact = boxqp.solve(prob, lo[b], hi[b])
        N = p["N"]
        wb = got[b]["w"][n:].reshape(N - 1, m) if N > 1 else np.zeros((0, m))
        assert np.all(wb > lo[b]) and np.all(wb < hi[b]), b
        # the dynamics hold
        xb = got[b]["x"]
        for t in range(N):
            wt = got[b]["w"][:n] if t == 0 else wb[t - 1]
            assert np.abs(prob.A[t] @ xb[t] + prob.B[t] @ wt + prob.a[t] - xb[t + 1]).max() <= 1e-11 * (
                1 + np.abs(xb).max())
        f_ip = boxqp.objective_of(prob, got[b]["x"], got[b]["w"])
        f_ex = boxqp.objective_of(prob, exact["x"], exact["w"])
        gap = 10 * 2 * (N - 1) * m * mu_final
        assert -1e-11 * (1 + abs(f_ex)) <= f_ip - f_ex <= gap + 1e-11 * (1 + abs(f_ex)), (b, f_ip - f_ex)
        assert np.abs(got[b]["w"] - exact["w"]).max() <= 1e-4 * (1 + np.abs(exact["w"]).max()), b
        assert np.abs(got[b]["x"] - exact["x"]).max() <= 1e-4 * (1 + np.abs(exact["x"]).max()), b
    if sum(len(boxqp.solve(r[0], lo[b], hi[b])["active"]) for b, r in enumerate(refs)) == 0:
        pytest.fail("the boxes bind nowhere: the case tests nothing")


def test_loose_bounds_give_the_unconstrained_step():
    n, m = 6, 3
    Ns = [3, 40, 100]
    insts = [synth.mhe_instance(2400 + i, n, m, m, N) for i, N in enumerate(Ns)]
    lo, hi, refs = _bounds(insts, 1e3, 11)
    got, steps, info = _run(insts, lo, hi)
    assert [int(v) for v in info["status"]] == [0] * len(Ns)
    for b in range(len(Ns)):
        ref = refs[b][1]
        assert rel_err(dict(x=got[b]["x"], w=got[b]["w"], lam=ref["lam"]), ref) <= 1e-6, b


def _barrier_certificate(prob, sol, lo, hi, mu_final):
    """Equality rows of the plain KKT system at (x, w, lam) and, for every bounded
    input, |gradient| <= 10 mu_final (1/(w-lo) + 1/(hi-w)) with the barrier's sign."""
    n, N = prob.n, prob.N
    r = oracle.kkt_residual(prob, sol["x"], sol["w"], sol["lam"])
    scale = r["K_inf"] * r["z_inf"] + r["b_inf"]
    assert np.abs(r["rx0"]).max() <= 1e-12 * scale
    assert np.abs(r["ra"]).max() <= 1e-11 * scale
    assert np.abs(r["rlN"]).max() <= 1e-11 * scale
    off = 0
    wo = np.concatenate([[0], np.cumsum(prob.m)])
    worst = 0.0
    for t in range(N):
        assert np.abs(r["rl"][off:off + n]).max() <= 1e-10 * scale, t
        g = r["rl"][off + n:off + n + prob.m[t]]          # gradient of the Lagrangian in w_t
        if t == 0:
            assert np.abs(g).max() <= 1e-10 * scale
        else:
            w = sol["w"][wo[t]:wo[t + 1]]
            dl, dh = w - lo, hi - w
            assert np.all(dl > 0) and np.all(dh > 0), t
            allow = 10 * mu_final * (1 / dl + 1 / dh) + 1e-10 * scale
            worst = max(worst, float(np.max(np.abs(g) / allow)))
            assert np.all(np.abs(g) <= allow), (t, g, allow)
            # the barrier's sign: an input nearer its lower bound has a gradient >= 0
            near_lo = dl < 1e-3 * dh
            near_hi = dh < 1e-3 * dl
            assert np.all(g[near_lo] >= -1e-10 * scale) and np.all(g[near_hi] <= 1e-10 * scale), t
        off += n + prob.m[t]
    return worst


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("n,m", [(12, 6), (20, 10)])
def test_ip_optimality_conditions_at_larger_sizes(n, m, method):
    rng = np.random.default_rng(31 + n)
    Ns = [int(v) for v in rng.integers(50, 300, size=12)]
    insts = [synth.mhe_instance(2500 + 3 * i + n, n, m, m, N) for i, N in enumerate(Ns)]
    lo, hi, refs = _bounds(insts, 0.5, 13 + n)
    mu_final = 1e-9
    got, steps, info = _run(insts, lo, hi, mu_final=mu_final, method=method)
    assert [int(v) for v in info["status"]] == [0] * len(Ns)
    for b in (0, 5, 11):
        _barrier_certificate(refs[b][0], got[b], lo[b], hi[b], mu_final)


def test_predictor_corrector_takes_fewer_factorisations():
    """Mehrotra's predictor-corrector reaches the same solution as barrier path
    following in fewer iterations (each one factorisation)."""
    n, m = 6, 3
    rng = np.random.default_rng(41)
    Ns = [int(v) for v in rng.integers(20, 200, size=16)]
    insts = [synth.mhe_instance(2550 + i, n, m, m, N) for i, N in enumerate(Ns)]
    lo, hi, _ = _bounds(insts, 0.5, 19)
    pc, k_pc, i1 = _run(insts, lo, hi, mu_final=1e-9, method=mhe.MHE_IP_PREDICTOR_CORRECTOR)
    pf, k_pf, i2 = _run(insts, lo, hi, mu_final=1e-9, method=mhe.MHE_IP_PATH_FOLLOWING)
    assert [int(v) for v in i1["status"]] == [0] * len(Ns) and [int(v) for v in i2["status"]] == [0] * len(Ns)
    assert 0 < k_pc < k_pf, (k_pc, k_pf)
    for b in range(len(Ns)):
        assert np.abs(pc[b]["w"] - pf[b]["w"]).max() <= 1e-5 * (1 + np.abs(pf[b]["w"]).max()), b


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("n,m", [(4, 2), (12, 6)])
def test_ip_in_mixed_precision_matches_fp64(n, m, method):
    """An FP32 tree with FP64 refinement of every Newton step takes the FP64
    context's iterations and ends on its solution, within the loop's own
    stopping tolerance (a full step shorter than 1e-6 of the iterate)."""
    Ns = [5, 17, 33, 120]
    insts = [synth.mhe_instance(2800 + 7 * i + n, n, m, m, N) for i, N in enumerate(Ns)]
    lo, hi, _ = _bounds(insts, 0.6, 23 + n)
    f64, k64, i64 = _run(insts, lo, hi, mu_final=1e-9, method=method)
    f32, k32, i32 = _run(insts, lo, hi, prec=mhe.MHE_FP32_IR, mu_final=1e-9, method=method,
                         refine_tol=1e-12, max_refine=16)
    assert [int(v) for v in i32["status"]] == [0] * len(Ns)
    assert np.all(i32["relres"] <= 1e-12)
    assert abs(k32 - k64) <= 2, (k32, k64)
    for b, N in enumerate(Ns):
        wb = f32[b]["w"][n:].reshape(N - 1, m)
        assert np.all(wb > lo[b]) and np.all(wb < hi[b]), b
        assert np.abs(f32[b]["w"] - f64[b]["w"]).max() <= 1e-6 * (1 + np.abs(f64[b]["w"]).max()), b


def test_ip_on_a_tree_plan_equals_the_serial_plan():
    """The Newton steps go through whichever plan the context holds."""
    n, m = 6, 3
    Ns = [64, 200]
    insts = [synth.mhe_instance(2600 + i, n, m, m, N) for i, N in enumerate(Ns)]
    lo, hi, _ = _bounds(insts, 0.5, 17)
    tree, _, i1 = _run(insts, lo, hi, leaf_len=4, branching=4, top_len=4)
    ser, _, i2 = _run(insts, lo, hi, top_len=100000)
    for b in range(len(Ns)):
        assert np.abs(tree[b]["w"] - ser[b]["w"]).max() <= 1e-6 * (1 + np.abs(ser[b]["w"]).max())


@pytest.mark.parametrize("method", METHODS)
def test_ip_with_arrival_only_instances(method):
    """Instances with N = 1 (the arrival stage alone: nothing bounded) in a batch
    with bounded ones: they end on the unconstrained step, the others inside their
    boxes, every instance with status 0."""
    n, m = 6, 3
    Ns = [1, 12, 1, 40]
    insts = [synth.mhe_instance(2900 + i, n, m, m, N) for i, N in enumerate(Ns)]
    lo, hi, refs = _bounds(insts, 0.5, 29)
    got, steps, info = _run(insts, lo, hi, mu_final=1e-9, method=method)
    assert [int(v) for v in info["status"]] == [0] * len(Ns)
    for b, N in enumerate(Ns):
        if N == 1:
            assert rel_err(got[b], refs[b][1]) <= 1e-10, b
        else:
            wb = got[b]["w"][n:].reshape(N - 1, m)
            assert np.all(wb > lo[b]) and np.all(wb < hi[b]), b


def test_ip_iteration_limit_reports_no_convergence():
    """max_newton reached before every instance has converged: MHE_E_NO_CONVERGE
    for the call, and in info for each instance still iterating."""
    import torch
    n, m = 6, 3
    Ns = [20, 60]
    insts = [synth.mhe_instance(2950 + i, n, m, m, N) for i, N in enumerate(Ns)]
    lo, hi, _ = _bounds(insts, 0.5, 31)
    d = device_inputs(insts)
    s = mhe.Solver(n, m, Ns)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float64).reshape(-1)).cuda()  # noqa: E731
    with pytest.raises(mhe.MheError) as e:
        s.ip_solve(d["A"], d["B"], d["Q"], d["P0inv"], d["l"], d["a"], d["x0"], t(lo), t(hi), max_newton=2)
    assert e.value.code == -6
    torch.cuda.synchronize()
    assert [int(v) for v in s.infos()["status"]] == [-6, -6]
    s.close()


def test_ip_argument_errors():
    import torch
    n, m = 4, 2
    insts = [synth.mhe_instance(2700, n, m, m, 10)]
    d = device_inputs(insts)
    s = mhe.Solver(n, m, [10])
    lo = torch.full((m,), -1.0, dtype=torch.float64, device="cuda")
    with pytest.raises(mhe.SizeError):
        s.ip_solve(d["A"], d["B"], d["Q"], d["P0inv"], d["l"], d["a"], d["x0"], lo[:1], lo)
    with pytest.raises(mhe.MheError):
        s.ip_solve(d["A"], d["B"], d["Q"], d["P0inv"], d["l"], d["a"], d["x0"], None, lo)
    hi = torch.full((m,), 1.0, dtype=torch.float64, device="cuda")
    with pytest.raises(mhe.MheError):
        s.ip_solve(d["A"], d["B"], d["Q"], d["P0inv"], d["l"], d["a"], d["x0"], lo, hi, method=7)
    s.close()
