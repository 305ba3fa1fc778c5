"""GPU parity: the CUDA tree (through the C-ABI) against the FP64 oracle.

Tolerances: FP64 mode <= 1e-10 relative per instance (max over x, w, lambda of
||z - z_oracle||_inf / ||z_oracle||_inf); FP32 + refinement <= 1e-8 relative
error and relative KKT residual <= the requested refine_tol.
"""
import numpy as np
import pytest

import oracle
from paper_1510_03110_gb300 import mhe, synth

from gpu_util import device_inputs, rel_err, split

pytestmark = pytest.mark.gpu


def _oracle(insts):
    out = []
    for p in insts:
        r = oracle.riccati(oracle.mhe_to_uftoc(p))
        assert r["status"] == 0
        out.append(r)
    return out


def _run(insts, fused=True, **kw):
    d = device_inputs(insts)
    s = mhe.Solver(d["n"], d["m"], d["N"], **kw)
    if fused:
        x, w, lam = s.factor_solve(d["A"], d["B"], d["Q"], d["P0inv"], d["l"], d["a"], d["x0"])
    else:
        s.factor(d["A"], d["B"], d["Q"], d["P0inv"])
        x, w, lam = s.solve(d["l"], d["a"], d["x0"])
    import torch
    torch.cuda.synchronize()
    sols = split(x, w, lam, d["N"], d["n"], d["m"])
    info = s.infos()
    s.close()
    return sols, info


def test_assembly_matches_oracle():
    """Step a0 on the GPU vs the oracle's Section II stage data."""
    p = synth.mhe_instance(3, 4, 2, 2, 9)
    d = device_inputs([p])
    u = oracle.mhe_to_uftoc(p)
    Q = d["Q"].cpu().numpy().reshape(-1, 6, 6)
    l = d["l"].cpu().numpy().reshape(-1, 6)
    for s in range(p["N"] - 1):
        Qo = u.Q[s + 1]
        assert np.abs(Q[s].T - Qo).max() <= 1e-13 * np.abs(Qo).max()
        assert np.abs(l[s] - u.l[s + 1]).max() <= 1e-13 * np.abs(u.l[s + 1]).max()


PLANS = [dict(), dict(leaf_len=2, branching=2, top_len=2), dict(leaf_len=3, branching=3, top_len=1),
         dict(leaf_len=5, branching=4, top_len=3), dict(top_len=1000)]


@pytest.mark.parametrize("plan", PLANS)
@pytest.mark.parametrize("fused", [True, False])
def test_fp64_small_case_nx4_N64(plan, fused):
    """nx=4, nw=2, ny=2, N=64, seed 0: tree and serial plans vs the oracle."""
    insts = [synth.mhe_instance(0, 4, 2, 2, 64)]
    sols, info = _run(insts, fused=fused, prec=mhe.MHE_FP64, **plan)
    ref = _oracle(insts)
    assert info["status"][0] == 0
    assert rel_err(sols[0], ref[0]) <= 1e-10
    assert info["relres"][0] <= 1e-12


@pytest.mark.parametrize("n,m", [(1, 1), (2, 1), (3, 2), (6, 3), (12, 6), (20, 10), (24, 12)])
def test_fp64_uneven_batch(n, m):
    """Uneven horizons (edge cases N = 1, 2, 3 and ragged last chunks) in one batch."""
    Ns = [1, 2, 3, 7, 17, 64, 101, 250]
    insts = [synth.mhe_instance(100 + i, n, m, m, N) for i, N in enumerate(Ns)]
    sols, info = _run(insts, prec=mhe.MHE_FP64, leaf_len=max(4, -(-n // m)), branching=3, top_len=2)
    ref = _oracle(insts)
    for b in range(len(Ns)):
        assert info["status"][b] == 0, b
        assert rel_err(sols[b], ref[b]) <= 1e-10, (b, rel_err(sols[b], ref[b]))


@pytest.mark.parametrize("n,m", [(6, 3), (12, 6), (24, 12)])
def test_fp32_refined_uneven_batch(n, m):
    Ns = [2, 5, 33, 64, 200, 301]
    insts = [synth.mhe_instance(200 + i, n, m, m, N) for i, N in enumerate(Ns)]
    sols, info = _run(insts, prec=mhe.MHE_FP32_IR, refine_tol=1e-12, max_refine=8)
    ref = _oracle(insts)
    for b in range(len(Ns)):
        assert info["status"][b] == 0, (b, info[b])
        assert info["relres"][b] <= 1e-12
        assert rel_err(sols[b], ref[b]) <= 1e-8, (b, rel_err(sols[b], ref[b]))


def test_fp64_long_horizon_nx20_sampled():
    """nx=20, nw=10, ny=10, N=1024: full parity against the oracle."""
    insts = [synth.mhe_instance(1, 20, 10, 10, 1024)]
    sols, info = _run(insts, prec=mhe.MHE_FP64, leaf_len=16, branching=8, top_len=4)
    ref = _oracle(insts)
    assert info["status"][0] == 0
    assert rel_err(sols[0], ref[0]) <= 1e-10
    assert info["relres"][0] <= 1e-12


def test_factor_once_solve_twice():
    """The stored factors serve several right-hand sides."""
    insts = [synth.mhe_instance(7, 6, 3, 3, 90)]
    d = device_inputs(insts)
    s = mhe.Solver(6, 3, d["N"], prec=mhe.MHE_FP64, leaf_len=4, branching=2, top_len=2)
    s.factor(d["A"], d["B"], d["Q"], d["P0inv"])
    x1, w1, l1 = s.solve(d["l"], d["a"], d["x0"])
    x2, w2, l2 = s.solve(2.0 * d["l"], -d["a"], d["x0"] * 0.5)
    import torch
    torch.cuda.synchronize()
    u = oracle.mhe_to_uftoc(insts[0])
    r1 = oracle.riccati(u)
    u2 = u.with_rhs(l=[2.0 * v for v in u.l], a=[-v for v in u.a], x0=u.x0 * 0.5)
    r2 = oracle.riccati(u2)
    assert rel_err(split(x1, w1, l1, d["N"], 6, 3)[0], r1) <= 1e-10
    assert rel_err(split(x2, w2, l2, d["N"], 6, 3)[0], r2) <= 1e-10
    s.close()


def test_not_factored_and_bad_shape_errors():
    d, _ = mhe.make_dims(5, 4, [10])
    with pytest.raises(mhe.MheError):
        mhe.mhe_create(d)
    s = mhe.Solver(4, 2, [8])
    import torch
    z = torch.zeros(64, dtype=torch.float64, device="cuda")
    x, w, lam = s.outputs()
    with pytest.raises(mhe.MheError) as e:
        mhe.mhe_solve(s.ctx, z, z, z, x, w, lam)
    assert e.value.code == -5
    s.close()


def test_non_pd_stage_is_reported():
    """A stage Hessian with a negative definite Q_w block: MHE_E_NOT_PD with its location."""
    import torch
    p = synth.mhe_instance(9, 4, 2, 2, 20)
    d = device_inputs([p])
    Q = d["Q"].view(19, 6, 6)
    Q[10, 4:, 4:] = -1e6 * torch.eye(2, dtype=torch.float64, device="cuda")
    s = mhe.Solver(4, 2, d["N"], prec=mhe.MHE_FP64, top_len=1000)
    s.factor_solve(d["A"], d["B"], d["Q"], d["P0inv"], d["l"], d["a"], d["x0"])
    info = s.infos()
    assert info["status"][0] == -3
    assert info["stage"][0] == 11
    s.close()


def test_autotuner_returns_a_working_plan():
    insts = [synth.mhe_instance(300 + i, 6, 3, 3, N) for i, N in enumerate([40, 90, 130, 257])]
    d = device_inputs(insts)
    dims, _keep = mhe.make_dims(6, 3, d["N"], mhe.MHE_FP64)
    best = mhe.mhe_autotune(dims, d["A"], d["B"], d["Q"], d["P0inv"], d["l"], d["a"], d["x0"], reps=1)
    assert best["ms"] > 0
    assert best["leaf_len"] * 3 >= 6 and best["branching"] >= 2 and best["top_len"] >= 1
    sols, info = _run(insts, prec=mhe.MHE_FP64, leaf_len=best["leaf_len"], branching=best["branching"],
                      top_len=best["top_len"])
    ref = _oracle(insts)
    for b in range(len(insts)):
        assert rel_err(sols[b], ref[b]) <= 1e-10
