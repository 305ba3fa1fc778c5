"""FP64 at nx = 64 and FP64 master levels in the mixed precisions (GPU).

The FP64 reduction workspace of an nx = 64 subproblem (about 342 KB) exceeds an
SM's shared memory; its reduction keeps the workspace in global memory.  FP64
mode at nx = 64 must match the FP64 oracle to 1e-10 like every other shape, for
the serial plan and for tree plans (uneven horizons incl. N = 1, 2, 3 and
ragged last chunks).

fp64_masters = 1 runs the master problems of the levels k >= 1 (Eq.
red_mpc_problem, Algorithm 5) in FP64 -- their Cholesky factorisations
included -- on top of an FP32 (or TF32 tensor-core) level 0.  Results must meet
the mixed-precision bar against the oracle (1e-8 after refinement, relres at
the requested tolerance), and at nx = 64 with short leaves, where the FP32
master levels make the refinement contract slowly, the FP64 master levels must
reach relres <= 1e-12 within three corrections.
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


def _estimate(d, s):
    return s.estimate(d["q"], d["A"], d["B"], d["C"], d["R"], d["a"], d["yt"], d["wt"], d["x0"], d["P0inv"])


NS64 = [1, 2, 3, 17, 64, 130]


@pytest.fixture(scope="module")
def nx64():
    insts = [synth.mhe_instance(600 + i, 64, 32, 32, N) for i, N in enumerate(NS64)]
    return insts, device_inputs(insts), _oracle(insts)


@pytest.mark.parametrize("plan", [dict(top_len=1000), dict(), dict(leaf_len=5, branching=3, top_len=2)])
def test_nx64_fp64_matches_oracle(nx64, plan):
    """FP64 mode at nx = 64 through both entries (UFTOC form and MHE form)."""
    import torch
    insts, d, ref = nx64
    for entry in ("factor_solve", "estimate"):
        s = mhe.Solver(64, 32, d["N"], prec=mhe.MHE_FP64, **plan)
        if entry == "factor_solve":
            x, w, lam = s.factor_solve(d["A"], d["B"], d["Q"], d["P0inv"], d["l"], d["a"], d["x0"])
        else:
            x, w, lam = _estimate(d, s)
        torch.cuda.synchronize()
        info = s.infos()
        sols = split(x, w, lam, d["N"], 64, 32)
        for b in range(len(NS64)):
            assert info["status"][b] == 0, (entry, b, info[b])
            assert rel_err(sols[b], ref[b]) <= 1e-10, (entry, b, rel_err(sols[b], ref[b]))
        s.close()


@pytest.mark.parametrize("n,m", [(6, 3), (12, 6), (24, 12), (20, 10)])
def test_fp64_masters_match_oracle(n, m):
    """FP32 level 0 + FP64 master levels, several levels deep, against the oracle;
    factor once and solve a second right-hand side with the stored mixed factors."""
    import torch
    Ns = [1, 2, 3, 9, 40, 257, 600]
    insts = [synth.mhe_instance(800 + i, n, m, m, N) for i, N in enumerate(Ns)]
    d = device_inputs(insts)
    ref = _oracle(insts)
    plan = dict(leaf_len=max(4, -(-n // m)), branching=3, top_len=2)
    s = mhe.Solver(n, m, d["N"], prec=mhe.MHE_FP32_IR, refine_tol=1e-12, fp64_masters=True, **plan)
    assert len(mhe.mhe_plan_info(s.ctx)) >= 4
    x, w, lam = _estimate(d, s)
    torch.cuda.synchronize()
    info = s.infos()
    sols = split(x, w, lam, d["N"], n, m)
    for b in range(len(Ns)):
        assert info["status"][b] == 0, (b, info[b])
        assert info["relres"][b] <= 1e-12
        assert rel_err(sols[b], ref[b]) <= 1e-8, (b, rel_err(sols[b], ref[b]))
    # a second right-hand side on the same factorisation (the FP64 levels' stored factors reused)
    l2 = d["l"] * 0.5 + 0.25
    x2, w2, lam2 = s.solve(l2, d["a"], d["x0"])
    torch.cuda.synchronize()
    info2 = s.infos()
    sols2 = split(x2, w2, lam2, d["N"], n, m)
    s.close()
    s64 = mhe.Solver(n, m, d["N"], prec=mhe.MHE_FP64, **plan)
    x3, w3, lam3 = s64.factor_solve(d["A"], d["B"], d["Q"], d["P0inv"], l2, d["a"], d["x0"])
    torch.cuda.synchronize()
    ref2 = split(x3, w3, lam3, d["N"], n, m)
    s64.close()
    for b in range(len(Ns)):
        assert info2["status"][b] == 0, (b, info2[b])
        assert rel_err(sols2[b], ref2[b]) <= 1e-8


@pytest.mark.parametrize("prec", [mhe.MHE_FP32_IR, mhe.MHE_TF32_IR])
def test_nx64_fp64_masters_converge_in_three_corrections(prec):
    """nx = 64 with short leaves (8, branching 4, top 4): with FP32 master levels the
    refinement contracts slowly; with FP64 master levels relres <= 1e-12 within three
    corrections, and the result matches the oracle."""
    import torch
    Ns = [256, 256, 200, 37]
    insts = [synth.mhe_instance(900 + i, 64, 32, 32, N) for i, N in enumerate(Ns)]
    d = device_inputs(insts)
    ref = _oracle(insts)
    plan = dict(leaf_len=8, branching=4, top_len=4)
    iters = {}
    for masters in (True, False):
        s = mhe.Solver(64, 32, d["N"], prec=prec, refine_tol=1e-12, max_refine=3 if masters else 60,
                       fp64_masters=masters, **plan)
        x, w, lam = _estimate(d, s)
        torch.cuda.synchronize()
        info = s.infos()
        sols = split(x, w, lam, d["N"], 64, 32)
        s.close()
        iters[masters] = int(np.max(info["refine_iters"]))
        if masters:
            for b in range(len(Ns)):
                assert info["status"][b] == 0, (b, info[b])
                assert info["relres"][b] <= 1e-12
                assert rel_err(sols[b], ref[b]) <= 1e-8, (b, rel_err(sols[b], ref[b]))
    assert iters[True] <= 3 and iters[True] < iters[False], iters
