"""mhe_estimate (steps a0..a7 from the MHE data of Eq. org_mhe) on the GPU.

FP64 contexts assemble Q and l internally and run the same kernels as
mhe_assemble + mhe_factor_solve, so their results are bit-identical to that
path.  FP32_IR contexts form Q only in FP32 and apply it in its factors C, R
in the FP64 residual: checked against the FP64 oracle at 1e-8 relative error
and the requested relative residual.
"""
import numpy as np
import pytest

import oracle
from paper_1510_03110_gb300 import mhe, synth

from gpu_util import device_inputs, rel_err, split

pytestmark = pytest.mark.gpu


def _estimate(d, s):
    return s.estimate(d["q"], d["A"], d["B"], d["C"], d["R"], d["a"], d["yt"], d["wt"], d["x0"], d["P0inv"])


def _oracle(insts):
    out = []
    for p in insts:
        r = oracle.riccati(oracle.mhe_to_uftoc(p))
        assert r["status"] == 0
        out.append(r)
    return out


@pytest.mark.parametrize("n,m", [(1, 1), (3, 2), (6, 3), (24, 12)])
def test_fp64_estimate_is_assemble_plus_factor_solve(n, m):
    import torch
    Ns = [1, 2, 3, 9, 40, 130]
    insts = [synth.mhe_instance(300 + i, n, m, m, N) for i, N in enumerate(Ns)]
    d = device_inputs(insts)
    plan = dict(leaf_len=max(4, -(-n // m)), branching=3, top_len=2)
    s1 = mhe.Solver(n, m, d["N"], prec=mhe.MHE_FP64, **plan)
    x1, w1, l1 = _estimate(d, s1)
    s2 = mhe.Solver(n, m, d["N"], prec=mhe.MHE_FP64, **plan)
    x2, w2, l2 = s2.factor_solve(d["A"], d["B"], d["Q"], d["P0inv"], d["l"], d["a"], d["x0"])
    torch.cuda.synchronize()
    assert torch.equal(x1, x2) and torch.equal(w1, w2) and torch.equal(l1, l2)
    ref = _oracle(insts)
    sols = split(x1, w1, l1, d["N"], n, m)
    info = s1.infos()
    for b in range(len(Ns)):
        assert info["status"][b] == 0
        assert rel_err(sols[b], ref[b]) <= 1e-10
    s1.close()
    s2.close()


@pytest.mark.parametrize("n,m", [(1, 1), (4, 2), (6, 3), (12, 6), (20, 10), (24, 12)])
@pytest.mark.parametrize("s_zero", [False, True])
def test_fp32_estimate_matches_oracle(n, m, s_zero):
    import torch
    Ns = [1, 2, 3, 33, 64, 257]
    insts = [synth.mhe_instance(400 + i, n, m, m, N, s_zero=s_zero) for i, N in enumerate(Ns)]
    d = device_inputs(insts)
    s = mhe.Solver(n, m, d["N"], prec=mhe.MHE_FP32_IR, refine_tol=1e-12, max_refine=8)
    x, w, lam = _estimate(d, s)
    torch.cuda.synchronize()
    sols = split(x, w, lam, d["N"], n, m)
    info = s.infos()
    ref = _oracle(insts)
    for b in range(len(Ns)):
        assert info["status"][b] == 0, (b, info[b])
        assert info["relres"][b] <= 1e-12
        assert rel_err(sols[b], ref[b]) <= 1e-8, (b, rel_err(sols[b], ref[b]))
    s.close()


def test_fp32_estimate_then_solve_new_rhs():
    """The factorisation from mhe_estimate serves mhe_solve; the residual still
    applies Q in its factors C, R, against the caller's l."""
    import torch
    insts = [synth.mhe_instance(9, 12, 6, 6, 150), synth.mhe_instance(10, 12, 6, 6, 31)]
    d = device_inputs(insts)
    s = mhe.Solver(12, 6, d["N"], prec=mhe.MHE_FP32_IR, refine_tol=1e-12, max_refine=8)
    _estimate(d, s)
    x, w, lam = s.solve(-0.5 * d["l"], 3.0 * d["a"], d["x0"] + 1.0)
    torch.cuda.synchronize()
    info = s.infos()
    sols = split(x, w, lam, d["N"], 12, 6)
    for b, p in enumerate(insts):
        u = oracle.mhe_to_uftoc(p)
        u2 = u.with_rhs(l=[-0.5 * v for v in u.l], a=[3.0 * v for v in u.a], x0=u.x0 + 1.0)
        r = oracle.riccati(u2)
        assert info["status"][b] == 0
        assert info["relres"][b] <= 1e-12
        assert rel_err(sols[b], r) <= 1e-8
    s.close()


def test_estimate_argument_errors():
    insts = [synth.mhe_instance(1, 6, 3, 3, 20)]
    d = device_inputs(insts)
    s = mhe.Solver(6, 3, d["N"], prec=mhe.MHE_FP32_IR)
    with pytest.raises(mhe.MheError) as e:
        s.estimate(4, d["A"], d["B"], d["C"], d["R"], d["a"], d["yt"], d["wt"], d["x0"], d["P0inv"])
    assert e.value.code == -1
    with pytest.raises(mhe.MheError) as e:
        s.estimate(3, d["A"], d["B"], None, d["R"], d["a"], d["yt"], d["wt"], d["x0"], d["P0inv"])
    assert e.value.code == -1
    s.close()


@pytest.mark.parametrize("prec,pieces", [(mhe.MHE_FP32_IR, 3), (mhe.MHE_FP32_IR, 1), (mhe.MHE_FP64, 4),
                                         (mhe.MHE_FP32_IR, 100)])
def test_estimate_host_equals_device(prec, pieces):
    """mhe_estimate_host (host buffers, pieces pipelined over two streams) gives
    the device-buffer result bit for bit: every instance's computation depends
    on its own data and plan only."""
    import torch
    n, m = 6, 3
    Ns = [1, 2, 40, 77, 3, 130, 64, 9, 200, 31]
    insts = [synth.mhe_instance(500 + i, n, m, m, N) for i, N in enumerate(Ns)]
    d = device_inputs(insts)
    kw = dict(prec=prec, refine_tol=1e-12, leaf_len=4, branching=3, top_len=2)
    s1 = mhe.Solver(n, m, d["N"], **kw)
    x1, w1, l1 = _estimate(d, s1)
    torch.cuda.synchronize()
    info1 = s1.infos()
    s2 = mhe.Solver(n, m, d["N"], **kw)
    h = {k: d[k].cpu().pin_memory() for k in ("A", "B", "C", "R", "a", "yt", "wt", "x0", "P0inv")}
    x2 = torch.zeros(x1.shape, dtype=torch.float64).pin_memory()
    w2 = torch.zeros(w1.shape, dtype=torch.float64).pin_memory()
    l2 = torch.zeros(l1.shape, dtype=torch.float64).pin_memory()
    info2 = np.zeros(len(Ns), dtype=mhe.INFO_DTYPE)
    mhe.mhe_estimate_host(s2.ctx, m, h["A"], h["B"], h["C"], h["R"], h["a"], h["yt"], h["wt"], h["x0"], h["P0inv"],
                          x2, w2, l2, info2, pieces=pieces)
    assert torch.equal(x1.cpu(), x2) and torch.equal(w1.cpu(), w2) and torch.equal(l1.cpu(), l2)
    assert np.array_equal(info1["status"], info2["status"]) and np.array_equal(info1["relres"], info2["relres"])
    ref = _oracle(insts)
    sols = split(x2, w2, l2, d["N"], n, m)
    for b in range(len(Ns)):
        assert rel_err(sols[b], ref[b]) <= (1e-10 if prec == mhe.MHE_FP64 else 1e-8)
    # a second call reuses the pipeline's engines and buffers; other piece counts re-plan
    # the engines whose instances change; inputs read in place give the same bits
    for pc, in_place in ((pieces, False), (pieces + 2, False), (pieces, False), (pieces, True)):
        s2.set_host_in_place(in_place)
        x2.zero_()
        mhe.mhe_estimate_host(s2.ctx, m, h["A"], h["B"], h["C"], h["R"], h["a"], h["yt"], h["wt"], h["x0"],
                              h["P0inv"], x2, w2, l2, info2, pieces=pc)
        assert torch.equal(x1.cpu(), x2), (pc, in_place)
    # with timing enabled the call records its pipeline's timeline: every piece's events in order
    mhe.mhe_timing_enable(s2.ctx, True)
    s2.set_host_in_place(False)
    mhe.mhe_estimate_host(s2.ctx, m, h["A"], h["B"], h["C"], h["R"], h["a"], h["yt"], h["wt"], h["x0"], h["P0inv"],
                          x2, w2, l2, info2, pieces=pieces)
    tl = mhe.mhe_pipe_timeline(s2.ctx)
    assert 1 <= len(tl) <= min(pieces, len(Ns)) and tl[0][1] == 0 and tl[-1][2] == len(Ns)
    for k, row in enumerate(tl):
        assert 0 <= row[4] <= row[5] <= row[6] <= row[7]
        if k + 1 < len(tl):
            assert row[2] == tl[k + 1][1]   # the pieces tile the batch in order
    mhe.mhe_timing_enable(s2.ctx, False)
    mhe.mhe_timing_read(s2.ctx)
    s1.close()
    s2.close()


def test_estimate_host_in_place_refuses_pageable_inputs():
    import torch
    n, m = 4, 2
    insts = [synth.mhe_instance(590, n, m, m, 12)]
    d = device_inputs(insts)
    s = mhe.Solver(n, m, d["N"], prec=mhe.MHE_FP32_IR)
    s.set_host_in_place(True)
    h = {k: d[k].cpu() for k in ("A", "B", "C", "R", "a", "yt", "wt", "x0", "P0inv")}   # pageable
    x = torch.zeros((13 * n,), dtype=torch.float64)
    w = torch.zeros((n + 11 * m,), dtype=torch.float64)
    lam = torch.zeros((13 * n,), dtype=torch.float64)
    with pytest.raises(mhe.MheError) as e:
        mhe.mhe_estimate_host(s.ctx, m, h["A"], h["B"], h["C"], h["R"], h["a"], h["yt"], h["wt"], h["x0"],
                              h["P0inv"], x, w, lam, None, pieces=2)
    assert e.value.code == -1
    s.close()


@pytest.mark.parametrize("plan", [dict(), dict(top_len=1000)])
def test_nx64_team_of_four_warps_matches_oracle(plan):
    """nx=64, nw=ny=32 (128-thread teams per subproblem, FP32 tree + FP64
    refinement): uneven horizons incl. N = 1, 2, 3 against the FP64 oracle, with
    the default tree plan and the serial plan.  The FP32 tree at this size
    contracts the residual by only ~0.5 per correction (the serial plan by
    ~1e-4), hence the generous correction budget."""
    import torch
    n, m = 64, 32
    Ns = [1, 2, 3, 17, 64, 130]
    insts = [synth.mhe_instance(600 + i, n, m, m, N) for i, N in enumerate(Ns)]
    d = device_inputs(insts)
    s = mhe.Solver(n, m, d["N"], prec=mhe.MHE_FP32_IR, refine_tol=1e-13, max_refine=60, **plan)
    x, w, lam = _estimate(d, s)
    torch.cuda.synchronize()
    info = s.infos()
    sols = split(x, w, lam, d["N"], n, m)
    ref = _oracle(insts)
    for b in range(len(Ns)):
        assert info["status"][b] == 0, (b, info[b])
        assert info["relres"][b] <= 1e-13
        assert rel_err(sols[b], ref[b]) <= 1e-8, (b, rel_err(sols[b], ref[b]))
    s.close()


@pytest.mark.parametrize("tc_prec", [mhe.MHE_TF32_IR, mhe.MHE_BF16_IR])
@pytest.mark.parametrize("plan", [dict(top_len=1000), dict()])
def test_nx64_tensor_core_products_match_oracle(plan, tc_prec):
    """MHE_TF32_IR and MHE_BF16_IR at nx=64, nw=ny=32: the stage products F, G, H
    of the reductions on the tensor cores (tcgen05 kind::tf32 with operands split
    into TF32 hi + lo, or kind::f16 with BF16 operands split three ways), with the
    serial plan (every stage) and the default tree plan (the last chunk of each
    level; the others in FP32).  Same bar as MHE_FP32_IR against the FP64 oracle;
    the solution differs bitwise from the FP32 run's (another product path ran)."""
    import torch
    n, m = 64, 32
    Ns = [1, 2, 3, 17, 64, 130]
    insts = [synth.mhe_instance(600 + i, n, m, m, N) for i, N in enumerate(Ns)]
    d = device_inputs(insts)
    ref = _oracle(insts)
    xs = {}
    for prec in (tc_prec, mhe.MHE_FP32_IR):
        s = mhe.Solver(n, m, d["N"], prec=prec, refine_tol=1e-13, max_refine=60, **plan)
        x, w, lam = _estimate(d, s)
        torch.cuda.synchronize()
        info = s.infos()
        sols = split(x, w, lam, d["N"], n, m)
        for b in range(len(Ns)):
            assert info["status"][b] == 0, (prec, b, info[b])
            assert info["relres"][b] <= 1e-13
            assert rel_err(sols[b], ref[b]) <= 1e-8, (prec, b, rel_err(sols[b], ref[b]))
        xs[prec] = x.clone()
        s.close()
    assert not torch.equal(xs[tc_prec], xs[mhe.MHE_FP32_IR])


def test_tensor_precisions_on_a_shape_without_tensor_products_are_fp32():
    """MHE_TF32_IR and MHE_BF16_IR on a shape compiled without a tensor-core
    reduction compute exactly as MHE_FP32_IR."""
    import torch
    n, m = 24, 12
    insts = [synth.mhe_instance(700 + i, n, m, m, N) for i, N in enumerate([5, 40, 99])]
    d = device_inputs(insts)
    out = []
    for prec in (mhe.MHE_TF32_IR, mhe.MHE_BF16_IR, mhe.MHE_FP32_IR):
        s = mhe.Solver(n, m, d["N"], prec=prec, refine_tol=1e-12)
        x, w, lam = _estimate(d, s)
        torch.cuda.synchronize()
        out.append(x.clone())
        s.close()
    assert torch.equal(out[0], out[2]) and torch.equal(out[1], out[2])


@pytest.mark.parametrize("prec", [mhe.MHE_FP32_IR, mhe.MHE_FP64])
def test_error_estimate_per_instance(prec):
    """mhe_info.est_relerr = ||dz_last||_inf / ||z||_inf of the last correction applied to the
    instance: zero for an instance that took no correction, positive otherwise, and at least
    the remaining error against the FP64 oracle (a correction that contracts the error shrinks
    it below the size of that correction)."""
    import torch
    n, m = 24, 12
    Ns = [1, 5, 40, 99, 300, 1000, 2045]
    insts = [synth.mhe_instance(1100 + i, n, m, m, N) for i, N in enumerate(Ns)]
    d = device_inputs(insts)
    ref = _oracle(insts)
    s = mhe.Solver(n, m, d["N"], prec=prec, refine_tol=1e-12 if prec == mhe.MHE_FP32_IR else 1e-15,
                   max_refine=8 if prec == mhe.MHE_FP32_IR else 2, leaf_len=8, branching=4, top_len=4)
    x, w, lam = _estimate(d, s)
    torch.cuda.synchronize()
    info = s.infos()
    sols = split(x, w, lam, d["N"], n, m)
    s.close()
    refined = 0
    for b in range(len(Ns)):
        est, it = float(info["est_relerr"][b]), int(info["refine_iters"][b])
        assert np.isfinite(est) and est >= 0
        if it == 0:
            assert est == 0.0
            continue
        refined += 1
        assert est > 0
        z = np.concatenate([np.ravel(sols[b][k]) for k in ("x", "w", "lam")])
        zr = np.concatenate([np.ravel(ref[b][k]) for k in ("x", "w", "lam")])
        assert np.abs(z - zr).max() / np.abs(zr).max() <= est, (b, est)
    if prec == mhe.MHE_FP32_IR:
        assert refined == len(Ns)


def test_tensor_core_wait_that_runs_out_is_reported_and_the_context_recovers():
    """The failure path of the tensor-core reductions: with the product waits limited to
    0 tries the first wait of every team runs out; the instance reports MHE_E_TIMEOUT
    with the place (level 0, its chunk, the chunk's first stage), the team issues no
    further products and waits once more (default limit) before freeing its tensor
    memory.  After the default limit is restored the same context solves correctly."""
    import torch
    n, m = 64, 32
    insts = [synth.mhe_instance(1500 + i, n, m, m, N) for i, N in enumerate([9, 20])]
    d = device_inputs(insts)
    ref = _oracle(insts)
    s = mhe.Solver(n, m, d["N"], prec=mhe.MHE_TF32_IR, top_len=1000, refine_tol=1e-12, max_refine=8)
    try:
        mhe.mhe_debug_set_tc_wait_limit(0)
        _estimate(d, s)
        torch.cuda.synchronize()
        info = s.infos()
    finally:
        mhe.mhe_debug_set_tc_wait_limit(-1)
    for b in range(2):
        assert info["status"][b] == -7, info[b]
        assert info["level"][b] == 0 and info["chunk"][b] == b and info["stage"][b] == 0, info[b]
    x, w, lam = _estimate(d, s)
    torch.cuda.synchronize()
    info = s.infos()
    sols = split(x, w, lam, d["N"], n, m)
    s.close()
    for b in range(2):
        assert info["status"][b] == 0, info[b]
        assert rel_err(sols[b], ref[b]) <= 1e-8


@pytest.mark.parametrize("n,m", [(6, 3), (12, 6), (24, 12), (20, 10), (64, 32)])
def test_double_float_residual_equals_fp64_residual(n, m):
    """The MHE-form residual of the mixed precisions in double-float arithmetic against the
    same residual with FP64 instructions: on the same iterate (the first solve, no correction)
    both report the same relres to 1e-13 absolute (the pairs carry 48 bits), and with
    refinement both reach relres <= 1e-12 and the oracle's solution within 1e-8."""
    import torch
    Ns = [1, 2, 5, 40, 300]
    insts = [synth.mhe_instance(1600 + i, n, m, m, N) for i, N in enumerate(Ns)]
    d = device_inputs(insts)
    ref = _oracle(insts)
    rel = {}
    for df in (True, False):
        s = mhe.Solver(n, m, d["N"], prec=mhe.MHE_FP32_IR, max_refine=0)
        mhe.mhe_set_double_float_residual(s.ctx, df)
        _estimate(d, s)
        torch.cuda.synchronize()
        rel[df] = np.array(s.infos()["relres"])
        s.close()
    assert np.all(rel[True] > 0)
    assert np.all(np.abs(rel[True] - rel[False]) <= 1e-13 + 1e-6 * rel[False]), (rel[True], rel[False])
    # nx = 64: the serial plan (its FP32 tree plans contract by only ~0.5 per correction)
    plan = dict(top_len=1000) if n == 64 else dict()
    for df in (True, False):
        s = mhe.Solver(n, m, d["N"], prec=mhe.MHE_FP32_IR, refine_tol=1e-12, max_refine=30, **plan)
        mhe.mhe_set_double_float_residual(s.ctx, df)
        x, w, lam = _estimate(d, s)
        torch.cuda.synchronize()
        info = s.infos()
        sols = split(x, w, lam, d["N"], n, m)
        s.close()
        for b in range(len(Ns)):
            assert info["status"][b] == 0 and info["relres"][b] <= 1e-12, (df, b, info[b])
            assert rel_err(sols[b], ref[b]) <= 1e-8, (df, b, rel_err(sols[b], ref[b]))


def test_estimate_host_async_two_contexts_from_one_thread():
    """mhe_estimate_host_async on two contexts, then mhe_estimate_host_wait on each:
    the results of the synchronous call, bit for bit."""
    import torch
    outs = []
    for n, m, seed in ((6, 3, 600), (12, 6, 700)):
        Ns = [5, 40, 200, 77, 1, 130]
        insts = [synth.mhe_instance(seed + i, n, m, m, N) for i, N in enumerate(Ns)]
        d = device_inputs(insts)
        s = mhe.Solver(n, m, d["N"], prec=mhe.MHE_FP32_IR, refine_tol=1e-12)
        h = {k: d[k].cpu().pin_memory() for k in ("A", "B", "C", "R", "a", "yt", "wt", "x0", "P0inv")}
        X, W = int(sum(N + 1 for N in Ns)), int(sum(n + (N - 1) * m for N in Ns))
        ref = [torch.zeros(X * n, dtype=torch.float64).pin_memory(), torch.zeros(W, dtype=torch.float64).pin_memory(),
               torch.zeros(X * n, dtype=torch.float64).pin_memory()]
        got = [torch.zeros_like(t).pin_memory() for t in ref]
        mhe.mhe_estimate_host(s.ctx, m, *[h[k] for k in ("A", "B", "C", "R", "a", "yt", "wt", "x0", "P0inv")],
                              *ref, None, pieces=3)
        outs.append((s, h, m, ref, got))
    for s, h, m, ref, got in outs:
        mhe.mhe_estimate_host_async(s.ctx, m, *[h[k] for k in ("A", "B", "C", "R", "a", "yt", "wt", "x0", "P0inv")],
                                    *got, None, pieces=3)
    for s, h, m, ref, got in outs:
        mhe.mhe_estimate_host_wait(s.ctx)
        for a, b in zip(ref, got):
            assert torch.equal(a, b)
        s.close()
