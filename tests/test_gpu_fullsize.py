"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (mhe_estimate with the same plans; FP32 tree + FP64 refinement for the
batched and nx=64 workloads, the nx=64 stage products also on the tensor
cores, FP64 for the long horizon).  With the bench's
refinement tolerance (relres <= 1e-9): every instance's status and relative
KKT residual, a property that holds at any size.  Sampled instances are
compared with the FP64 oracle solved one by one after refining to relres <=
1e-12: relres 1e-9 bounds the backward error only, and the worst-conditioned
instances of the batch (cond ~1e3 in the forward/backward ratio) then sit
~2e-6 from the oracle; at 1e-12 every sample is within the 1e-8 bar."""
import numpy as np
import pytest

import oracle
from paper_1510_03110_gb300 import mhe, synth

from gpu_util import device_from_pool, rel_err, split

pytestmark = pytest.mark.gpu


def _estimate(n, m, q, N, d, prec, tol, max_refine, plan):
    import torch
    s = mhe.Solver(n, m, N, prec=prec, refine_tol=tol, max_refine=max_refine, **plan)
    x, w, lam = s.estimate(q, d["A"], d["B"], d["C"], d["R"], d["a"], d["yt"], d["wt"], d["x0"], d["P0inv"])
    torch.cuda.synchronize()
    info = s.infos()
    sols = split(x, w, lam, N, n, m)
    s.close()
    return sols, info


def _check_sample(sols, info, b, inst, bound):
    r = oracle.riccati(oracle.mhe_to_uftoc(inst))
    assert r["status"] == 0
    assert rel_err(sols[b], r) <= bound, (b, rel_err(sols[b], r))


def test_batched_uneven_4096_full_size():
    """4096 instances, nx ~ U{6,12,24}, nw = ny = nx/2, N ~ U[32,2048], seed 3."""
    w = synth.batch_uneven(seed=3)
    plans = {6: dict(leaf_len=32, branching=4, top_len=4), 12: dict(leaf_len=64, branching=8, top_len=4),
             24: dict(leaf_len=32, branching=4, top_len=4)}
    for n, bk in sorted(w["buckets"].items()):
        m, q, N = bk["m"], bk["q"], [int(v) for v in bk["N"]]
        d = device_from_pool(n, m, q, bk["pool"], bk["idx"], bk["x0"])
        sols, info = _estimate(n, m, q, N, d, mhe.MHE_FP32_IR, 1e-9, 16, plans[n])
        assert np.all(info["status"] == 0), n
        assert np.max(info["relres"]) <= 1e-9, n
        sols, info = _estimate(n, m, q, N, d, mhe.MHE_FP32_IR, 1e-12, 24, plans[n])
        assert np.all(info["status"] == 0), n
        assert np.max(info["relres"]) <= 1e-12, n
        for j in (int(np.argmax(bk["N"])), int(np.argmin(bk["N"])), len(N) // 2, 137):
            _check_sample(sols, info, j, synth.bucket_instance(bk, j), 1e-8)


def test_long_horizon_nx20_N131072_full_size():
    """One instance, nx=20, nw=ny=10, N=131072, FP64, seed 1: the whole solution."""
    p = synth.mhe_instance(1, 20, 10, 10, 131072)
    pool = {k: p[k] for k in ("A", "B", "C", "R", "a", "yt", "wt")}
    d = device_from_pool(20, 10, 10, pool, np.arange(131071), p["x0"])
    sols, info = _estimate(20, 10, 10, [131072], d, mhe.MHE_FP64, 1e-9, 2,
                           dict(leaf_len=64, branching=4, top_len=16))
    assert info["status"][0] == 0 and info["relres"][0] <= 1e-12
    _check_sample(sols, info, 0, p, 1e-10)


@pytest.mark.parametrize("prec", [mhe.MHE_TF32_IR, mhe.MHE_BF16_IR, mhe.MHE_FP32_IR])
def test_nx64_256_instances_full_size(prec):
    """256 instances of nx=64, nw=ny=32, N=1024 (the serial plan the autotuner
    picks), with the stage products on the tensor cores (the bench's default for
    this workload) and in FP32 on the CUDA cores."""
    rng = np.random.default_rng(5)
    count, N, n, m = 256, 1024, 64, 32
    pool = synth.stage_pool(np.random.default_rng([5, n]), n, m, m, 2048)
    idx = rng.integers(0, 2048, size=count * (N - 1))
    x0 = rng.standard_normal((count, n))
    d = device_from_pool(n, m, m, pool, idx, x0)
    plan = dict(leaf_len=64, branching=4, top_len=N + 1)
    sols, info = _estimate(n, m, m, [N] * count, d, prec, 1e-9, 16, plan)
    assert np.all(info["status"] == 0)
    assert np.max(info["relres"]) <= 1e-9
    sols, info = _estimate(n, m, m, [N] * count, d, prec, 1e-12, 24, plan)
    assert np.all(info["status"] == 0)
    assert np.max(info["relres"]) <= 1e-12
    for j in (0, 137):
        inst = synth.instance_from_pool(pool, idx[j * (N - 1):(j + 1) * (N - 1)], x0[j], n, m, m)
        _check_sample(sols, info, j, inst, 1e-8)
