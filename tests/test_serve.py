"""Serving (continuous batching) on the GPU through the C-ABI.

Each request shifts an estimator's window by one sample; the arrival state of
the shifted window is the previous solution's x_2.  The oracle replays the
same sequence on the CPU.  The result of a request must equal the oracle's,
and an estimator's results must not depend on what else is in the batch.
"""
import numpy as np
import pytest

import oracle
from paper_1510_03110_gb300 import mhe, synth

pytestmark = pytest.mark.gpu


def _stage(stream, k):
    return mhe.pack_stage(stream["A"][k], stream["B"][k], stream["C"][k], stream["R"][k], stream["a"][k],
                          stream["yt"][k], stream["wt"][k])


def _oracle_sequence(stream, N, x0, requests, n, m, q):
    """Request j solves the window of stream stages j+1 .. j+N-1; x~0 of request 0 is
    the given x0, afterwards the previous solution's x_2.  Returns x_{N-1} per request."""
    out, x0j = [], np.asarray(x0, float)
    for j in range(requests):
        p = synth.window_of(stream, j + 1, N, x0j, n, m, q)
        r = oracle.riccati(oracle.mhe_to_uftoc(p))
        assert r["status"] == 0
        out.append(r["x"][N - 1].copy())
        x0j = r["x"][2].copy()
    return out


def _run_alone(prec, stream, N, x0, requests, n, m, q, tol, plan=None, reuse=True, stats=None):
    srv = mhe.Server(1 << 30, prec=prec, refine_tol=tol)
    if plan:
        srv.set_plan(**plan)
    srv.set_reuse(reuse)
    e = srv.open(synth.window_of(stream, 0, N, x0, n, m, q))
    res = []
    for j in range(requests):
        t = srv.submit(e, _stage(stream, N - 1 + j))
        res.append(srv.wait(t, n))
    if stats is not None:
        stats.update(srv.stats())
    srv.close()
    return res


PLANS = [dict(leaf_len=8, branching=4, top_len=4), dict(leaf_len=4, branching=2, top_len=2),
         dict(leaf_len=0, branching=0, top_len=1 << 20)]


@pytest.mark.parametrize("plan", PLANS, ids=["tree", "short_leaves", "serial"])
@pytest.mark.parametrize("prec,tol,bound", [(mhe.MHE_FP64, 1e-12, 1e-10), (mhe.MHE_FP32_IR, 1e-12, 1e-8)])
def test_served_estimates_match_oracle(prec, tol, bound, plan):
    """K = 70 consecutive shifts of one estimator (N = 40): the windows cross many chunk
    boundaries and wrap the level rings, so most rounds reuse the reductions of chunks
    kept from earlier rounds.  Every result equals the oracle's from-scratch solve of
    that window.  FP32_IR refines to relres 1e-12, the residual at which the forward
    error of the worst-conditioned windows meets 1e-8 (relres 1e-11 left 1.02e-8 on one
    of these 70)."""
    n, m, q, N, K = 4, 2, 2, 40, 70
    st = synth.plant_stream(1, n, m, q, N - 1 + K)
    x0 = np.zeros(n)
    got = _run_alone(prec, st, N, x0, K, n, m, q, tol, plan=plan)
    ref = _oracle_sequence(st, N, x0, K, n, m, q)
    for j in range(K):
        assert got[j]["status"] == 0
        err = np.abs(got[j]["x"] - ref[j]).max() / np.abs(ref[j]).max()
        assert err <= bound, (j, err)


@pytest.mark.parametrize("prec", [mhe.MHE_FP64, mhe.MHE_FP32_IR])
def test_reuse_equals_full_refactorisation_and_reduces_little(prec):
    """The same request sequence served with factorisation reuse and with every chunk
    reduced again gives the same estimates (the kept reductions are exactly what a fresh
    reduction computes); with reuse the stages reduced per request are a few chunks per
    level, O(leaf_len * levels), against N per request without it."""
    n, m, q, N, K = 12, 6, 6, 1000, 30
    st = synth.plant_stream(21, n, m, q, N - 1 + K)
    x0 = np.zeros(n)
    plan = dict(leaf_len=8, branching=4, top_len=4)
    s_on, s_off = {}, {}
    on = _run_alone(prec, st, N, x0, K, n, m, q, 1e-11, plan=plan, reuse=True, stats=s_on)
    off = _run_alone(prec, st, N, x0, K, n, m, q, 1e-11, plan=plan, reuse=False, stats=s_off)
    for j in range(K):
        assert on[j]["status"] == 0 and off[j]["status"] == 0
        err = np.abs(on[j]["x"] - off[j]["x"]).max() / np.abs(off[j]["x"]).max()
        assert err <= 1e-13, (j, err)
    assert s_on["requests"] == s_off["requests"] == K
    assert s_on["stages_solved"] == s_off["stages_solved"] == K * N
    # without reuse every stage of every level is reduced in every round (level 0's N and the
    # master stages above); with it, after the first round, a few chunks per level
    assert s_off["stages_reduced"] >= K * N
    first = s_off["stages_reduced"] / K
    per = (s_on["stages_reduced"] - first) / (K - 1)
    assert per <= 3 * (8 + 1) + 3 * 4 * 6, per
    assert per < N / 10


def test_result_is_the_same_alone_and_in_the_mix():
    """Estimator E's answers when it is served alone and when its requests share
    rounds with many other estimators of several shapes (submitted all at once,
    so they overlap on the device)."""
    n, m, q, N, K = 6, 3, 3, 60, 5
    tol = 1e-10
    st = synth.plant_stream(7, n, m, q, N - 1 + K)
    x0 = np.zeros(n)
    alone = _run_alone(mhe.MHE_FP32_IR, st, N, x0, K, n, m, q, tol)

    srv = mhe.Server(2 << 30, prec=mhe.MHE_FP32_IR, refine_tol=tol, max_refine=16)
    others = []
    for i, (nn, NN) in enumerate([(6, 50), (12, 200), (6, 120), (24, 90), (12, 60)] * 4):
        ss = synth.plant_stream(100 + i, nn, nn // 2, nn // 2, NN - 1 + K)
        others.append((srv.open(synth.window_of(ss, 0, NN, np.zeros(nn), nn, nn // 2, nn // 2)), ss, NN, nn))
    e = srv.open(synth.window_of(st, 0, N, x0, n, m, q))
    tickets_e, tickets_o = [], []
    for j in range(K):
        for (oe, ss, NN, nn) in others:
            tickets_o.append((srv.submit(oe, _stage(ss, NN - 1 + j)), nn))
        tickets_e.append(srv.submit(e, _stage(st, N - 1 + j)))
    mixed = [srv.wait(t, n) for t in tickets_e]
    for t, nn in tickets_o:
        r = srv.wait(t, nn)
        assert r["status"] == 0 and r["relres"] <= tol
    srv.close()
    for j in range(K):
        err = np.abs(mixed[j]["x"] - alone[j]["x"]).max() / np.abs(alone[j]["x"]).max()
        assert err <= 1e-8, (j, err)
        assert mixed[j]["latency"] > 0


def test_admission_by_device_memory():
    n, m, q = 24, 12, 12
    srv = mhe.Server(64 << 20, prec=mhe.MHE_FP32_IR)   # 64 MiB
    small = synth.plant_stream(3, n, m, q, 60)
    srv.open(synth.window_of(small, 0, 50, np.zeros(n), n, m, q))
    big = synth.plant_stream(4, n, m, q, 1100)
    with pytest.raises(mhe.MheError) as e:
        for i in range(40):
            srv.open(synth.window_of(big, 0, 1000, np.zeros(n), n, m, q))
    assert e.value.code == -9
    assert srv.used_bytes() <= 64 << 20
    srv.close()
