"""CUDA-graph replay of the entry points (mhe_set_graph): a replayed launch
sequence gives bit for bit what the eager calls give on the same data, after
the data in the same buffers has changed, and it counts its launches."""
import numpy as np
import pytest

from paper_1510_03110_gb300 import mhe, synth

from gpu_util import device_inputs, rel_err, split

pytestmark = pytest.mark.gpu


def _perturb(d, k):
    """Change the contents of the problem's buffers in place (same pointers)."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(100 + k)
    for key in ("l", "a", "x0", "yt", "wt"):
        d[key].add_(0.1 * torch.randn(d[key].shape, generator=g, device="cuda", dtype=torch.float64))
    d["A"].mul_(1.0 - 0.01 * k)


@pytest.mark.parametrize("prec", [mhe.MHE_FP64, mhe.MHE_FP32_IR])
@pytest.mark.parametrize("plan", [dict(leaf_len=4, branching=4, top_len=4), dict(top_len=100000)])
def test_factor_solve_replay_equals_eager(prec, plan):
    import torch
    n, m = 6, 3
    Ns = [2, 17, 64, 130]
    insts = [synth.mhe_instance(3100 + i, n, m, m, N) for i, N in enumerate(Ns)]
    d = device_inputs(insts)
    st = torch.cuda.Stream()
    kw = dict(prec=prec, refine_tol=1e-12, max_refine=8, **plan)
    g = mhe.Solver(n, m, Ns, stream=st, **kw)
    e = mhe.Solver(n, m, Ns, stream=st, **kw)
    g.set_graph(True)
    out_g, out_e = g.outputs(), e.outputs()
    counts = []
    for k in range(4):
        if k >= 2:
            with torch.cuda.stream(st):
                _perturb(d, k)
                mhe.mhe_assemble(n, m, m, d["C"].view(d["S"], -1), d["R"], d["yt"], d["wt"], d["Q"], d["l"],
                                 stream=st)
        before = mhe.mhe_launch_count(g.ctx)
        with torch.cuda.stream(st):
            g.factor_solve(d["A"], d["B"], d["Q"], d["P0inv"], d["l"], d["a"], d["x0"], out=out_g)
            e.factor_solve(d["A"], d["B"], d["Q"], d["P0inv"], d["l"], d["a"], d["x0"], out=out_e)
        st.synchronize()
        counts.append(mhe.mhe_launch_count(g.ctx) - before)
        for a, b in zip(out_g, out_e):
            assert torch.equal(a, b), k
        ig, ie = g.infos(), e.infos()
        assert np.array_equal(ig["status"], ie["status"]) and np.array_equal(ig["relres"], ie["relres"])
        assert list(ig["status"]) == [0] * len(Ns)
    # calls 1.. replay the same sequence: the same launches as the eager first call
    assert counts[1] == counts[2] == counts[3] == counts[0] > 0
    g.close()
    e.close()


def test_estimate_replay_and_new_pointers():
    import torch
    n, m = 12, 6
    Ns = [40, 333]
    insts = [synth.mhe_instance(3200 + i, n, m, m, N) for i, N in enumerate(Ns)]
    d = device_inputs(insts)
    st = torch.cuda.Stream()
    g = mhe.Solver(n, m, Ns, prec=mhe.MHE_FP32_IR, refine_tol=1e-12, max_refine=8, stream=st)
    g.set_graph(True)
    ref = mhe.Solver(n, m, Ns, prec=mhe.MHE_FP32_IR, refine_tol=1e-12, max_refine=8, stream=st)
    outs = [g.outputs(), g.outputs()]
    for k in range(6):
        out = outs[k % 2 if k >= 3 else 0]   # new output pointers from the fourth call on, alternating
        if k == 4:
            with torch.cuda.stream(st):
                _perturb(d, k)
        with torch.cuda.stream(st):
            x, w, lam = g.estimate(m, d["A"], d["B"], d["C"], d["R"], d["a"], d["yt"], d["wt"], d["x0"], d["P0inv"],
                                   out=out)
            xr, wr, lr = ref.estimate(m, d["A"], d["B"], d["C"], d["R"], d["a"], d["yt"], d["wt"], d["x0"],
                                      d["P0inv"])
        st.synchronize()
        assert torch.equal(x, xr) and torch.equal(w, wr) and torch.equal(lam, lr), k
        assert list(g.infos()["status"]) == [0, 0]
    g.close()
    ref.close()


def test_factor_then_solve_replays_follow_the_factorised_problem():
    """mhe_solve's graph reads the problem the last factorisation left in the
    context; a factorisation of other buffers must not replay a stale residual."""
    import torch
    n, m = 4, 2
    Ns = [9, 50]
    st = torch.cuda.Stream()
    probs = []
    for s in (3300, 3400):
        insts = [synth.mhe_instance(s + i, n, m, m, N) for i, N in enumerate(Ns)]
        probs.append(device_inputs(insts))
    g = mhe.Solver(n, m, Ns, stream=st)
    g.set_graph(True)
    e = mhe.Solver(n, m, Ns, stream=st)
    outs = g.outputs()
    for k in range(6):
        d = probs[(k // 2) % 2]
        with torch.cuda.stream(st):
            g.factor(d["A"], d["B"], d["Q"], d["P0inv"])
            g.solve(d["l"], d["a"], d["x0"], out=outs)
            ref = e.factor_solve(d["A"], d["B"], d["Q"], d["P0inv"], d["l"], d["a"], d["x0"])
        st.synchronize()
        got = split(*outs, Ns, n, m)
        want = split(*ref, Ns, n, m)
        for b in range(len(Ns)):
            assert rel_err(got[b], want[b]) <= 1e-13, (k, b)
        assert list(g.infos()["status"]) == [0, 0]
    g.close()
    e.close()


def test_default_stream_stays_eager():
    """The legacy default stream cannot be captured: calls run eagerly and
    every call counts its own launches."""
    import torch
    n, m = 4, 2
    insts = [synth.mhe_instance(3500, n, m, m, 30)]
    d = device_inputs(insts)
    g = mhe.Solver(n, m, [30])
    g.set_graph(True)
    counts = []
    for _ in range(3):
        before = mhe.mhe_launch_count(g.ctx)
        g.factor_solve(d["A"], d["B"], d["Q"], d["P0inv"], d["l"], d["a"], d["x0"])
        torch.cuda.synchronize()
        counts.append(mhe.mhe_launch_count(g.ctx) - before)
    assert counts[0] == counts[1] == counts[2] > 0
    g.set_graph(False)
    g.close()


def test_ip_solve_with_replayed_newton_steps_equals_eager():
    """mhe_ip_solve on a context with graphs on: its factor and solve calls (the
    same pointers every iteration) replay, with the same iterations and bits."""
    import torch
    n, m = 6, 3
    Ns = [9, 40, 130]
    insts = [synth.mhe_instance(3900 + i, n, m, m, N) for i, N in enumerate(Ns)]
    d = device_inputs(insts)
    rng = np.random.default_rng(3)
    lo = -0.05 - 0.02 * rng.random((len(Ns), m))
    hi = 0.05 + 0.02 * rng.random((len(Ns), m))
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float64).reshape(-1)).cuda()  # noqa: E731
    st = torch.cuda.Stream()
    outs = []
    for graph in (False, True):
        s = mhe.Solver(n, m, Ns, stream=st)
        s.set_graph(graph)
        with torch.cuda.stream(st):
            x, w, lam, k = s.ip_solve(d["A"], d["B"], d["Q"], d["P0inv"], d["l"], d["a"], d["x0"], t(lo), t(hi))
        st.synchronize()
        assert list(s.infos()["status"]) == [0] * len(Ns)
        outs.append((x.clone(), w.clone(), lam.clone(), k))
        s.set_graph(False)
        s.close()
    assert outs[0][3] == outs[1][3] > 2
    for a, b in zip(outs[0][:3], outs[1][:3]):
        assert torch.equal(a, b)
