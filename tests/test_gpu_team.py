"""Team-width variants of a shape (mhe_dims.team): the same problems solved with
every compiled width agree with the oracle, and the autotuner returns a
compiled width."""
import numpy as np
import pytest

import oracle
from paper_1510_03110_gb300 import mhe, synth

from gpu_util import device_inputs, rel_err, split

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,m", [(4, 2), (6, 3), (12, 6)])
@pytest.mark.parametrize("prec,tol", [(mhe.MHE_FP64, 1e-10), (mhe.MHE_FP32_IR, 1e-8)])
def test_every_team_width_matches_the_oracle(n, m, prec, tol):
    import torch
    Ns = [1, 2, 3, 17, 130, 257]
    insts = [synth.mhe_instance(3600 + 11 * i + n, n, m, m, N) for i, N in enumerate(Ns)]
    d = device_inputs(insts)
    refs = [oracle.riccati(oracle.mhe_to_uftoc(p)) for p in insts]
    teams = mhe.shape_teams(n, m)
    assert len(teams) >= 2
    for team in teams:
        for plan in (dict(leaf_len=4, branching=4, top_len=4), dict(top_len=1000)):
            s = mhe.Solver(n, m, Ns, prec=prec, refine_tol=1e-12 if prec else 0.0, max_refine=16 if prec else -1,
                           team=team, **plan)
            x, w, lam = s.factor_solve(d["A"], d["B"], d["Q"], d["P0inv"], d["l"], d["a"], d["x0"])
            torch.cuda.synchronize()
            got = split(x, w, lam, Ns, n, m)
            assert list(s.infos()["status"]) == [0] * len(Ns), (team, plan)
            for b in range(len(Ns)):
                assert rel_err(got[b], refs[b]) <= tol, (team, plan, b)
            s.close()


def test_autotuner_returns_a_compiled_team_width():
    import torch
    n, m = 6, 3
    rng = np.random.default_rng(7)
    Ns = [int(v) for v in rng.integers(32, 400, size=64)]
    insts = [synth.mhe_instance(3700 + i, n, m, m, N) for i, N in enumerate(Ns)]
    d = device_inputs(insts)
    dims, _keep = mhe.make_dims(n, m, Ns, mhe.MHE_FP32_IR, refine_tol=1e-12, max_refine=16)
    r = mhe.mhe_autotune(dims, d["A"], d["B"], d["Q"], d["P0inv"], d["l"], d["a"], d["x0"])
    assert r["team"] == 0 or r["team"] in mhe.shape_teams(n, m)
    s = mhe.Solver(n, m, Ns, prec=mhe.MHE_FP32_IR, refine_tol=1e-12, max_refine=16,
                   **{k: r[k] for k in ("leaf_len", "branching", "top_len", "down_pass", "team")})
    s.factor_solve(d["A"], d["B"], d["Q"], d["P0inv"], d["l"], d["a"], d["x0"])
    torch.cuda.synchronize()
    assert list(s.infos()["status"]) == [0] * len(Ns)
    s.close()
