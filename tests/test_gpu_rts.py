"""The Kalman filter + RTS smoother on the GPU (mhe_rts_smooth), the method the
paper compares its parallel Riccati recursion with (Section VI).

For uncorrelated noises (S = 0) the smoothed means are the x and w of the MHE
Newton step, so the GPU smoother must agree with the oracle's textbook RTS
recursion (oracle/rts.py, a CPU pin of the Section II transform) and with the
library's own tree solution, to 1e-10 in FP64."""
import numpy as np
import pytest

import oracle
from oracle import rts
from paper_1510_03110_gb300 import mhe, synth

from gpu_util import device_inputs, rel_err, split

pytestmark = pytest.mark.gpu


def _rel(a, b):
    a, b = np.asarray(a).ravel(), np.asarray(b).ravel()
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("n,m", [(4, 2), (6, 3), (12, 6), (20, 10), (24, 12), (2, 1)])
def test_gpu_rts_equals_oracle_rts_and_tree(n, m):
    import torch
    Ns = [2, 3, 17, 120, 333]
    insts = [synth.mhe_instance(1900 + 5 * i + n, n, m, m, N, s_zero=True) for i, N in enumerate(Ns)]
    d = device_inputs(insts)
    X = int(sum(N + 1 for N in Ns))
    W = int(sum(n + (N - 1) * m for N in Ns))
    x = torch.full((X * n,), float("nan"), dtype=torch.float64, device="cuda")
    w = torch.full((W,), float("nan"), dtype=torch.float64, device="cuda")
    status = torch.full((len(Ns),), 7, dtype=torch.int32, device="cuda")
    mhe.mhe_rts_smooth(n, m, m, Ns, d["A"], d["B"], d["C"], d["R"], d["a"], d["yt"], d["wt"], d["x0"], d["P0inv"],
                       x, w, status=status)
    torch.cuda.synchronize()
    assert status.cpu().tolist() == [0] * len(Ns)
    lam = torch.zeros_like(x)
    got = split(x, w, lam, Ns, n, m)
    s = mhe.Solver(n, m, Ns, prec=mhe.MHE_FP64)
    xt, wt, lt = s.factor_solve(d["A"], d["B"], d["Q"], d["P0inv"], d["l"], d["a"], d["x0"])
    torch.cuda.synchronize()
    tree = split(xt, wt, lt, Ns, n, m)
    s.close()
    for b, p in enumerate(insts):
        xs, ws = rts.smooth(p)
        # the oracle's RTS gives x_1 .. x_N and w_1 .. w_{N-1} (UFTOC indexing)
        assert _rel(got[b]["x"][1:], xs) <= 1e-10, b
        if Ns[b] > 1:
            assert _rel(got[b]["w"][n:], ws.ravel()) <= 1e-10, b
        for k in ("x", "w"):
            assert _rel(got[b][k], tree[b][k]) <= 1e-10, (b, k)
        ref = oracle.riccati(oracle.mhe_to_uftoc(p))
        assert _rel(got[b]["x"], ref["x"]) <= 1e-10 and _rel(got[b]["w"], ref["w"]) <= 1e-10
