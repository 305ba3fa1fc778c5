"""Algorithm 6 as printed on the GPU (mhe_dims.down_pass = 1): every subproblem of
every level solved again with Algorithms 1-3 from its parent's P^, Psi^ and x^,
the cost-to-go written at every state for the level below.  It must give the
same Newton step as the back-substitution down pass (the default) and as the
FP64 oracle -- the oracle pins the same equality on the CPU
(tests/test_oracle.py::test_backsubstitution_equals_literal_alg6)."""
import numpy as np
import pytest

import oracle
from paper_1510_03110_gb300 import mhe, synth

from gpu_util import device_inputs, rel_err, split

pytestmark = pytest.mark.gpu


def _solve(d, n, m, **kw):
    import torch
    s = mhe.Solver(n, m, d["N"], **kw)
    x, w, lam = s.factor_solve(d["A"], d["B"], d["Q"], d["P0inv"], d["l"], d["a"], d["x0"])
    torch.cuda.synchronize()
    out = split(x, w, lam, d["N"], n, m)
    info = s.infos()
    s.close()
    return out, info


# leaf_len * nw above nx in every case but the rank-revealing one (6, 3, leaf 1): at exactly nx the FP32
# Cholesky of a square B^ can fail where FP64's does not (reported as MHE_E_NOT_PD, seen at nx=20, leaf 2)
@pytest.mark.parametrize("n,m,leaf,br,top", [(4, 2, 4, 3, 2), (6, 3, 8, 4, 4), (12, 6, 3, 2, 1), (24, 12, 8, 4, 4),
                                             (20, 10, 3, 3, 2), (6, 3, 1, 2, 2)])
@pytest.mark.parametrize("prec,bound", [(mhe.MHE_FP64, 1e-10), (mhe.MHE_FP32_IR, 1e-8)])
def test_literal_algorithm6_equals_backsubstitution_and_oracle(n, m, leaf, br, top, prec, bound):
    Ns = [1, 2, 3, 17, 64, 201]
    insts = [synth.mhe_instance(1700 + 3 * i + n, n, m, m, N) for i, N in enumerate(Ns)]
    d = device_inputs(insts)
    ref = [oracle.riccati(oracle.mhe_to_uftoc(p)) for p in insts]
    kw = dict(prec=prec, leaf_len=leaf, branching=br, top_len=top,
              refine_tol=1e-12 if prec == mhe.MHE_FP32_IR else 0.0, max_refine=-1 if prec == 0 else 30)
    lit, ilit = _solve(d, n, m, down_pass=1, **kw)
    bs, ibs = _solve(d, n, m, down_pass=0, **kw)
    for b in range(len(Ns)):
        assert ilit["status"][b] == 0 and ibs["status"][b] == 0, (b, ilit[b], ibs[b])
        assert rel_err(lit[b], ref[b]) <= bound, (b, rel_err(lit[b], ref[b]))
        if prec == mhe.MHE_FP64:
            assert rel_err(lit[b], bs[b]) <= 1e-10


def test_autotuner_considers_both_down_passes():
    insts = [synth.mhe_instance(1800 + i, 6, 3, 3, N) for i, N in enumerate([40, 90, 130])]
    d = device_inputs(insts)
    dims, _keep = mhe.make_dims(6, 3, d["N"], mhe.MHE_FP64)
    best = mhe.mhe_autotune(dims, d["A"], d["B"], d["Q"], d["P0inv"], d["l"], d["a"], d["x0"], reps=1)
    assert best["down_pass"] in (0, 1) and best["ms"] > 0
