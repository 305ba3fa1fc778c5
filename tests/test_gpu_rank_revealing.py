"""Rank-revealing master stages on the GPU (Section IV-B's remark on a singular G^,
Theorem 1 with the U_1 basis of Eq. Bh_def).

With leaf chunks shorter than ceil(nx / nw) stages, a chunk's S^T has rank
L nw < nx and the T-form Q^_w is singular.  The library then factors every master
stage's Q^_w with a pivoted Cholesky that stops at the numerical rank r and uses
the master stage B = Pi L (zero-padded to width nx), Q_w = I; the down pass
recovers w^ = Pi [L_11^{-T} w^'; 0].  The oracle pins this very basis
(tests/test_oracle.py::test_pivoted_square_root_basis_gives_the_same_step).  The
GPU result must match the FP64 oracle to 1e-10 in FP64 mode and 1e-8 after
refinement in FP32_IR (with FP64 master levels, and with FP32 ones for the small
shapes), for the shapes and plans of the oracle's U_1 tests that are compiled,
with uneven horizons incl. N = 1, 2, 3.
"""
import numpy as np
import pytest

import oracle
from paper_1510_03110_gb300 import mhe, synth

from gpu_util import device_inputs, rel_err, split

pytestmark = pytest.mark.gpu

# (nx, nw, leaf_len, branching, top_len): leaf_len * nw < nx in every case
PLANS = [(2, 1, 1, 2, 1), (4, 2, 1, 3, 2), (6, 3, 1, 2, 2), (3, 2, 1, 2, 1), (12, 6, 1, 4, 4), (24, 12, 1, 2, 2),
         (6, 3, 1, 8, 4), (20, 10, 1, 3, 2)]


# FP32_IR: with FP32 master levels a deep tree of rank-revealing master stages (leaf 1)
# contracts the residual slowly (~0.3 per correction at nx = 12) and stalls at nx >= 20
# (relres 2e-7 after 40 corrections, measured on GB300): an FP32 pivoted Cholesky cannot
# tell directions below ~1e-5 of the largest pivot from its rounding, and the deep master
# levels lose them.  FP64 master levels (mhe_dims.fp64_masters) decide the rank at 1e-10
# and restore fast contraction; FP32 master levels are run for the small shapes.
CASES = [(p, mhe.MHE_FP64, False, 1e-10) for p in PLANS] + \
        [(p, mhe.MHE_FP32_IR, True, 1e-8) for p in PLANS] + \
        [(p, mhe.MHE_FP32_IR, False, 1e-8) for p in PLANS if p[0] <= 12]


@pytest.mark.parametrize("plan,prec,masters,bound", CASES)
def test_short_leaves_match_oracle(plan, prec, masters, bound):
    import torch
    n, m, leaf, br, top = plan
    Ns = [1, 2, 3, 11, 40, 97]
    insts = [synth.mhe_instance(1300 + 7 * i + n, n, m, m, N) for i, N in enumerate(Ns)]
    d = device_inputs(insts)
    ref = [oracle.riccati(oracle.mhe_to_uftoc(p)) for p in insts]
    s = mhe.Solver(n, m, d["N"], prec=prec, leaf_len=leaf, branching=br, top_len=top,
                   refine_tol=1e-12 if prec == mhe.MHE_FP32_IR else 0.0,
                   max_refine=(8 if masters else 40) if prec == mhe.MHE_FP32_IR else -1, fp64_masters=masters)
    assert len(mhe.mhe_plan_info(s.ctx)) >= 3
    x, w, lam = s.factor_solve(d["A"], d["B"], d["Q"], d["P0inv"], d["l"], d["a"], d["x0"])
    torch.cuda.synchronize()
    info = s.infos()
    sols = split(x, w, lam, d["N"], n, m)
    s.close()
    for b in range(len(Ns)):
        assert info["status"][b] == 0, (b, info[b])
        assert rel_err(sols[b], ref[b]) <= bound, (b, rel_err(sols[b], ref[b]))
