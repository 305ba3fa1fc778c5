"""The allocation-free entry point against the regular one (GPU).

mhe_solve_serial_noalloc serves callers that cannot allocate device memory
(hard real-time loops, hosts that own the memory budget): it keeps its stored
factors in a fixed library scratch array.  Its answers must equal those of
mhe_factor_solve on the same instance within the FP64 tolerance of the other
parity tests (1e-10 relative), on two calls in a row with different data, so
that nothing of the first call leaks into the second.  This file is collected
last on purpose.
"""
import numpy as np
import pytest

from paper_1510_03110_gb300 import mhe, synth

from gpu_util import device_inputs, rel_err, split

pytestmark = pytest.mark.gpu


def _regular(d):
    s = mhe.Solver(d["n"], d["m"], d["N"], prec=mhe.MHE_FP64, top_len=int(max(d["N"])) + 1)
    x, w, lam = s.factor_solve(d["A"], d["B"], d["Q"], d["P0inv"], d["l"], d["a"], d["x0"])
    import torch
    torch.cuda.synchronize()
    out = split(x, w, lam, d["N"], d["n"], d["m"])[0]
    st = int(s.infos()["status"][0])
    s.close()
    return out, st


def _noalloc(d):
    import torch
    n, m, N = d["n"], d["m"], d["N"][0]
    x = torch.full(((N + 1) * n,), float("nan"), dtype=torch.float64, device="cuda")
    w = torch.full((n + (N - 1) * m,), float("nan"), dtype=torch.float64, device="cuda")
    lam = torch.full(((N + 1) * n,), float("nan"), dtype=torch.float64, device="cuda")
    status = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    mhe.mhe_solve_serial_noalloc(n, m, N, d["A"], d["B"], d["Q"], d["P0inv"], d["l"], d["a"], d["x0"],
                                 x, w, lam, status)
    torch.cuda.synchronize()
    return split(x, w, lam, d["N"], n, m)[0], int(status.item())


@pytest.mark.parametrize("n,m,N", [(6, 3, 300), (20, 10, 257)])
def test_noalloc_matches_regular_entry_two_calls(n, m, N):
    first = device_inputs([synth.mhe_instance(31, n, m, m, N)])
    second = device_inputs([synth.mhe_instance(32, n, m, m, N - 17)])
    for d in (first, second):
        ref, st_ref = _regular(d)
        got, st = _noalloc(d)
        assert st_ref == 0 and st == 0
        for k in ("x", "w", "lam"):
            assert np.all(np.isfinite(got[k])), k
        assert rel_err(got, ref) <= 1e-10


def test_noalloc_rejects_sizes_beyond_the_scratch():
    import torch
    d = device_inputs([synth.mhe_instance(33, 24, 12, 12, 4)])
    z = torch.zeros(8, dtype=torch.float64, device="cuda")
    too_long = 1 << 20
    with pytest.raises(mhe.MheError) as e:
        mhe.mhe_solve_serial_noalloc(24, 12, too_long, d["A"], d["B"], d["Q"], d["P0inv"], d["l"], d["a"],
                                     d["x0"], z, z, z)
    assert e.value.code == -1
