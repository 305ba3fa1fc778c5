"""The allocation-free entry point against the regular one (GPU).

mhe_solve_serial_noalloc serves callers that cannot allocate device memory
(hard real-time loops, where cudaMalloc can stall a sample instant, and hosts
that own the device-memory budget): it keeps its stored factors in a fixed
library scratch array.  Its answers must equal those of mhe_factor_solve on the
same instance within the FP64 tolerance of the other parity tests (1e-10
relative), on two calls in a row with different data, so that nothing of the
first call leaks into the second; after its first (warm-up) call on a device
it must not change the device's free memory.  This file is collected last on
purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_1510_03110_gb300 import mhe, synth

from gpu_util import device_inputs, rel_err, split

pytestmark = pytest.mark.gpu


def _regular(d):
    import torch
    s = mhe.Solver(d["n"], d["m"], d["N"], prec=mhe.MHE_FP64, top_len=int(max(d["N"])) + 1)
    x, w, lam = s.factor_solve(d["A"], d["B"], d["Q"], d["P0inv"], d["l"], d["a"], d["x0"])
    torch.cuda.synchronize()
    out = split(x, w, lam, d["N"], d["n"], d["m"])[0]
    st = int(s.infos()["status"][0])
    s.close()
    return out, st


def _buffers(d):
    import torch
    n, m, N = d["n"], d["m"], d["N"][0]
    x = torch.full(((N + 1) * n,), float("nan"), dtype=torch.float64, device="cuda")
    w = torch.full((n + (N - 1) * m,), float("nan"), dtype=torch.float64, device="cuda")
    lam = torch.full(((N + 1) * n,), float("nan"), dtype=torch.float64, device="cuda")
    status = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    return x, w, lam, status


def _call(d, bufs, with_status=True):
    x, w, lam, status = bufs
    mhe.mhe_solve_serial_noalloc(d["n"], d["m"], d["N"][0], d["A"], d["B"], d["Q"], d["P0inv"], d["l"], d["a"],
                                 d["x0"], x, w, lam, status if with_status else None)


def _noalloc(d, with_status=True):
    import torch
    bufs = _buffers(d)
    _call(d, bufs, with_status)
    torch.cuda.synchronize()
    x, w, lam, status = bufs
    return split(x, w, lam, d["N"], d["n"], d["m"])[0], int(status.item())


@pytest.mark.parametrize("n,m,N", [(1, 1, 40), (3, 2, 90), (6, 3, 300), (20, 10, 257), (24, 12, 130),
                                   (6, 3, 1), (24, 12, 2), (4, 2, 1), (20, 20, 3)])
def test_noalloc_matches_regular_entry_two_calls(n, m, N):
    first = device_inputs([synth.mhe_instance(31, n, m, m, N)])
    second = device_inputs([synth.mhe_instance(32, n, m, m, max(1, N - 17))])
    for d in (first, second):
        ref, st_ref = _regular(d)
        got, st = _noalloc(d)
        assert st_ref == 0 and st == 0
        for k in ("x", "w", "lam"):
            assert np.all(np.isfinite(got[k])), k
        assert rel_err(got, ref) <= 1e-10


def test_noalloc_without_status_word():
    d = device_inputs([synth.mhe_instance(34, 6, 3, 3, 77)])
    ref, _ = _regular(d)
    got, st = _noalloc(d, with_status=False)
    assert st == 7                                  # the status word was not passed, so it is untouched
    assert rel_err(got, ref) <= 1e-10


def test_noalloc_reports_a_non_pd_stage():
    """A stage Hessian with a negative definite Q_w block: MHE_E_NOT_PD, as the regular entry reports;
    a good instance right after it solves correctly (the scratch keeps no error state)."""
    import torch
    p = synth.mhe_instance(9, 4, 2, 2, 20)
    d = device_inputs([p])
    Q = d["Q"].view(19, 6, 6)
    Q[10, 4:, 4:] = -1e6 * torch.eye(2, dtype=torch.float64, device="cuda")
    _, st_ref = _regular(d)
    _, st = _noalloc(d)
    assert st_ref == -3 and st == -3
    good = device_inputs([synth.mhe_instance(10, 4, 2, 2, 20)])
    ref, _ = _regular(good)
    got, st = _noalloc(good)
    assert st == 0 and rel_err(got, ref) <= 1e-10


def test_noalloc_allocates_nothing_after_the_warm_up():
    import torch
    d = device_inputs([synth.mhe_instance(35, 20, 10, 10, 400)])
    bufs = _buffers(d)
    _call(d, bufs)                                  # warm-up: may load the device code and its scratch
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        _call(d, bufs)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert int(bufs[3].item()) == 0


def test_noalloc_rejects_sizes_beyond_the_scratch():
    """The library's own check, called through the C-ABI with raw pointers (the binding's size
    checks would refuse the short buffers first)."""
    import torch
    d = device_inputs([synth.mhe_instance(33, 24, 12, 12, 4)])
    z = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    too_long = 1 << 20
    rc = mhe.lib().mhe_solve_serial_noalloc(24, 12, too_long, p(d["A"]), p(d["B"]), p(d["Q"]), p(d["P0inv"]),
                                            p(d["l"]), p(d["a"]), p(d["x0"]), p(z), p(z), p(z), None,
                                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == -1
    assert b"exceeds the fixed scratch" in mhe.lib().mhe_last_error()
