"""The ctypes binding's marshalling on the CPU: every wrapper of
paper_1510_03110_gb300/mhe.py called against a stand-in library object that
records its arguments and writes what the C function would write, with the
device-pointer check relaxed to host tensors.  This exercises the argument
packing and the unpacking of outputs (structures, buffers, out-parameters),
which the GPU tests exercise only on the paths they take."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1510_03110_gb300 import mhe


class Fake:
    def __init__(self):
        self.calls = {}

    def _rec(self, name, args):
        self.calls[name] = args
        return 0

    def mhe_last_error(self):
        return b"fake"

    def mhe_create(self, dims, stream, out):
        self._rec("mhe_create", (dims, stream))
        out._obj.value = 1234
        return 0

    def mhe_workspace_bytes(self, dims):
        self._rec("mhe_workspace_bytes", (dims,))
        return 4096

    def mhe_shapes(self, nx, nw, cap):
        for i, (a, b) in enumerate([(4, 2), (24, 12)]):
            nx[i], nw[i] = a, b
        return 2

    def mhe_timing_read(self, ctx, buf, cap):
        vals = [0, 0, 1, 2.5, 2.5, 3, 0, 17, 8.0, 1.0]
        for k, v in enumerate(vals):
            buf[k] = v
        return 2

    def mhe_autotune(self, dims, m, r, stream, reps, best, ms):
        self._rec("mhe_autotune", (dims, m, r, reps))
        best._obj.leaf_len, best._obj.branching, best._obj.top_len, best._obj.down_pass = 16, 4, 3, 1
        best._obj.team = 16
        ms._obj.value = 1.5
        return 0

    def mhe_launch_count(self, ctx):
        return 77

    def mhe_assemble_count(self):
        return 5

    def mhe_estimator_open(self, s, n, m, q, N, *rest):
        rest[-1]._obj.value = 3
        return 0

    def mhe_submit(self, s, est, packed, ticket):
        ticket._obj.value = 99
        return 0

    def mhe_poll(self, s, ticket, x, info, lat):
        info._obj.relres = 1e-12
        info._obj.refine_iters = 2
        lat._obj.value = 0.004
        return 0

    def __getattr__(self, name):
        if not name.startswith("mhe_"):
            raise AttributeError(name)
        return lambda *args: self._rec(name, args)


@pytest.fixture
def fake(monkeypatch):
    f = Fake()
    monkeypatch.setattr(mhe, "lib", lambda: f)
    monkeypatch.setattr(mhe, "_ptr", lambda t: None if t is None else ctypes.c_void_p(t.data_ptr()))
    monkeypatch.setattr(mhe, "_stream", lambda s: ctypes.c_void_p(0))
    return f


def test_dims_and_context(fake):
    d, N32 = mhe.make_dims(24, 12, [5, 9, 3], prec=mhe.MHE_FP32_IR, leaf_len=8, branching=4, top_len=2,
                           refine_tol=1e-11, max_refine=3)
    assert (d.nx, d.nw, d.batch, d.prec, d.leaf_len, d.branching, d.top_len) == (24, 12, 3, 1, 8, 4, 2)
    assert d.refine_tol == 1e-11 and d.max_refine == 3 and list(N32) == [5, 9, 3]
    assert [d.N[i] for i in range(3)] == [5, 9, 3]
    ctx = mhe.mhe_create(d)
    assert ctx.value == 1234
    assert mhe.mhe_workspace_bytes(d) == 4096
    assert mhe.shapes() == [(4, 2), (24, 12)]
    assert mhe.mhe_launch_count(ctx) == 77 and mhe.mhe_assemble_count() == 5
    assert mhe.mhe_destroy(ctx) == 0


def test_factor_solve_estimate_marshalling(fake):
    t = {k: torch.zeros(8, dtype=torch.float64) for k in
         ("A", "B", "Q", "P0", "l", "a", "x0", "x", "w", "lam", "C", "R", "yt", "wt")}
    info = torch.zeros(64, dtype=torch.uint8)
    mhe.mhe_factor(1, t["A"], t["B"], t["Q"], t["P0"])
    m = fake.calls["mhe_factor"][1]._obj
    assert m.A == t["A"].data_ptr() and m.P0inv == t["P0"].data_ptr()
    mhe.mhe_solve(1, t["l"], t["a"], t["x0"], t["x"], t["w"], t["lam"], info)
    args = fake.calls["mhe_solve"]
    assert args[1]._obj.x0 == t["x0"].data_ptr() and args[2].value == t["x"].data_ptr()
    assert args[5].value == info.data_ptr()
    mhe.mhe_factor_solve(1, t["A"], t["B"], t["Q"], t["P0"], t["l"], t["a"], t["x0"], t["x"], t["w"], t["lam"])
    assert fake.calls["mhe_factor_solve"][6] is None            # no info buffer
    mhe.mhe_estimate(1, 3, t["A"], t["B"], t["C"], t["R"], t["a"], t["yt"], t["wt"], t["x0"], t["P0"],
                     t["x"], t["w"], t["lam"], info)
    p = fake.calls["mhe_estimate"][1]._obj
    assert p.ny == 3 and p.C == t["C"].data_ptr() and p.wt == t["wt"].data_ptr()


def test_host_estimate_marshalling(fake):
    h = {k: np.zeros(8) for k in ("A", "B", "C", "R", "a", "yt", "wt", "x0", "P0", "x", "w", "lam")}
    info = np.zeros(64, dtype=np.uint8)
    mhe.mhe_estimate_host(1, 3, h["A"], h["B"], h["C"], h["R"], h["a"], h["yt"], h["wt"], h["x0"], h["P0"],
                          h["x"], h["w"], h["lam"], info, pieces=3)
    args = fake.calls["mhe_estimate_host"]
    assert args[1]._obj.A == h["A"].ctypes.data and args[5].value == info.ctypes.data and args[6] == 3


def test_timing_autotune_assemble(fake):
    assert mhe.mhe_timing_read(1) == [("reduce", 0, 1, 2.5, 2.5), ("resid", 0, 17, 8.0, 1.0)]
    d, _ = mhe.make_dims(4, 2, [10])
    z = torch.zeros(64, dtype=torch.float64)
    r = mhe.mhe_autotune(d, z, z, z, z, z, z, z, reps=3)
    assert r == dict(leaf_len=16, branching=4, top_len=3, down_pass=1, team=16, ms=1.5) and fake.calls["mhe_autotune"][3] == 3
    S, nx, nw, ny = 5, 4, 2, 2
    C = torch.zeros(S, ny * nx, dtype=torch.float64)
    R = torch.zeros(S * (nw + ny) ** 2, dtype=torch.float64)
    Q = torch.zeros(S * (nx + nw) ** 2, dtype=torch.float64)
    v = torch.zeros(S * (nx + nw), dtype=torch.float64)
    mhe.mhe_assemble(nx, nw, ny, C, R, v, v, Q, v)
    assert fake.calls["mhe_assemble"][3] == S
    with pytest.raises(mhe.MheError):                       # a flat C does not fix S
        mhe.mhe_assemble(nx, nw, ny, C.reshape(-1), R, v, v, Q, v)
    with pytest.raises(mhe.MheError):
        mhe.mhe_assemble(nx, nw, ny, C, R[:-1], v, v, Q, v)
    arrs = _noalloc_arrays(4, 2, 10)
    mhe.mhe_solve_serial_noalloc(4, 2, 10, *arrs)
    assert fake.calls["mhe_solve_serial_noalloc"][:3] == (4, 2, 10)
    assert fake.calls["mhe_solve_serial_noalloc"][13] is None    # no status word: NULL


def _noalloc_arrays(n, m, N):
    """Arrays of exactly the batch = 1 layout: A B Q P0inv l a x0 x w lam."""
    S, nq = N - 1, n + m
    z = lambda k: torch.zeros(k, dtype=torch.float64)  # noqa: E731
    return [z(S * n * n), z(S * n * m), z(S * nq * nq), z(n * n), z(S * nq), z(S * n), z(n),
            z((N + 1) * n), z(n + S * m), z((N + 1) * n)]


@pytest.mark.parametrize("short", range(10))
def test_noalloc_refuses_short_arrays(fake, short):
    """Every array of mhe_solve_serial_noalloc is checked against the batch = 1 layout before the
    call: one element short is refused (SizeError, MHE_E_ARG) and the library is not called."""
    arrs = _noalloc_arrays(6, 3, 12)
    arrs[short] = arrs[short][:-1]
    with pytest.raises(mhe.SizeError):
        mhe.mhe_solve_serial_noalloc(6, 3, 12, *arrs)
    assert "mhe_solve_serial_noalloc" not in fake.calls


@pytest.mark.parametrize("status", [torch.zeros(1, dtype=torch.int32),          # host memory
                                    torch.zeros(1, dtype=torch.int64),          # wrong type
                                    torch.zeros(0, dtype=torch.int32),          # empty
                                    np.zeros(1, dtype=np.int32)])               # not a tensor
def test_noalloc_refuses_a_bad_status_buffer(fake, status):
    """The status word must be None or a contiguous int32 CUDA tensor (the kernel writes it)."""
    with pytest.raises(TypeError):
        mhe.mhe_solve_serial_noalloc(4, 2, 10, *_noalloc_arrays(4, 2, 10), status=status)
    assert "mhe_solve_serial_noalloc" not in fake.calls


def test_info_records():
    rec = np.zeros(2, dtype=mhe.INFO_DTYPE)
    rec["status"] = [0, -3]
    rec["relres"] = [1e-12, 2e-3]
    t = torch.from_numpy(rec.view(np.uint8).copy())
    out = mhe.info_array(t)
    assert list(out["status"]) == [0, -3] and out["relres"][1] == 2e-3
    assert mhe.INFO_DTYPE.itemsize == ctypes.sizeof(mhe.mhe_info)


def test_server_marshalling(fake):
    from paper_1510_03110_gb300 import synth
    srv = mhe.Server(1 << 30)
    st = synth.plant_stream(2, 4, 2, 2, 30)
    e = srv.open(synth.window_of(st, 0, 12, np.zeros(4), 4, 2, 2))
    assert e == 3 and srv.nx[3] == 4
    tk = srv.submit(e, mhe.pack_stage(*(st[f][12] for f in ("A", "B", "C", "R", "a", "yt", "wt"))))
    assert tk == 99
    r = srv.poll(tk, 4)
    assert r["status"] == 0 and r["iters"] == 2 and r["latency"] == 0.004 and r["x"].shape == (4,)
    srv.set_plan(8, 4, 2)
    srv.close()


def _cpu_solver(nx, nw, N):
    """A Solver with its context and info buffer stood in on the host (the fake
    library never touches them), for marshalling checks."""
    s = object.__new__(mhe.Solver)
    s.nx, s.nw, s.N = nx, nw, np.asarray(N, dtype=np.int64)
    s.batch = int(s.N.size)
    s.X, s.S = int(np.sum(s.N + 1)), int(np.sum(s.N - 1))
    s.W = int(np.sum(nx + (s.N - 1) * nw))
    s.ctx, s.info = 1, torch.zeros(s.batch * mhe.INFO_DTYPE.itemsize, dtype=torch.uint8)
    return s


def test_ip_solve_marshalling(fake):
    nx, nw = 4, 2
    s = _cpu_solver(nx, nw, [3, 5])
    nq = nx + nw
    z = lambda k: torch.zeros(k, dtype=torch.float64)  # noqa: E731
    arr = dict(A=z(s.S * nx * nx), B=z(s.S * nx * nw), Q=z(s.S * nq * nq), P0inv=z(s.batch * nx * nx),
               l=z(s.S * nq), a=z(s.S * nx), x0=z(s.batch * nx))
    out = (z(s.X * nx), z(s.W), z(s.X * nx))
    lo, hi = z(s.batch * nw), torch.ones(s.batch * nw, dtype=torch.float64)
    args = [arr[k] for k in ("A", "B", "Q", "P0inv", "l", "a", "x0")]
    s.ip_solve(*args, lo, hi, mu0=0.5, mu_final=1e-8, max_newton=30, out=out, method=mhe.MHE_IP_PATH_FOLLOWING)
    call = fake.calls["mhe_ip_solve"]
    o = call[3]._obj
    assert (o.w_lo, o.w_hi) == (lo.data_ptr(), hi.data_ptr())
    assert (o.mu0, o.mu_final, o.max_newton, o.method) == (0.5, 1e-8, 30, mhe.MHE_IP_PATH_FOLLOWING)
    assert call[4].value == out[0].data_ptr() and call[7].value == s.info.data_ptr()
    s.ip_solve(*args, lo, hi, out=out)
    assert fake.calls["mhe_ip_solve"][3]._obj.method == mhe.MHE_IP_PREDICTOR_CORRECTOR
    # short bounds or outputs are refused before the library is called
    del fake.calls["mhe_ip_solve"]
    with pytest.raises(mhe.SizeError):
        s.ip_solve(*args, lo[:-1], hi, out=out)
    with pytest.raises(mhe.SizeError):
        s.ip_solve(*args, lo, hi, out=(out[0], out[1][:-1], out[2]))
    assert "mhe_ip_solve" not in fake.calls
