"""CPU checks of the C-ABI library: it loads without a GPU, exports every
symbol include/mhe.h declares, and its host-side planning answers."""
import os
import re

import pytest

from paper_1510_03110_gb300 import build, mhe

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return mhe.lib()


def declared():
    txt = open(os.path.join(ROOT, "include", "mhe.h")).read()
    return sorted(set(re.findall(r"\b(mhe_[a-z_0-9]+)\s*\(", txt)))


def test_header_symbols_are_exported(L):
    names = declared()
    assert "mhe_create" in names and "mhe_solve" in names
    for n in names:
        assert hasattr(L, n), n


def test_binding_declares_every_signature(L):
    """Every function of the header has argtypes (as many as the declaration has
    parameters) and a restype in the binding, so no 64-bit pointer or size is
    passed through ctypes' default int conversion."""
    txt = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "mhe.h")).read(), flags=re.S)
    decls = re.findall(r"\b(mhe_[a-z_0-9]+)\s*\(([^()]*)\)\s*;", txt)
    assert len(decls) == len(declared())
    for name, params in decls:
        params = params.strip()
        count = 0 if params in ("", "void") else params.count(",") + 1
        fn = getattr(L, name)
        assert fn.argtypes is not None and len(fn.argtypes) == count, (name, count, fn.argtypes)
        assert fn.restype is not None, name


def test_shapes_listed(L):
    s = mhe.shapes()
    for need in [(4, 2), (6, 3), (12, 6), (20, 10), (24, 12)]:
        assert need in s


def test_workspace_bytes_host_only(L):
    d, _ = mhe.make_dims(20, 10, [131072], prec=mhe.MHE_FP64, leaf_len=16, branching=8, top_len=4)
    b64 = mhe.mhe_workspace_bytes(d)
    d32, _ = mhe.make_dims(20, 10, [131072], prec=mhe.MHE_FP32_IR, leaf_len=16, branching=8, top_len=4)
    b32 = mhe.mhe_workspace_bytes(d32)
    # stored factors per stage: P n^2, chol G m^2, K and L m n, k m
    per_stage = 400 + 100 + 200 + 200 + 10
    assert b64 > 131072 * per_stage * 8
    assert b64 < 4 * 131072 * per_stage * 8
    # FP32 mode: the factors in FP32 plus FP32 copies of A, B, Q (n^2 + nm + (n+m)^2 per stage)
    copies = 131071 * (400 + 200 + 900) * 4
    assert b32 > 131072 * per_stage * 4 + copies
    assert b32 < 4 * 131072 * per_stage * 4 + 2 * copies


def test_zero_plan_fields_are_the_documented_defaults(L):
    """leaf_len = branching = top_len = 0 select max(8, ceil(nx / nw)), 4 and 4
    (the sizes of the workspace agree with the explicit plan)."""
    for nx, nw, N in [(24, 12, [100, 2000, 37]), (6, 3, [5000]), (64, 32, [1024] * 4), (1, 1, [3, 4])]:
        d0, _ = mhe.make_dims(nx, nw, N, prec=mhe.MHE_FP32_IR)
        de, _ = mhe.make_dims(nx, nw, N, prec=mhe.MHE_FP32_IR, leaf_len=max(8, -(-nx // nw)), branching=4,
                              top_len=4)
        assert mhe.mhe_workspace_bytes(d0) == mhe.mhe_workspace_bytes(de) > 0


def test_bad_dims_rejected_on_host(L):
    d, _ = mhe.make_dims(5, 4, [10])        # shape not compiled
    assert mhe.mhe_workspace_bytes(d) == 0
    d, _ = mhe.make_dims(4, 2, [10], leaf_len=1)   # leaf_len * nw < nx: rank-revealing master stages
    assert mhe.mhe_workspace_bytes(d) > 0
    d, _ = mhe.make_dims(4, 2, [10], leaf_len=-1)
    assert mhe.mhe_workspace_bytes(d) > 0            # negative = the default plan
    d, _ = mhe.make_dims(4, 2, [10], branching=1)    # branching must be >= 2
    assert mhe.mhe_workspace_bytes(d) == 0
    d, _ = mhe.make_dims(4, 2, [0])         # horizon must be >= 1
    assert mhe.mhe_workspace_bytes(d) == 0


def test_product_path_has_no_fallback(tmp_path, monkeypatch):
    """Without libmhe.so the binding raises instead of computing anything."""
    monkeypatch.setattr(mhe, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(mhe, "_lib", None)
    with pytest.raises(RuntimeError):
        mhe.lib()


def test_precision_enum_matches_the_binding():
    """The mhe_precision values of include/mhe.h and the binding's constants agree."""
    txt = open(os.path.join(ROOT, "include", "mhe.h")).read()
    body = txt[txt.index("typedef enum {\n    MHE_FP64"):]
    body = body[:body.index("} mhe_precision;")]
    vals = dict((k, int(v)) for k, v in re.findall(r"\b(MHE_[A-Z0-9_]+)\s*=\s*(\d+)", body))
    assert vals == {"MHE_FP64": mhe.MHE_FP64, "MHE_FP32_IR": mhe.MHE_FP32_IR,
                    "MHE_TF32_IR": mhe.MHE_TF32_IR, "MHE_BF16_IR": mhe.MHE_BF16_IR}


def test_tensor_core_precisions_share_the_fp32_workspace(L):
    """The tensor-core precisions change only the products of the reductions:
    the same workspace as MHE_FP32_IR; an unknown precision is refused."""
    d32, _ = mhe.make_dims(64, 32, [100, 7], prec=mhe.MHE_FP32_IR)
    dtf, _ = mhe.make_dims(64, 32, [100, 7], prec=mhe.MHE_TF32_IR)
    dbf, _ = mhe.make_dims(64, 32, [100, 7], prec=mhe.MHE_BF16_IR)
    dno, _ = mhe.make_dims(64, 32, [100, 7], prec=7)
    assert mhe.mhe_workspace_bytes(dtf) == mhe.mhe_workspace_bytes(d32) > 0
    assert mhe.mhe_workspace_bytes(dbf) == mhe.mhe_workspace_bytes(d32)
    assert mhe.mhe_workspace_bytes(dno) == 0


def test_pointer_checks_raise_without_asserts():
    """The binding's pointer checks are real checks (they survive python -O): a
    host tensor where a device pointer is expected, or the wrong dtype or
    layout, raises TypeError before anything reaches the library."""
    import numpy as np
    import torch
    with pytest.raises(TypeError):
        mhe._ptr(torch.zeros(4, dtype=torch.float64))          # host memory
    with pytest.raises(TypeError):
        mhe._ptr(np.zeros(4))
    with pytest.raises(TypeError):
        mhe._hptr(np.zeros(4, dtype=np.float32))
    with pytest.raises(TypeError):
        mhe._hptr(np.zeros((4, 4))[:, 1])                      # not contiguous
    with pytest.raises(TypeError):
        mhe._hptr(torch.zeros(4, dtype=torch.float32))
    assert mhe._hptr(np.zeros(4)) is not None and mhe._hptr(torch.zeros(4, dtype=torch.float64)) is not None
    assert mhe._ptr(None) is None and mhe._hptr(None) is None


def test_size_checks_of_the_binding():
    """Arrays shorter than the problem's layout are refused with MHE_E_ARG before
    the library sees their pointers; None is left to the library (NULL check)."""
    import numpy as np
    import torch
    nx, nw, ny, N = 4, 2, 2, [5, 9]
    S, batch, X, W = sum(v - 1 for v in N), len(N), sum(v + 1 for v in N), sum(nx + (v - 1) * nw for v in N)
    ok = dict(A=torch.zeros(S * nx * nx), B=torch.zeros(S * nx * nw), C=torch.zeros(S * ny * nx),
              R=torch.zeros(S * (nw + ny) ** 2), a=torch.zeros(S * nx), yt=torch.zeros(S * ny),
              wt=torch.zeros(S * nw), x0=torch.zeros(batch * nx), P0inv=torch.zeros(batch * nx * nx),
              Q=torch.zeros(S * (nx + nw) ** 2), l=torch.zeros(S * (nx + nw)), x=torch.zeros(X * nx),
              w=torch.zeros(W), lam=torch.zeros(X * nx))
    mhe.check_sizes(nx, nw, S, batch, X, W, ny, **ok)
    mhe.check_sizes(nx, nw, S, batch, X, W, ny, **dict(ok, C=None))
    for name in ok:
        short = dict(ok)
        short[name] = torch.zeros(ok[name].numel() - 1)
        with pytest.raises(mhe.MheError) as e:
            mhe.check_sizes(nx, nw, S, batch, X, W, ny, **short)
        assert e.value.code == -1 and isinstance(e.value, ValueError) and name in str(e.value)
    # a wrong ny makes the MHE-form arrays too short: refused the same way
    with pytest.raises(mhe.MheError):
        mhe.check_sizes(nx, nw, S, batch, X, W, ny + 1, C=ok["C"])
    mhe.check_sizes(nx, nw, 0, 2, 4, 2 * nx, ny, A=np.zeros(0), x0=np.zeros(2 * nx))   # N = 1: no stages


def test_server_size_checks_of_the_binding():
    """The serving binding refuses a window or a packed stage shorter than the
    estimator's shape needs, before the library reads the host arrays."""
    import numpy as np
    from paper_1510_03110_gb300 import synth
    srv = mhe.Server.__new__(mhe.Server)      # the checks run before any library call
    srv.s, srv.nx, srv.stage_len = None, {}, {}
    n, m, q = 4, 2, 2
    st = synth.plant_stream(1, n, m, q, 30)
    win = synth.window_of(st, 0, 20, np.zeros(n), n, m, q)
    short = dict(win, C=win["C"][:-1])
    with pytest.raises(mhe.MheError) as e:
        srv.open(short)
    assert e.value.code == -1 and "C" in str(e.value)
    with pytest.raises(mhe.MheError):
        srv.open(dict(win, N=25))             # more stages claimed than given
    srv.stage_len[7] = n * n + n * m + q * n + (m + q) ** 2 + n + q + m
    packed = mhe.pack_stage(*(st[f][0] for f in ("A", "B", "C", "R", "a", "yt", "wt")))
    assert packed.size == srv.stage_len[7]
    with pytest.raises(mhe.MheError):
        srv.submit(7, packed[:-1])


def test_plan_info_unpacks_the_levels(monkeypatch):
    """mhe_plan_info's buffer: 3 long longs per level, read back as (level, chunks, stages)."""
    class Fake:
        def mhe_plan_info(self, ctx, buf, cap):
            assert cap == 256
            for k, v in enumerate([0, 40, 1000, 1, 9, 39, 2, 1, 8]):
                buf[k] = v
            return 3
    monkeypatch.setattr(mhe, "lib", lambda: Fake())
    assert mhe.mhe_plan_info(None) == [(0, 40, 1000), (1, 9, 39), (2, 1, 8)]


def test_fp64_workspace_at_nx64_and_fp64_master_levels(L):
    """FP64 at nx = 64 is accepted: its workspace includes the reduction's global-memory
    team slots (two 128-thread teams per SM of 152, ~342 KB each).  FP64 master levels
    enlarge the FP32 workspace by the FP64 copies of the upper levels' arrays."""
    d64, _ = mhe.make_dims(64, 32, [100, 7], prec=mhe.MHE_FP64)
    d32, _ = mhe.make_dims(64, 32, [100, 7], prec=mhe.MHE_FP32_IR)
    assert mhe.mhe_workspace_bytes(d64) > 304 * 342 * 1024 > mhe.mhe_workspace_bytes(d32) > 0
    for nx, nw in [(24, 12), (64, 32), (6, 3)]:
        plain, _ = mhe.make_dims(nx, nw, [2000, 300], prec=mhe.MHE_FP32_IR, leaf_len=8, branching=4, top_len=4)
        mixed, _ = mhe.make_dims(nx, nw, [2000, 300], prec=mhe.MHE_FP32_IR, leaf_len=8, branching=4, top_len=4,
                                 fp64_masters=True)
        assert mhe.mhe_workspace_bytes(mixed) > mhe.mhe_workspace_bytes(plain) > 0
    assert ctypes_sizeof_dims_matches_header()


def ctypes_sizeof_dims_matches_header():
    """The binding's mhe_dims has every field of the header's struct, in order."""
    txt = open(os.path.join(ROOT, "include", "mhe.h")).read()
    body = txt[txt.index("typedef struct {\n    int nx;"):]
    body = body[:body.index("} mhe_dims;")]
    names = re.findall(r"^\s+(?:const\s+)?(?:int|double)\*?\s+(\w+);", body, re.M)
    return names == [f[0] for f in mhe.mhe_dims._fields_]


def test_team_width_variants_listed_and_validated(L):
    """Every compiled shape lists its team widths, the default first; a width that
    is not compiled for the shape is refused on the host; the registry of shapes
    lists each shape once."""
    shapes = mhe.shapes()
    assert len(set(shapes)) == len(shapes)
    for nx, nw in shapes:
        teams = mhe.shape_teams(nx, nw)
        assert teams and len(set(teams)) == len(teams), (nx, nw)
        for t in teams:
            d, _keep = mhe.make_dims(nx, nw, [40, 7], mhe.MHE_FP32_IR, team=t)
            assert mhe.mhe_workspace_bytes(d) > 0, (nx, nw, t)
        for t in (1, 3, 4096):
            d, _keep = mhe.make_dims(nx, nw, [40, 7], mhe.MHE_FP32_IR, team=t)
            assert mhe.mhe_workspace_bytes(d) == 0, (nx, nw, t)
    assert mhe.shape_teams(6, 3) == [8, 16, 32]
    assert mhe.shape_teams(12, 6) == [16, 32]
    assert mhe.shape_teams(5, 5) == []


def test_ip_opts_fields_match_header():
    """The binding's mhe_ip_opts has every field of the header's struct, in order,
    and the header names both interior-point methods with the binding's values."""
    txt = open(os.path.join(ROOT, "include", "mhe.h")).read()
    end = txt.index("} mhe_ip_opts;")
    body = txt[txt.rindex("typedef struct {", 0, end):end]
    names = re.findall(r"^\s+(?:const\s+)?(?:int|double)\*?\s+(\w+);", body, re.M)
    assert names == [f[0] for f in mhe.mhe_ip_opts._fields_]
    assert f"MHE_IP_PREDICTOR_CORRECTOR = {mhe.MHE_IP_PREDICTOR_CORRECTOR}" in txt
    assert f"MHE_IP_PATH_FOLLOWING = {mhe.MHE_IP_PATH_FOLLOWING}" in txt
