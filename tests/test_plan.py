"""The host-side tree planner (csrc/plan.cpp, Algorithm 5's levels and chunk
lists) against the structure the method fixes, for many horizons and plans:

* at every level each instance's horizon is tiled by its chunks in order; all
  chunks have the level's length (leaf_len at level 0, branching above) except
  the last, which takes the remainder (1..L stages; reading R9);
* the p non-last chunks of a level become the p stages of the next level's
  master problem (Eq. red_mpc_problem), so N_{k+1} = chunks_k - 1, and chunk i
  of level k is master stage i of level k+1 (its parent link);
* the top problem (horizon <= top_len) is one chunk, flagged last and top, and
  only level 0's first chunk holds the arrival stage;
* the depth is logarithmic in N; invalid plans are refused.

The planner is compiled for the host with the system C++ compiler."""
import ctypes
import math
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1510_03110_gb300", "csrc")

SHIM = r'''
#include "plan.h"
// per chunk: level, inst, t0, len, flags, g0, parent; per (level, inst): N
extern "C" int plan_chunks(int n, int m, const int* N, int batch, int leaf, int br, int top,
                           long long* out, int cap, int* levN, int levcap)
{
    mhe::Plan p;
    const char* err = nullptr;
    if (mhe::make_plan(n, m, N, batch, leaf, br, top, p, &err) != 0) return -1;
    int k = 0;
    for (int lv = 0; lv < (int)p.levels.size(); ++lv) {
        for (const auto& c : p.levels[lv].chunks) {
            if (k < cap) {
                long long* o = out + 7 * k;
                o[0] = lv; o[1] = c.inst; o[2] = c.t0; o[3] = c.len; o[4] = c.flags; o[5] = c.g0; o[6] = c.parent;
            }
            ++k;
        }
        for (int b = 0; b < batch && lv * batch + b < levcap; ++b) levN[lv * batch + b] = p.levels[lv].li[b].N;
    }
    return k;
}
extern "C" int plan_levels(int n, int m, const int* N, int batch, int leaf, int br, int top)
{
    mhe::Plan p;
    const char* err = nullptr;
    if (mhe::make_plan(n, m, N, batch, leaf, br, top, p, &err) != 0) return -1;
    return (int)p.levels.size();
}
'''

CH_LAST, CH_TOP, CH_ARRIVAL = 1, 2, 4


@pytest.fixture(scope="module")
def planner():
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    d = tempfile.mkdtemp()
    src = os.path.join(d, "shim.cpp")
    so = os.path.join(d, "shim.so")
    open(src, "w").write(SHIM)
    subprocess.run([cxx, "-std=c++17", "-O1", "-shared", "-fPIC", "-I", CSRC, src, os.path.join(CSRC, "plan.cpp"),
                    "-o", so], check=True)
    L = ctypes.CDLL(so)
    I, P = ctypes.c_int, ctypes.c_void_p
    L.plan_chunks.restype = I
    L.plan_chunks.argtypes = [I, I, P, I, I, I, I, P, I, P, I]
    L.plan_levels.restype = I
    L.plan_levels.argtypes = [I, I, P, I, I, I, I]

    def run(n, m, Ns, leaf, br, top):
        Ns = np.ascontiguousarray(Ns, dtype=np.int32)
        nl = L.plan_levels(n, m, Ns.ctypes.data, len(Ns), leaf, br, top)
        if nl < 0:
            return None
        cap = 4 * int(Ns.sum()) + 64
        out = np.zeros(7 * cap, dtype=np.int64)
        levN = np.zeros(nl * len(Ns), dtype=np.int32)
        k = L.plan_chunks(n, m, Ns.ctypes.data, len(Ns), leaf, br, top, out.ctypes.data, cap,
                          levN.ctypes.data, levN.size)
        assert 0 <= k <= cap
        return out[:7 * k].reshape(k, 7), levN.reshape(nl, len(Ns))
    yield run
    shutil.rmtree(d, ignore_errors=True)


def check_tree(chunks, levN, Ns, leaf, br, top, n, m):
    nl = levN.shape[0]
    for b, N0 in enumerate(Ns):
        assert levN[0, b] == N0
        for k in range(nl):
            Nk = int(levN[k, b])
            mine = chunks[(chunks[:, 0] == k) & (chunks[:, 1] == b)]
            if Nk == 0:   # the instance's tree ended below this level
                assert len(mine) == 0
                continue
            mine = mine[np.argsort(mine[:, 2])]
            # the chunks tile [0, Nk) in order
            assert mine[0, 2] == 0
            assert np.all(mine[1:, 2] == mine[:-1, 2] + mine[:-1, 3])
            assert mine[-1, 2] + mine[-1, 3] == Nk
            assert np.all(mine[:, 3] >= 1)
            last = (mine[:, 4] & CH_LAST) != 0
            assert last[-1] and not last[:-1].any()
            # arrival stage only in level 0's first chunk
            arr = (mine[:, 4] & CH_ARRIVAL) != 0
            assert arr[0] == (k == 0) and not arr[1:].any()
            if Nk <= top:
                assert len(mine) == 1 and (mine[0, 4] & CH_TOP)
                assert mine[0, 6] == -1
                assert all(levN[j, b] == 0 for j in range(k + 1, nl))
                continue
            if len(mine) == 1:   # the planner made it the top (the leaf rank rule)
                assert mine[0, 4] & CH_TOP
                continue
            assert not (mine[:, 4] & CH_TOP).any()
            # equal lengths but the last (chunk_bounds halves L when Nk <= L)
            L = leaf if k == 0 else br
            if Nk <= L:
                L = (Nk + 1) // 2
            assert np.all(mine[:-1, 3] == L) and 1 <= mine[-1, 3] <= L
            # the p non-last chunks are the next level's stages, chunk i -> master stage i
            p = len(mine) - 1
            assert k + 1 < nl and levN[k + 1, b] == p
            base = mine[0, 6]
            assert np.all(mine[:-1, 6] == base + np.arange(p)) and mine[-1, 6] == -1
            up = chunks[(chunks[:, 0] == k + 1) & (chunks[:, 1] == b)]
            up_first_stage = up[np.argsort(up[:, 2])][0]
            assert up_first_stage[5] == base   # the master problem's stages start at the parents' index
            # global stage index of a chunk = the level's base of the instance + t0
            assert np.all(mine[:, 5] - mine[:, 2] == mine[0, 5])
    # depth: each level shrinks the horizon by the chunk length
    depth_bound = 2 + math.ceil(math.log(max(Ns) / max(2, leaf) + 1, 2))
    assert nl <= depth_bound + 1


@pytest.mark.parametrize("leaf,br,top", [(8, 4, 4), (32, 8, 4), (3, 2, 2), (64, 16, 1), (4, 4, 10)])
def test_tree_structure_over_many_horizons(planner, leaf, br, top):
    rng = np.random.default_rng(leaf * 100 + br)
    Ns = [1, 2, 3, 4, 5, 7, 8, 9, 16, 17, 31, 33, 64, 65, 127, 250, 1000, 2047] + list(rng.integers(1, 3000, 40))
    r = planner(6, 3, Ns, leaf, br, top)
    assert r is not None
    check_tree(*r, Ns, leaf, br, top, 6, 3)


def test_serial_plan_is_one_chunk_per_instance(planner):
    Ns = [1, 5, 99, 1024]
    chunks, levN = planner(24, 12, Ns, 32, 4, max(Ns) + 1)
    assert levN.shape[0] == 1 and len(chunks) == len(Ns)
    assert np.all(chunks[:, 4] == (CH_LAST | CH_TOP | CH_ARRIVAL))
    assert np.all(chunks[:, 3] == Ns)


def test_invalid_plans_are_refused(planner):
    assert planner(24, 12, [100], 1, 4, 4) is None    # leaf_len * nw < nx: the chunk's B^ is singular
    assert planner(24, 12, [100], 8, 1, 4) is None    # branching < 2
    assert planner(24, 12, [100], 8, 4, 0) is None    # top_len < 1
    assert planner(24, 12, [0, 5], 8, 4, 4) is None   # a horizon of 0
