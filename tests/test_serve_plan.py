"""The serving planner with factorisation reuse (csrc/plan.cpp: make_serve_plan)
on the host, against a symbolic model of what each chunk's Algorithm 4 output
depends on.

A chunk's stored factors and its master stage (Eq. red_mpc_problem) depend on
exactly its stages' data and, for a level's last chunk, on the terminal the
level below hands up.  The model gives every chunk a signature built from
those inputs, recursively from the measured samples, and replays the rounds of
several estimators whose windows shift by one sample per round (Section II's
receding horizon): a chunk the planner marks dirty writes its signature into
its ring slots; a chunk it keeps must find there the signature a fresh
reduction would write; every chunk above level 0 must read, at its ring slots,
the master data of exactly its stages.  The per-round checks also cover the
tree's shape (each level's chunks tile its horizon in order, the arrival stage
in level 0's first chunk, the top problem one chunk) and that the re-reduced
stages per shift stay near 3 chunks per level, not O(N).

The planner is compiled for the host with the system C++ compiler."""
import ctypes
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
#include <stdio.h>
#include <vector>
static std::vector<std::vector<mhe::ServeLevelHist>> H(64);
extern "C" void reset() { for (auto& h : H) h.clear(); }
// caps and tail for horizon N
extern "C" int caps(int N, int leaf, int br, int top, long long* cap, int capn, long long* tail)
{
    std::vector<long long> c;
    int k = mhe::serve_caps(N, leaf, br, top, c, tail);
    for (int i = 0; i < k && i < capn; ++i) cap[i] = c[i];
    return k;
}
// one round over `batch` windows; per chunk 11 long longs:
// level, inst, t0, len, flags, g0, parent, parent2, pw, px, dirty
extern "C" int round_plan(int n, int m, int batch, const int* N, const long long* k0, const int* est,
                          const long long* base, const long long* cap, int nlev, int leaf, int br, int top,
                          long long* out, int outcap, int* levN, long long* reduced)
{
    std::vector<mhe::ServeWindow> w(batch);
    for (int b = 0; b < batch; ++b) {
        w[b].N = N[b]; w[b].k0 = k0[b]; w[b].in_off = 0;
        w[b].base = base + (long long)b * nlev; w[b].cap = cap + (long long)b * nlev; w[b].nlev = nlev;
        w[b].hist = &H[est[b]];
    }
    mhe::Plan p;
    std::vector<std::vector<mhe::ChunkDesc>> dirty;
    const char* err = nullptr;
    *reduced = 0;
    if (mhe::make_serve_plan(n, m, w, leaf, br, top, p, dirty, reduced, &err) != 0) {
        fprintf(stderr, "make_serve_plan: %s\n", err);
        return -1;
    }
    int q = 0;
    for (int lv = 0; lv < (int)p.levels.size(); ++lv) {
        for (const auto& c : p.levels[lv].chunks) {
            int d = 0;
            for (const auto& x : dirty[lv]) if (x.inst == c.inst && x.t0 == c.t0 && x.g0 == c.g0) d = 1;
            if (q < outcap) {
                long long* o = out + 11 * q;
                o[0] = lv; o[1] = c.inst; o[2] = c.t0; o[3] = c.len; o[4] = c.flags; o[5] = c.g0; o[6] = c.parent;
                o[7] = c.parent2; o[8] = c.pw; o[9] = c.px; o[10] = d;
            }
            ++q;
        }
        for (int b = 0; b < batch; ++b) levN[lv * batch + b] = p.levels[lv].li[b].N;
    }
    return q;
}
'''

CH_LAST, CH_TOP, CH_ARRIVAL = 1, 2, 4


@pytest.fixture(scope="module")
def lib():
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    d = tempfile.mkdtemp()
    src = os.path.join(d, "shim.cpp")
    open(src, "w").write(SHIM)
    so = os.path.join(d, "libsp.so")
    subprocess.run([cxx, "-std=c++17", "-O1", "-shared", "-fPIC", "-I", CSRC, src, os.path.join(CSRC, "plan.cpp"),
                    "-o", so], check=True, capture_output=True, text=True)
    return ctypes.CDLL(so)


def P(a, t=ctypes.c_longlong):
    return a.ctypes.data_as(ctypes.POINTER(t))


def run_rounds(lib, n, m, Ns, leaf, br, top, rounds, seed=0):
    """Replay `rounds` rounds; in each a random subset of the estimators shifts by one."""
    rng = np.random.default_rng(seed)
    lib.reset()   # the shim keeps each estimator's history between rounds; start afresh
    E = len(Ns)
    caps, tails = [], []
    for N in Ns:
        c = np.zeros(64, dtype=np.int64)
        t = np.zeros(1, dtype=np.int64)
        k = lib.caps(int(N), leaf, br, top, P(c), 64, P(t))
        assert k >= 1
        caps.append(c[:k])
        tails.append(int(t[0]))
    nlev = max(len(c) for c in caps)
    # per level a store shared by the estimators: estimator e's slots start at base[e][k]
    base = np.zeros((E, nlev), dtype=np.int64)
    capa = np.ones((E, nlev), dtype=np.int64)
    total = np.zeros(nlev, dtype=np.int64)
    for e in range(E):
        for k in range(nlev):
            ck = int(caps[e][k]) if k < len(caps[e]) else int(caps[e][-1])
            capa[e, k] = ck
            base[e, k] = total[k]
            total[k] += ck + tails[e]
    fac = [dict() for _ in range(nlev)]      # level k: slot -> signature of the chunk that stored factors there
    mst = [dict() for _ in range(nlev)]      # level k: slot -> signature of the master stage stored there
    k0 = np.zeros(E, dtype=np.int64)
    first_round = np.ones(E, dtype=bool)
    stats = []
    for r in range(rounds):
        who = [e for e in range(E) if first_round[e] or rng.random() < 0.7]
        if not who:
            continue
        for e in who:
            if not first_round[e]:
                k0[e] += 1
        batch = len(who)
        N = np.array([Ns[e] for e in who], dtype=np.int32)
        K0 = np.array([k0[e] for e in who], dtype=np.int64)
        est = np.array(who, dtype=np.int32)
        b_ = np.ascontiguousarray(base[who]).reshape(-1)
        c_ = np.ascontiguousarray(capa[who]).reshape(-1)
        out = np.zeros(11 * 200000, dtype=np.int64)
        levN = np.zeros(64 * batch, dtype=np.int32)
        red = np.zeros(1, dtype=np.int64)
        q = lib.round_plan(n, m, batch, P(N, ctypes.c_int), P(K0), P(est, ctypes.c_int), P(b_), P(c_), nlev,
                           leaf, br, top, P(out), 200000, P(levN, ctypes.c_int), P(red))
        assert q > 0
        ch = out[:11 * q].reshape(q, 11)
        check_round(ch, who, Ns, k0, base, capa, tails, fac, mst, nlev, batch, levN)
        for e in who:
            first_round[e] = False
        stats.append((batch, int(red[0]), sum(Ns[e] for e in who)))
    return stats


def check_round(ch, who, Ns, k0, base, capa, tails, fac, mst, nlev, batch, levN):
    for b, e in enumerate(who):
        mine = ch[ch[:, 1] == b]
        levels = int(mine[:, 0].max()) + 1
        # fresh signatures bottom-up: a level-0 stage is its sample (or the arrival stage)
        stage_sig = [("arrival",)] + [("s", int(k0[e]) + t) for t in range(Ns[e] - 1)]
        terminal = ("zero",)
        for lv in range(levels):
            rows = mine[mine[:, 0] == lv]
            rows = rows[np.argsort(rows[:, 2])]
            Nk = int(levN[lv * batch + b])
            assert Nk == len(stage_sig), (lv, Nk, len(stage_sig))
            # tiling in order; flags
            t = 0
            for i, r in enumerate(rows):
                _, _, t0, ln, fl, g0, par, par2, pw, px, d = (int(v) for v in r)
                assert t0 == t and ln >= 1
                t += ln
                assert bool(fl & CH_LAST) == (i == len(rows) - 1)
                assert bool(fl & CH_ARRIVAL) == (lv == 0 and i == 0)
                assert bool(fl & CH_TOP) == (len(rows) == 1)
            assert t == Nk
            lo, hi = base[e, lv], base[e, lv] + capa[e, lv] + tails[e]
            next_sig = []
            for i, r in enumerate(rows):
                _, _, t0, ln, fl, g0, par, par2, pw, px, d = (int(v) for v in r)
                last = bool(fl & CH_LAST)
                sig = (lv, tuple(stage_sig[t0:t0 + ln]), last, terminal if last else None)
                slots = [g0 + tt for tt in range(ln) if not (lv == 0 and t0 + tt == 0)]
                for s in slots:
                    assert lo <= s < hi, (lv, s, lo, hi)
                if lv >= 1:   # the master data read at the chunk's slots are its stages'
                    for tt, s in enumerate(slots):
                        assert mst[lv].get(s) == stage_sig[t0 + tt], (lv, s)
                if d:
                    for s in slots:
                        fac[lv][s] = sig
                else:
                    assert not last and i > 0, "first, last and top chunks are reduced every round"
                    for s in slots:
                        assert fac[lv].get(s) == sig, (lv, s, "kept chunk's stored factors are stale")
                if not last:
                    msig = ("m", sig)
                    pl, ph = base[e, lv + 1], base[e, lv + 1] + capa[e, lv + 1] + tails[e]
                    assert pl <= par < ph
                    if d:
                        mst[lv + 1][par] = msig
                        if par2 >= 0:
                            assert pl <= par2 < ph
                            mst[lv + 1][par2] = msig
                    else:
                        assert mst[lv + 1].get(par) == msig
                    next_sig.append(sig)
                else:
                    terminal = ("t", sig)
            stage_sig = [("m", s_) for s_ in next_sig]
        # within the round, distinct stages of one level never share a factor slot
        for lv in range(levels):
            rows = mine[mine[:, 0] == lv]
            slots = [int(r[5]) + tt for r in rows for tt in range(int(r[3])) if not (lv == 0 and int(r[2]) + tt == 0)]
            assert len(slots) == len(set(slots))


@pytest.mark.parametrize("Ns,leaf,br,top", [([50, 200, 1000], 8, 4, 4), ([40, 61, 300], 4, 2, 2),
                                            ([1000, 77], 16, 8, 4), ([12, 9, 30], 3, 3, 4)])
def test_reuse_keeps_only_what_a_fresh_reduction_would_give(lib, Ns, leaf, br, top):
    stats = run_rounds(lib, 6, 3, Ns, leaf, br, top, rounds=150)
    # after the first round, the re-reduced stages per shifted window are a few chunks per level
    later = stats[1:]
    per = sum(s[1] for s in later) / sum(s[0] for s in later)
    levels = np.ceil(np.log(max(Ns)) / np.log(br)) + 2
    assert per <= 3 * (leaf + 1) + 3 * br * levels + top, per
    assert per < 0.5 * np.mean(Ns) or max(Ns) < 60


def test_serial_plan_rereduces_everything(lib):
    """top_len >= N: the serial recursion has one chunk, which every shift changes."""
    stats = run_rounds(lib, 6, 3, [50, 80], 8, 4, 1000, rounds=20)
    for batch, red, total in stats:
        assert red == total
