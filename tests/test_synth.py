"""The seeded input generators (paper_1510_03110_gb300/synth.py) against the
recipe they document: draw order and distributions of one MHE stage, the
spectral radius of A, SPD weights, the S = 0 variant, the batched workload's
shapes and horizons, the pool expansion, and the serving plant's weights.
Every input of the tests and the bench comes from these functions, so the
recipe stated for the workloads is pinned here."""
import numpy as np
import pytest

from paper_1510_03110_gb300 import synth


@pytest.mark.parametrize("n,m,q,N", [(4, 2, 2, 64), (1, 1, 1, 3), (6, 3, 3, 10)])
def test_mhe_instance_follows_the_documented_draw_order(n, m, q, N):
    p = synth.mhe_instance(17, n, m, q, N)
    S = N - 1
    rng = np.random.default_rng(17)
    A_raw = rng.standard_normal((S, n, n))
    B = rng.standard_normal((S, n, m))
    C = rng.standard_normal((S, q, n))
    M = rng.standard_normal((S, m + q, m + q))
    a = rng.standard_normal((S, n))
    yt = rng.standard_normal((S, q))
    wt = rng.standard_normal((S, m))
    x0 = rng.standard_normal(n)
    rho = np.max(np.abs(np.linalg.eigvals(A_raw)), axis=-1)
    assert np.array_equal(p["B"], B) and np.array_equal(p["C"], C)
    assert np.array_equal(p["a"], a) and np.array_equal(p["yt"], yt) and np.array_equal(p["wt"], wt)
    assert np.array_equal(p["x0"], x0) and np.array_equal(p["P0inv"], np.eye(n))
    assert np.allclose(p["A"], 0.95 * A_raw / rho[:, None, None], rtol=0, atol=1e-15)
    assert np.allclose(p["R"], M @ M.transpose(0, 2, 1) + 0.1 * np.eye(m + q), rtol=0, atol=1e-13)
    assert p["N"] == N and (p["n"], p["m"], p["q"]) == (n, m, q)


def test_stage_properties():
    p = synth.mhe_instance(3, 6, 3, 3, 200)
    rho = np.max(np.abs(np.linalg.eigvals(p["A"])), axis=-1)
    assert np.allclose(rho, 0.95, rtol=0, atol=1e-12)
    assert np.allclose(p["R"], p["R"].transpose(0, 2, 1))
    assert np.linalg.eigvalsh(p["R"]).min() >= 0.1 - 1e-12      # R = M M^T + 0.1 I
    z = synth.mhe_instance(3, 6, 3, 3, 200, s_zero=True)
    assert np.all(z["R"][:, :3, 3:] == 0) and np.all(z["R"][:, 3:, :3] == 0)
    assert np.array_equal(z["R"][:, :3, :3], p["R"][:, :3, :3])   # only S is zeroed
    again = synth.mhe_instance(3, 6, 3, 3, 200)
    assert all(np.array_equal(p[k], again[k]) for k in ("A", "B", "C", "R", "a", "yt", "wt", "x0"))


def test_colmajor_layout():
    X = np.arange(24, dtype=float).reshape(2, 3, 4)
    cm = synth.colmajor(X)
    assert cm.shape == (2, 4, 3) and cm.flags["C_CONTIGUOUS"]
    # element (i, j) of matrix s sits at s * 12 + i + j * 3
    flat = cm.reshape(-1)
    for s in range(2):
        for i in range(3):
            for j in range(4):
                assert flat[s * 12 + i + j * 3] == X[s, i, j]


def test_batched_uneven_workload():
    w = synth.batch_uneven(3, count=300, pool_size=4096)
    assert len(w["nx"]) == 300 and set(np.unique(w["nx"])) <= {6, 12, 24}
    assert w["N"].min() >= 32 and w["N"].max() <= 2048
    members = np.sort(np.concatenate([b["members"] for b in w["buckets"].values()]))
    assert np.array_equal(members, np.arange(300))              # the buckets partition the batch
    for n, b in w["buckets"].items():
        assert b["m"] == b["q"] == n // 2 and np.all(w["nx"][b["members"]] == n)
        assert np.array_equal(b["N"], w["N"][b["members"]])
        S = int(np.sum(b["N"] - 1))
        assert len(b["idx"]) == S and b["idx"].min() >= 0 and b["idx"].max() < len(b["pool"]["A"])
        assert b["x0"].shape == (len(b["members"]), n)
        inst = synth.bucket_instance(b, 1)
        off = int(b["N"][0] - 1)
        assert inst["N"] == b["N"][1]
        assert np.array_equal(inst["A"], b["pool"]["A"][b["idx"][off:off + inst["N"] - 1]])
        assert np.array_equal(inst["x0"], b["x0"][1])
    again = synth.batch_uneven(3, count=300, pool_size=4096)
    assert np.array_equal(again["N"], w["N"]) and np.array_equal(again["nx"], w["nx"])


def test_serving_plant():
    n, m, q = 4, 2, 2
    s = synth.plant_stream(5, n, m, q, 30)
    assert np.all(s["wt"] == 0)
    assert np.all(s["R"][:, :m, m:] == 0) and np.all(s["R"][:, m:, :m] == 0)          # S = 0
    assert np.allclose(s["R"][:, m:, m:], 100.0 * np.eye(q))                          # V = (0.01 I)^{-1}
    assert np.linalg.eigvalsh(s["R"][:, :m, :m]).min() >= 0.1 - 1e-12                 # W = M M^T + 0.1 I
    assert s["x_true"].shape == (31, n)
    win = synth.window_of(s, 3, 10, np.zeros(n), n, m, q)
    assert win["N"] == 10 and np.array_equal(win["A"], s["A"][3:12])
    ps = synth.plant_streams(5, n, m, q, E=8, length=20, pool_size=64)
    e = synth.stream_of(ps, 3)
    assert e["A"].shape == (20, n, n) and np.array_equal(e["A"], ps["pool"]["A"][ps["idx"][3]])
    assert np.allclose(ps["pool"]["R"][:, m:, m:], 100.0 * np.eye(q))
