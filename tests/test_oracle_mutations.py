"""Planted mistakes: each plausible slip in the C oracle must fail a pin.

A mutated copy of the oracle source is compiled into a temporary library on
the CPU, swapped in, and the relevant pin is shown to fail.  Nothing here
touches a GPU.
"""
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from oracle import core, dense
from paper_1510_03110_gb300 import synth

from test_golden import as_float, load  # noqa: E402
from test_oracle import _mhe_cost, random_uftoc, rel  # noqa: E402

SRC = open(core._SRC).read()

MUTATIONS = {
    # Alg 1: F = Q_x + A^T P A loses its Q_x term
    "drop_Qx_in_F": ("AT(F, i, j, n) += AT(Qt, i, j, nq);", "(void)0;"),
    # Alg 1: F = Q_x + A P A (transposed operand)
    "transpose_A_in_F": ("mm(n, n, n, At, n, 1, PA, n, 0, F, n);", "mm(n, n, n, At, n, 0, PA, n, 0, F, n);"),
    # Alg 1: H = Q_xw + A P B (transposed operand)
    "wrong_operand_in_H": ("mm(n, mt, n, At, n, 1, PB, n, 0, H, n);", "mm(n, mt, n, At, n, 0, PB, n, 0, H, n);"),
    # Alg 2: sign of l_x in Psi
    "sign_lx_in_Psi": ("Psit[i] -= tv[i] + lx[i];", "Psit[i] -= tv[i] - lx[i];"),
    # Alg 2: the cbar recursion drops -1/2 k^T G k
    "drop_kGk_in_cbar": ("- 0.5 * kGk", "- 0.0 * kGk"),
    # Alg 3: lambda_t = P_t x_t + Psi_t
    "sign_Psi_in_lambda": ("tv[i] - Psi[(size_t)t * n + i]", "tv[i] + Psi[(size_t)t * n + i]"),
    # Section II: Q_xw = +(S C)^T
    "sign_Qxw_assembly": ("AT(Q, i, n + j, nq) = -AT(SC, j, i, m);", "AT(Q, i, n + j, nq) = AT(SC, j, i, m);"),
    # Section II: l_w = S y~ + W w~
    "sign_lw_assembly": ("l[n + i] = t1[i] - t2[i];", "l[n + i] = t1[i] + t2[i];"),
    # Alg 1: P_t = F - K^T G K stored as computed, not its symmetric part
    "drop_symmetrisation_of_P": ("0.5 * ((AT(F, i, j, n) - AT(KGK, i, j, n)) +\n                                         (AT(F, j, i, n) - AT(KGK, j, i, n)));",
                                 "(AT(F, i, j, n) - AT(KGK, i, j, n));"),
    # Section II: l_w = S^T y~ (S and S^T confused; type-checks when nw = ny)
    "transpose_S_in_lw": ("/* l_w = S y~ - W w~ */\n    mv(m, q, S, m, 0, yt, t1);",
                          "/* l_w = S y~ - W w~ */\n    mv(m, q, S, m, 1, yt, t1);"),
    # residual: the -lambda_t term of the x-stationarity row is dropped
    "drop_lambda_in_residual": ("if (i < n) { s -= ltt[i]; rs += 1.0; }", "if (i < n) { rs += 1.0; }"),
}


@pytest.fixture(scope="module")
def tmpdir_mod():
    with tempfile.TemporaryDirectory() as d:
        yield d


def _mutant(tmpdir, name):
    old, new = MUTATIONS[name]
    assert SRC.count(old) == 1, name
    path_c = os.path.join(tmpdir, f"{name}.c")
    path_so = os.path.join(tmpdir, f"{name}.so")
    with open(path_c, "w") as f:
        f.write(SRC.replace(old, new))
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c99", "-o", path_so, path_c, "-lm"])
    return core.load(path_so)


# the mistakes that change the Newton step itself (the rest touch only the
# objective's constant, the residual routine or rounding)
STEP_CHANGING = ["drop_Qx_in_F", "transpose_A_in_F", "wrong_operand_in_H", "sign_lx_in_Psi",
                 "sign_Psi_in_lambda", "sign_Qxw_assembly", "sign_lw_assembly", "transpose_S_in_lw"]


def _golden_fails(lib_mut) -> bool:
    """The exact golden steps (n = 2, nw = ny = 1, N = 6 and n = 4, nw = ny = 2, N = 5
    with a non-symmetric S) against a library."""
    saved = core._lib
    core._lib = lib_mut
    try:
        for name in ("mhe_2x1x1_N6_exact", "mhe_4x2x2_N5_exact"):
            pf, sol = as_float(load(name))
            r = oracle.riccati(oracle.mhe_to_uftoc(pf))
            if r["status"] != 0 or any(rel(r[k], sol[k]) > 1e-12 for k in ("x", "w", "lam")):
                return True
        return False
    finally:
        core._lib = saved


def _pins_fail(lib_mut) -> list:
    """Run the core pins against a mutated library; return those that fail."""
    saved = core._lib
    core._lib = lib_mut
    failed = []
    try:
        p = random_uftoc(3, 3, 6, [2, 3])
        r = oracle.riccati(p)
        d = dense.solve(p)
        if r["status"] != 0 or rel(r["x"], d["x"]) > 1e-10 or rel(r["lam"], d["lam"]) > 1e-10 \
                or rel(r["w"], d["w"]) > 1e-10:
            failed.append("lu")
        dz = dense.solve(p)
        z = np.concatenate([dz["x"].ravel(), dz["w"], dz["lam"].ravel()])
        res = oracle.kkt_residual(p, dz["x"], dz["w"], dz["lam"])
        if res["relres"] > 1e-12 or abs(res["r_inf"] - np.abs(dz["b"] - dz["K"] @ z).max()) > 1e-12:
            failed.append("residual")
        # perturbed point: the residual routine must agree with b - K z
        zp = z + 1e-3
        xp = zp[:len(dz["x"].ravel())].reshape(dz["x"].shape)
        res2 = oracle.kkt_residual(p, xp, zp[xp.size:xp.size + dz["w"].size],
                                   zp[xp.size + dz["w"].size:].reshape(dz["lam"].shape))
        if abs(res2["r_inf"] - np.abs(dz["b"] - dz["K"] @ zp).max()) > 1e-10:
            failed.append("residual_vs_dense")
        v1 = 0.5 * p.x0 @ r["P0"] @ p.x0 - r["Psi0"] @ p.x0 + r["cbar0"]
        if abs(v1 - oracle.objective(p, r["x"], r["w"])) > 1e-9 * (1 + abs(v1)):
            failed.append("objective")
        q = synth.mhe_instance(8, 3, 2, 2, 6)
        u = oracle.mhe_to_uftoc(q)
        rng = np.random.default_rng(0)
        xm0 = rng.standard_normal(3)
        wm = [rng.standard_normal(2) for _ in range(5)]
        xm = [xm0]
        for k in range(5):
            xm.append(q["A"][k] @ xm[k] + q["B"][k] @ wm[k] + q["a"][k])
        xu = np.vstack([q["x0"]] + xm)
        wu = np.concatenate([xm0 - q["x0"]] + wm)
        if abs(oracle.objective(u, xu, wu) - _mhe_cost(q, xm, wm)) > 1e-10 * abs(_mhe_cost(q, xm, wm)):
            failed.append("mhe_cost")
        lp = oracle.mhe_to_uftoc(synth.mhe_instance(105, 20, 10, 10, 600))
        lr = oracle.riccati(lp)
        if lr["status"] != 0 or oracle.relres(lp, lr["x"], lr["w"], lr["lam"]) > 1e-13:
            failed.append("long_horizon")
    finally:
        core._lib = saved
    if _golden_fails(lib_mut):
        failed.append("golden")
    return failed


def test_unmutated_oracle_passes_all_pins():
    assert _pins_fail(core.lib()) == []


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmpdir_mod, name):
    assert _pins_fail(_mutant(tmpdir_mod, name)) != []


@pytest.mark.parametrize("name", STEP_CHANGING)
def test_exact_golden_step_alone_catches_step_changing_mistakes(tmpdir_mod, name):
    assert _golden_fails(_mutant(tmpdir_mod, name))


# Planted mistakes in the U_1 form of the reduction (Eq. Bh_def), made in a
# wrapper around the oracle's reduce_u1: each must fail the U_1 tree pin.
U1_MUTATIONS = {
    # B^ = S U_1 (Qbar^{-1} dropped)
    "u1_drop_qbar_in_Bhat": lambda d: dict(d, Bhat=d["S"] @ d["U1"]),
    # Q^_w = I (U_1 taken as Qbar^{-1}-orthonormal)
    "u1_Qw_identity": lambda d: dict(d, Qw=np.eye(d["Qw"].shape[0])),
    # wbar = U_1 w^ (Qbar^{-1} dropped in the chunk's inputs)
    "u1_wbar_without_qbar": lambda d: dict(d, Qbar_inv=np.eye(d["Qbar_inv"].shape[0])),
    # Q^_w = 2 U_1^T Qbar^{-1} U_1 (the reduced input's cost scaled, e.g. a dropped 1/2)
    "u1_Qw_scaled": lambda d: dict(d, Qw=2.0 * d["Qw"]),
}


def _u1_pins_fail():
    from oracle import tree
    u = oracle.mhe_to_uftoc(synth.mhe_instance(7, 6, 1, 1, 40))
    r = oracle.riccati(u)
    t = tree.tree_solve(u, 2, 2, 2, "backsub", form="U1")
    return rel(t["x"], r["x"]) > 1e-9 or rel(np.concatenate(t["w"]), r["w"]) > 1e-9 or rel(t["lam"], r["lam"]) > 1e-9


def test_unmutated_u1_form_passes():
    assert not _u1_pins_fail()


@pytest.mark.parametrize("name", sorted(U1_MUTATIONS))
def test_planted_u1_mistake_is_caught(monkeypatch, name):
    from oracle import tree
    good = tree.reduce_u1
    monkeypatch.setattr(tree, "reduce_u1", lambda *a: U1_MUTATIONS[name](good(*a)))
    assert _u1_pins_fail()
