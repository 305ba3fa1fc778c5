"""Planted mistakes in the RTS smoother oracle (oracle/rts.py, the Section VI
comparison and the independent pin of the MHE -> UFTOC transform with S = 0):
a copy of the module with one plausible slip must disagree with the Riccati
oracle's MHE solution on at least one of the shapes the pin runs."""
import importlib.util
import os
import tempfile

import numpy as np
import pytest

import oracle
from oracle import rts
from paper_1510_03110_gb300 import synth

RTS_MUTATIONS = {
    # the process noise left out of the predicted covariance
    "drop_process_noise": ("Pp[k + 1] = A @ Pf[k] @ A.T + B @ Winv @ B.T", "Pp[k + 1] = A @ Pf[k] @ A.T"),
    # the measurement weight used as the noise covariance (V for V^{-1})
    "measurement_weight_for_covariance": ("S = C @ Pp[k] @ C.T + np.linalg.inv(V)", "S = C @ Pp[k] @ C.T + V"),
    # the smoother gain with A instead of A^T
    "smoother_gain_transposed": ("J = Pf[k] @ A.T @ Ppi", "J = Pf[k] @ A @ Ppi"),
    # the noise estimate without its prior mean
    "noise_prior_mean_dropped": ('ws[k] = p["wt"][k] + np.linalg.inv(W) @ B.T @ Ppi @ d',
                                 "ws[k] = np.linalg.inv(W) @ B.T @ Ppi @ d"),
}

SHAPES = [(4, 2, 2, 20), (3, 3, 1, 9), (1, 1, 1, 6)]


def _mutant(name, tmp):
    src = open(rts.__file__).read()
    old, new = RTS_MUTATIONS[name]
    assert src.count(old) == 1, name
    path = os.path.join(tmp, f"rts_{name}.py")
    open(path, "w").write(src.replace(old, new))
    spec = importlib.util.spec_from_file_location(f"rts_{name}", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _agrees(mod):
    """The pin of tests/test_oracle.py: the smoothed means equal the MHE solution."""
    for n, m, q, N in SHAPES:
        p = synth.mhe_instance(11 + n, n, m, q, N, s_zero=True)
        u = oracle.mhe_to_uftoc(p)
        r = oracle.riccati(u)
        try:
            xs, ws = mod.smooth(p)
        except np.linalg.LinAlgError:   # a slip that makes a covariance singular fails the pin too
            return False
        wsol = oracle.split_solution(u, r["w"])
        ex = np.abs(r["x"][1:] - xs).max() / np.abs(xs).max()
        ew = np.abs(np.array(wsol[1:]) - ws).max() / np.abs(ws).max()
        if not (ex < 1e-9 and ew < 1e-9):
            return False
    return True


def test_the_unmutated_smoother_agrees():
    assert _agrees(rts)


@pytest.mark.parametrize("name", sorted(RTS_MUTATIONS))
def test_planted_rts_mistake_is_caught(name):
    with tempfile.TemporaryDirectory() as tmp:
        assert not _agrees(_mutant(name, tmp)), name
