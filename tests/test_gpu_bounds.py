"""The bounds-checked debug build (libmhe_bounds.so, MHE_BOUNDS_CHECK): the tree
passes check every chunk descriptor and caller-stage index against the extents
of its arrays and report MHE_E_BOUNDS instead of making the access.  On valid
plans no check may fire: the GPU parity, estimate, rank-revealing, literal
Algorithm 6, team-width and golden suites run again in a child process against
the bounds-checked library (every test there asserts status 0 per instance)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SUITES = ["test_gpu_parity.py", "test_gpu_estimate.py", "test_gpu_rank_revealing.py", "test_gpu_literal_alg6.py",
          "test_gpu_team.py", "test_golden.py", "test_gpu_fp64_masters.py"]


def test_suites_pass_against_the_bounds_checked_build():
    sys.path.insert(0, ROOT)
    from paper_1510_03110_gb300 import build
    lib = build.build(bounds_check=True)
    assert lib.endswith("libmhe_bounds.so") and os.path.exists(lib)
    env = dict(os.environ, MHE_BOUNDS_CHECK="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
                        *[os.path.join(HERE, s) for s in SUITES]],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    tail = "\n".join((r.stdout + r.stderr).splitlines()[-15:])
    assert r.returncode == 0, tail
    assert " passed" in tail


def test_binding_loads_the_bounds_checked_library():
    env = dict(os.environ, MHE_BOUNDS_CHECK="1")
    code = "from paper_1510_03110_gb300 import mhe; print(mhe.LIB_PATH); mhe.lib(); print(mhe.shapes()[0])"
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.splitlines()[0].endswith("libmhe_bounds.so")
