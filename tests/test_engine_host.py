"""The solver engine's orchestration on the CPU (tests/host/engine_orchestration.cpp):
engine.cpp and plan.cpp built with the system C++ compiler against a runtime
table of host memory and a kernel table that records launches.  It checks the
order and data flow of Algorithm 5 (reduce level 0 up, each level reading the
master data the level below wrote), Algorithm 6 (down pass top level first,
each level reading the solution of the level above) and of the refinement
loop, the MHE-form entry and a re-planned serving context, plus the host-side
errors.  Planted mistakes in a copy of engine.cpp must each make it fail."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1510_03110_gb300", "csrc")
HARNESS = os.path.join(ROOT, "tests", "host", "engine_orchestration.cpp")
ENGINE = open(os.path.join(CSRC, "engine.cpp")).read()

MUTATIONS = {
    # Algorithm 6 run bottom-up instead of top level first
    "down_pass_bottom_up": ("for (int k = (int)lv.size() - 1; k >= 0; --k) {\n        if (m64 && k >= 1) {\n"
                            "            down_level",
                            "for (int k = 0; k < (int)lv.size(); ++k) {\n        if (m64 && k >= 1) {\n"
                            "            down_level"),
    # a level reads the wrong part of its parent's solution
    "parent_w_for_x": ("a.xd_up = static_cast<const T*>(st ? U.xd32 : U.xd);",
                       "a.xd_up = static_cast<const T*>(st ? U.xd32 : U.wd);"),
    # a level reads its own master data instead of the data the level below wrote
    "master_data_not_chained": ("a.Ah_up = static_cast<T*>(st ? U.Ah32 : U.Ah);", "a.Ah_up = static_cast<T*>(L.Pst);"),
    # FP64 master levels: level 1 reads its FP32 master data without the widening
    "fp64_masters_not_widened": ("        wid(U.Bh, U.Bh32, ns * n * n);\n", ""),
    # FP64 master levels: level 0's down pass reads a stale FP32 copy of level 1's solution
    "fp64_masters_not_narrowed": ("            if (k == 1) narrow_solution();\n", ""),
    # FP64 master levels: the corrections' top chunks read the first solve's x~0
    "fp64_masters_correction_x0": ("            x0_hi = rx0_64;\n", ""),
    # the master-problem variant not selected at level 1
    "upper_from_level_2": ("launch<T>(ops->reduce64, r32, g, k >= 1, stream);",
                           "launch<T>(ops->reduce64, r32, g, k >= 2, stream);"),
    # corrections read in the caller's layout instead of the compact one
    "corrections_in_input_layout": ("        rhs_compact = true;\n        pass_rhs<T>(crl, cra, crl0, cra0, crlN);",
                                    "        rhs_compact = false;\n        pass_rhs<T>(crl, cra, crl0, cra0, crlN);"),
    # the MHE-form estimate's residual loses its factors C, R (would read the unformed Q)
    "estimate_residual_without_C": ("    mheC = p.C; mheR = p.R;", "    mheC = nullptr; mheR = p.R;"),
    # a re-planned serving batch ignores the resident stage offsets
    "replan_drops_offsets": ("    if (in_off_custom) p.in_off.assign(in_off_custom, in_off_custom + batch);\n", ""),
    # the corrections lose the active mask
    "refinement_without_mask": ("        active_mask = active;\n        rhs_compact = true;",
                                "        active_mask = nullptr;\n        rhs_compact = true;"),
}


def _build_and_run(tmp, engine_src):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    eng = os.path.join(tmp, "engine.cpp")
    with open(eng, "w") as f:
        f.write(engine_src)
    exe = os.path.join(tmp, "eo")
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, HARNESS, eng, os.path.join(CSRC, "plan.cpp"), "-o", exe],
                   check=True, capture_output=True, text=True)
    return subprocess.run([exe], capture_output=True, text=True, timeout=60)


def test_engine_orchestration():
    with tempfile.TemporaryDirectory() as tmp:
        r = _build_and_run(tmp, ENGINE)
    assert r.returncode == 0 and r.stdout.strip() == "OK", r.stdout + r.stderr


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_orchestration_mistake_is_caught(name):
    old, new = MUTATIONS[name]
    assert ENGINE.count(old) == 1, name
    with tempfile.TemporaryDirectory() as tmp:
        r = _build_and_run(tmp, ENGINE.replace(old, new))
    assert r.returncode == 1 and "FAIL" in r.stdout, (name, r.stdout)
