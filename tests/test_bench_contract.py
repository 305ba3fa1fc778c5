"""bench.py's command-line contract, the parts that need no GPU: the reference
arm (the oracle timed on the host cores) prints one JSON line with the keys
the line must carry, and under a multi-process launch the ranks other than 0
exit 0 without work or output, for both arms."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(args, env_extra=None, timeout=300):
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=timeout)


def test_reference_arm_prints_one_json_line():
    r = _bench(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference"
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["steps"] == 1 and d["warmup"] == 0
    assert d["higher_is_better"] is True and d["vs_baseline"] is None and d["data"] == "synthetic"
    assert d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_ranks_other_than_zero_exit_without_work():
    env = dict(RANK="1", LOCAL_RANK="1", WORLD_SIZE="2")
    for arm in ("gpu", "reference"):
        r = _bench(["--impl", arm, "--gpus", "2", "--steps", "1", "--warmup", "3"], env, timeout=120)
        assert r.returncode == 0, (arm, r.stderr[-2000:])
        assert r.stdout.strip() == "", (arm, r.stdout)


def _bench_module():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_clock_samples_and_rule():
    """The clock record of the timed region: nvidia-smi rows parsed into the median
    SM clock, the maximum and the active reasons, and the timing rule applied
    (slowdowns and unexplained low clocks reject the run; the power cap is noted)."""
    b = _bench_module()
    c = b.Clocks()

    class Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0
    rows = ["0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "0, 2055, 2070, 1100.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 950.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"]
    c.f.write("\n".join(rows) + "\n")
    c.p = Done()
    clk = c.stop()
    assert clk["samples"] == 3 and clk["sm_mhz"] == 2070.0 and clk["sm_max_mhz"] == 2070.0
    assert clk["reasons"] == ["sw_power_cap"]
    assert b.clocks_check(clk).startswith("ok")
    assert b.clocks_check(dict(clk, reasons=["hw_slowdown"])).startswith("rejected")
    assert b.clocks_check(dict(clk, reasons=["sw_thermal_slowdown", "sw_power_cap"])).startswith("rejected")
    assert b.clocks_check(dict(clk, reasons=[], sm_mhz=1200.0)).startswith("rejected")
    assert b.clocks_check(dict(clk, reasons=["sw_power_cap"], sm_mhz=1700.0)).startswith("ok")
    assert b.clocks_check(None) == "no clock samples"
