"""Measure the GPU's FP64 and FP32 FMA peaks with probes/alu_peaks.cu.

    python -m paper_1510_03110_gb300.peaks        # prints one JSON line

The ALU rooflines of bench.py use the FP64 and FP32 FMA rates; this probe
checks them against the part (build-time nvcc, one GPU)."""
import os
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))


def main() -> int:
    from .build import ARCH, nvcc
    src = os.path.join(HERE, "probes", "alu_peaks.cu")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "alu_peaks")
        subprocess.run([nvcc(), "-O3", *ARCH, "-o", exe, src], check=True)
        r = subprocess.run([exe], capture_output=True, text=True)
        sys.stdout.write(r.stdout)
        sys.stderr.write(r.stderr)
        return r.returncode


if __name__ == "__main__":
    raise SystemExit(main())
