"""The transform arithmetic of the CUDA path on the CPU: tests/cpp/fft_passes.cu
compiles the pass sequence of fft_core.cuh (radix plan, register codelets,
twiddles, Stockham index map) as host code and compares every compiled grid
length (16, 24, 32, 48, 72, 96, 120), in both directions, with the DFT sum
written out in extended precision.  FP64 bar: 1e-14 relative to the largest
output (the measured errors are near 3e-16)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_pass_arithmetic_all_grid_lengths(tmp_path):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = tmp_path / "fft_passes"
    src = os.path.join(ROOT, "tests", "cpp", "fft_passes.cu")
    inc = os.path.join(ROOT, "paper_2605_28637_gb300", "csrc")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a", "-I", inc, src,
                    "-o", str(exe)], check=True, capture_output=True, timeout=600)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=300).stdout
    seen = set()
    for line in out.strip().splitlines():
        n, d, err = line.split()
        seen.add((int(n), int(d)))
        assert float(err) < 1e-14, line
    assert seen == {(n, d) for n in (16, 24, 32, 48, 72, 96, 120) for d in (-1, 1)}
