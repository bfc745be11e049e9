"""The compensated FP32 density accumulator of the mixed path
(DensAcc<float>, roks_impl.cuh) on the CPU, compiled for the host by
tests/cpp/dens_acc.cu: positive terms of mixed magnitude (|psi|^2
contributions of many bands to one grid point) summed term by term with
Knuth's two-sum, and in eight groups merged in order (the band-group slots),
against the FP64 sum.

Bars: up to 1e5 terms, the (hi, lo) pair is within 1e-9 of the FP64 sum. That
is below a thousandth of the plain FP32 sum's error whenever that error is
nonzero; one grid point of mgo-120 sums 430 bands. At 1e6 terms it is within
1e-7, where the plain sum is off by about 1e-3. The FP32 value hi + lo is the
FP64 sum rounded to within one unit in the last place."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_compensated_density_sums(tmp_path):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = tmp_path / "dens_acc"
    src = os.path.join(ROOT, "tests", "cpp", "dens_acc.cu")
    csrc = os.path.join(ROOT, "paper_2605_28637_gb300", "csrc")
    inc = os.path.join(ROOT, "include")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a", "-I", csrc, "-I", inc,
                    src, "-o", str(exe)], check=True, capture_output=True, timeout=600)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=300).stdout
    seen = set()
    for line in out.strip().splitlines():
        n, err_pair, err_plain, ulp_ok = line.split()
        n, err_pair, err_plain = int(n), float(err_pair), float(err_plain)
        seen.add(n)
        assert int(ulp_ok) == 1, line
        if n <= 100000:
            assert err_pair < 1e-9, line
            if err_plain > 0.0:
                assert err_pair < 1e-3 * err_plain, line
        else:
            assert err_pair < 1e-7 and err_plain > 1e-4, line
    assert seen == {10, 1000, 100000, 1000000}
