"""The transform arithmetic of the CUDA path on the CPU: tests/cpp/fft_passes.cu
compiles the pass sequence of fft_core.cuh (radix plan, register codelets,
twiddles, Stockham index map) as host code and compares every compiled grid
length (16, 24, 32, 48, 72, 96, 120), in both directions, with the DFT sum
written out in extended precision.  FP64 bar: 1e-14 relative to the largest
output (the measured errors are near 3e-16).

The sphere-pruned first pass (inputs known to be zero left out, for the
frequencies |i| <= (N - 1) / 4) against the same sums at the same bar, with
every dropped input checked to lie outside that range and the number of
dropped inputs of the 120-, 96- and 72-point plans fixed (7 of 15, 6 of 12,
3 of 9).  Every pruned codelet (radix 2, 3, 4, 5, 8) for every mask it
accepts equals the plain codelet on inputs with zeros at the mask, exactly:
it only leaves out additions of zeros."""
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
    seen, pruned, codelets = set(), {}, {}
    for line in out.strip().splitlines():
        f = line.split()
        if f[0] == "prune":
            n, d, err, nz, ok = int(f[1]), int(f[2]), float(f[3]), int(f[4]), int(f[5])
            assert err < 1e-14 and ok == 1, line
            pruned[(n, d)] = nz
        elif f[0] == "codelet":
            r, d, err, count = int(f[1]), int(f[2]), float(f[3]), int(f[4])
            assert err == 0.0, line
            codelets[(r, d)] = count
        else:
            n, d, err = f
            seen.add((int(n), int(d)))
            assert float(err) < 1e-14, line
    lengths = (16, 24, 32, 48, 72, 96, 120)
    assert seen == {(n, d) for n in lengths for d in (-1, 1)}
    assert set(pruned) == seen
    assert all(pruned[(n, d)] > 0 for n, d in pruned)
    assert (pruned[(120, 1)], pruned[(96, 1)], pruned[(72, 1)]) == (7, 6, 3)
    assert codelets == {(r, d): c for r, c in ((2, 2), (3, 4), (4, 8), (5, 16), (8, 64)) for d in (-1, 1)}


def test_full_size_workloads_take_the_pruned_first_pass():
    """The pruned first pass applies to spheres with nmax <= (N - 1) / 4 (the
    density fits the grid without aliasing).  The full-size workloads are such
    spheres, so the benchmark runs the pruned instances; tiny-16 (nmax 6 on a
    16-point grid) is not, and its parity cases run the full first pass."""
    import math

    from paper_2605_28637_gb300 import synthetic as syn

    def nmax(cfg):
        m = math.floor(2.0 * cfg["ecut"] * (cfg["L"] / (2.0 * math.pi)) ** 2)
        return math.isqrt(m)

    for name in ("organic-96", "mgo-120", "hybrid-72", "mgo-72", "mgo-32"):
        cfg = syn.make_config(name, 0)
        assert nmax(cfg) <= (cfg["grid"] - 1) // 4, name
    tiny = syn.make_config("tiny-16", 0)
    assert nmax(tiny) > (tiny["grid"] - 1) // 4
