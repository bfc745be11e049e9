"""The DIIS window test and coefficient solve of the CUDA path
(diis_window_coefficients, compiled for the host from roks_diis.cuh by
tests/cpp/diis_window.cu) against the DIIS oracle's window() and
coefficients() on Gram matrices of random error vectors: shrinking norms as
in a converging run, a newest vector nearly in the span of older ones, a
repeated vector, and a one-pair history.  The window must match exactly; the
coefficients to 1e-8 relative to the largest (the oracle solves Pulay's
bordered system, the CUDA path a Cholesky solve of the normalised Gram matrix:
two routes to the same minimiser)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import diis as D

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def cases():
    rng = np.random.default_rng(11)
    out = []
    for n in range(1, 9):
        E = rng.standard_normal((60, n)) * np.logspace(0, -4, n)[None, :]
        out.append(E)
    v = rng.standard_normal((60, 5))
    dep = v.copy()
    dep[:, 4] = v[:, 0] - 0.3 * v[:, 2] + 1e-9 * rng.standard_normal(60)   # newest in the span of older
    out.append(dep)
    rep = rng.standard_normal((60, 4))
    rep[:, 3] = rep[:, 1]                                                   # a repeated vector
    out.append(rep)
    near = rng.standard_normal((60, 6))
    near[:, 5] = near[:, 4] + 1e-2 * rng.standard_normal(60)                # close but well conditioned
    out.append(near)
    return [E.T @ E for E in out]


def test_window_and_coefficients_match_the_oracle(tmp_path):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = tmp_path / "diis_window"
    subprocess.run([nvcc, "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-I", os.path.join(ROOT, "paper_2605_28637_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "cpp", "diis_window.cu"), "-o", str(exe)],
                   check=True, capture_output=True, timeout=600)
    Bs = cases()
    text = [str(len(Bs))]
    for B in Bs:
        text.append(f"{B.shape[0]} {D.COND_TOL!r}")
        text += [" ".join(repr(float(x)) for x in row) for row in B]
    out = subprocess.run([str(exe)], input="\n".join(text) + "\n", check=True, capture_output=True, text=True,
                         timeout=120).stdout.strip().splitlines()
    assert len(out) == len(Bs)
    windows = []
    for B, line in zip(Bs, out):
        vals = line.split()
        h = int(vals[0])
        d = np.array([float(x) for x in vals[1:]])
        n = B.shape[0]
        h_ref = D.window(B, D.COND_TOL)
        assert h == h_ref, (n, h, h_ref)
        d_ref = D.coefficients(B[n - h:, n - h:])
        assert np.abs(d - d_ref).max() <= 1e-8 * max(1.0, np.abs(d_ref).max()), (d, d_ref)
        windows.append(h)
    # the constructed cases exercise both outcomes of the window test
    assert windows[8] < 5 and windows[9] < 4 and windows[10] == 6 and windows[7] == 8
