"""Pins of the oracle's Fourier transforms against the DFT definition."""
import numpy as np
import pytest

from oracle import fft as F


@pytest.mark.parametrize("n", list(range(1, 17)) + [18, 20, 24, 25, 27, 30, 36, 45])
@pytest.mark.parametrize("sign", [-1, +1])
def test_fft_matches_definition(n, sign):
    rng = np.random.default_rng(n)
    x = rng.standard_normal((3, n)) + 1j * rng.standard_normal((3, n))
    ref = np.array([[sum(x[b, j] * np.exp(sign * 2j * np.pi * j * k / n) for j in range(n))
                     for k in range(n)] for b in range(3)])
    assert np.allclose(F.fft(x, sign), ref, atol=1e-12 * n, rtol=0)
    assert np.allclose(F.dft(x, sign), ref, atol=1e-12 * n, rtol=0)


@pytest.mark.parametrize("n", [4, 5, 6, 8, 9, 10, 12])
def test_fft3_brute_force(n):
    rng = np.random.default_rng(100 + n)
    x = rng.standard_normal((n, n, n)) + 1j * rng.standard_normal((n, n, n))
    idx = np.arange(n)
    W = np.exp(-2j * np.pi * np.outer(idx, idx) / n)
    W3 = np.kron(np.kron(W, W), W)               # acts on the C-order flattened grid
    ref = (W3 @ x.reshape(-1)).reshape(n, n, n)
    assert np.allclose(F.fft3(x, -1), ref, atol=1e-11 * n ** 3, rtol=0)


@pytest.mark.parametrize("n", [16, 24, 30])
def test_parseval_and_roundtrip(n):
    rng = np.random.default_rng(7)
    x = rng.standard_normal((n, n, n)) + 1j * rng.standard_normal((n, n, n))
    X = F.fft3(x, -1)
    assert np.isclose((np.abs(X) ** 2).sum(), n ** 3 * (np.abs(x) ** 2).sum(), rtol=1e-12)
    back = F.fft3(X, +1) / n ** 3
    assert np.allclose(back, x, atol=1e-12, rtol=0)


def test_single_mode_is_plane_wave():
    n = 12
    x = np.zeros((n, n, n), complex)
    x[2, 11, 5] = 1.0
    y = F.fft3(x, +1)
    a, b, c = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ref = np.exp(2j * np.pi * (2 * a + 11 * b + 5 * c) / n)
    assert np.allclose(y, ref, atol=1e-12)
