"""Textbook discrete Fourier transforms for the oracle.

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg may import this package; the product path never does.

The plane-wave method needs 3D transforms between the coefficient grid and
real space (orbitals are expanded in plane waves, Sec. II; grids of 16, 72,
96 and 120 points per side, which are 2^a 3^b 5^c).  Two definitions are
given here:

* `dft`: the sum X[k] = sum_n x[n] exp(sign * 2 pi i n k / N), written out as
  a matrix product (the definition itself);
* `fft`: recursive mixed-radix Cooley-Tukey decimation in time.  N = p*m with
  p the smallest prime factor; X[k] = sum_r W_N^{r k} Y_r[k mod m], where
  Y_r is the length-m transform of x[r::p].  Prime lengths fall back to `dft`.

Both are unnormalised; sign=-1 is the forward transform, sign=+1 the inverse.
"""
from __future__ import annotations

import numpy as np


def smallest_prime_factor(n: int) -> int:
    p = 2
    while p * p <= n:
        if n % p == 0:
            return p
        p += 1
    return n


def dft(x: np.ndarray, sign: int, axis: int = -1) -> np.ndarray:
    """Direct O(N^2) DFT along `axis` (the definition)."""
    x = np.moveaxis(np.asarray(x, dtype=np.complex128), axis, -1)
    n = x.shape[-1]
    idx = np.arange(n)
    W = np.exp(sign * 2j * np.pi * np.outer(idx, idx) / n)
    out = x @ W.T
    return np.moveaxis(out, -1, axis)


def _fft_last(x: np.ndarray, sign: int) -> np.ndarray:
    n = x.shape[-1]
    if n == 1:
        return x.copy()
    p = smallest_prime_factor(n)
    if p == n:
        return dft(x, sign, -1)
    m = n // p
    k = np.arange(n)
    out = np.zeros(x.shape, dtype=np.complex128)
    for r in range(p):
        y = _fft_last(x[..., r::p], sign)
        tw = np.exp(sign * 2j * np.pi * r * k / n)
        out += tw * np.tile(y, p)
    return out


def fft(x: np.ndarray, sign: int, axis: int = -1) -> np.ndarray:
    """Mixed-radix Cooley-Tukey along `axis`; same result as `dft`."""
    x = np.moveaxis(np.asarray(x, dtype=np.complex128), axis, -1)
    return np.moveaxis(_fft_last(x, sign), -1, axis)


def fft3(x: np.ndarray, sign: int) -> np.ndarray:
    """Unnormalised 3D transform over the last three axes."""
    y = fft(x, sign, -1)
    y = fft(y, sign, -2)
    return fft(y, sign, -3)
