"""Plain FP64 CPU oracle of the Gamma-point real-orbital representation
(the half sphere of plane waves).

TEST INFRASTRUCTURE, like the rest of this package: only tests/,
__graft_entry__.smoke() and bench.py's CPU-baseline leg may import it.

At the Gamma point (the only k-point the paper samples, Sec. III) the
orbitals can be chosen real in real space.  Their coefficients then satisfy
c(-G) = conj(c(G)) and c(0) real, so half of the sphere carries all of
them: the kept set is G = 0 and every G whose Miller triple (i, j, k) is
lexicographically positive, in the order of the full basis.  Plain
definitions:

* expand: c_full(G) = c(G), c_full(-G) = conj(c(G)) for kept G;
* restrict: the kept rows of a full coefficient vector;
* overlap of two real orbitals: sum over the full sphere of conj(a) b
  = 2 Re sum_half conj(a) b - a(0) b(0)  (a real number);
* seeded start: c(G) = (u_re + i u_im) / (1 + |G|^2) on the half sphere,
  c(0) = its real part, expanded and S-orthonormalised by the full oracle.

Every step of the method maps real orbitals to real orbitals here (real
potentials, projectors real in real space, a real symmetric overlap and
real multipliers), so the full-sphere oracle run from a symmetric start IS
the Gamma-point method: the pins (tests/test_oracle_gamma.py) check the
counts, the maps, the overlap identity and that PCG keeps the symmetry.
"""
from __future__ import annotations

import numpy as np

from . import roks as R


def half_index(sys_: R.System) -> np.ndarray:
    """Rows of the full basis kept in the half sphere (G = 0 and (i, j, k) > 0)."""
    m = sys_.miller
    pos = (m[:, 0] > 0) | ((m[:, 0] == 0) & ((m[:, 1] > 0) | ((m[:, 1] == 0) & (m[:, 2] >= 0))))
    return np.where(pos)[0]


def partner_index(sys_: R.System) -> np.ndarray:
    """For every full row g, the row of -G."""
    lookup = {tuple(v): i for i, v in enumerate(sys_.miller)}
    return np.array([lookup[tuple(-v)] for v in sys_.miller])


def expand(sys_: R.System, C_half: np.ndarray) -> np.ndarray:
    """Full coefficients of real orbitals from their half-sphere coefficients."""
    h = half_index(sys_)
    p = partner_index(sys_)
    C = np.zeros((sys_.npw,) + C_half.shape[1:], dtype=np.complex128)
    C[h] = C_half
    C[p[h]] = np.conj(C_half)
    return C


def restrict(sys_: R.System, C_full: np.ndarray) -> np.ndarray:
    return C_full[half_index(sys_)].copy()


def overlap_half(sys_: R.System, A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """A^H B over the full sphere from the half-sphere coefficients of real orbitals."""
    h = half_index(sys_)
    g0 = int(np.where(np.all(sys_.miller[h] == 0, axis=1))[0][0])
    return 2.0 * np.real(A.conj().T @ B) - np.outer(A[g0].real, B[g0].real)


def initial_orbitals(sys_: R.System, u_half: np.ndarray) -> np.ndarray:
    """Seeded real orbitals (full coefficients): u_half is nbands x npw_half x 2."""
    h = half_index(sys_)
    c = (u_half[..., 0] + 1j * u_half[..., 1]).T / (1.0 + sys_.g2[h])[:, None]
    g0 = int(np.where(np.all(sys_.miller[h] == 0, axis=1))[0][0])
    c[g0] = c[g0].real
    return sys_.orthonormalize(expand(sys_, c))


def realness(sys_: R.System, C_full: np.ndarray) -> float:
    """Largest |Im psi_n(r)| relative to the largest |psi_n(r)| over the bands."""
    worst = 0.0
    for n in range(C_full.shape[1]):
        psi = sys_.to_real(C_full[:, n])
        worst = max(worst, float(np.abs(psi.imag).max() / max(np.abs(psi).max(), 1e-300)))
    return worst
