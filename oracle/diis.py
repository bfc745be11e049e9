"""Plain FP64 CPU oracle of the DIIS solver for the ROKS functional.

TEST INFRASTRUCTURE, like the rest of this package: only tests/,
__graft_entry__.smoke() and bench.py's CPU-baseline leg may import it.  It
shares no code with the CUDA path.

The paper minimises E_S with PCG and also with a DIIS solver (Sec. II A,
the residual of Frank et al. with coupling coefficients lambda), whose
details it leaves to Hutter, Luthi and Parrinello (1994).  Steps, in order:

* residual  R_n = F^n|n> - sum_m S|m> Lambda_mn,
            Lambda_mn = theta_mn - lambda_mn (theta_mn - theta_nm^*),
            theta_mn = <m|F^n|n>                               (Sec. II A)
* error vector  e = tau K R, K the TPA preconditioner (Eqs. 17, 18 with R1)
  applied to the whole residual: the paper's DIIS uses K alone, without the
  out-of-subspace split of the PCG path
* DIIS: keep the last m pairs (Psi_j, e_j); B_jk = sum_n Re<e_jn|e_kn>;
  real coefficients d minimising |sum_j d_j e_j|^2 with sum_j d_j = 1
  (the bordered linear system of Pulay's method);
  Psi' = orth(sum_j d_j (Psi_j + e_j))   (Cholesky S-orthonormalisation, R6)

Readings where the paper is silent or garbled (each also applied by the CUDA
path, which implements them independently):
  R8   sign of lambda: the printed bracket theta_mn + lambda (theta_mn -
       theta_nm^*) is read with a minus, so that lambda = 1/2 for every pair
       turns Lambda into gamma of Eq. 11 and R into the gradient g of Eq. 7,
       which is what the text states for lambda = 1/2.
  R9   lambda_ab is the coefficient of the component along |a> in the
       residual of band b; lambda_ba that along |b> in the residual of a.
       Every other pair takes 1/2 (within a shell the bracket vanishes).
  R10  coefficients are real and shared by all bands; e = tau K R with
       tau = 1/2 by default; history m = 6 by default.
  R11  conditioning: with D = diag(B) over the h most recent pairs and
       Bn = D^-1/2 B D^-1/2, the window is accepted when every Cholesky
       pivot of Bn satisfies L_kk^2 >= tol (1e-7); otherwise the oldest
       pair is dropped and the test repeated (h = 1 always passes).
  R12  convergence as R7: |E_i+1 - E_i| < e_tol on two consecutive steps,
       and the residual norm |R| < g_tol at the start of the last step when
       g_tol > 0.

Pins (tests/test_oracle_diis.py): lambda = 1/2 reproduces the gradient of
Eq. 7 (itself pinned by finite differences of E); the in-subspace part of R
and its out-of-subspace part against the split of Eq. 12; the coefficients
against a brute-force constrained least-squares solve; a one-pair window
against preconditioned steepest descent written out; the converged closed
shell against the dense generalised eigenproblem; the converged singlet
against the stationarity conditions and the PCG energy.
"""
from __future__ import annotations

from collections import deque
from dataclasses import dataclass

import numpy as np

from . import roks as R

TAU = 0.5
HISTORY = 6
COND_TOL = 1e-7


def coupling_table(sys_: R.System, lambda_ab: float = 0.5, lambda_ba: float = 0.5) -> np.ndarray:
    """lambda_mn for every band pair: 1/2, except the open pair (R9)."""
    lam = np.full((sys_.nb, sys_.nb), 0.5)
    if sys_.mode == 1:
        a, b = sys_.n_closed, sys_.n_closed + 1
        lam[a, b] = lambda_ab
        lam[b, a] = lambda_ba
    return lam


def multipliers(Theta: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """Lambda_mn = theta_mn - lambda_mn (theta_mn - theta_nm^*) (R8)."""
    return Theta - lam * (Theta - Theta.conj().T)


def residual(Psi, FPsi, SPsi, lam):
    """theta = Psi^H F Psi, Lambda and R = F Psi - S Psi Lambda."""
    Theta = Psi.conj().T @ FPsi
    Lam = multipliers(Theta, lam)
    return Theta, Lam, FPsi - SPsi @ Lam


def error_vector(sys_: R.System, Rres, tau: float = TAU):
    """e = tau K R, K the TPA factor with X from the residual itself (R1, R10)."""
    KR, _ = R.tpa_step(sys_, Rres)
    return tau * KR


def window(B: np.ndarray, tol: float = COND_TOL) -> int:
    """Largest h such that the h most recent pairs pass the pivot test (R11)."""
    n = B.shape[0]
    for h in range(n, 0, -1):
        Bh = B[n - h:, n - h:]
        dsq = np.sqrt(np.diag(Bh))
        Bn = Bh / np.outer(dsq, dsq)
        try:
            Lc = np.linalg.cholesky(Bn)
        except np.linalg.LinAlgError:
            continue
        if np.min(np.diag(Lc) ** 2) >= tol:
            return h
    return 1


def coefficients(B: np.ndarray) -> np.ndarray:
    """Pulay's bordered system [B 1; 1^T 0] [d; mu] = [0; 1]."""
    h = B.shape[0]
    M = np.zeros((h + 1, h + 1))
    M[:h, :h] = B
    M[:h, h] = 1.0
    M[h, :h] = 1.0
    rhs = np.zeros(h + 1)
    rhs[h] = 1.0
    return np.linalg.solve(M, rhs)[:h]


@dataclass
class DiisInfo:
    E: float
    E_new: float
    res_norm: float
    grad_norm: float
    window: int
    coef: np.ndarray


class DIIS:
    """DIIS on the ROKS residual (Sec. II A, Hutter et al. 1994), steps in
    the order of the module docstring."""

    def __init__(self, sys_: R.System, history: int = HISTORY, tau: float = TAU,
                 lambda_ab: float = 0.5, lambda_ba: float = 0.5, e_tol: float = 1e-6, tol: float = COND_TOL,
                 g_tol: float = 0.0):
        if sys_.n_empty:
            raise ValueError("the DIIS solver takes occupied bands only (no empty shell)")
        self.sys = sys_
        self.tau = tau
        self.tol = tol
        self.e_tol = e_tol
        self.g_tol = g_tol
        self.lam = coupling_table(sys_, lambda_ab, lambda_ba)
        self.hist = deque(maxlen=history)
        self.n_small = 0
        self.converged = False

    def step(self, Psi):
        sy = self.sys
        pot = sy.potentials(sy.class_densities(Psi))
        E0 = sy.energies(Psi, pot)["total"]
        FPsi, SPsi = sy.apply(Psi, pot)
        Theta, _, Rres = residual(Psi, FPsi, SPsi, self.lam)
        G = FPsi - SPsi @ (0.5 * (Theta + Theta.conj().T))
        e = error_vector(sy, Rres, self.tau)
        self.hist.append((Psi, e))
        n = len(self.hist)
        B = np.zeros((n, n))
        for j in range(n):
            for k in range(n):
                B[j, k] = float(np.real(np.vdot(self.hist[j][1], self.hist[k][1])))
        h = window(B, self.tol)
        d = coefficients(B[n - h:, n - h:])
        X = np.zeros_like(Psi)
        for c, (P, ej) in zip(d, list(self.hist)[n - h:]):
            X = X + c * (P + ej)
        Psi_new = sy.orthonormalize(X)
        E_new = sy.energy(Psi_new)
        if abs(E_new - E0) < self.e_tol:
            self.n_small += 1
        else:
            self.n_small = 0
        self.converged = self.n_small >= 2 and (self.g_tol <= 0.0 or float(np.linalg.norm(Rres)) < self.g_tol)
        return Psi_new, DiisInfo(E=E0, E_new=E_new, res_norm=float(np.linalg.norm(Rres)),
                                 grad_norm=float(np.linalg.norm(G)), window=h, coef=d)


def run(sys_: R.System, Psi, max_iter=100, callback=None, **kw):
    """DIIS to convergence (R12) or max_iter; returns (Psi, list of DiisInfo)."""
    dz = DIIS(sys_, **kw)
    hist = []
    for _ in range(max_iter):
        Psi, info = dz.step(Psi)
        hist.append(info)
        if callback is not None:
            callback(info)
        if dz.converged:
            break
    return Psi, hist
