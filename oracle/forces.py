"""Plain FP64 CPU oracle of the ROKS forces (Sec. II B, the force equations).

TEST INFRASTRUCTURE, like the rest of this package: only tests/,
__graft_entry__.smoke() and bench.py's CPU-baseline leg may import it.  It
shares no code with the CUDA path.

The derivative of E_S with respect to the position R_I of atom I follows
from the generalised Hellmann-Feynman theorem at stationary orbitals:

  dE/dR_Inu = sum_{L sigma n} c_L f_n^{sigma L} <n|dH^{sigma L}/dR_Inu|n>
              - sum_{m,n occ} gamma_mn <m|dS/dR_Inu|n>,       F_Inu = -dE/dR_Inu.

In the model Hamiltonian only the local wells and the projectors depend on
the atoms; Hartree, exchange and exact exchange depend on them through the
density alone.  With w_n = sum_{L sigma} c_L f_n^{sigma L} and rho_w =
sum_n w_n |psi_n|^2:

  local       Omega sum_G (-i G_nu) v_I(G) e^{-iG.R_I} conj(rho_w(G))
              (grid G, Nyquist planes excluded as in the local potential)
  non-local   sum_n w_n <n| dP D P^H + P D dP^H |n>
  overlap     - sum_mn gamma_mn <m| dP Q P^H + P Q dP^H |n>

with dP_i(G) = -i G_nu p_i(G) for the projectors of atom I (zero for the
others).  gamma is the multiplier matrix of the constraint <m|S|n> = delta_mn
(Eq. 11): gamma_nm = (theta_mn + theta_nm^*)/2, theta_mn = <m|F^n|n>.

The paper evaluates the overlap term in the basis that diagonalises gamma;
here it is the double sum as written, which is the same number up to
rounding (a diagonalisation changes how the sum is formed, not its value).

Pins (tests/test_oracle_forces.py): at fixed orbitals and fixed gamma the
expression is the derivative of L(R) = E(Psi; R) - sum gamma_mn (<m|S(R)|n>
- delta_mn), checked by central differences for every term and both the
singlet and the ground state; at converged closed-shell orbitals it is the
total derivative of the minimised energy, checked by re-minimising at
displaced positions.
"""
from __future__ import annotations

import numpy as np

from . import roks as R


def gamma_matrix(Psi, FPsi) -> np.ndarray:
    """gamma_mn, row m, column n, of the constraint sum (Eq. 11)."""
    Theta = Psi.conj().T @ FPsi
    Gam = 0.5 * (Theta + Theta.conj().T)     # Gam_mn = gamma_nm
    return Gam.T.copy()


def projector_owner(sys_: R.System) -> np.ndarray:
    """Atom index of every projector column, in the order of sys_.P."""
    own = []
    for a, at in enumerate(sys_.cfg["atoms"]):
        own += [a] * len(sys_.cfg["species"][at["species"]]["l"])
    return np.array(own, dtype=int)


def well_fourier(sys_: R.System, a: int) -> np.ndarray:
    """v_a(G) e^{-iG.R_a} of one Gaussian well on the grid, Nyquist planes zero."""
    at = sys_.cfg["atoms"][a]
    d, w = at["depth"], at["width"]
    Ra = np.asarray(at["pos"], dtype=np.float64)
    ph = [np.exp(-1j * sys_.gx * Ra[c]) for c in range(3)]
    sf = (ph[0][:, None, None] * ph[1][None, :, None] * ph[2][None, None, :]).reshape(-1)
    v = -(d * (R.TWO_PI * w * w) ** 1.5 / sys_.omega) * np.exp(-0.5 * sys_.G2grid * w * w) * sf
    v[sys_.nyq] = 0.0
    return v


def energy_gradient(sys_: R.System, Psi, gamma=None) -> np.ndarray:
    """dE/dR_Inu (natoms x 3) by the Hellmann-Feynman expression above; gamma
    defaults to that of Psi.  Only the occupied bands enter (empty bands, the
    columns after them, carry no occupation)."""
    Psi = Psi[:, :sys_.n_occ]
    pot = sys_.potentials(sys_.class_densities(Psi))
    if gamma is None:
        FPsi, _ = sys_.apply(Psi, pot)
        gamma = gamma_matrix(Psi, FPsi)
    wn = sys_.w[sys_.cls[:sys_.n_occ]]
    rho_w = (sys_.w[:, None] * pot.rho_k).sum(axis=0)
    rG = sys_.grid_fourier(rho_w)
    N = sys_.N
    gvec = [np.broadcast_to(sys_.gx[:, None, None], (N, N, N)).reshape(-1),
            np.broadcast_to(sys_.gx[None, :, None], (N, N, N)).reshape(-1),
            np.broadcast_to(sys_.gx[None, None, :], (N, N, N)).reshape(-1)]
    own = projector_owner(sys_)
    natoms = len(sys_.cfg["atoms"])
    dE = np.zeros((natoms, 3))
    for a in range(natoms):
        va = well_fourier(sys_, a)
        cols = np.where(own == a)[0]
        for nu in range(3):
            loc = sys_.omega * np.sum(-1j * gvec[nu] * va * np.conj(rG))
            dE[a, nu] = loc.real
            if len(cols) == 0:
                continue
            # <p_i|n> and <dp_i|n> for the projectors of atom a (the others do
            # not move); D and Q are block diagonal, so their block suffices
            Pa = sys_.P[:, cols]
            dPa = -1j * sys_.G[:, nu][:, None] * Pa
            Ba = Pa.conj().T @ Psi
            dBa = dPa.conj().T @ Psi
            Da = sys_.D[np.ix_(cols, cols)]
            Qa = sys_.Q[np.ix_(cols, cols)]
            # <n|dV_nl|n> = <n|dP D P^H + P D dP^H|n>
            nl = sum(wn[n] * (np.vdot(dBa[:, n], Da @ Ba[:, n]) + np.vdot(Ba[:, n], Da @ dBa[:, n]))
                     for n in range(sys_.n_occ))
            # C_mn = <m|dP Q P^H + P Q dP^H|n>
            C = dBa.conj().T @ Qa @ Ba + Ba.conj().T @ Qa @ dBa
            ov = np.sum(gamma * C)
            dE[a, nu] += nl.real - ov.real
    return dE


def forces(sys_: R.System, Psi) -> np.ndarray:
    """F_Inu = -dE/dR_Inu (Ha/Bohr)."""
    return -energy_gradient(sys_, Psi)
