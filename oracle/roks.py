"""Plain FP64 CPU oracle for the ROKS plane-wave hot path.

TEST INFRASTRUCTURE: this package exists to check the CUDA path.  Only
tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import
it; the library and its Python binding never do.  It shares no code with the
CUDA path; the only common input is the seeded random numbers.

What it computes, in the paper's order and notation:

* ROKS singlet functional E_S = 2 E(Phi_1) - E(Phi_3)            (Eq. 1)
  minimised over one set of spatial orbitals shared by the mixed-spin (M)
  and triplet (T) configurations, c_M = 2, c_T = -1                (Sec. II A)
* overlap S = 1 + sum |beta> q <beta|                             (Eq. 3)
* configuration/spin Hamiltonians H^{sigma L}                      (Eq. 8)
* shell operators F^n = sum_{sigma L} c_L f_n^{sigma L} H^{sigma L} (Eq. 13)
* Lagrange multipliers gamma                                       (Eq. 11, SI S1)
* gradient, split into out-of-subspace (I) and in-subspace (II)    (Eqs. 7, 12)
* preconditioned gradient with the TPA kinetic preconditioner      (Eqs. 17, 18)
* ROKS R matrix and the Jacobi-like in-subspace rotation           (Eqs. 20-23)
* Fletcher-Reeves CG with the two-step update                      (Eqs. 5, 6, 24)

The model behind the Hamiltonian (not given by the paper, whose PAW data
sets are not available): Gaussian local wells, Gaussian s/p projectors with
fixed D and Q matrices, LSDA Slater exchange, an optional exact-exchange
fraction alpha with a spherically truncated Coulomb kernel.

Readings where the paper is silent or garbled (each is also applied by the
CUDA path, which implements them independently):
  R1  TPA scale X: the constant printed as "10" in Eq. 18 is read as
      X_n = 1.5 * E_kin(g_nI) in Rydberg (kinetic energy of the residual),
      with K carrying the minus sign.
  R2  denominator in Eq. 23: d_m - d_n with d_m = <m| sum_{sigma L} c_L H |m>,
      i.e. the diagonal of the closed-shell operator F^c.
  R3  sign of A (Eq. 22): chosen so that U = exp(A) with |n'> = sum_m U_mn |m>
      diagonalises a 2x2 block exactly; A_mn = -atan(2|x|)/2 * x/|x|.
  R4  the Fletcher-Reeves ratio sums Re<p_n|g_n> over all bands; p_II = Psi A.
  R5  line search: parabola through E(0), E'(0), E(dt); dt starts at 0.3 and
      is then the previous step clamped to [0.05, 2]; curvature <= 0 takes dt;
      the step is capped at 3 dt.  The same step scales the rotation (Eq. 24).
  R6  the search direction is projected S-orthogonal to the current orbitals
      before the step; orbitals are S-orthonormalised by Cholesky in the
      order closed, a, b, empty after each step.
  R7  convergence: |E_i+1 - E_i| < e_tol on two consecutive iterations and,
      when a gradient tolerance g_tol > 0 is given, |g| < g_tol at the start
      of the last step (the stationarity the energy criterion stands for,
      Eq. 15 and SI S1, made explicit).
  R13 the empty shell (Eq. 20, fourth row and column): n_empty unoccupied
      bands follow a, b.  They carry no occupation in any configuration, so
      F^e = 0 in the energy and its gradient: theta_mn = <m|F^e|n> = 0 for an
      empty n in gamma, the full gradient g and the in-subspace gradient, and
      R_mn = <m|F^s|n> between an occupied shell s and the empty shell.  The
      empty-empty block of R is F^c.  The paper leaves the rest open; read
      here: an empty band's own out-of-subspace direction is the
      preconditioned F^c residual (1 - S Psi Psi^H) F^c|e>, so the empty bands
      relax to the lowest eigenvectors of F^c outside the occupied space; it
      moves with the accepted step, while the trial point of the line search
      moves the occupied bands alone (the empty directions add nothing to
      E'(0), and their second order through the rotation would distort the
      parabola); the Fletcher-Reeves ratio (R4) takes the occupied bands.  An
      occupied band m of class k and an empty band rotate by the angle that
      turns m to the lower eigenvector of the pair's 2 x 2 block of F^k,
      (1/2) atan2(2|R|, <e|F^k|e> - <m|F^k|m>): the Jacobi angle of Eq. 22
      when m lies lower, past pi/4 (an exchange) when the empty band does, so
      the occupied bands take the lowest states.  Not combined with exact
      exchange.

What pins each part (tests/test_oracle_*.py; none compares the oracle with
itself): the transforms against the DFT sum and brute force; the basis
against brute-force counts; kinetic, Hartree, Slater exchange, truncated
Coulomb kernel, wells and projectors against closed forms; H against
Hermiticity and the gradient against finite differences of E; E_S = 2 E_M -
E_T term by term; gamma, the gradient split, p_I and the R-matrix rotation
against their defining identities; the line-search slope against finite
differences along the path taken; the converged result against the dense
generalised eigenproblem (closed shell) and the stationarity conditions
(singlet); the Fletcher-Reeves numerator (R4) against central differences
of the energy along a fresh steepest-descent path, and each accepted step
(R5) against the energy along its own path (a local minimum on +-25%, or
still descending where the 3 dt cap applies).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg

from . import fft as _fft

TWO_PI = 2.0 * np.pi

# Occupation table f_k^{sigma L} of the three orbital classes (rows: closed,
# open a, open b) in the four channels (up M, down M, up T, down T).  The
# mixed configuration Phi_1 has a-up, b-down; the triplet Phi_3 has a-up,
# b-up (Fig. 1A; Eq. 7 uses f in {0, 1}).
F_TABLE = np.array([[1.0, 1.0, 1.0, 1.0],
                    [1.0, 0.0, 1.0, 0.0],
                    [0.0, 1.0, 1.0, 0.0]])


def config_coefficients(mode: int) -> np.ndarray:
    """c_L for (M, T).  mode 1: ROKS singlet, c = (2, -1) (Eq. 1 and Eq. 2).
    mode 2: the triplet alone, c = (0, 1).  mode 0: closed-shell ground state
    (no open bands), one configuration with c = 1."""
    return {0: np.array([1.0, 0.0]), 1: np.array([2.0, -1.0]),
            2: np.array([0.0, 1.0])}[mode]


def slater_prefactor() -> float:
    return 0.75 * (6.0 / np.pi) ** (1.0 / 3.0)


# PBE exchange (the GGA of Sec. III; Perdew, Burke and Ernzerhof 1996):
# enhancement factor F_x(s) = 1 + kappa - kappa / (1 + mu s^2 / kappa), with
# mu = beta pi^2 / 3 the gradient-expansion coefficient.
PBE_KAPPA = 0.804
PBE_MU = 0.06672455060314922 * np.pi ** 2 / 3.0
RHO_MIN = 1e-10        # a spin-channel density at or below this carries no exchange


def pbe_enhancement(s2):
    """F_x and dF_x/d(s^2) of PBE exchange at s^2."""
    den = 1.0 + PBE_MU * s2 / PBE_KAPPA
    return 1.0 + PBE_MU * s2 / den, PBE_MU / (den * den)


@dataclass
class Potentials:
    rho_k: np.ndarray          # (3, N^3) class densities closed, a, b
    rho_ch: np.ndarray         # (4, N^3) channel densities
    rho: np.ndarray            # (N^3,) total density
    VH: np.ndarray             # Hartree potential
    vx: np.ndarray             # (4, N^3) exchange potentials per channel
    Vk: np.ndarray             # (3, N^3) class local potentials
    E: dict = field(default_factory=dict)


class System:
    """One model system: cubic cell, Gamma point, plane-wave basis."""

    def __init__(self, cfg: dict, *, hartree: bool = True, xc: bool = True):
        self.cfg = cfg
        self.L = float(cfg["L"])
        self.N = int(cfg["grid"])
        self.ecut = float(cfg["ecut"])
        self.omega = self.L ** 3
        self.alpha = float(cfg.get("alpha", 0.0))
        self.mode = int(cfg["mode"])
        self.n_closed = int(cfg["n_closed"])
        self.n_open = 0 if self.mode == 0 else 2
        self.n_empty = int(cfg.get("n_empty", 0))
        self.n_occ = self.n_closed + self.n_open
        self.nb = self.n_occ + self.n_empty
        if self.n_empty and self.alpha != 0.0:
            raise ValueError("empty bands are not modelled with exact exchange")
        self.hartree = hartree
        self.xc = xc
        # exchange functional: "slater" (LSDA) or "pbe_x" (PBE exchange, the GGA)
        self.xc_kind = str(cfg.get("xc", "slater"))
        if self.xc_kind not in ("slater", "pbe_x"):
            raise ValueError("unknown exchange functional " + self.xc_kind)
        self._occupations()
        self._basis()
        self._grid_vectors()
        self._local_potential()
        self._projectors()

    # ----------------------------------------------------------- a1: occupations
    def _occupations(self):
        """Weights that follow from f_n^{sigma L} and c_L (Eqs. 7, 13)."""
        self.cL = config_coefficients(self.mode)
        c_ch = np.repeat(self.cL, 2)                 # c_L per channel
        self.C = F_TABLE * c_ch[None, :]              # c_L f_k^{sigma L}
        self.w = self.C.sum(axis=1)                   # weight of T, V_ext, V_H in F^k
        self.WX = (F_TABLE * c_ch) @ F_TABLE.T        # sum c_L f_k f_k' (exchange pairs)
        # class of the operator applied to each band: closed 0, open a 1 and
        # b 2; an empty band takes F^c (R13) but no occupation
        self.cls = np.array([0] * self.n_closed + list(range(1, self.n_open + 1)) + [0] * self.n_empty)
        self.empty = np.arange(self.nb) >= self.n_occ

    # ----------------------------------------------------------- plane-wave basis
    def _basis(self):
        """Miller indices (i,j,k) with (2 pi/L)^2 (i^2+j^2+k^2)/2 <= Ecut, tested
        in integers; loops over i, then j, then k ascending (full sphere)."""
        q = self.L / TWO_PI
        M = int(np.floor(2.0 * self.ecut * q * q))
        n = int(np.floor(np.sqrt(M)))
        while (n + 1) * (n + 1) <= M:
            n += 1
        while n * n > M:
            n -= 1
        if self.N < 2 * n + 1:
            raise ValueError("grid too small for the sphere")
        mil = [(i, j, k) for i in range(-n, n + 1) for j in range(-n, n + 1)
               for k in range(-n, n + 1) if i * i + j * j + k * k <= M]
        self.M = M
        self.nmax = n
        self.miller = np.array(mil, dtype=np.int64)
        self.npw = len(mil)
        N = self.N
        m = self.miller % N
        self.gidx = (m[:, 0] * N + m[:, 1]) * N + m[:, 2]
        b = TWO_PI / self.L
        self.G = self.miller * b
        self.g2 = (self.G ** 2).sum(axis=1)

    def _grid_vectors(self):
        N = self.N
        mt = np.arange(N)
        mt = np.where(mt <= N // 2, mt, mt - N)      # index N/2 maps to +N/2
        self.mt = mt
        b = TWO_PI / self.L
        gx = b * mt
        self.G2grid = (gx[:, None, None] ** 2 + gx[None, :, None] ** 2
                       + gx[None, None, :] ** 2).reshape(-1)
        self.gx = gx
        nyq = np.zeros(N, dtype=bool)
        if N % 2 == 0:
            nyq[N // 2] = True
        self.nyq = (nyq[:, None, None] | nyq[None, :, None] | nyq[None, None, :]).reshape(-1)

    # ----------------------------------------------------------- model V_ext
    def _local_potential(self):
        """Periodic Gaussian wells: V(G) = -(1/Omega) sum_a d_a (2 pi w^2)^{3/2}
        exp(-G^2 w^2/2) exp(-i G.R_a) on every grid G except the Nyquist
        planes (zeroed so that V(r) is real), then V(r) = sum_G V(G) e^{iGr}."""
        N = self.N
        VG = np.zeros(N ** 3, dtype=np.complex128)
        for at in self.cfg["atoms"]:
            d, w = at["depth"], at["width"]
            R = np.asarray(at["pos"], dtype=np.float64)
            ph = [np.exp(-1j * self.gx * R[c]) for c in range(3)]
            sf = (ph[0][:, None, None] * ph[1][None, :, None] * ph[2][None, None, :]).reshape(-1)
            VG += -(d * (TWO_PI * w * w) ** 1.5 / self.omega) * np.exp(-0.5 * self.G2grid * w * w) * sf
        VG[self.nyq] = 0.0
        Vr = _fft.fft3(VG.reshape(N, N, N), +1).reshape(-1)
        if np.abs(Vr.imag).max() > 1e-10 * max(1.0, np.abs(Vr.real).max()):
            raise AssertionError("local potential not real")
        self.Vloc = Vr.real.copy()

    # ----------------------------------------------------------- projectors
    def _projectors(self):
        """p_i(G) = Omega^{-1/2} N_l (2 pi rc^2)^{3/2} e^{-G^2 rc^2/2} Y(G) e^{-iG.R},
        Y = 1 for s and -i rc^2 G_m for p_m; N_l gives unit norm in the
        continuum.  V_nl = sum |p_i> D_ij <p_j|,  S = 1 + sum |p_i> Q_ij <p_j| (Eq. 3)."""
        cols, Dblocks, Qblocks, owner = [], [], [], []
        for a, at in enumerate(self.cfg["atoms"]):
            sp = self.cfg["species"][at["species"]]
            R = np.asarray(at["pos"], dtype=np.float64)
            phase = np.exp(-1j * (self.G @ R))
            for l, m, rc in zip(sp["l"], sp["m"], sp["rc"]):
                norm = (np.pi * rc * rc) ** -0.75
                if l == 1:
                    norm *= np.sqrt(2.0 / (rc * rc))
                pref = norm * (TWO_PI * rc * rc) ** 1.5 / np.sqrt(self.omega)
                radial = np.exp(-0.5 * self.g2 * rc * rc)
                ang = 1.0 if l == 0 else (-1j * rc * rc * self.G[:, m])
                cols.append(pref * ang * radial * phase)
                owner.append(a)
            Dblocks.append(np.asarray(sp["D"], dtype=np.float64))
            Qblocks.append(np.asarray(sp["Q"], dtype=np.float64))
        self.P = np.array(cols).T.copy() if cols else np.zeros((self.npw, 0), complex)
        self.nproj = self.P.shape[1]
        self.D = scipy.linalg.block_diag(*Dblocks) if Dblocks else np.zeros((0, 0))
        self.Q = scipy.linalg.block_diag(*Qblocks) if Qblocks else np.zeros((0, 0))

    # ----------------------------------------------------------- grid transforms
    def to_real(self, c: np.ndarray) -> np.ndarray:
        """psi(r) = Omega^{-1/2} sum_G c_G e^{iG.r} on the N^3 grid."""
        N = self.N
        g = np.zeros(N ** 3, dtype=np.complex128)
        g[self.gidx] = c
        return _fft.fft3(g.reshape(N, N, N), +1).reshape(-1) / np.sqrt(self.omega)

    def to_pw(self, f: np.ndarray) -> np.ndarray:
        """<e_G|f> = Omega^{-1/2} int e^{-iG.r} f(r) dr on the grid, G in the sphere."""
        N = self.N
        F = _fft.fft3(f.reshape(N, N, N), -1).reshape(-1)
        return F[self.gidx] * (np.sqrt(self.omega) / N ** 3)

    def grid_fourier(self, f: np.ndarray) -> np.ndarray:
        """f(G) = N^{-3} sum_r f(r) e^{-iG.r} on every grid G."""
        N = self.N
        return _fft.fft3(f.reshape(N, N, N), -1).reshape(-1) / N ** 3

    def grid_synth(self, FG: np.ndarray) -> np.ndarray:
        """f(r) = sum_G f(G) e^{iG.r}."""
        N = self.N
        return _fft.fft3(FG.reshape(N, N, N), +1).reshape(-1)

    def dvol(self) -> float:
        return self.omega / self.N ** 3

    # ----------------------------------------------------------- a2, a3: densities
    def class_densities(self, Psi: np.ndarray, bands=None) -> np.ndarray:
        """rho_k(r) = sum_{n in k} |psi_n(r)|^2 for k = closed, a, b (the
        occupied bands; empty ones carry no density).  With `bands`, the
        columns of Psi are those bands only (their share of the sums, for
        callers that split the bands over processes)."""
        bands = range(self.n_occ) if bands is None else [n for n in bands if n < self.n_occ]
        rho = np.zeros((3, self.N ** 3))
        for col, n in enumerate(bands):
            psi = self.to_real(Psi[:, col])
            rho[self.cls[n]] += (psi.conj() * psi).real
        return rho

    # ----------------------------------------------------------- a4-a6: potentials
    def potentials(self, rho_k: np.ndarray) -> Potentials:
        """Channel densities rho^{sigma L} = sum_k f_k^{sigma L} rho_k; one
        Hartree solve (rho_M = rho_T, Eq. 8); Slater exchange per channel;
        class potentials V^k = w_k (V_loc + V_H) + sum c_L f_k v_x^{sigma L}."""
        rho_ch = F_TABLE.T @ rho_k                    # (4, N^3)
        rho = rho_ch[0] + rho_ch[1]
        E = {}
        if self.hartree:
            rG = self.grid_fourier(rho)
            VG = np.zeros_like(rG)
            nz = self.G2grid > 0
            VG[nz] = 4.0 * np.pi * rG[nz] / self.G2grid[nz]
            VH = self.grid_synth(VG).real
            E["H"] = 0.5 * self.omega * float((4.0 * np.pi * np.abs(rG[nz]) ** 2
                                               / self.G2grid[nz]).sum())
        else:
            VH = np.zeros_like(rho)
            E["H"] = 0.0
        scale = (1.0 - self.alpha) if self.xc else 0.0
        vx, ex = self.exchange_channels(rho_ch, scale)
        E["x_M"] = float(ex[0] + ex[1])
        E["x_T"] = float(ex[2] + ex[3])
        E["loc"] = self.dvol() * float((self.Vloc * rho).sum())
        V0 = self.Vloc + VH
        Vk = self.w[:, None] * V0[None, :] + self.C @ vx
        return Potentials(rho_k=rho_k, rho_ch=rho_ch, rho=rho, VH=VH, vx=vx, Vk=Vk, E=E)

    def grid_derivative(self, f: np.ndarray, axis: int) -> np.ndarray:
        """d f / d r_axis of a real grid field by the spectral derivative:
        i G_axis f(G), with the Nyquist index of that axis left out (so the
        derivative of a real field stays real)."""
        N = self.N
        g = np.where(self.mt == N // 2, 0.0, self.gx) if N % 2 == 0 else self.gx
        shape = [1, 1, 1]
        shape[axis] = N
        mult = np.broadcast_to(g.reshape(shape), (N, N, N)).reshape(-1)
        return self.grid_synth(1j * mult * self.grid_fourier(f)).real

    def exchange_channels(self, rho_ch: np.ndarray, scale: float = 1.0):
        """Exchange potential v^{ch} (4, N^3) and energies (4,) of the channel
        densities, each a spin density, times `scale` (1 - alpha).

        Slater (LSDA): e = -(3/4) (6/pi)^{1/3} rho^{4/3}, v = -(6 rho / pi)^{1/3}.
        PBE exchange: e = e_Slater F_x(s), s^2 = |grad rho|^2 / (4 (6 pi^2)^{2/3}
        rho^{8/3}) (the spin-scaled reduced gradient, E_x[rho_up, rho_dn] =
        (E_x[2 rho_up] + E_x[2 rho_dn]) / 2), and v = de/drho - div(2
        de/d|grad rho|^2 grad rho), with spectral derivatives."""
        dv = self.dvol()
        r = np.maximum(rho_ch, 0.0)
        cx = slater_prefactor()
        if self.xc_kind == "slater":
            v = -scale * np.cbrt(6.0 * r / np.pi)
            return v, -scale * cx * dv * (np.cbrt(r) * r).sum(axis=1)
        k2 = (6.0 * np.pi ** 2) ** (2.0 / 3.0)
        vx = np.zeros_like(r)
        ex = np.zeros(r.shape[0])
        for ch in range(r.shape[0]):
            rr = r[ch]
            grad = [self.grid_derivative(rr, c) for c in range(3)]
            g = grad[0] ** 2 + grad[1] ** 2 + grad[2] ** 2
            on = rr > RHO_MIN
            c = np.cbrt(np.where(on, rr, 1.0))
            s2 = np.where(on, g / (4.0 * k2 * np.where(on, rr, 1.0) ** 2 * c * c), 0.0)
            F, dF = pbe_enhancement(s2)
            eL = -cx * rr * c
            e = np.where(on, eL * F, 0.0)
            v1 = np.where(on, -(4.0 / 3.0) * cx * c * (F - 2.0 * s2 * dF), 0.0)
            f = np.where(on, -cx * dF / (2.0 * k2 * np.where(on, rr, 1.0) * c), 0.0)   # 2 de/dg
            div = sum(self.grid_derivative(f * grad[c], c) for c in range(3))
            vx[ch] = scale * (v1 - div)
            ex[ch] = scale * dv * float(e.sum())
        return vx, ex

    # ----------------------------------------------------------- a11: exact exchange
    def coulomb_trunc(self) -> np.ndarray:
        """Exchange kernel on the grid.  Default (cfg exx_kernel 0): the
        spherically truncated Coulomb kernel v(G) = 4 pi (1 - cos(|G| Rc))/G^2,
        v(0) = 2 pi Rc^2, Rc = (3 Omega / 4 pi)^{1/3}.  exx_kernel 1: the bare
        Coulomb kernel 4 pi / G^2 with the G = 0 term left out."""
        Rc = (3.0 * self.omega / (4.0 * np.pi)) ** (1.0 / 3.0)
        g2 = self.G2grid
        v = np.empty_like(g2)
        nz = g2 > 0
        g = np.sqrt(g2[nz])
        if int(self.cfg.get("exx_kernel", 0)) == 1:
            v[nz] = 4.0 * np.pi / g2[nz]
            v[~nz] = 0.0
        else:
            v[nz] = 4.0 * np.pi * (1.0 - np.cos(g * Rc)) / g2[nz]
            v[~nz] = 2.0 * np.pi * Rc * Rc
        return v

    def exchange(self, Occ: np.ndarray, X: np.ndarray | None = None, classes=None, pair_integrals: bool = True):
        """Pair terms W_jn(r) = sum_G v(G) rho_jn(G) e^{iGr}, rho_jn = psi_j^* x_n,
        psi_j the occupied orbitals Occ.  Returns the operator part
        -alpha sum_j wx(k,k_j) psi_j W_jn for each column x_n of X (default Occ),
        as plane-wave coefficients, and the pair integrals of the occupied set
        K_ij = Omega sum_G v(G) |rho_ij(G)|^2 (None when pair_integrals is
        False: the operator alone)."""
        if X is None:
            X = Occ
        if classes is None:
            classes = self.cls
        v = self.coulomb_trunc()
        nb = X.shape[1]
        psis = [self.to_real(Occ[:, n]) for n in range(self.nb)]
        targets = [self.to_real(X[:, n]) for n in range(nb)]
        out = np.zeros_like(X)
        for n in range(nb):
            X = np.zeros(self.N ** 3, dtype=np.complex128)
            for j in range(self.nb):
                rG = self.grid_fourier(psis[j].conj() * targets[n])
                W = self.grid_synth(v * rG)
                X += self.WX[classes[n], self.cls[j]] * psis[j] * W
            out[:, n] = -self.alpha * self.to_pw(X)
        if not pair_integrals:
            return out, None
        K = np.zeros((self.nb, self.nb))
        for i in range(self.nb):
            for j in range(self.nb):
                rG = self.grid_fourier(psis[i].conj() * psis[j])
                K[i, j] = self.omega * float((v * np.abs(rG) ** 2).sum())
        return out, K

    # ----------------------------------------------------------- a7-a10: apply
    def apply(self, Psi: np.ndarray, pot: Potentials, classes=None, occ=None):
        """F^{k}|n> for each column (k = class of band n unless `classes` is
        given) and S|n>.  F^k = w_k (T + V_loc + V_nl + V_H) + sum c_L f v_x
        (+ exact exchange built from the occupied orbitals `occ`, default the
        columns themselves), Eq. 13 with Eq. 8."""
        if classes is None:
            classes = self.cls
        if occ is None:
            occ = Psi
        F = np.zeros_like(Psi)
        S = np.zeros_like(Psi)
        B = self.P.conj().T @ Psi
        for n in range(Psi.shape[1]):
            k = classes[n]
            psi = self.to_real(Psi[:, n])
            loc = self.to_pw(pot.Vk[k] * psi)
            kin = self.w[k] * 0.5 * self.g2 * Psi[:, n]
            nl = self.w[k] * (self.P @ (self.D @ B[:, n]))
            F[:, n] = kin + loc + nl
            S[:, n] = Psi[:, n] + self.P @ (self.Q @ B[:, n])
        if self.alpha != 0.0:
            X, _ = self.exchange(occ, Psi, classes, pair_integrals=False)
            F += X
        return F, S

    def apply_S(self, X: np.ndarray) -> np.ndarray:
        return X + self.P @ (self.Q @ (self.P.conj().T @ X))

    # ----------------------------------------------------------- a18: energies
    def energies(self, Psi: np.ndarray, pot: Potentials | None = None) -> dict:
        """E_L = sum f <n|T+V_loc+V_nl|n> + E_H + E_x^L (+ alpha E_HF^L);
        E = sum_L c_L E_L, which is E_S = 2 E_M - E_T for the singlet (Eq. 1)."""
        if pot is None:
            pot = self.potentials(self.class_densities(Psi))
        Psi = Psi[:, :self.n_occ]               # empty bands carry no energy
        wn = self.w[self.cls[:self.n_occ]]
        kin = float((wn[None, :] * 0.5 * self.g2[:, None] * np.abs(Psi) ** 2).sum())
        B = self.P.conj().T @ Psi
        nl = float(sum(wn[n] * (B[:, n].conj() @ self.D @ B[:, n]).real for n in range(self.n_occ)))
        E = dict(pot.E)
        E["kin"] = kin
        E["nl"] = nl
        if self.alpha != 0.0:
            _, K = self.exchange(Psi)
            fM = F_TABLE[self.cls[:self.n_occ]][:, 0:2]
            fT = F_TABLE[self.cls[:self.n_occ]][:, 2:4]
            E["hf_M"] = -0.5 * float(((fM @ fM.T) * K).sum())
            E["hf_T"] = -0.5 * float(((fT @ fT.T) * K).sum())
        else:
            E["hf_M"] = E["hf_T"] = 0.0
        one = kin + E["loc"] + nl + E["H"]
        E["M"] = one + E["x_M"] + self.alpha * E["hf_M"]
        E["T"] = one + E["x_T"] + self.alpha * E["hf_T"]
        E["total"] = self.cL[0] * E["M"] + self.cL[1] * E["T"]
        return E

    def energy(self, Psi: np.ndarray) -> float:
        return self.energies(Psi)["total"]

    # ----------------------------------------------------------- a17: orthonormalise
    def overlap(self, Psi: np.ndarray) -> np.ndarray:
        B = self.P.conj().T @ Psi
        O = Psi.conj().T @ Psi + B.conj().T @ self.Q @ B
        return 0.5 * (O + O.conj().T)

    def orthonormalize(self, Psi: np.ndarray) -> np.ndarray:
        """<m|S|n> = delta_mn (the constraint of Eq. 2) by Cholesky O = L L^H,
        Psi <- Psi L^{-H}, bands in the order closed, a, b."""
        O = self.overlap(Psi)
        Lc = np.linalg.cholesky(O)
        Linv = scipy.linalg.solve_triangular(Lc, np.eye(Lc.shape[0]), lower=True)
        return Psi @ Linv.conj().T

    def initial_orbitals(self, u: np.ndarray) -> np.ndarray:
        """c_nG = (u_re + i u_im)/(1 + |G|^2), then S-orthonormalised."""
        c = (u[..., 0] + 1j * u[..., 1]).T / (1.0 + self.g2)[:, None]
        return self.orthonormalize(c)


# =========================================================== a12-a16: PCG pieces
def gradient_parts(Psi, FPsi, SPsi, empty=None):
    """theta_mn = <m|F^n|n>; gamma (Eq. 11) as Gam_mn = gamma_nm =
    (theta_mn + theta_nm^*)/2; full gradient g = F Psi - S Psi Gam (Eq. 7);
    out-of-subspace part g_I = F Psi - S Psi theta and in-subspace matrix
    Gin_mn = theta_mn - theta_nm^* = 2 <m|g_n> (Eq. 12).

    empty (bool per band, R13): those columns of F Psi hold F^c|e>; the
    energy's operator there is F^e = 0, so gamma, g and Gin take theta and
    F Psi with those columns zero, while g_I keeps the F^c residual (the
    empty bands' own direction).  theta is returned as computed."""
    Theta = Psi.conj().T @ FPsi
    gI = FPsi - SPsi @ Theta
    ThE, FE = Theta, FPsi
    if empty is not None and np.any(empty):
        ThE = Theta.copy()
        ThE[:, empty] = 0.0
        FE = FPsi.copy()
        FE[:, empty] = 0.0
    Gam = 0.5 * (ThE + ThE.conj().T)
    G = FE - SPsi @ Gam
    Gin = ThE - ThE.conj().T
    return Theta, G, gI, Gin


def tpa_factor(x: np.ndarray) -> np.ndarray:
    """(27 + 18x + 12x^2 + 8x^3) / (27 + 18x + 12x^2 + 8x^3 + 16x^4) (Eq. 17)."""
    num = 27.0 + 18.0 * x + 12.0 * x * x + 8.0 * x ** 3
    return num / (num + 16.0 * x ** 4)


def tpa_step(sys_: System, gI):
    """K g_I with K = -(2/X) tpa(x) (Eq. 17), x = E_kin(G)/X with E_kin(G) =
    |G|^2 in Rydberg and X_n = 1.5 E_kin(g_nI) (Eq. 18 with R1); returns
    (K g_I, X)."""
    g2ry = sys_.g2
    w = np.abs(gI) ** 2
    X = 1.5 * (g2ry[:, None] * w).sum(axis=0) / np.maximum(w.sum(axis=0), 1e-300)
    x = g2ry[:, None] / X[None, :]
    K = -(2.0 / X)[None, :] * tpa_factor(x)
    return K * gI, X


def precondition(sys_: System, Psi, SPsi, gI):
    """p_I = K g_I - sum_m |m><m|S K|g_I> (Eq. 16) with the TPA step of tpa_step."""
    KgI, X = tpa_step(sys_, gI)
    pI = KgI - Psi @ (SPsi.conj().T @ KgI)
    return pI, X


def shell_of(cls: np.ndarray, mode: int, empty=None) -> np.ndarray:
    """Shell index per band: closed = 0; singlet: a = 1, b = 2; triplet: a, b
    share shell 1 (one open shell, Eq. 20 for high-spin states); empty = 3."""
    sh = np.minimum(cls, 1) if mode == 2 else cls.copy()
    if empty is not None:
        sh = np.where(empty, 3, sh)
    return sh


def r_matrix(Theta, cls, mode, suppress_ab=False, empty=None):
    """Off-diagonal R_mn of Eq. 20 from theta: same shell <m|F^s|n> = theta_mn;
    shells s < t: <m|F^s - F^t|n> = theta_nm^* - theta_mn; s > t the conjugate
    relation.  The a-b element is zeroed when the coupling is suppressed.
    With empty bands (R13) theta_mn = <m|F^c|n> in their columns: F^e = 0
    between shells (so R_mn = <m|F^s|n> there) and F^c within the empty
    shell, as in the fourth row and column of Eq. 20."""
    sh = shell_of(cls, mode, empty)
    nb = len(cls)
    ThE = Theta
    if empty is not None and np.any(empty):
        ThE = Theta.copy()
        ThE[:, empty] = 0.0
    R = np.zeros_like(Theta)
    for m in range(nb):
        for n in range(nb):
            if sh[m] == sh[n]:
                R[m, n] = Theta[m, n]
            elif sh[m] < sh[n]:
                R[m, n] = np.conj(ThE[n, m]) - ThE[m, n]
            else:
                R[m, n] = ThE[m, n] - np.conj(ThE[n, m])
    if suppress_ab and mode == 1:
        ia = np.where(cls == 1)[0]
        ib = np.where(cls == 2)[0]
        for a in ia:
            for b in ib:
                R[a, b] = R[b, a] = 0.0
    np.fill_diagonal(R, 0.0)
    return R


def rotation_generator(R, d, empty=None, dk=None, cls=None, Theta=None):
    """A_mn = -(1/2) atan(2|x|) x/|x|, x = R_mn/(d_m - d_n) (Eqs. 22-23 with R2, R3);
    computed for m < n and completed anti-Hermitian.

    An occupied band m of class k and an empty band n (R13, the empty bands
    come last): A_mn = (1/2) atan2(2|R_mn|, <n|F^k|n> - <m|F^k|m>) R_mn/|R_mn|
    (R_mn = <m|F^k|n>, dk[k, n] = <n|F^k|n>, Theta_mm = <m|F^k|m>), the
    rotation that takes m to the lower eigenvector of the 2 x 2 block of its
    own operator F^k.  Where m lies lower this is a Jacobi angle; where the
    empty band does, the angle exceeds pi/4 and exchanges the two, so the
    occupied bands end on the lowest states (aufbau), which a Jacobi step,
    never past pi/4, cannot reach."""
    nb = R.shape[0]
    A = np.zeros_like(R)
    for m in range(nb):
        for n in range(m + 1, nb):
            r = abs(R[m, n])
            if r < 1e-14:
                continue
            dd = d[m] - d[n]
            if empty is not None and empty[n] and not empty[m]:
                k = cls[m]
                gap = dk[k, n] - Theta[m, m].real
                A[m, n] = 0.5 * np.arctan2(2.0 * r, gap) * R[m, n] / r
            else:
                sg = 1.0 if dd >= 0.0 else -1.0
                phi = 0.5 * np.arctan2(2.0 * r, abs(dd))
                A[m, n] = -phi * sg * R[m, n] / r
            A[n, m] = -np.conj(A[m, n])
    return A


def closed_shell_diagonal(sys_: System, Psi, pot):
    """d_m = <m|F^c|m> for every band, by applying the closed-shell operator."""
    Fc, _ = sys_.apply(Psi, pot, classes=np.zeros(Psi.shape[1], dtype=int), occ=Psi)
    return np.real(np.einsum("gm,gm->m", Psi.conj(), Fc))


@dataclass
class StepInfo:
    E: float
    E_new: float
    step: float
    grad_norm: float
    coupling: complex
    beta: float
    dE0: float
    restarted: bool


class PCG:
    """All-band preconditioned Fletcher-Reeves CG (Eqs. 5, 6) with the ROKS
    two-step update: out-of-subspace step, then U = exp(step (A^i + beta A^{i-1}))
    (Eq. 24)."""

    def __init__(self, sys_: System, e_tol: float = 1e-6, suppress_ab: bool = False,
                 dt0: float = 0.3, g_tol: float = 0.0):
        self.sys = sys_
        self.e_tol = e_tol
        self.g_tol = g_tol
        self.suppress_ab = suppress_ab
        self.dt = dt0
        self.s_prev = None
        self.pg_prev = None
        self.A_prev = None
        self.E_prev = None
        self.n_small = 0
        self.converged = False

    def trial(self, Psi, s, A, step):
        U = scipy.linalg.expm(step * A)
        return self.sys.orthonormalize((Psi + step * s) @ U)

    def step(self, Psi):
        sy = self.sys
        pot = sy.potentials(sy.class_densities(Psi))
        E0 = sy.energies(Psi, pot)["total"]
        FPsi, SPsi = sy.apply(Psi, pot)
        empty = sy.empty if sy.n_empty else None
        Theta, G, gI, Gin = gradient_parts(Psi, FPsi, SPsi, empty)
        pI, _ = precondition(sy, Psi, SPsi, gI)
        d = closed_shell_diagonal(sy, Psi, pot)
        R = r_matrix(Theta, sy.cls, sy.mode, self.suppress_ab, empty)
        dk = None
        if sy.n_empty:
            # <e|F^k|e> of the empty bands for the three classes (R13)
            Pe = Psi[:, sy.empty]
            dk = np.zeros((3, sy.nb))
            for k in range(3):
                Fe, _ = sy.apply(Pe, pot, classes=np.full(Pe.shape[1], k, dtype=int), occ=Psi[:, :sy.n_occ])
                dk[k, sy.empty] = np.real(np.einsum("gm,gm->m", Pe.conj(), Fe))
        A = rotation_generator(R, d, empty, dk, sy.cls, Theta)
        no = sy.n_occ       # R13: the ratio of the energy's gradient (occupied bands)
        pg = float(np.real(np.vdot(pI[:, :no], gI[:, :no]))) + 0.5 * float(np.real(np.vdot(A, Gin)))
        beta = 0.0 if self.pg_prev is None else pg / self.pg_prev
        restarted = False

        def direction(beta_):
            s = pI if self.s_prev is None or beta_ == 0.0 else pI + beta_ * self.s_prev
            s = s - Psi @ (SPsi.conj().T @ s)
            At = A if self.A_prev is None or beta_ == 0.0 else A + beta_ * self.A_prev
            dE = 2.0 * float(np.real(np.vdot(s, G))) + float(np.real(np.vdot(At, Gin)))
            return s, At, dE

        s, At, dE0 = direction(beta)
        if dE0 >= 0.0 and beta != 0.0:
            beta, restarted = 0.0, True
            s, At, dE0 = direction(0.0)
        if dE0 >= 0.0:
            At = np.zeros_like(A)
            dE0 = 2.0 * float(np.real(np.vdot(s, G)))
            restarted = True
        dt = self.dt
        # the trial point moves the occupied bands only: the empty bands'
        # direction does not change the energy to first order, and its second
        # order (through the rotation) would distort the parabola (R13)
        s_t = s
        if sy.n_empty:
            s_t = s.copy()
            s_t[:, sy.empty] = 0.0
        Et = sy.energy(self.trial(Psi, s_t, At, dt))
        c = (Et - E0 - dE0 * dt) / (dt * dt)
        step = -dE0 / (2.0 * c) if c > 0.0 else dt
        step = min(step, 3.0 * dt)
        Psi_new = self.trial(Psi, s, At, step)
        E_new = sy.energy(Psi_new)
        self.dt = min(max(step, 0.05), 2.0)
        self.s_prev, self.pg_prev, self.A_prev = s, pg, A
        if abs(E_new - E0) < self.e_tol:
            self.n_small += 1
        else:
            self.n_small = 0
        grad_norm = float(np.linalg.norm(G))
        self.converged = self.n_small >= 2 and (self.g_tol <= 0.0 or grad_norm < self.g_tol)
        coupling = 0.0
        if sy.mode == 1:
            ia, ib = sy.n_closed, sy.n_closed + 1
            coupling = np.conj(Theta[ib, ia]) - Theta[ia, ib]
        info = StepInfo(E=E0, E_new=E_new, step=step,
                        grad_norm=grad_norm, coupling=coupling,
                        beta=beta, dE0=dE0, restarted=restarted)
        return Psi_new, info


def run(sys_: System, Psi, max_iter=50, e_tol=1e-6, suppress_ab=False, callback=None, g_tol=0.0):
    """PCG to convergence (R7) or max_iter; returns (Psi, list of StepInfo)."""
    pcg = PCG(sys_, e_tol=e_tol, suppress_ab=suppress_ab, g_tol=g_tol)
    hist = []
    for _ in range(max_iter):
        Psi, info = pcg.step(Psi)
        hist.append(info)
        if callback is not None:
            callback(info)
        if pcg.converged:
            break
    return Psi, hist
