"""Pins of the oracle's empty shell (Eq. 20, fourth row and column; reading
R13): unoccupied bands after a, b that carry no occupation, the 4 x 4 shell
structure of R, and triplet runs with unoccupied bands.

What fixes the oracle here, without comparing it with itself:
* the empty bands leave the densities and every energy term unchanged, and
  the Cholesky order keeps the occupied start of the run without them;
* every block of R equals the matrix element of the operator Eq. 20 puts
  there, each operator applied to the bands directly (F^k on every band);
* the line-search slope E'(0) is the derivative of the energy along the path
  taken, so the empty bands' F^c direction adds nothing to it;
* the converged closed-shell ground state with empty bands spans the lowest
  eigenvectors of the dense generalised problem F^c x = e S x, and the empty
  bands the next ones (the aufbau order of the Kohn-Sham virtual orbitals);
* a converged triplet with unoccupied bands is a stationary state of the
  triplet without them, its empty bands are eigenvectors of F^c outside the
  occupied space, and none lies below an occupied band in that band's own
  operator (aufbau);
* the occupied-empty rotation reaches the lower eigenvalue of a 2 x 2 block
  whichever of the two lies lower."""
import numpy as np
import pytest
import scipy.linalg

from oracle import roks as R
from paper_2605_28637_gb300 import synthetic as syn


def tiny(**kw):
    return syn.with_changes(syn.make_config("tiny-16", 0), **kw)


def start(cfg):
    s = R.System(cfg)
    return s, s.initial_orbitals(syn.orbital_uniforms(cfg, s.npw))


def test_empty_bands_carry_no_density_or_energy():
    s0, P0 = start(tiny())
    s, P = start(tiny(n_empty=3))
    assert (s.nb, s.n_occ) == (s0.nb + 3, s0.nb)
    # the occupied start does not depend on the bands after it
    assert np.abs(P[:, :s.n_occ] - P0).max() < 1e-12
    assert np.abs(s.overlap(P) - np.eye(s.nb)).max() < 1e-12
    rho = s.class_densities(P)
    assert np.abs(rho - s0.class_densities(P0)).max() < 1e-12 * np.abs(rho).max()
    E, E0 = s.energies(P), s0.energies(P0)
    for k in ("kin", "nl", "H", "x_M", "x_T", "loc", "M", "T", "total"):
        assert E[k] == pytest.approx(E0[k], rel=1e-13, abs=1e-13), k


def operator_on_bands(s, P, pot, k):
    """F^k applied to every band (class k for all columns)."""
    F, _ = s.apply(P, pot, classes=np.full(P.shape[1], k, dtype=int), occ=P[:, :s.n_occ])
    return F


@pytest.mark.parametrize("mode", [1, 2])
def test_r_matrix_blocks_of_the_four_shells(mode):
    """Eq. 20 block by block: F^c within closed and within empty; F^s - F^t
    between occupied shells s < t; F^s between occupied shell s and the
    empty shell; the triplet's a and b form one open shell (F^a = F^b)."""
    s, P = start(tiny(mode=mode, n_empty=3))
    pot = s.potentials(s.class_densities(P))
    F, S = s.apply(P, pot)
    Th, G, gI, Gin = R.gradient_parts(P, F, S, s.empty)
    Rm = R.r_matrix(Th, s.cls, s.mode, empty=s.empty)
    assert np.allclose(Rm, Rm.conj().T, atol=1e-12)
    Fk = [operator_on_bands(s, P, pot, k) for k in range(3)]
    M = [P.conj().T @ Fk[k] for k in range(3)]          # M[k]_mn = <m|F^k|n>
    nc = s.n_closed
    c = list(range(nc))
    a, b = nc, nc + 1
    e = list(range(s.n_occ, s.nb))
    off = ~np.eye(s.nb, dtype=bool)
    blocks = {("c", "c"): M[0], ("c", "e"): M[0], ("e", "e"): M[0], ("a", "e"): M[1], ("b", "e"): M[2]}
    if mode == 1:
        blocks.update({("c", "a"): M[0] - M[1], ("c", "b"): M[0] - M[2], ("a", "b"): M[1] - M[2]})
    else:
        blocks.update({("c", "a"): M[0] - M[1], ("c", "b"): M[0] - M[2], ("a", "b"): M[1]})
    idx = {"c": c, "a": [a], "b": [b], "e": e}
    for (x, y), ref in blocks.items():
        rows, cols = idx[x], idx[y]
        want = ref[np.ix_(rows, cols)] * off[np.ix_(rows, cols)]
        got = Rm[np.ix_(rows, cols)]
        assert np.abs(got - want).max() < 1e-10 * max(1.0, np.abs(ref).max()), (x, y)
    if mode == 2:
        # one open shell: F^a = F^b in the triplet (c_M = 0)
        assert np.abs(M[1] - M[2]).max() < 1e-12 * np.abs(M[1]).max()
    # the energy's gradient vanishes in the empty columns outside the subspace
    Q = G[:, e] - S @ (P.conj().T @ G[:, e])
    assert np.abs(Q).max() < 1e-12 * max(1.0, np.abs(G).max())
    # while the empty bands' own direction is the F^c residual
    ge = Fk[0][:, e] - S @ (P.conj().T @ Fk[0][:, e])
    assert np.abs(gI[:, e] - ge).max() < 1e-10 * np.abs(ge).max()


def test_line_search_slope_with_empty_bands():
    """E'(0) is the derivative of E along orth((Psi + h s) exp(h A_tot)),
    both along the trial path (the occupied bands' directions) and along the
    accepted one (with the empty bands' F^c directions): had those entered
    the slope, central differences of the energy would disagree."""
    s, Psi = start(tiny(n_empty=3))
    pcg = R.PCG(s)
    seen = []
    trial = pcg.trial

    def spy(P, d, A, h):
        seen.append((P, d, A))
        return trial(P, d, A, h)

    pcg.trial = spy
    for it in range(3):
        P0 = Psi
        Psi, info = pcg.step(Psi)
        calls = [x for x in seen if x[0] is P0]
        # the trial point (occupied bands) and the accepted one (all bands:
        # the empty bands move out of the subspace as well)
        assert len(calls) == 2
        assert np.abs(calls[0][1][:, s.n_occ:]).max() == 0.0
        assert np.abs(calls[1][1][:, s.n_occ:]).max() > 1e-8
        for P, d, A in calls:
            h = 1e-4
            fd = (s.energy(trial(P, d, A, h)) - s.energy(trial(P, d, A, -h))) / (2 * h)
            assert abs(fd - info.dE0) < 1e-6 * max(1.0, abs(info.dE0)), (it, fd, info.dE0)


def dense_fc(s, Psi):
    pot = s.potentials(s.class_densities(Psi))
    I = np.eye(s.npw, dtype=complex)
    H, Sm = s.apply(I, pot, classes=np.zeros(s.npw, dtype=int), occ=Psi[:, :s.n_occ])
    return pot, 0.5 * (H + H.conj().T), 0.5 * (Sm + Sm.conj().T)


@pytest.mark.slow
def test_ground_state_empty_bands_are_the_next_eigenvectors():
    """Closed shell with 2 empty bands, converged: the occupied Ritz values
    are the 5 lowest eigenvalues of the dense F^c x = e S x, the empty bands'
    the next 2, and the empty bands span those eigenvectors.  The energy is
    that of the run without empty bands."""
    cfg = tiny(mode=0, n_closed=5, n_empty=2)
    s, Psi = start(cfg)
    Psi, hist = R.run(s, Psi, max_iter=600, e_tol=1e-11)
    s0, P0 = start(syn.with_changes(cfg, n_empty=0))
    P0, h0 = R.run(s0, P0, max_iter=600, e_tol=1e-11)
    assert hist[-1].E_new == pytest.approx(h0[-1].E_new, abs=1e-9)
    assert hist[-1].E_new <= hist[0].E
    pot, H, Sm = dense_fc(s, Psi)
    ev, X = scipy.linalg.eigh(H, Sm)
    Fc = operator_on_bands(s, Psi, pot, 0)
    Th = Psi.conj().T @ Fc
    occ = np.sort(np.linalg.eigvalsh(0.5 * (Th[:5, :5] + Th[:5, :5].conj().T)))
    emp = np.sort(np.linalg.eigvalsh(0.5 * (Th[5:, 5:] + Th[5:, 5:].conj().T)))
    assert np.allclose(occ, ev[:5], atol=2e-6)
    assert np.allclose(emp, ev[5:7], atol=2e-6), (emp, ev[5:8])
    # the empty span is that of eigenvectors 5, 6 (S-orthonormal projectors)
    Pe = Psi[:, 5:] @ Psi[:, 5:].conj().T
    Px = X[:, 5:7] @ X[:, 5:7].conj().T
    assert np.abs((Pe - Px) @ Sm).max() < 1e-3


@pytest.mark.slow
def test_triplet_with_empty_bands_is_stationary_with_aufbau_empty_bands():
    """Triplet (one open shell in R) with 2 empty bands, converged:
    * its occupied orbitals are a stationary state of the triplet without
      empty bands (PCG on them alone changes the energy by < 1e-7 Ha);
    * the empty bands are eigenvectors of F^c outside the occupied space:
      their residual (1 - S Psi Psi^H) F^c|e> and the off-diagonal of
      <e|F^c|e'> vanish;
    * aufbau: no empty band lies below an occupied band in that band's own
      operator, <e|F^k|e> > <m|F^k|m> for every occupied m of class k.
    (The triplet has more than one stationary state; which one a run
    reaches depends on the start and the band set, as for the singlet.)"""
    cfg = tiny(mode=2, n_closed=4, n_empty=2)
    s, P = start(cfg)
    P, h = R.run(s, P, max_iter=600, e_tol=1e-10)
    assert h[-1].E_new < h[0].E
    s0 = R.System(syn.with_changes(cfg, n_empty=0))
    P0, h0 = R.run(s0, P[:, :s.n_occ].copy(), max_iter=50, e_tol=1e-10)
    assert abs(h0[-1].E_new - h[-1].E_new) < 1e-7
    pot = s.potentials(s.class_densities(P))
    F, S = s.apply(P, pot)
    Th, G, gI, Gin = R.gradient_parts(P, F, S, s.empty)
    e = slice(s.n_occ, s.nb)
    assert np.linalg.norm(G) < 1e-3
    assert np.linalg.norm(gI[:, e]) < 1e-3 * np.linalg.norm(F[:, e])
    Te = Th[e, e]
    assert np.abs(Te - np.diag(np.diag(Te))).max() < 1e-4 * np.abs(Te).max()
    for k in range(3):
        Fe = operator_on_bands(s, P[:, e], pot, k)
        de = np.real(np.einsum("gm,gm->m", P[:, e].conj(), Fe))
        own = [Th[m, m].real for m in range(s.n_occ) if s.cls[m] == k]
        assert de.min() > max(own), (k, de, own)


@pytest.mark.parametrize("d_occ,d_emp", [(-1.0, -0.4), (-0.4, -1.0), (0.3, 0.2)])
def test_occupied_empty_rotation_reaches_the_lower_state(d_occ, d_emp):
    """The occupied-empty generator (R13) turns the occupied band to the lower
    eigenvector of the pair's 2 x 2 block, whichever of the two lies lower:
    with |m'> = sum_k U_km |k>, U = exp(A), <m'|H|m'> is H's lower
    eigenvalue; a Jacobi angle (never past pi/4) would leave the occupied
    band on the upper one when the empty band lies lower."""
    r = 0.05 * np.exp(0.7j)
    H = np.array([[d_occ, r], [np.conj(r), d_emp]])
    Rm = np.array([[0.0, r], [np.conj(r), 0.0]])
    Theta = np.diag([d_occ, 0.0]).astype(complex)
    dk = np.zeros((3, 2))
    dk[0, 1] = d_emp
    A = R.rotation_generator(Rm, np.array([d_occ, d_emp]), np.array([False, True]), dk, np.array([0, 0]), Theta)
    U = scipy.linalg.expm(A)
    m = U[:, 0]
    assert np.allclose(A, -A.conj().T)
    assert np.real(m.conj() @ H @ m) == pytest.approx(np.linalg.eigvalsh(H)[0], abs=1e-12)
