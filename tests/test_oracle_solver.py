"""Pins of the oracle's PCG pieces: gamma/gradient split (Eqs. 7, 11, 12),
TPA (Eqs. 17, 18), the R-matrix rotation (Eqs. 20-23), orthonormalisation, the
line search and the converged solutions (stationarity, closed-shell limit)."""
import json
import os

import numpy as np
import pytest
import scipy.linalg

from oracle import roks as R
from paper_2605_28637_gb300 import synthetic as syn

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def tiny(**kw):
    return syn.with_changes(syn.make_config("tiny-16", 0), **kw)


def start(cfg):
    s = R.System(cfg)
    return s, s.initial_orbitals(syn.orbital_uniforms(cfg, s.npw))


def test_orthonormal_start():
    s, Psi = start(tiny())
    assert np.abs(s.overlap(Psi) - np.eye(s.nb)).max() < 1e-12


def test_gradient_split_identities():
    """g = g_I + g_II; g_I is S-orthogonal... to the subspace in the sense
    Psi^H g_I = 0; <m|g_n> = Gin_mn / 2; gamma Hermitian."""
    s, Psi = start(tiny())
    pot = s.potentials(s.class_densities(Psi))
    F, S = s.apply(Psi, pot)
    Th, G, gI, Gin = R.gradient_parts(Psi, F, S)
    gII = S @ (0.5 * Gin)
    assert np.allclose(G, gI + gII, atol=1e-12)
    assert np.abs(Psi.conj().T @ gI).max() < 1e-11
    assert np.allclose(Psi.conj().T @ G, 0.5 * Gin, atol=1e-11)
    # the SI S1 conditions: <g_m|n> + <m|g_n> = 0 holds for the gamma choice
    M = Psi.conj().T @ G
    assert np.abs(M + M.conj().T).max() < 1e-11


def test_preconditioned_gradient_is_s_orthogonal_and_descent():
    s, Psi = start(tiny())
    pot = s.potentials(s.class_densities(Psi))
    F, S = s.apply(Psi, pot)
    Th, G, gI, Gin = R.gradient_parts(Psi, F, S)
    pI, X = R.precondition(s, Psi, S, gI)
    assert np.abs(S.conj().T @ pI).max() < 1e-11     # Psi^H S p_I = 0 (Eq. 16)
    assert np.real(np.vdot(pI, gI)) < 0


def test_tpa_limits():
    x = np.array([0.0, 1e-8])
    assert np.allclose(R.tpa_factor(x), 1.0)
    big = np.array([1e4, 1e6])
    assert np.allclose(R.tpa_factor(big) * 2 * big, 1.0, rtol=1e-3)
    # hand values: x = 1 -> 65/81, x = 2 -> (27+36+48+64)/(175+256)
    assert np.isclose(R.tpa_factor(np.array([1.0]))[0], 65 / 81)
    assert np.isclose(R.tpa_factor(np.array([2.0]))[0], 175 / 431)


def test_jacobi_rotation_diagonalises_2x2():
    rng = np.random.default_rng(0)
    for _ in range(20):
        a, d = rng.normal(size=2)
        b = rng.normal() + 1j * rng.normal()
        H = np.array([[a, b], [np.conj(b), d]])
        Rm = H.copy()
        np.fill_diagonal(Rm, 0)
        A = R.rotation_generator(Rm, np.real(np.diag(H)))
        U = scipy.linalg.expm(A)
        Hp = U.conj().T @ H @ U                      # |n'> = sum_m U_mn |m>
        assert abs(Hp[0, 1]) < 1e-12
        assert np.allclose(A, -A.conj().T)


def test_rotation_derivative_matches_in_subspace_gradient():
    """d/dh E(Psi exp(hA)) at 0 = Re sum A^* Gin (the in-subspace part of Eq. 12)."""
    s, Psi = start(tiny())
    pot = s.potentials(s.class_densities(Psi))
    F, S = s.apply(Psi, pot)
    Th, G, gI, Gin = R.gradient_parts(Psi, F, S)
    d = R.closed_shell_diagonal(s, Psi, pot)
    A = R.rotation_generator(R.r_matrix(Th, s.cls, s.mode), d)
    h = 1e-4
    fd = (s.energy(Psi @ scipy.linalg.expm(h * A)) - s.energy(Psi @ scipy.linalg.expm(-h * A))) / (2 * h)
    an = float(np.real(np.vdot(A, Gin)))
    assert abs(fd - an) < 1e-7 * max(1e-6, abs(an))
    assert an < 0                                    # descent for this start (R2)


def test_r_matrix_structure():
    """R is Hermitian; inter-shell entries are -+ 2 <m|g_n> (Eq. 20 with Eq. 12)."""
    s, Psi = start(tiny())
    pot = s.potentials(s.class_densities(Psi))
    F, S = s.apply(Psi, pot)
    Th, G, gI, Gin = R.gradient_parts(Psi, F, S)
    Rm = R.r_matrix(Th, s.cls, s.mode)
    assert np.allclose(Rm, Rm.conj().T, atol=1e-13)
    c, a, b = 0, s.n_closed, s.n_closed + 1
    assert np.isclose(Rm[c, a], -Gin[c, a])
    assert np.isclose(Rm[a, b], -Gin[a, b])
    Rs = R.r_matrix(Th, s.cls, s.mode, suppress_ab=True)
    assert Rs[a, b] == 0 and Rs[b, a] == 0 and np.isclose(Rs[c, a], Rm[c, a])


def test_orthonormalize_cholesky_order():
    s, Psi = start(tiny())
    X = Psi + 0.3 * syn.random_vectors(9, s.npw, s.nb)
    Y = s.orthonormalize(X)
    assert np.abs(s.overlap(Y) - np.eye(s.nb)).max() < 1e-12
    # Cholesky keeps the span of the first k bands for every k
    for k in range(1, s.nb + 1):
        Qx, _ = np.linalg.qr(X[:, :k])
        Qy, _ = np.linalg.qr(Y[:, :k])
        assert np.abs(Qx @ (Qx.conj().T @ Qy) - Qy).max() < 1e-10


def test_pcg_trace_golden_and_monotone():
    with open(os.path.join(GOLDEN, "tiny16_pcg_trace.json")) as f:
        gold = json.load(f)
    s, Psi = start(tiny())
    _, hist = R.run(s, Psi, max_iter=len(gold["E"]), e_tol=0.0)
    E = [h.E for h in hist]
    assert np.allclose(E, gold["E"], rtol=0, atol=1e-10)
    En = [h.E_new for h in hist]
    assert all(b < a for a, b in zip(E, En))


@pytest.mark.slow
def test_closed_shell_reduction():
    """Ground state (no open shell): the converged orbitals span the lowest
    eigenvectors of the dense generalised problem F^c x = e S x."""
    s, Psi = start(tiny(mode=0, n_closed=5))
    Psi, hist = R.run(s, Psi, max_iter=400, e_tol=1e-11)
    pot = s.potentials(s.class_densities(Psi))
    I = np.eye(s.npw, dtype=complex)
    H, Sm = s.apply(I, pot, classes=np.zeros(s.npw, dtype=int), occ=Psi)
    H = 0.5 * (H + H.conj().T)
    Sm = 0.5 * (Sm + Sm.conj().T)
    ev = scipy.linalg.eigh(H, Sm, eigvals_only=True)[: s.nb]
    Th = Psi.conj().T @ s.apply(Psi, pot)[0]
    sub = np.sort(np.linalg.eigvalsh(0.5 * (Th + Th.conj().T)))
    assert np.allclose(sub, ev, atol=2e-6)


@pytest.mark.slow
def test_singlet_stationarity():
    """Converged singlet: |g| small and the inter-shell conditions
    <m|F^n - F^m|n> = 0 (Eq. 15, SI S1) hold."""
    s, Psi = start(tiny())
    Psi, hist = R.run(s, Psi, max_iter=400, e_tol=1e-9)
    pot = s.potentials(s.class_densities(Psi))
    F, S = s.apply(Psi, pot)
    Th, G, gI, Gin = R.gradient_parts(Psi, F, S)
    assert np.linalg.norm(G) < 2e-3
    c, a, b = np.arange(s.n_closed), s.n_closed, s.n_closed + 1
    assert np.abs(Gin[np.ix_(c, [a, b])]).max() < 1e-4
    assert abs(Gin[a, b]) < 1e-4
    E = s.energies(Psi)
    assert E["total"] == pytest.approx(2 * E["M"] - E["T"], abs=1e-12)


def test_line_search_slope_matches_finite_difference():
    """E'(0) used by the line search (R5) is the derivative of E along the
    path actually taken, orth((Psi + h s) exp(h A_tot)) (Eqs. 5, 24), with
    and without the Fletcher-Reeves history: central differences of the
    energy agree, so a wrong sign, a dropped in-subspace term or a missing
    factor 2 in 2 Re<s|g> would show."""
    s, Psi = start(tiny())
    pcg = R.PCG(s)
    seen = []
    trial = pcg.trial

    def spy(P, d, A, h):
        if len(seen) == 0 or seen[-1][0] is not P:
            seen.append((P, d, A))
        return trial(P, d, A, h)

    pcg.trial = spy
    checked = 0
    for it in range(3):
        P0 = Psi
        Psi, info = pcg.step(Psi)
        P, d, A = [x for x in seen if x[0] is P0][0]
        h = 1e-4
        fd = (s.energy(trial(P, d, A, h)) - s.energy(trial(P, d, A, -h))) / (2 * h)
        assert abs(fd - info.dE0) < 1e-6 * max(1.0, abs(info.dE0)), (it, fd, info.dE0)
        checked += info.beta != 0.0
    assert checked >= 1          # at least one step used the Fletcher-Reeves history


@pytest.mark.parametrize("mode_kw", [dict(), dict(mode=0, n_closed=5), dict(mode=2)],
                         ids=["singlet", "ground-state", "triplet"])
def test_line_search_step_and_fr_numerator_against_the_energy_curve(mode_kw):
    """The step lengths (R5) and the Fletcher-Reeves ratios (R4), each
    against the energy along a path rather than against the formulas.

    * Fletcher-Reeves numerator: the ratio of step i is pg_i / pg_{i-1}, with
      pg = Re<p_I|g_I> + 1/2 Re<A|G_in> at the step's start.  A fresh solver
      at that start takes the preconditioned steepest-descent direction, and
      central differences of the energy along its path give the slope.  The
      slope equals 2 pg, so both factors of every ratio are fixed by energies.
      A dropped 1/2 on the in-subspace term, a sign, or the full gradient in
      place of g_I would break it.
    * Step: the accepted step minimises the energy along the accepted path
      to within the quadratic model's error.  The energy at 0.75 and 1.25
      times the step lies above the energy at the step.  A step off by a
      factor of two from the parabola's vertex fails this.  The first step
      is capped at 3 dt (R5), and there the energy still falls past the
      step."""
    s, Psi = start(tiny(**mode_kw))
    pcg = R.PCG(s)
    seen = []
    trial = pcg.trial

    def spy(P, d, A, h):
        seen.append((P, d, A))
        return trial(P, d, A, h)

    pcg.trial = spy
    h = 1e-4
    for it in range(6):
        fresh = R.PCG(s)
        fresh_calls = []

        def fresh_spy(P, d, A, t, calls=fresh_calls):
            calls.append((P, d, A))
            return trial(P, d, A, t)

        fresh.trial = fresh_spy
        _, finfo = fresh.step(Psi)
        assert finfo.beta == 0.0 and not finfo.restarted
        P0, d0, A0 = fresh_calls[0]
        slope = (s.energy(trial(P0, d0, A0, h)) - s.energy(trial(P0, d0, A0, -h))) / (2 * h)

        dt = pcg.dt
        start_psi = Psi
        Psi, info = pcg.step(Psi)
        assert abs(slope - 2.0 * pcg.pg_prev) < 1e-7 * abs(slope), (it, slope, pcg.pg_prev)

        Pa, da, Aa = [x for x in seen if x[0] is start_psi][-1]
        st = info.step
        e_at = s.energy(trial(Pa, da, Aa, st))
        e_lo = s.energy(trial(Pa, da, Aa, 0.75 * st))
        e_hi = s.energy(trial(Pa, da, Aa, 1.25 * st))
        assert e_at == pytest.approx(info.E_new, abs=1e-12)
        if abs(st - 3.0 * dt) < 1e-15:
            assert e_hi < e_at < e_lo, (it, e_lo, e_at, e_hi)      # capped: still descending
        else:
            assert e_at < e_lo and e_at < e_hi, (it, e_lo, e_at, e_hi)
