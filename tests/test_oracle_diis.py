"""Pins of the DIIS oracle (oracle/diis.py) against what the paper and the
mathematics fix; none compares the oracle with itself.

* lambda = 1/2 for every pair turns the residual into the gradient of Eq. 7
  (pinned by finite differences of E in test_oracle_model.py).
* lambda_ba = -1/2 changes exactly one in-subspace component of the residual
  of band a, the one along |b>, and flips its sign (reading R9).
* The coefficients of the bordered system minimise |sum d_j e_j| under
  sum d_j = 1: checked against a least-squares solve on the null space of the
  constraint, computed from the vectors themselves.
* The window test drops the oldest pairs when a later error vector lies in
  their span.
* A one-pair history is preconditioned steepest descent, written out.
* The converged closed shell spans the lowest eigenvectors of the dense
  generalised eigenproblem; the converged singlet is stationary (Eq. 15 and
  |g| small) and PCG started there keeps its energy (the paper's check that
  CG and DIIS agree on E_S).
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import diis as D
from oracle import roks as R
from paper_2605_28637_gb300 import synthetic as syn


def tiny(**kw):
    return syn.with_changes(syn.make_config("tiny-16", 0), **kw)


def start(cfg):
    s = R.System(cfg)
    return s, s.initial_orbitals(syn.orbital_uniforms(cfg, s.npw))


def fields(s, Psi):
    pot = s.potentials(s.class_densities(Psi))
    F, S = s.apply(Psi, pot)
    return F, S


def test_half_coupling_residual_is_the_gradient():
    s, Psi = start(tiny())
    F, S = fields(s, Psi)
    _, G, _, _ = R.gradient_parts(Psi, F, S)
    _, _, Rres = D.residual(Psi, F, S, D.coupling_table(s))
    assert np.abs(Rres - G).max() < 1e-12 * np.abs(G).max()


def test_open_pair_coupling_flips_one_component():
    s, Psi = start(tiny())
    F, S = fields(s, Psi)
    _, G, _, _ = R.gradient_parts(Psi, F, S)
    _, _, Rres = D.residual(Psi, F, S, D.coupling_table(s, 0.5, -0.5))
    a, b = s.n_closed, s.n_closed + 1
    # every column but a is the gradient
    others = [n for n in range(s.nb) if n != a]
    assert np.abs(Rres[:, others] - G[:, others]).max() < 1e-12
    # column a differs by a multiple of S|b> only, and <b|R_a> = -<b|g_a>
    diff = Rres[:, a] - G[:, a]
    Sb = S[:, b]
    c = np.vdot(Sb, diff) / np.vdot(Sb, Sb)
    assert np.abs(diff - c * Sb).max() < 1e-12
    gb = np.vdot(Psi[:, b], G[:, a])
    assert abs(gb) > 1e-6
    assert abs(np.vdot(Psi[:, b], Rres[:, a]) + gb) < 1e-10


def test_coefficients_minimise_the_combined_error():
    rng = np.random.default_rng(3)
    for h in (1, 2, 4, 7):
        E = rng.standard_normal((40, h)) + 1j * rng.standard_normal((40, h))
        E *= np.logspace(0, -3, h)[None, :]     # shrinking errors, as in a converging run
        B = np.real(E.conj().T @ E)
        d = D.coefficients(B)
        assert abs(d.sum() - 1.0) < 1e-12
        if h == 1:
            assert d[0] == pytest.approx(1.0)
            continue
        # d = d0 + N y, N a basis of {sum y = 0}; minimise |E d| over real y
        d0 = np.zeros(h)
        d0[-1] = 1.0
        N = scipy.linalg.null_space(np.ones((1, h)))
        Er = np.vstack([E.real, E.imag])
        y, *_ = np.linalg.lstsq(Er @ N, -Er @ d0, rcond=None)
        assert np.allclose(d, d0 + N @ y, atol=1e-9)


def test_window_drops_pairs_spanned_later():
    rng = np.random.default_rng(4)
    v = rng.standard_normal((30, 3))
    # the newest vector lies (almost) in the span of the two oldest
    E = np.column_stack([v[:, 0], v[:, 1], v[:, 2], v[:, 0] - 0.5 * v[:, 1] + 1e-6 * v[:, 2]])
    B = E.T @ E
    assert D.window(B) == 3          # the oldest pair goes; the rest is independent
    assert D.window(E[:, :3].T @ E[:, :3]) == 3
    same = np.column_stack([v[:, 0], v[:, 0]])
    assert D.window(same.T @ same) == 1


def test_one_pair_history_is_preconditioned_steepest_descent():
    s, Psi = start(tiny())
    F, S = fields(s, Psi)
    _, G, _, _ = R.gradient_parts(Psi, F, S)
    KG, _ = R.tpa_step(s, G)
    expect = s.orthonormalize(Psi + 0.5 * KG)
    dz = D.DIIS(s, history=1, tau=0.5)
    P1, info = dz.step(Psi)
    assert info.window == 1 and info.coef[0] == 1.0
    assert np.abs(P1 - expect).max() < 1e-12
    # the second step again forgets the first pair
    P2, info = dz.step(P1)
    F1, S1 = fields(s, P1)
    _, G1, _, _ = R.gradient_parts(P1, F1, S1)
    KG1, _ = R.tpa_step(s, G1)
    assert np.abs(P2 - s.orthonormalize(P1 + 0.5 * KG1)).max() < 1e-12


@pytest.mark.slow
def test_closed_shell_diis_reaches_the_ground_state():
    s, Psi = start(tiny(mode=0, n_closed=5))
    Psi, hist = D.run(s, Psi, max_iter=150, e_tol=1e-11)
    assert hist[-1].grad_norm < 1e-4
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
def test_singlet_diis_fixed_point_is_stationary_and_pcg_keeps_it():
    s, Psi = start(tiny(n_closed=2, ecut=5.0))
    Psi, hist = D.run(s, Psi, max_iter=400, e_tol=1e-10)
    assert hist[-1].grad_norm < 1e-4
    F, S = fields(s, Psi)
    _, G, _, Gin = R.gradient_parts(Psi, F, S)
    c, a, b = np.arange(s.n_closed), s.n_closed, s.n_closed + 1
    assert np.abs(Gin[np.ix_(c, [a, b])]).max() < 1e-5
    assert abs(Gin[a, b]) < 1e-5
    E_diis = s.energy(Psi)
    P = Psi
    pcg = R.PCG(s, e_tol=0.0)
    for _ in range(5):
        P, info = pcg.step(P)
    assert abs(info.E_new - E_diis) < 1e-8
