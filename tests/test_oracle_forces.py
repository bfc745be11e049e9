"""Pins of the force oracle (oracle/forces.py).

* At fixed orbitals and fixed gamma the Hellmann-Feynman expression is the
  exact derivative of L(R) = E(Psi; R) - sum gamma_mn (<m|S(R)|n> - delta_mn):
  central differences of L with displaced atoms (the whole model rebuilt:
  wells and projectors) agree to 1e-7 for every atom and direction, in the
  singlet and the ground state.  The local, non-local and overlap terms are
  each of size 1e-2 or more there, and transposing gamma moves the result by
  about 4e-3, so a dropped term, a sign or a transposed index fails.
* At converged closed-shell orbitals it is the total derivative of the
  minimised energy: re-minimising at R +- h gives the same slope to 2e-6
  (the paper checks its forces against finite differences of the energy).
"""
import copy

import numpy as np
import pytest

from oracle import forces as Fo
from oracle import roks as R
from paper_2605_28637_gb300 import synthetic as syn


def tiny(**kw):
    return syn.with_changes(syn.make_config("tiny-16", 0), **kw)


def displaced(cfg, a, nu, h):
    c = copy.deepcopy(cfg)
    pos = list(c["atoms"][a]["pos"])
    pos[nu] += h
    c["atoms"][a]["pos"] = tuple(pos)
    return c


@pytest.mark.parametrize("kw", [dict(), dict(mode=0, n_closed=5)], ids=["singlet", "ground-state"])
def test_fixed_orbital_derivative_matches_finite_differences(kw):
    cfg = tiny(**kw)
    s = R.System(cfg)
    P = s.initial_orbitals(syn.orbital_uniforms(cfg, s.npw))
    pcg = R.PCG(s)
    for _ in range(5):
        P, _ = pcg.step(P)
    pot = s.potentials(s.class_densities(P))
    F, _ = s.apply(P, pot)
    gam = Fo.gamma_matrix(P, F)
    dE = Fo.energy_gradient(s, P, gam)
    assert np.abs(Fo.energy_gradient(s, P, gam.T) - dE).max() > 1e-3

    def lagrangian(c):
        s2 = R.System(c)
        B = s2.P.conj().T @ P
        Smat = P.conj().T @ P + B.conj().T @ s2.Q @ B
        return s2.energy(P) - float(np.sum(gam * (Smat - np.eye(s.nb))).real)

    h = 1e-4
    for a in range(len(cfg["atoms"])):
        for nu in range(3):
            fd = (lagrangian(displaced(cfg, a, nu, h)) - lagrangian(displaced(cfg, a, nu, -h))) / (2 * h)
            assert abs(dE[a, nu] - fd) < 1e-7, (a, nu, dE[a, nu], fd)
    assert np.array_equal(Fo.forces(s, P), -Fo.energy_gradient(s, P))


@pytest.mark.slow
def test_converged_forces_are_the_energy_slope():
    cfg = tiny(mode=0, n_closed=5)
    s = R.System(cfg)
    P = s.initial_orbitals(syn.orbital_uniforms(cfg, s.npw))
    P, hist = R.run(s, P, max_iter=400, e_tol=1e-12)
    assert hist[-1].grad_norm < 1e-5
    dE = Fo.energy_gradient(s, P)
    a, nu, h = 2, 2, 2e-3
    E = []
    for sg in (1, -1):
        s2 = R.System(displaced(cfg, a, nu, sg * h))
        _, h2 = R.run(s2, s2.orthonormalize(P), max_iter=400, e_tol=1e-12)
        E.append(h2[-1].E_new)
    fd = (E[0] - E[1]) / (2 * h)
    assert abs(dE[a, nu] - fd) < 2e-6, (dE[a, nu], fd)
