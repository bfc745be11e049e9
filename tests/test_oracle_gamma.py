"""Pins of the Gamma-point half-sphere oracle (oracle/gamma.py)."""
import json
import os

import numpy as np

from oracle import gamma as Gm
from oracle import roks as R
from paper_2605_28637_gb300 import synthetic as syn

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def tiny(**kw):
    return syn.with_changes(syn.make_config("tiny-16", 0), **kw)


def test_half_sphere_count_and_partners():
    with open(os.path.join(GOLDEN, "basis_counts.json")) as f:
        gold = json.load(f)["workloads"]["tiny-16"]
    s = R.System(tiny())
    h = Gm.half_index(s)
    assert len(h) == (s.npw + 1) // 2 == gold["npw_half"]
    p = Gm.partner_index(s)
    assert np.array_equal(p[p], np.arange(s.npw))                      # -(-G) = G
    assert np.array_equal(s.miller[p], -s.miller)
    fixed = np.where(p == np.arange(s.npw))[0]
    assert len(fixed) == 1 and np.all(s.miller[fixed[0]] == 0)          # only G = 0 is its own partner
    # the kept set and its mirror image cover the sphere, meeting only at G = 0
    assert len(np.union1d(h, p[h])) == s.npw


def test_expand_restrict_and_realness():
    s = R.System(tiny())
    rng = np.random.default_rng(5)
    nh = len(Gm.half_index(s))
    C = rng.standard_normal((nh, 3)) + 1j * rng.standard_normal((nh, 3))
    g0 = int(np.where(np.all(s.miller[Gm.half_index(s)] == 0, axis=1))[0][0])
    C[g0] = C[g0].real
    F = Gm.expand(s, C)
    assert np.array_equal(Gm.restrict(s, F), C)
    assert Gm.realness(s, F) < 1e-13
    # a vector that is not symmetric is not real in real space
    G = F.copy()
    G[Gm.partner_index(s)[Gm.half_index(s)[1]]] += 0.3
    assert Gm.realness(s, G) > 1e-3


def test_overlap_from_the_half_sphere():
    s = R.System(tiny())
    rng = np.random.default_rng(6)
    h = Gm.half_index(s)
    g0 = int(np.where(np.all(s.miller[h] == 0, axis=1))[0][0])
    A = rng.standard_normal((len(h), 4)) + 1j * rng.standard_normal((len(h), 4))
    B = rng.standard_normal((len(h), 3)) + 1j * rng.standard_normal((len(h), 3))
    A[g0] = A[g0].real
    B[g0] = B[g0].real
    full = Gm.expand(s, A).conj().T @ Gm.expand(s, B)
    assert np.abs(full.imag).max() < 1e-12
    assert np.abs(Gm.overlap_half(s, A, B) - full.real).max() < 1e-12
    # projector coefficients of real orbitals are real (real projectors)
    Bp = s.P.conj().T @ Gm.expand(s, A)
    assert np.abs(Bp.imag).max() < 1e-12 * max(1.0, np.abs(Bp).max())


def test_pcg_keeps_real_orbitals():
    cfg = tiny()
    s = R.System(cfg)
    u = syn.orbital_uniforms(cfg, len(Gm.half_index(s)))
    P = Gm.initial_orbitals(s, u)
    assert Gm.realness(s, P) < 1e-12
    assert np.abs(s.overlap(P) - np.eye(s.nb)).max() < 1e-12
    pcg = R.PCG(s)
    E = []
    for _ in range(6):
        P, info = pcg.step(P)
        E.append(info.E_new)
    assert Gm.realness(s, P) < 1e-10
    assert all(b < a for a, b in zip(E, E[1:]))
    # the multipliers of real orbitals are real
    F, _ = s.apply(P, s.potentials(s.class_densities(P)))
    Theta = P.conj().T @ F
    assert np.abs(Theta.imag).max() < 1e-10 * np.abs(Theta).max()
