"""The C++ oracle (oracle/cpp/roks_oracle.cpp) against the NumPy oracle
(oracle/roks.py): two independent FP64 restatements of the model and of the
apply path, which must agree to rounding.

Compared on tiny-16 (singlet, ground state with an odd band count), a 24^3
triplet and a 32^3 case with more bands: the basis rows bit for bit, the
local potential and the projector columns, the class densities of the
seeded start, the potentials and the energies, and F, S of every band, all
within 1e-12 relative (observed near 1e-15).  F and S do not depend on the
thread count (each band is one thread's work)."""
import numpy as np
import pytest

from oracle import cpp_oracle as CO
from oracle import roks as R
from paper_2605_28637_gb300 import synthetic as syn

CASES = {
    "tiny16-singlet": dict(),
    "tiny16-gs-odd": dict(mode=0, n_closed=5),
    "grid24-triplet": dict(grid=24, L=11.0, ecut=12.0, n_closed=5, mode=2),
    "grid32": dict(grid=32, L=12.0, ecut=20.0, n_closed=10),
}


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


@pytest.mark.parametrize("name", list(CASES))
def test_cpp_oracle_matches_numpy_oracle(name):
    cfg = syn.with_changes(syn.make_config("tiny-16", 0), **CASES[name])
    s = R.System(cfg)
    c = CO.CppSystem(cfg, threads=2)
    assert (c.npw, c.nproj, c.nb) == (s.npw, s.nproj, s.nb)
    assert np.array_equal(c.miller, s.miller)
    assert rel(c.vloc(), s.Vloc) < 1e-12
    assert rel(c.projectors(), s.P) < 1e-12
    P = s.initial_orbitals(syn.orbital_uniforms(cfg, s.npw))
    rho = c.class_densities(P)
    rho_ref = s.class_densities(P)
    assert rel(rho, rho_ref) < 1e-12
    Vk, E = c.potentials(rho_ref)
    pot = s.potentials(rho_ref)
    assert rel(Vk, pot.Vk) < 1e-12
    for k in ("H", "x_M", "x_T", "loc"):
        assert abs(E[k] - pot.E[k]) <= 1e-12 * max(1.0, abs(pot.E[k])), k
    F, S = c.apply(P, pot.Vk)
    F_ref, S_ref = s.apply(P, pot)
    assert rel(F, F_ref) < 1e-12
    assert rel(S, S_ref) < 1e-12
    c1 = CO.CppSystem(cfg, threads=1)
    F1, S1 = c1.apply(P, pot.Vk)
    assert np.array_equal(F1, F) and np.array_equal(S1, S)
    c.close()
    c1.close()


def test_cpp_oracle_rejects_a_small_grid():
    cfg = syn.with_changes(syn.make_config("tiny-16", 0), ecut=40.0)
    with pytest.raises(ValueError):
        CO.CppSystem(cfg)


@pytest.mark.parametrize("change", [dict(n_empty=2), dict(xc="pbe_x")])
def test_cpp_oracle_refuses_what_it_does_not_model(change):
    cfg = syn.with_changes(syn.make_config("tiny-16", 0), **change)
    with pytest.raises(ValueError):
        CO.CppSystem(cfg)
