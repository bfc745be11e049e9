"""Degenerate systems on the GPU against the FP64 oracle (1e-9 relative on
the energies of three PCG steps and one DIIS step): a singlet with no closed
band (only the open pair a, b), a system without atoms (no wells, no
projectors: the free-electron gas with Hartree and exchange), and a ground
state with a single band."""
import numpy as np
import pytest

from oracle import diis as D
from oracle import roks as R
from paper_2605_28637_gb300 import synthetic as syn
from tests.gpu_helpers import built, rel, to_np

pytestmark = pytest.mark.gpu

CASES = {
    "open-pair-only": dict(n_closed=0),
    "no-atoms": dict(atoms=[]),
    "one-band": dict(mode=0, n_closed=1),
}


@pytest.mark.parametrize("name", list(CASES))
def test_degenerate_systems_fp64(name):
    cfg = syn.with_changes(syn.make_config("tiny-16", 0), **CASES[name])
    roks = built()
    ctx = roks.Context(cfg, "fp64")
    s = R.System(cfg)
    u = syn.orbital_uniforms(cfg, ctx.npw)
    psi = ctx.init_orbitals(u)
    P = s.initial_orbitals(u)
    assert rel(to_np(psi, s.npw), P) < 1e-10
    pcg = R.PCG(s)
    for it in range(3):
        info = ctx.pcg_step(psi)
        P, ref = pcg.step(P)
        assert abs(info["E_new"] - ref.E_new) <= 1e-9 * max(1.0, abs(ref.E_new)), (it, info["E_new"], ref.E_new)
    P0 = s.initial_orbitals(u)
    psi = ctx.init_orbitals(u)
    dinfo = ctx.diis_step(psi)
    _, dref = D.DIIS(s).step(P0)
    assert abs(dinfo["E_new"] - dref.E_new) <= 1e-9 * max(1.0, abs(dref.E_new))
    F = ctx.forces(psi)
    assert F.shape == (len(cfg["atoms"]), 3) and np.all(np.isfinite(F))
    # the forces of the DIIS result against the force oracle on the same orbitals
    from oracle import forces as Fo
    Fref = Fo.forces(s, to_np(psi, s.npw))
    assert Fref.shape == F.shape
    if F.size:
        assert np.abs(F - Fref).max() <= 1e-9 * max(np.abs(Fref).max(), 1e-12), (F, Fref)
    ctx.close()
