"""Parity at the full size of the MgO-vacancy workload (mgo-120: 215 atoms,
428 + 2 bands, 120^3 grid, 37,705 plane waves, 1288 projectors), mixed path,
in the benchmark's launch configuration (PCG steps captured as a CUDA graph
and replayed; tensor-core contractions), against the FP64 oracle evaluating
the GPU's own orbitals.

The oracle forms the class densities of all 430 bands (spread over host
processes), the potentials and the energies, and applies F and S to sampled
bands.  Tolerances as for organic-96 (FP32 rounding): S-orthonormality 5e-6,
densities and S|n> 2e-6 relative, F|n> 2e-5 relative, the energy 2e-7 of the
sum of the energy terms' magnitudes.  The steps descend, and each starts at
the previous step's energy."""
import numpy as np
import pytest

from oracle import roks as R
from paper_2605_28637_gb300 import synthetic as syn
from tests import oracle_pool
from tests.gpu_helpers import built, rel, to_np

pytestmark = pytest.mark.gpu

TERMS = ("kin", "loc", "nl", "H", "x_M", "x_T")


def test_mgo120_full_size_against_oracle():
    roks = built()
    cfg = syn.make_config("mgo-120", 0)
    ctx = roks.Context(cfg, "mixed")
    assert (ctx.nb, ctx.nproj, ctx.npw) == (430, 1288, 37705)
    psi = ctx.init_orbitals(None)
    infos = [ctx.pcg_step(psi) for _ in range(3)]      # eager, captured, replayed
    for a, b in zip(infos, infos[1:]):
        assert b["E"] == a["E_new"]
    assert all(i["E_new"] < i["E"] for i in infos)
    # GPU evaluation of the final orbitals
    rho = ctx.density(psi, want_rho=True).cpu().numpy()
    E = ctx.potential()
    f, sp, _ = ctx.apply_h(psi)
    P = to_np(psi, ctx.npw)
    # oracle on the same orbitals
    s = R.System(cfg)
    rho_ref = oracle_pool.class_densities(cfg, P)
    assert rel(rho, rho_ref) < 2e-6
    pot = s.potentials(rho_ref)
    Eref = s.energies(P, pot)
    scale = sum(abs(Eref[k]) for k in TERMS)
    assert abs(E["E_total"] - Eref["total"]) < 2e-7 * scale, (E["E_total"], Eref["total"], scale)
    assert abs(infos[-1]["E_new"] - Eref["total"]) < 2e-7 * scale
    sel = [0, 211, 427, 428, 429]                       # closed bands, then a and b
    F_ref, S_ref = s.apply(P[:, sel], pot, classes=s.cls[sel])
    Fg, Sg = to_np(f, ctx.npw)[:, sel], to_np(sp, ctx.npw)[:, sel]
    assert rel(Fg, F_ref) < 2e-5
    assert rel(Sg, S_ref) < 2e-6
    O = P.conj().T @ s.apply_S(P)
    assert np.abs(O - np.eye(ctx.nb)).max() < 5e-6
    ctx.close()
