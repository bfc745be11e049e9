"""GPU parity of PBE exchange (roks_options.xc = ROKS_XC_PBE_X, the GGA of
Sec. III) through the C ABI against the oracle (oracle/roks.py,
System.exchange_channels, pinned in tests/test_oracle_gga.py).

* FP64, 1e-10 relative, on tiny-16 (singlet, triplet, ground state) and on
  the 24^3, 32^3 and 48^3 variants (several tiles and ragged tails):
  - the class potentials V^k, with the divergence of the exchange flux;
  - every energy term and the gradient;
  - F|n> and S|n>;
* FP64 8-step PCG trajectories (singlet, triplet, with empty bands);
* the forces, in FP64, of orbitals after three steps;
* the Gamma-point form: the half-sphere step against the oracle's
  full-sphere step from the same real start, in FP64;
* mixed precision:
  - V^k and F|n> within the mixed bars (2e-6 and 2e-5 relative of the
    largest entry), the energy within 2e-7 of the sum of the terms'
    magnitudes;
  - 20 singlet steps within 1e-6 of that sum;
* the hybrid: PBE exchange scaled by (1 - alpha) beside exact exchange."""
import numpy as np
import pytest

from oracle import forces as Fo
from oracle import gamma as Gm
from oracle import roks as R
from paper_2605_28637_gb300 import synthetic as syn
from tests.gpu_helpers import built, rel, to_dev, to_np

pytestmark = pytest.mark.gpu

TOL64 = 1e-10

CASES = {
    "tiny16-singlet": dict(),
    "tiny16-triplet": dict(mode=2),
    "tiny16-gs": dict(mode=0, n_closed=5),
    "grid24": dict(grid=24, L=11.0, ecut=12.0, n_closed=5),
    "grid32": dict(grid=32, L=12.0, ecut=20.0, n_closed=6),
    "grid48": dict(grid=48, L=12.0, ecut=35.0, n_closed=3),
}


def cfg_of(**kw):
    return syn.with_changes(syn.make_config("tiny-16", 0), xc="pbe_x", **kw)


def terms(E):
    return sum(abs(E[k]) for k in ("kin", "loc", "nl", "H", "x_M", "x_T"))


@pytest.mark.parametrize("name", list(CASES))
def test_pbe_exchange_potentials_energies_apply_fp64(name):
    cfg = cfg_of(**CASES[name])
    roks = built()
    ctx = roks.Context(cfg, "fp64")
    s = R.System(cfg)
    u = syn.orbital_uniforms(cfg, ctx.npw)
    psi = ctx.init_orbitals(u)
    P = s.initial_orbitals(u)
    rho = ctx.density(psi, want_rho=True).cpu().numpy()
    rho_ref = s.class_densities(P)
    assert rel(rho, rho_ref) < TOL64
    E, V = ctx.potential(want_v=True)
    pot = s.potentials(rho_ref)
    Eref = s.energies(P, pot)
    assert rel(V.cpu().numpy(), pot.Vk) < TOL64
    # the gradient correction is really there
    sl = R.System(syn.with_changes(cfg, xc="slater"))
    assert abs(Eref["x_M"] - sl.energies(P)["x_M"]) > 1e-3 * abs(Eref["x_M"])
    for k_gpu, k_ref in (("E_kin", "kin"), ("E_loc", "loc"), ("E_nl", "nl"), ("E_H", "H"), ("E_x_M", "x_M"),
                         ("E_x_T", "x_T"), ("E_total", "total")):
        assert abs(E[k_gpu] - Eref[k_ref]) <= TOL64 * max(1.0, abs(Eref[k_ref])), k_gpu
    f, sp, g = ctx.apply_h(psi, want_s=True, want_grad=True)
    F_ref, S_ref = s.apply(P, pot)
    assert rel(to_np(f, s.npw), F_ref) < TOL64
    assert rel(to_np(sp, s.npw), S_ref) < TOL64
    _, G_ref, _, _ = R.gradient_parts(P, F_ref, S_ref)
    assert rel(to_np(g, s.npw), G_ref) < 1e-9


@pytest.mark.parametrize("variant", ["singlet", "triplet", "empty"])
def test_pbe_exchange_trajectory_fp64(variant):
    kw = {"singlet": {}, "triplet": dict(mode=2), "empty": dict(n_empty=2)}[variant]
    cfg = cfg_of(**kw)
    roks = built()
    ctx = roks.Context(cfg, "fp64")
    s = R.System(cfg)
    u = syn.orbital_uniforms(cfg, ctx.npw)
    psi = ctx.init_orbitals(u)
    P = s.initial_orbitals(u)
    pcg = R.PCG(s)
    for it in range(8):
        info = ctx.pcg_step(psi)
        P, ref = pcg.step(P)
        assert abs(info["E_new"] - ref.E_new) <= TOL64 * max(1, abs(ref.E_new)), (it, info["E_new"], ref.E_new)
        assert abs(info["step"] - ref.step) <= 1e-8 * ref.step
        assert abs(info["grad_norm"] - ref.grad_norm) <= 1e-9 * ref.grad_norm
    assert rel(to_np(psi, s.npw), P) < 1e-8


def test_pbe_exchange_forces_fp64():
    cfg = cfg_of()
    roks = built()
    ctx = roks.Context(cfg, "fp64")
    s = R.System(cfg)
    psi = ctx.init_orbitals(syn.orbital_uniforms(cfg, ctx.npw))
    for _ in range(3):
        ctx.pcg_step(psi)
    Fgpu = ctx.forces(psi)
    Fref = Fo.forces(s, to_np(psi, s.npw))
    assert np.abs(Fgpu - Fref).max() < 1e-9 * max(1.0, np.abs(Fref).max())


def test_pbe_exchange_gamma_point_fp64():
    """Half-sphere (real orbitals) steps against the oracle's full-sphere
    steps from the same real start: the exchange grid pass is the complex
    path's, on the packed transforms' densities."""
    from tests.test_gpu_gamma import to_full
    cfg = cfg_of()
    roks = built()
    ctx = roks.Context(cfg, "fp64", gamma=1)
    s = R.System(cfg)
    u = syn.orbital_uniforms(cfg, ctx.npw)
    psi = ctx.init_orbitals(u)
    P = Gm.initial_orbitals(s, u)
    pcg = R.PCG(s)
    for it in range(6):
        info = ctx.pcg_step(psi)
        P, ref = pcg.step(P)
        assert abs(info["E_new"] - ref.E_new) <= TOL64 * max(1, abs(ref.E_new)), (it, info["E_new"], ref.E_new)
    assert rel(to_full(s, to_np(psi, ctx.npw)), P) < 1e-8


@pytest.mark.parametrize("name", ["tiny16-singlet", "grid32"])
def test_pbe_exchange_mixed(name):
    cfg = cfg_of(**CASES[name])
    roks = built()
    ctx = roks.Context(cfg, "mixed")
    s = R.System(cfg)
    u = syn.orbital_uniforms(cfg, ctx.npw)
    P = s.initial_orbitals(u)
    psi = to_dev(ctx, P)
    rho_ref = s.class_densities(P)
    ctx.density(psi)
    E, V = ctx.potential(want_v=True)
    pot = s.potentials(rho_ref)
    Eref = s.energies(P, pot)
    assert rel(V.cpu().numpy(), pot.Vk) < 2e-6
    assert abs(E["E_total"] - Eref["total"]) < 2e-7 * terms(Eref)
    assert abs(E["E_x_M"] - Eref["x_M"]) < 2e-7 * terms(Eref)
    f, sp, _ = ctx.apply_h(psi)
    F_ref, S_ref = s.apply(P, pot)
    assert rel(to_np(f, s.npw), F_ref) < 2e-5


def test_pbe_exchange_mixed_trajectory():
    cfg = cfg_of()
    roks = built()
    ctx = roks.Context(cfg, "mixed")
    s = R.System(cfg)
    u = syn.orbital_uniforms(cfg, ctx.npw)
    psi = ctx.init_orbitals(u)
    P = s.initial_orbitals(u)
    pcg = R.PCG(s)
    for it in range(20):
        info = ctx.pcg_step(psi)
        P, ref = pcg.step(P)
        assert abs(info["E_new"] - ref.E_new) < 1e-6 * terms(s.energies(P)), (it, info["E_new"], ref.E_new)


def test_pbe_exchange_with_exact_exchange_fp64():
    """The hybrid: (1 - alpha) PBE exchange beside alpha exact exchange."""
    cfg = cfg_of(alpha=1.0 / 3.0)
    roks = built()
    ctx = roks.Context(cfg, "fp64")
    s = R.System(cfg)
    u = syn.orbital_uniforms(cfg, ctx.npw)
    psi = ctx.init_orbitals(u)
    P = s.initial_orbitals(u)
    ctx.density(psi)
    E, V = ctx.potential(want_v=True)
    pot = s.potentials(s.class_densities(P))
    Eref = s.energies(P, pot)
    assert rel(V.cpu().numpy(), pot.Vk) < TOL64
    assert abs(E["E_total"] - Eref["total"]) <= TOL64 * max(1.0, abs(Eref["total"]))
    f, _, _ = ctx.apply_h(psi)
    F_ref, _ = s.apply(P, pot)
    assert rel(to_np(f, s.npw), F_ref) < TOL64
