"""GPU parity of the Gamma-point path (roks_options.gamma): real orbitals on
the half sphere, two per complex transform, against the full-sphere FP64
oracle run from the same symmetric start (oracle/gamma.py).

Every step of the method maps real orbitals to real orbitals (real
potentials, real-space-real projectors, real band-space matrices), so the
oracle's full-sphere computation from a start with c(-G) = conj c(G) is the
Gamma-point method; the library stores c(0) and sqrt(2) c(G) for the other
half-sphere G, and the tests convert between the two forms (to_full,
to_half).  Bars: FP64 1e-10 relative as on the complex path; mixed
precision the complex path's mixed bars."""
import numpy as np
import pytest

from oracle import diis as D
from oracle import forces as Fo
from oracle import gamma as Gm
from oracle import roks as R
from paper_2605_28637_gb300 import synthetic as syn
from tests.gpu_helpers import built, rel, to_dev, to_np

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
SQ2 = np.sqrt(2.0)

VARIANTS = {
    "tiny16-singlet": dict(),
    "tiny16-triplet": dict(mode=2),
    "tiny16-gs-odd": dict(mode=0, n_closed=5),      # one packed band holds a single orbital
    "grid24": dict(grid=24, L=11.0, ecut=12.0, n_closed=4),
    "grid32": dict(grid=32, L=12.0, ecut=20.0, n_closed=6),
}


def cfg_of(**kw):
    return syn.with_changes(syn.make_config("tiny-16", 0), **kw)


def to_full(s, Xh):
    """Stored half-sphere form (rows 1.. times sqrt 2) -> full coefficients."""
    c = np.array(Xh, dtype=np.complex128)
    c[1:] /= SQ2
    return Gm.expand(s, c)


def to_half(s, Xf):
    c = Gm.restrict(s, Xf)
    c[1:] *= SQ2
    return c


def start(cfg, precision="fp64", **opt):
    roks = built()
    ctx = roks.Context(cfg, precision, gamma=1, **opt)
    s = R.System(cfg)
    u = syn.orbital_uniforms(cfg, ctx.npw)
    psi = ctx.init_orbitals(u)
    return roks, ctx, s, psi, Gm.initial_orbitals(s, u)


@pytest.mark.parametrize("name", list(VARIANTS))
def test_gamma_basis_is_the_half_sphere(name):
    cfg = cfg_of(**VARIANTS[name])
    roks = built()
    ctx = roks.Context(cfg, "fp64", gamma=1)
    s = R.System(cfg)
    h = Gm.half_index(s)
    assert ctx.npw == len(h) == (s.npw + 1) // 2
    assert np.array_equal(ctx.miller, s.miller[h])
    assert np.all(ctx.miller[0] == 0)             # G = 0 first
    ctx.close()


@pytest.mark.parametrize("name", list(VARIANTS))
def test_gamma_density_potential_apply_fp64(name):
    cfg = cfg_of(**VARIANTS[name])
    roks, ctx, s, psi, P_ref = start(cfg)
    P = to_np(psi, ctx.npw)
    assert np.all(P[0].imag == 0.0)                # c(0) real
    assert rel(to_full(s, P), P_ref) < TOL64
    rho = ctx.density(psi, want_rho=True).cpu().numpy()
    rho_ref = s.class_densities(P_ref)
    assert rel(rho, rho_ref) < TOL64
    E, V = ctx.potential(want_v=True)
    pot = s.potentials(rho_ref)
    Eref = s.energies(P_ref, pot)
    assert rel(V.cpu().numpy(), pot.Vk) < TOL64
    for k_gpu, k_ref in (("E_kin", "kin"), ("E_loc", "loc"), ("E_nl", "nl"), ("E_H", "H"), ("E_x_M", "x_M"),
                         ("E_x_T", "x_T"), ("E_M", "M"), ("E_T", "T"), ("E_total", "total")):
        assert abs(E[k_gpu] - Eref[k_ref]) <= TOL64 * max(1.0, abs(Eref[k_ref])), k_gpu
    f, sp, g = ctx.apply_h(psi, want_s=True, want_grad=True)
    F_ref, S_ref = s.apply(P_ref, pot)
    assert rel(to_np(f, ctx.npw), to_half(s, F_ref)) < TOL64
    assert rel(to_np(sp, ctx.npw), to_half(s, S_ref)) < TOL64
    _, G_ref, _, _ = R.gradient_parts(P_ref, F_ref, S_ref)
    assert rel(to_np(g, ctx.npw), to_half(s, G_ref)) < 1e-9
    ctx.close()


@pytest.mark.parametrize("name", ["tiny16-singlet", "tiny16-triplet", "tiny16-gs-odd", "grid32"])
def test_gamma_pcg_trajectory_fp64(name):
    cfg = cfg_of(**VARIANTS[name])
    roks, ctx, s, psi, P = start(cfg)
    pcg = R.PCG(s)
    for it in range(8):
        info = ctx.pcg_step(psi)
        P, ref = pcg.step(P)
        assert abs(info["E"] - ref.E) <= TOL64 * max(1, abs(ref.E)), (it, info["E"], ref.E)
        assert abs(info["E_new"] - ref.E_new) <= TOL64 * max(1, abs(ref.E_new)), (it, info["E_new"], ref.E_new)
        assert abs(info["step"] - ref.step) <= 1e-8 * ref.step
        assert abs(info["beta"] - ref.beta) <= 1e-8 * max(1, abs(ref.beta))
        assert bool(info["restarted"]) == ref.restarted
        assert abs(info["grad_norm"] - ref.grad_norm) <= 1e-9 * ref.grad_norm
    assert rel(to_full(s, to_np(psi, ctx.npw)), P) < 1e-8
    # the oracle's full-sphere orbitals stayed real (the Gamma-point method)
    assert Gm.realness(s, P) < 1e-12
    ctx.close()


def test_gamma_matches_the_complex_path_on_the_gpu():
    """The same real start stepped by the complex path (full sphere) and by
    the Gamma-point path: the same energies step by step."""
    cfg = cfg_of()
    roks, ctx_g, s, psi_g, P0 = start(cfg)
    ctx_c = roks.Context(cfg, "fp64")
    psi_c = to_dev(ctx_c, P0)
    ctx_c.orthonormalize(psi_c)
    for it in range(10):
        a = ctx_g.pcg_step(psi_g)
        b = ctx_c.pcg_step(psi_c)
        assert abs(a["E_new"] - b["E_new"]) <= TOL64 * abs(b["E_new"]), (it, a["E_new"], b["E_new"])
    ctx_g.close()
    ctx_c.close()


@pytest.mark.parametrize("name", ["tiny16-singlet", "grid32"])
def test_gamma_mixed_precision(name):
    """Mixed path: densities 2e-6, F and S 2e-5 / 2e-6 relative, energies
    2e-5 Ha, against the oracle on the GPU's own (expanded) orbitals."""
    cfg = cfg_of(**VARIANTS[name])
    roks, ctx, s, psi, P_ref = start(cfg, "mixed")
    P = to_full(s, to_np(psi, ctx.npw))
    assert np.abs(s.overlap(P) - np.eye(s.nb)).max() < 3e-6
    rho = ctx.density(psi, want_rho=True).cpu().numpy()
    assert rel(rho, s.class_densities(P)) < 2e-6
    E = ctx.potential()
    assert abs(E["E_total"] - s.energy(P)) < 2e-5
    f, sp, _ = ctx.apply_h(psi)
    F_ref, S_ref = s.apply(P, s.potentials(s.class_densities(P)))
    assert rel(to_np(f, ctx.npw), to_half(s, F_ref)) < 2e-5
    assert rel(to_np(sp, ctx.npw), to_half(s, S_ref)) < 2e-6
    # a few steps stay real and descend
    e0 = E["E_total"]
    for _ in range(5):
        info = ctx.pcg_step(psi)
    assert info["E_new"] < e0
    assert np.all(to_np(psi, ctx.npw)[0].imag == 0.0)
    ctx.close()


def test_gamma_forces_fp64():
    cfg = cfg_of()
    roks, ctx, s, psi, _ = start(cfg)
    for _ in range(4):
        ctx.pcg_step(psi)
    F = ctx.forces(psi)
    ref = Fo.forces(s, to_full(s, to_np(psi, ctx.npw)))
    assert np.abs(F - ref).max() < 1e-9 * np.abs(ref).max(), (F, ref)
    ctx.close()


def test_gamma_diis_fp64():
    cfg = cfg_of()
    roks, ctx, s, psi, P = start(cfg)
    dz = D.DIIS(s)
    for it in range(6):
        info = ctx.diis_step(psi)
        P, ref = dz.step(P)
        assert abs(info["E_new"] - ref.E_new) <= TOL64 * max(1, abs(ref.E_new)), (it, info["E_new"], ref.E_new)
        assert abs(info["res_norm"] - ref.res_norm) <= 1e-9 * ref.res_norm
        assert info["window"] == ref.window
    assert rel(to_full(s, to_np(psi, ctx.npw)), P) < 1e-8
    ctx.close()


def test_gamma_rejects_what_it_does_not_pack():
    roks = built()
    with pytest.raises(roks.RoksError):
        roks.Context(cfg_of(alpha=0.25), "fp64", gamma=1)          # exact exchange: complex path only
    with pytest.raises(roks.RoksError):
        roks.Context(cfg_of(n_closed=5), "fp64", gamma=1)          # open pair split across packed bands
    ctx = roks.Context(cfg_of(mode=0, n_closed=5), "fp64", gamma=1)  # ground state: any count
    ctx.close()
