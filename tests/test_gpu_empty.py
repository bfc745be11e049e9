"""GPU parity of the empty shell (Eq. 20, fourth row and column): n_empty
unoccupied bands after a, b, through the C ABI against the oracle on the
same seeded start.

* FP64 (1e-10): the apply (F^c on the empty bands), the energy's gradient
  g (F^e = 0) and the empty bands' F^c residual g_I, the densities and
  energies (occupied bands only), and 8-step PCG trajectories (energies,
  step, Fletcher-Reeves ratio from the occupied bands, restarts, |g|) for
  the ground state, the singlet with and without the a-b coupling, and the
  triplet;
* the converged ground state with two empty bands: energy of the run
  without them, and the empty bands' Ritz values the next eigenvalues of
  the dense F^c x = e S x;
* forces: those of the occupied bands;
* mixed precision: after every one of 20 singlet steps, and of 2 steps
  with 72 bands (the blocked band-space kernels), the energy within 1e-6
  of the sum of the energy terms' magnitudes of the oracle's point (FP32
  arithmetic on a trajectory whose first steps drop E by several Ha); the
  converged ground state with two empty bands (|dE| < 1e-8 twice and
  |g| < 1e-4) within 1e-5 Ha of the FP64 oracle's, its empty bands' Ritz
  values within 1e-5 of the dense ones;
* what the empty shell does not combine with is refused: DIIS, exact
  exchange, the Gamma-point form."""
import numpy as np
import pytest
import scipy.linalg

from oracle import forces as Fo
from oracle import roks as R
from paper_2605_28637_gb300 import synthetic as syn
from tests.gpu_helpers import built, rel, to_dev, to_np

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


def cfg_of(**kw):
    return syn.with_changes(syn.make_config("tiny-16", 0), **kw)


VARIANTS = {
    "gs": dict(mode=0, n_closed=5, n_empty=2),
    "singlet": dict(n_empty=3),
    "suppress": dict(n_empty=2),
    "triplet": dict(mode=2, n_empty=2),
}


@pytest.mark.parametrize("variant", list(VARIANTS))
def test_empty_shell_trajectory_fp64(variant):
    cfg = cfg_of(**VARIANTS[variant])
    sup = variant == "suppress"
    roks = built()
    ctx = roks.Context(cfg, "fp64", suppress_ab=sup)
    s = R.System(cfg)
    assert ctx.nb == s.nb == s.n_occ + s.n_empty
    u = syn.orbital_uniforms(cfg, ctx.npw)
    psi = ctx.init_orbitals(u)
    P = s.initial_orbitals(u)
    assert rel(to_np(psi, s.npw), P) < 1e-12
    pcg = R.PCG(s, suppress_ab=sup)
    for it in range(8):
        info = ctx.pcg_step(psi)
        P, ref = pcg.step(P)
        assert abs(info["E"] - ref.E) <= TOL64 * max(1, abs(ref.E)), (it, info["E"], ref.E)
        assert abs(info["E_new"] - ref.E_new) <= TOL64 * max(1, abs(ref.E_new)), (it, info["E_new"], ref.E_new)
        assert abs(info["step"] - ref.step) <= 1e-8 * ref.step, (it, info["step"], ref.step)
        assert abs(info["beta"] - ref.beta) <= 1e-8 * max(1, abs(ref.beta)), (it, info["beta"], ref.beta)
        assert bool(info["restarted"]) == ref.restarted
        assert abs(info["grad_norm"] - ref.grad_norm) <= 1e-9 * ref.grad_norm
    assert rel(to_np(psi, s.npw), P) < 1e-8


def test_empty_shell_apply_gradient_density_fp64():
    cfg = cfg_of(n_empty=3)
    roks = built()
    ctx = roks.Context(cfg, "fp64")
    s = R.System(cfg)
    u = syn.orbital_uniforms(cfg, ctx.npw)
    psi = ctx.init_orbitals(u)
    P = s.initial_orbitals(u)
    rho = ctx.density(psi, want_rho=True).cpu().numpy()
    rho_ref = s.class_densities(P)
    assert rel(rho, rho_ref) < 1e-12
    E = ctx.potential()
    Eref = s.energies(P)
    assert abs(E["E_total"] - Eref["total"]) < TOL64 * abs(Eref["total"])
    pot = s.potentials(rho_ref)
    F_ref, S_ref = s.apply(P, pot)
    f, sp, g, gi = ctx.gradient_parts(psi)
    assert rel(to_np(f, s.npw), F_ref) < TOL64
    assert rel(to_np(sp, s.npw), S_ref) < TOL64
    Th, G, gI, Gin = R.gradient_parts(P, F_ref, S_ref, s.empty)
    assert rel(to_np(g, s.npw), G) < 1e-9
    assert rel(to_np(gi, s.npw), gI) < 1e-9
    # the occupied energy's operator of an empty band is zero: its gradient
    # column lies in the span of S Psi
    ge = to_np(g, s.npw)[:, s.n_occ:]
    assert np.abs(ge - S_ref @ (P.conj().T @ ge)).max() < 1e-10 * np.abs(G).max()


def test_empty_shell_ground_state_converges_to_the_next_eigenvectors():
    """FP64, 2 empty bands: converged to the energy of the run without them,
    with the empty bands' Ritz values the 6th and 7th eigenvalues of the
    dense F^c x = e S x at the GPU's converged density."""
    cfg = cfg_of(mode=0, n_closed=5, n_empty=2)
    roks = built()
    ctx = roks.Context(cfg, "fp64", e_tol=1e-11)
    s = R.System(cfg)
    psi = ctx.init_orbitals(syn.orbital_uniforms(cfg, ctx.npw))
    for _ in range(300):
        info = ctx.pcg_step(psi)
        if info["converged"]:
            break
    assert info["converged"]
    cfg0 = syn.with_changes(cfg, n_empty=0)
    s0 = R.System(cfg0)
    P0, h0 = R.run(s0, s0.initial_orbitals(syn.orbital_uniforms(cfg0, s0.npw)), max_iter=600, e_tol=1e-11)
    assert info["E_new"] == pytest.approx(h0[-1].E_new, abs=1e-8)
    P = to_np(psi, s.npw)
    pot = s.potentials(s.class_densities(P))
    I = np.eye(s.npw, dtype=complex)
    H, Sm = s.apply(I, pot, classes=np.zeros(s.npw, dtype=int), occ=P[:, :s.n_occ])
    ev = scipy.linalg.eigh(0.5 * (H + H.conj().T), 0.5 * (Sm + Sm.conj().T), eigvals_only=True)
    Fc, _ = s.apply(P, pot, classes=np.zeros(s.nb, dtype=int), occ=P[:, :s.n_occ])
    Th = P.conj().T @ Fc
    emp = np.sort(np.linalg.eigvalsh(0.5 * (Th[5:, 5:] + Th[5:, 5:].conj().T)))
    assert np.allclose(emp, ev[5:7], atol=2e-6), (emp, ev[5:8])


def test_empty_shell_forces_fp64():
    cfg = cfg_of(n_empty=2)
    roks = built()
    ctx = roks.Context(cfg, "fp64")
    s = R.System(cfg)
    u = syn.orbital_uniforms(cfg, ctx.npw)
    psi = ctx.init_orbitals(u)
    for _ in range(3):
        ctx.pcg_step(psi)
    Fgpu = ctx.forces(psi)
    Fref = Fo.forces(s, to_np(psi, s.npw))
    assert np.abs(Fgpu - Fref).max() < 1e-9 * max(1.0, np.abs(Fref).max())


def terms(s, P):
    E = s.energies(P)
    return sum(abs(E[k]) for k in ("kin", "loc", "nl", "H", "x_M", "x_T"))


def test_empty_shell_mixed_singlet():
    cfg = cfg_of(n_empty=3)
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
        assert abs(info["E_new"] - ref.E_new) < 1e-6 * terms(s, P), (it, info["E_new"], ref.E_new)


def test_empty_shell_mixed_ground_state_converged():
    cfg = cfg_of(mode=0, n_closed=5, n_empty=2)
    roks = built()
    ctx = roks.Context(cfg, "mixed", e_tol=1e-8, g_tol=1e-4)
    s = R.System(cfg)
    psi = ctx.init_orbitals(syn.orbital_uniforms(cfg, ctx.npw))
    for _ in range(600):
        info = ctx.pcg_step(psi)
        if info["converged"]:
            break
    assert info["converged"]
    P, h = R.run(s, s.initial_orbitals(syn.orbital_uniforms(cfg, s.npw)), max_iter=600, e_tol=1e-11)
    assert abs(info["E_new"] - h[-1].E_new) < 1e-5
    X = to_np(psi, s.npw)
    pot = s.potentials(s.class_densities(X))
    I = np.eye(s.npw, dtype=complex)
    H, Sm = s.apply(I, pot, classes=np.zeros(s.npw, dtype=int), occ=X[:, :s.n_occ])
    ev = scipy.linalg.eigh(0.5 * (H + H.conj().T), 0.5 * (Sm + Sm.conj().T), eigvals_only=True)
    Fc, _ = s.apply(X, pot, classes=np.zeros(s.nb, dtype=int), occ=X[:, :s.n_occ])
    Th = X.conj().T @ Fc
    emp = np.sort(np.linalg.eigvalsh(0.5 * (Th[5:, 5:] + Th[5:, 5:].conj().T)))
    assert np.allclose(emp, ev[5:7], atol=1e-5), (emp, ev[5:8])


def test_empty_shell_many_bands_mixed():
    """64 closed, a, b and 6 empty bands (72: the blocked Cholesky and
    exponential, the band-space products for more than 64 bands)."""
    cfg = cfg_of(grid=32, L=14.0, ecut=16.0, n_closed=64, n_empty=6)
    roks = built()
    ctx = roks.Context(cfg, "mixed")
    s = R.System(cfg)
    u = syn.orbital_uniforms(cfg, ctx.npw)
    psi = ctx.init_orbitals(u)
    assert np.abs(s.overlap(to_np(psi, s.npw)) - np.eye(s.nb)).max() < 5e-6
    P = s.initial_orbitals(u)
    pcg = R.PCG(s)
    for it in range(2):
        info = ctx.pcg_step(psi)
        P, ref = pcg.step(P)
        assert abs(info["E_new"] - ref.E_new) < 1e-6 * terms(s, P), (it, info["E_new"], ref.E_new)


def test_empty_shell_refusals():
    roks = built()
    cfg = cfg_of(n_empty=2)
    ctx = roks.Context(cfg, "fp64")
    psi = ctx.init_orbitals(syn.orbital_uniforms(cfg, ctx.npw))
    with pytest.raises(roks.RoksError) as ei:
        ctx.diis_step(psi)
    assert ei.value.status == roks.ROKS_EINVAL
    for bad in (dict(alpha=1.0 / 3.0), dict(gamma=1)):
        kw = {}
        c = cfg
        if "alpha" in bad:
            c = syn.with_changes(cfg, alpha=bad["alpha"])
        else:
            kw["gamma"] = 1
        with pytest.raises(roks.RoksError) as ei:
            roks.Context(c, "fp64", **kw)
        assert ei.value.status == roks.ROKS_EINVAL
