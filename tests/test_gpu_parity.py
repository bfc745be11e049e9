"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs.

FP64 path: 1e-10 relative (element by element on small cases).  Mixed path
(FP32 transforms and contractions, FP64 reductions and Cholesky): the
tolerances stated in each test, derived from FP32 rounding (2^-24 per
operation, a few hundred operations deep)."""
import numpy as np
import pytest

from oracle import roks as R
from paper_2605_28637_gb300 import synthetic as syn
from tests.gpu_helpers import built, rel, to_dev, to_np

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


def cfg_of(name="tiny-16", **kw):
    return syn.with_changes(syn.make_config(name, 0), **kw)


# variants spanning every compiled grid size that the oracle finishes quickly,
# with ragged tiles and both the singlet, triplet and ground-state modes
SMALL = {
    "tiny16-singlet": dict(),
    "tiny16-triplet": dict(mode=2),
    "tiny16-gs": dict(mode=0, n_closed=5),
    "grid24": dict(grid=24, L=11.0, ecut=12.0, n_closed=5),
    "grid32": dict(grid=32, L=12.0, ecut=20.0, n_closed=6),
    "grid48": dict(grid=48, L=12.0, ecut=35.0, n_closed=3),
}


def setup_pair(cfg, precision="fp64"):
    roks = built()
    ctx = roks.Context(cfg, precision)
    s = R.System(cfg)
    return roks, ctx, s


@pytest.mark.parametrize("name", list(SMALL))
def test_basis_bit_exact(name):
    cfg = cfg_of(**SMALL[name])
    roks, ctx, s = setup_pair(cfg)
    assert ctx.npw == s.npw
    assert np.array_equal(ctx.miller, s.miller)
    ctx.close()


@pytest.mark.parametrize("name", list(SMALL))
def test_density_potential_apply_fp64(name):
    cfg = cfg_of(**SMALL[name])
    roks, ctx, s = setup_pair(cfg)
    u = syn.orbital_uniforms(cfg, ctx.npw)
    psi = ctx.init_orbitals(u)
    P_ref = s.initial_orbitals(u)
    assert rel(to_np(psi, s.npw), P_ref) < TOL64
    # densities
    rho = ctx.density(psi, want_rho=True).cpu().numpy()
    rho_ref = s.class_densities(P_ref)
    assert rel(rho, rho_ref) < TOL64
    # potentials and energies
    E, V = ctx.potential(want_v=True)
    pot = s.potentials(rho_ref)
    Eref = s.energies(P_ref, pot)
    assert rel(V.cpu().numpy(), pot.Vk) < TOL64
    for k_gpu, k_ref in (("E_kin", "kin"), ("E_loc", "loc"), ("E_nl", "nl"), ("E_H", "H"), ("E_x_M", "x_M"),
                         ("E_x_T", "x_T"), ("E_M", "M"), ("E_T", "T"), ("E_total", "total")):
        assert abs(E[k_gpu] - Eref[k_ref]) <= TOL64 * max(1.0, abs(Eref[k_ref])), k_gpu
    # F|n>, S|n>, g_n
    f, sp, g = ctx.apply_h(psi, want_s=True, want_grad=True)
    F_ref, S_ref = s.apply(P_ref, pot)
    assert rel(to_np(f, s.npw), F_ref) < TOL64
    assert rel(to_np(sp, s.npw), S_ref) < TOL64
    _, G_ref, _, _ = R.gradient_parts(P_ref, F_ref, S_ref)
    assert rel(to_np(g, s.npw), G_ref) < 1e-9
    ctx.close()


def test_orthonormalize_fp64():
    cfg = cfg_of()
    roks, ctx, s = setup_pair(cfg)
    X = s.initial_orbitals(syn.orbital_uniforms(cfg, s.npw)) + 0.3 * syn.random_vectors(9, s.npw, s.nb)
    psi = to_dev(ctx, X)
    ctx.orthonormalize(psi)
    Y = to_np(psi, s.npw)
    assert rel(Y, s.orthonormalize(X)) < TOL64
    assert np.abs(s.overlap(Y) - np.eye(s.nb)).max() < 1e-12


def test_orthonormalize_rejects_singular_overlap():
    cfg = cfg_of()
    roks, ctx, s = setup_pair(cfg)
    X = s.initial_orbitals(syn.orbital_uniforms(cfg, s.npw))
    X[:, 1] = X[:, 0]                              # rank deficient
    psi = to_dev(ctx, X)
    with pytest.raises(roks.RoksError) as ei:
        ctx.orthonormalize(psi)
    assert ei.value.status == roks.ROKS_ENOTPOSDEF
    # the context stays usable
    psi = ctx.init_orbitals(syn.orbital_uniforms(cfg, s.npw))
    ctx.density(psi)
    ctx.potential()


def test_setup_rejects_bad_input():
    roks = built()
    with pytest.raises(roks.RoksError):
        roks.Context(cfg_of(grid=20))              # no compiled transform
    with pytest.raises(roks.RoksError):
        roks.Context(cfg_of(grid=16, ecut=40.0))   # sphere does not fit the grid
    ctx = roks.Context(cfg_of())
    import torch
    bad = torch.zeros((ctx.nb, ctx.npw - 1), dtype=torch.complex128, device="cuda")
    with pytest.raises(roks.RoksError):
        roks.roks_density(ctx.ctx, bad, ctx.npw - 1)


def test_no_projectors():
    cfg = cfg_of()
    cfg["species"] = [dict(l=[], m=[], rc=[], D=np.zeros((0, 0)), Q=np.zeros((0, 0)))]
    roks, ctx, s = setup_pair(cfg)
    assert s.nproj == 0
    u = syn.orbital_uniforms(cfg, ctx.npw)
    psi = ctx.init_orbitals(u)
    P_ref = s.initial_orbitals(u)
    ctx.density(psi)
    E = ctx.potential()
    assert abs(E["E_total"] - s.energy(P_ref)) < TOL64 * abs(s.energy(P_ref))


@pytest.mark.parametrize("variant", ["singlet", "suppress", "gs", "triplet"])
def test_pcg_trajectory_fp64(variant):
    kw = {"singlet": {}, "suppress": {}, "gs": dict(mode=0, n_closed=5), "triplet": dict(mode=2)}[variant]
    cfg = cfg_of(**kw)
    sup = variant == "suppress"
    roks = built()
    ctx = roks.Context(cfg, "fp64", suppress_ab=sup)
    s = R.System(cfg)
    u = syn.orbital_uniforms(cfg, ctx.npw)
    psi = ctx.init_orbitals(u)
    P = s.initial_orbitals(u)
    pcg = R.PCG(s, suppress_ab=sup)
    for it in range(8):
        info = ctx.pcg_step(psi)
        P, ref = pcg.step(P)
        assert abs(info["E"] - ref.E) <= TOL64 * max(1, abs(ref.E)), (it, info["E"], ref.E)
        assert abs(info["E_new"] - ref.E_new) <= TOL64 * max(1, abs(ref.E_new)), (it, info["E_new"], ref.E_new)
        assert abs(info["step"] - ref.step) <= 1e-8 * ref.step
        assert abs(info["beta"] - ref.beta) <= 1e-8 * max(1, abs(ref.beta))
        assert bool(info["restarted"]) == ref.restarted
        assert abs(info["grad_norm"] - ref.grad_norm) <= 1e-9 * ref.grad_norm
    assert rel(to_np(psi, s.npw), P) < 1e-8


def test_pcg_tiny_50_iterations_fp64():
    """The tiny workload's 50 iterations: energy after every step within
    1e-6 Ha of the oracle's trajectory (and 1e-9 relative for the first 20)."""
    cfg = cfg_of()
    roks = built()
    ctx = roks.Context(cfg, "fp64")
    s = R.System(cfg)
    u = syn.orbital_uniforms(cfg, ctx.npw)
    psi = ctx.init_orbitals(u)
    P = s.initial_orbitals(u)
    pcg = R.PCG(s)
    for it in range(50):
        info = ctx.pcg_step(psi)
        P, ref = pcg.step(P)
        tol = 1e-9 * abs(ref.E_new) if it < 20 else 1e-6
        assert abs(info["E_new"] - ref.E_new) <= tol, (it, info["E_new"], ref.E_new)


@pytest.mark.parametrize("name", ["tiny16-singlet", "grid32"])
def test_mixed_precision_apply(name):
    """FP32 path: densities to 2e-6 relative, F|n> and S|n> to 2e-5 relative
    (of the largest entry), energies to 2e-5 Ha."""
    cfg = cfg_of(**SMALL[name])
    roks, ctx, s = setup_pair(cfg, "mixed")
    u = syn.orbital_uniforms(cfg, ctx.npw)
    psi = ctx.init_orbitals(u)
    P_ref = s.initial_orbitals(u)
    assert rel(to_np(psi, s.npw), P_ref) < 2e-6
    rho = ctx.density(psi, want_rho=True).cpu().numpy()
    rho_ref = s.class_densities(P_ref)
    assert rel(rho, rho_ref) < 2e-6
    E = ctx.potential()
    Eref = s.energies(P_ref)
    assert abs(E["E_total"] - Eref["total"]) < 2e-5
    f, sp, _ = ctx.apply_h(to_dev(ctx, P_ref))
    pot = s.potentials(rho_ref)
    F_ref, S_ref = s.apply(P_ref, pot)
    assert rel(to_np(f, s.npw), F_ref) < 2e-5
    assert rel(to_np(sp, s.npw), S_ref) < 2e-6


@pytest.mark.parametrize("layout", ["odd_ld", "offset8"])
def test_mixed_apply_any_layout(layout):
    """The streamed FP32 contractions need 16-byte aligned blocks with an even
    leading dimension; other layouts take the general kernels.  Both give the
    oracle's F|n>, S|n> and orthonormal orbitals within the mixed tolerances."""
    import torch
    cfg = cfg_of(**SMALL["grid32"])
    roks, ctx, s = setup_pair(cfg, "mixed")
    u = syn.orbital_uniforms(cfg, ctx.npw)
    P_ref = s.initial_orbitals(u)
    ctx.density(to_dev(ctx, P_ref))
    ctx.potential()
    pad, off = (1, 0) if layout == "odd_ld" else (2, 1)
    ld = ctx.ld + pad
    if layout == "odd_ld":
        assert ld % 2 == 1

    def block(X=None):
        buf = torch.zeros((ctx.nb * ld + off,), dtype=ctx.cdtype, device="cuda")
        view = buf[off:].view(ctx.nb, ld)
        if X is not None:
            view[:, :s.npw] = torch.from_numpy(X.T.copy()).to(ctx.cdtype)
        return view

    psi = block(P_ref)
    f, sp = block(), block()
    roks.roks_apply_h(ctx.ctx, psi, ld, f, sp)
    F_ref, S_ref = s.apply(P_ref, s.potentials(s.class_densities(P_ref)))
    assert rel(to_np(f, s.npw), F_ref) < 2e-5
    assert rel(to_np(sp, s.npw), S_ref) < 2e-6
    # orthonormalisation in the same layout: Psi^H S Psi = 1
    roks.roks_orthonormalize(ctx.ctx, psi, ld)
    P = to_np(psi, s.npw)
    SP = s.apply(P, s.potentials(s.class_densities(P)))[1]
    assert np.abs(P.conj().T @ SP - np.eye(ctx.nb)).max() < 2e-6


def test_mixed_precision_pcg_tiny():
    """Mixed path follows the FP64 trajectory: |E_new - E_new(oracle)| < 1e-5 Ha
    over 20 iterations of the tiny workload."""
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
        assert abs(info["E_new"] - ref.E_new) < 1e-5, (it, info["E_new"], ref.E_new)


# ------------------------------------------------------------------ exact exchange
HYBRID = {
    "tiny16-hybrid": dict(alpha=1.0 / 3.0),
    "grid24-hybrid-2batches": dict(grid=24, L=11.0, ecut=12.0, n_closed=10, alpha=1.0 / 3.0),
}


@pytest.mark.parametrize("name", list(HYBRID))
def test_exact_exchange_fp64(name):
    """Pair integrals, exchange energies and F|n> with the exchange operator
    (truncated Coulomb kernel, alpha = 1/3) against the oracle, 1e-10."""
    cfg = cfg_of(**HYBRID[name])
    roks, ctx, s = setup_pair(cfg)
    u = syn.orbital_uniforms(cfg, ctx.npw)
    psi = ctx.init_orbitals(u)
    P_ref = s.initial_orbitals(u)
    ctx.density(psi)
    E = ctx.potential()
    Eref = s.energies(P_ref)
    for k_gpu, k_ref in (("E_hf_M", "hf_M"), ("E_hf_T", "hf_T"), ("E_x_M", "x_M"), ("E_total", "total")):
        assert abs(E[k_gpu] - Eref[k_ref]) <= TOL64 * max(1.0, abs(Eref[k_ref])), k_gpu
    f, sp, _ = ctx.apply_h(psi)
    pot = s.potentials(s.class_densities(P_ref))
    F_ref, _ = s.apply(P_ref, pot)
    assert rel(to_np(f, s.npw), F_ref) < TOL64


def test_exact_exchange_pcg_fp64():
    cfg = cfg_of(**HYBRID["tiny16-hybrid"])
    roks = built()
    ctx = roks.Context(cfg, "fp64")
    s = R.System(cfg)
    u = syn.orbital_uniforms(cfg, ctx.npw)
    psi = ctx.init_orbitals(u)
    P = s.initial_orbitals(u)
    pcg = R.PCG(s)
    for it in range(4):
        info = ctx.pcg_step(psi)
        P, ref = pcg.step(P)
        assert abs(info["E_new"] - ref.E_new) <= TOL64 * max(1, abs(ref.E_new)), (it, info["E_new"], ref.E_new)
        assert abs(info["step"] - ref.step) <= 1e-8 * ref.step


def test_exact_exchange_mixed():
    cfg = cfg_of(**HYBRID["grid24-hybrid-2batches"])
    roks, ctx, s = setup_pair(cfg, "mixed")
    u = syn.orbital_uniforms(cfg, ctx.npw)
    psi = ctx.init_orbitals(u)
    P_ref = s.initial_orbitals(u)
    ctx.density(psi)
    E = ctx.potential()
    Eref = s.energies(P_ref)
    assert abs(E["E_total"] - Eref["total"]) < 2e-5
    assert abs(E["E_hf_M"] - Eref["hf_M"]) < 2e-5
    f, _, _ = ctx.apply_h(to_dev(ctx, P_ref))
    pot = s.potentials(s.class_densities(P_ref))
    F_ref, _ = s.apply(P_ref, pot)
    assert rel(to_np(f, s.npw), F_ref) < 2e-5


# ------------------------------------------------------------------ more than 64 bands
def test_many_bands_blocked_paths_fp64():
    """70 bands (beyond the single-block band-space kernels): the blocked
    Cholesky inverse and the tiled exponential follow the oracle's PCG."""
    cfg = cfg_of(grid=32, L=14.0, ecut=16.0, n_closed=68)
    roks = built()
    ctx = roks.Context(cfg, "fp64")
    s = R.System(cfg)
    assert s.nb == 70
    u = syn.orbital_uniforms(cfg, ctx.npw)
    psi = ctx.init_orbitals(u)
    P = s.initial_orbitals(u)
    assert rel(to_np(psi, s.npw), P) < TOL64
    pcg = R.PCG(s)
    for it in range(2):
        info = ctx.pcg_step(psi)
        P, ref = pcg.step(P)
        assert abs(info["E_new"] - ref.E_new) <= TOL64 * max(1, abs(ref.E_new)), (it, info["E_new"], ref.E_new)


def test_many_bands_blocked_paths_mixed():
    cfg = cfg_of(grid=32, L=14.0, ecut=16.0, n_closed=68)
    roks = built()
    ctx = roks.Context(cfg, "mixed")
    s = R.System(cfg)
    u = syn.orbital_uniforms(cfg, ctx.npw)
    psi = ctx.init_orbitals(u)
    Y = to_np(psi, s.npw)
    assert np.abs(s.overlap(Y) - np.eye(s.nb)).max() < 5e-6
    P = s.initial_orbitals(u)
    pcg = R.PCG(s)
    for it in range(2):
        info = ctx.pcg_step(psi)
        P, ref = pcg.step(P)
        assert abs(info["E_new"] - ref.E_new) < 5e-5, (it, info["E_new"], ref.E_new)


def test_many_bands_ragged_orthonormalize_and_steps():
    """200 bands (six full 32-column blocks and a ragged one of 8): the
    blocked Cholesky with its inverse formed along the way, against the
    oracle's orthonormalisation (FP64, 1e-10) and two PCG steps (the
    Paterson-Stockmeyer exponential with the device's squarings); the mixed
    path's orthonormality at 200 bands."""
    cfg = cfg_of(grid=32, L=16.0, ecut=16.0, n_closed=198)
    roks = built()
    ctx = roks.Context(cfg, "fp64")
    s = R.System(cfg)
    assert s.nb == 200 and s.npw > 400
    X = s.initial_orbitals(syn.orbital_uniforms(cfg, s.npw)) + 0.3 * syn.random_vectors(4, s.npw, s.nb)
    psi = to_dev(ctx, X)
    ctx.orthonormalize(psi)
    assert rel(to_np(psi, s.npw), s.orthonormalize(X)) < TOL64
    u = syn.orbital_uniforms(cfg, ctx.npw)
    psi = ctx.init_orbitals(u)
    P = s.initial_orbitals(u)
    pcg = R.PCG(s)
    for it in range(2):
        info = ctx.pcg_step(psi)
        P, ref = pcg.step(P)
        assert abs(info["E_new"] - ref.E_new) <= TOL64 * max(1, abs(ref.E_new)), (it, info["E_new"], ref.E_new)
    ctx.close()
    ctx = roks.Context(cfg, "mixed")
    psi = to_dev(ctx, X)
    ctx.orthonormalize(psi)
    Y = to_np(psi, s.npw)
    assert np.abs(s.overlap(Y) - np.eye(s.nb)).max() < 5e-6
    ctx.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_gradient_parts(precision):
    """roks_gradient_parts: F, S, g = F - S gamma and g_I = F - S theta (Eqs. 7,
    11, 12) against the oracle on the GPU's own orbitals (FP64 1e-9, mixed
    2e-5 of the largest entry)."""
    cfg = cfg_of()
    roks, ctx, s = setup_pair(cfg, precision)
    psi = ctx.init_orbitals(syn.orbital_uniforms(cfg, ctx.npw))
    P = to_np(psi, s.npw)
    ctx.density(psi)
    ctx.potential()
    f, sp, g, gi = ctx.gradient_parts(psi)
    F_ref, S_ref = s.apply(P, s.potentials(s.class_densities(P)))
    _, G_ref, gI_ref, _ = R.gradient_parts(P, F_ref, S_ref)
    bar = 1e-9 if precision == "fp64" else 2e-5
    assert rel(to_np(f, s.npw), F_ref) < bar
    assert rel(to_np(g, s.npw), G_ref) < bar
    assert rel(to_np(gi, s.npw), gI_ref) < bar
    ctx.close()
