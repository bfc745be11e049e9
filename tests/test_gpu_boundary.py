"""The C-ABI options and failure handling on the GPU.

* Seeded start: orbitals drawn on the device from SplitMix64 (roks_init_orbitals
  without host numbers) equal, bit for bit, those built from the host draws.
* A wait cap below zero makes every bounded mbarrier wait of the streamed
  contractions give up at once: the step returns ROKS_ETIMEOUT (no GPU fault,
  no hang) and the GPU stays usable.
* A non-finite orbital coefficient written on the host gives ROKS_EDIVERGED.
* max_iter: ROKS_ENOCONV on the max_iter-th step without convergence.
* The gradient criterion g_tol holds convergence back until |g| < g_tol.
* Option and occupation checks return ROKS_EINVAL.
* The bare exact-exchange kernel against the oracle (1e-10).
* The learned preconditioner selected at setup with all-zero weights steps
  exactly like TPA (the network's output is zero, so its factor is one).
* More than 128 bands and 376 projectors: the tiled band-space products
  follow the oracle's PCG."""
import ctypes as C

import numpy as np
import pytest

from oracle import roks as R
from paper_2605_28637_gb300 import synthetic as syn
from tests.gpu_helpers import built, rel, to_np

pytestmark = pytest.mark.gpu


def tiny(**kw):
    return syn.with_changes(syn.make_config("tiny-16", 0), **kw)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_seeded_start_on_device_is_bit_exact(precision):
    roks = built()
    cfg = tiny()
    ctx = roks.Context(cfg, precision)
    a = ctx.init_orbitals(syn.orbital_uniforms(cfg, ctx.npw))
    b = ctx.new_bands()
    roks.roks_init_orbitals(ctx.ctx, None, b, ctx.ld)
    assert bool((a == b).all())
    ctx.close()


def test_wait_cap_timeout_returns_status():
    roks = built()
    cfg = tiny()
    ctx = roks.Context(cfg, "mixed", wait_cap=-1)
    with pytest.raises(roks.RoksError) as ei:
        ctx.init_orbitals(syn.orbital_uniforms(cfg, ctx.npw))
    assert ei.value.status == roks.ROKS_ETIMEOUT
    ctx.close()
    # the GPU and a context with the default cap work as before
    ctx = roks.Context(cfg, "mixed")
    psi = ctx.init_orbitals(syn.orbital_uniforms(cfg, ctx.npw))
    info = ctx.pcg_step(psi)
    assert np.isfinite(info["E_new"])
    ctx.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_nan_orbital_gives_ediverged(precision):
    import torch
    roks = built()
    cfg = tiny()
    ctx = roks.Context(cfg, precision)
    psi = ctx.init_orbitals(syn.orbital_uniforms(cfg, ctx.npw))
    ctx.pcg_step(psi)
    host = psi.cpu()
    host[1, 7] = complex(float("nan"), 0.0)
    psi.copy_(host)
    torch.cuda.synchronize()
    ctx.invalidate()
    with pytest.raises(roks.RoksError) as ei:
        ctx.pcg_step(psi)
    assert ei.value.status == roks.ROKS_EDIVERGED
    # new orbitals bring the context back
    psi = ctx.init_orbitals(syn.orbital_uniforms(cfg, ctx.npw))
    assert np.isfinite(ctx.pcg_step(psi)["E_new"])
    ctx.close()


def test_max_iter_gives_enoconv():
    roks = built()
    cfg = tiny()
    ctx = roks.Context(cfg, "fp64", max_iter=3)
    psi = ctx.init_orbitals(syn.orbital_uniforms(cfg, ctx.npw))
    ctx.pcg_step(psi)
    ctx.pcg_step(psi)
    with pytest.raises(roks.RoksError) as ei:
        ctx.pcg_step(psi)
    assert ei.value.status == roks.ROKS_ENOCONV
    ctx.close()


def test_gradient_criterion_holds_convergence_back():
    roks = built()
    cfg = tiny()
    loose = roks.Context(cfg, "fp64", e_tol=100.0)
    strict = roks.Context(cfg, "fp64", e_tol=100.0, g_tol=1e-3)
    u = syn.orbital_uniforms(cfg, loose.npw)
    p1, p2 = loose.init_orbitals(u), strict.init_orbitals(u)
    i1 = [loose.pcg_step(p1) for _ in range(3)]
    i2 = [strict.pcg_step(p2) for _ in range(3)]
    assert i1[1]["converged"] == 1                       # |dE| < 100 twice
    assert all(i["converged"] == 0 for i in i2)          # |g| is far above 1e-3
    assert all(i["grad_norm"] > 1e-3 for i in i2)
    loose.close()
    strict.close()


def test_bad_options_rejected():
    roks = built()
    lib = roks.load()
    cfg = tiny()
    cell = roks.roks_cell(cfg["L"], cfg["grid"])
    out = C.c_void_p()
    opt = roks.roks_options(roks.ROKS_FP64, 0.0, 0, 1e-6, 0.0, 0, 0, 0, 0, 0, 0)
    no_atoms = (roks.roks_atom * 1)()
    no_species = (roks.roks_species * 1)()
    for occ in (roks.roks_occ(4, 0, 1), roks.roks_occ(4, 2, 0), roks.roks_occ(4, 1, 2)):
        st = lib.roks_setup(C.byref(cell), cfg["ecut"], 0, no_atoms, 0, no_species, C.byref(occ), C.byref(opt),
                            None, C.byref(out))
        assert st == roks.ROKS_EINVAL
    occ = roks.roks_occ(4, 2, 1)
    for field, value in (("exx_kernel", 5), ("precond", 3), ("autotune", 2), ("max_iter", -1), ("g_tol", -1.0)):
        bad = roks.roks_options(roks.ROKS_FP64, 0.0, 0, 1e-6, 0.0, 0, 0, 0, 0, 0, 0)
        setattr(bad, field, value)
        st = lib.roks_setup(C.byref(cell), cfg["ecut"], 0, no_atoms, 0, no_species, C.byref(occ), C.byref(bad),
                            None, C.byref(out))
        assert st == roks.ROKS_EINVAL, field
    st = lib.roks_setup(C.byref(cell), cfg["ecut"], 0, no_atoms, 0, no_species, C.byref(occ), C.byref(opt), None,
                        C.byref(out))
    assert st == roks.ROKS_OK
    lib.roks_destroy(out)


def test_bare_exchange_kernel_fp64():
    roks = built()
    cfg = tiny(alpha=1.0 / 3.0, exx_kernel=1)
    ctx = roks.Context(cfg, "fp64", exx_kernel=1)
    s = R.System(cfg)
    u = syn.orbital_uniforms(cfg, ctx.npw)
    psi = ctx.init_orbitals(u)
    P = s.initial_orbitals(u)
    ctx.density(psi)
    E = ctx.potential()
    Eref = s.energies(P)
    for k_gpu, k_ref in (("E_hf_M", "hf_M"), ("E_hf_T", "hf_T"), ("E_total", "total")):
        assert abs(E[k_gpu] - Eref[k_ref]) <= 1e-10 * max(1.0, abs(Eref[k_ref])), k_gpu
    # the bare kernel differs from the truncated one
    Etr = R.System(tiny(alpha=1.0 / 3.0)).energies(P)
    assert abs(Etr["hf_M"] - Eref["hf_M"]) > 1e-3
    f, _, _ = ctx.apply_h(psi)
    F_ref, _ = s.apply(P, s.potentials(s.class_densities(P)))
    assert rel(to_np(f, s.npw), F_ref) < 1e-10
    ctx.close()


def test_learned_preconditioner_with_zero_weights_is_tpa():
    """With all-zero weights the network's output is 0 and its factor exp(0)
    is 1, so the preconditioner selected at setup steps like TPA.  The fused
    kernel evaluates the TPA factor K in FP32 (as the network), so on the FP64
    path the direction carries FP32 rounding of K: the energies agree to
    1e-7 relative over four steps, not bit for bit."""
    roks = built()
    cfg = tiny()
    a = roks.Context(cfg, "fp64")
    b = roks.Context(cfg, "fp64", precond=roks.ROKS_PRECOND_TPA_MLP)
    u = syn.orbital_uniforms(cfg, a.npw)
    pa, pb = a.init_orbitals(u), b.init_orbitals(u)
    for _ in range(4):
        ia, ib = a.pcg_step(pa), b.pcg_step(pb)
        assert ia["E"] == ib["E"] or abs(ia["E"] - ib["E"]) <= 1e-7 * abs(ia["E"])
        assert abs(ia["E_new"] - ib["E_new"]) <= 1e-7 * abs(ia["E_new"]), (ia, ib)
    a.close()
    b.close()


def energy_scale(s, P):
    """Sum of the magnitudes of the energy terms of orbitals P (the scale of
    the FP32 rounding of the energy on the mixed path)."""
    E = s.energies(P)
    return sum(abs(E[k]) for k in ("kin", "loc", "nl", "H", "x_M", "x_T"))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_many_bands_many_projectors(precision):
    """128 bands, 376 projectors (a 2x2x2 rocksalt cell on a 32^3 grid): the
    band-space products of this size (projector blocks B2^H Q B2, B2 L^-H)
    run in the tiled kernel, the contractions on the tensor cores (mixed).
    FP64: 1e-10 relative along the oracle's trajectory.  Mixed: each step's
    energy against the oracle's evaluation of the GPU's own orbitals to 2e-7
    of the sum of the energy terms' magnitudes (FP32 rounding), and the
    trajectory against the oracle's to 1e-6 of that sum (two steps whose line
    search amplifies the rounding of the search direction)."""
    cfg = syn.with_changes(syn.make_config("hybrid-72", 0), grid=32, ecut=12.0, alpha=0.0)
    roks = built()
    ctx = roks.Context(cfg, precision)
    s = R.System(cfg)
    assert s.nb == 128 and s.nproj == 376
    u = syn.orbital_uniforms(cfg, ctx.npw)
    psi = ctx.init_orbitals(u)
    P = s.initial_orbitals(u)
    if precision == "fp64":
        assert rel(to_np(psi, s.npw), P) < 1e-10
    else:
        assert np.abs(s.overlap(to_np(psi, s.npw)) - np.eye(s.nb)).max() < 5e-6
    pcg = R.PCG(s)
    for it in range(2):
        info = ctx.pcg_step(psi)
        P, ref = pcg.step(P)
        if precision == "fp64":
            assert abs(info["E_new"] - ref.E_new) <= 1e-10 * max(1, abs(ref.E_new)), (it, info["E_new"], ref.E_new)
        else:
            Pg = to_np(psi, s.npw)
            scale = energy_scale(s, Pg)
            assert abs(info["E_new"] - s.energy(Pg)) <= 2e-7 * scale, (it, info["E_new"], s.energy(Pg), scale)
            assert abs(info["E_new"] - ref.E_new) <= 1e-6 * scale, (it, info["E_new"], ref.E_new, scale)
    ctx.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_autotune_keeps_the_results(precision):
    """roks_options.autotune times the density's band grouping (2, 4, 8) and,
    on the mixed path, the tensor-core schedule (stream-K, or K split into
    2.5 or 4 waves), then keeps the fastest:
    the chosen shapes are valid and the energies and F|n> stay those of the
    default shapes (only the order of some sums changes: 1e-12 relative on
    the FP64 path, FP32 rounding on the mixed path)."""
    cfg = syn.with_changes(syn.make_config("mgo-72", 0), grid=32, ecut=12.0)
    roks = built()
    ref = roks.Context(cfg, precision)
    tuned = roks.Context(cfg, precision, autotune=1)
    t = tuned.tuning()
    assert t["density_groups"] in (2, 4, 8)
    assert t["tc_split_waves_x2"] in (2, 5, 8)
    assert all(ms > 0 for ms in t["candidate_ms"][:3])
    if precision == "mixed":
        assert all(ms > 0 for ms in t["candidate_ms"][3:])
    d = roks.Context(cfg, precision).tuning()
    assert (d["density_groups"], d["tc_split_waves_x2"]) == (4, 2)
    u = syn.orbital_uniforms(cfg, ref.npw)
    out = []
    for ctx in (ref, tuned):
        psi = ctx.init_orbitals(u)
        ctx.density(psi)
        e = ctx.potential()
        f, _, _ = ctx.apply_h(psi)
        out.append((e["E_total"], to_np(f, ctx.npw)))
    tol_e, tol_f = (1e-12, 1e-11) if precision == "fp64" else (2e-6, 2e-5)
    assert abs(out[0][0] - out[1][0]) <= tol_e * abs(out[0][0])
    assert rel(out[1][1], out[0][1]) < tol_f
    ref.close()
    tuned.close()
