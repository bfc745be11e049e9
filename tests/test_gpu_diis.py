"""GPU parity of the DIIS solver (roks_diis_step) against the DIIS oracle
(oracle/diis.py) on the same seeded inputs.

FP64 path: energies 1e-10 relative and residual norms 1e-9 relative at every
step, the same window, coefficients to 1e-7 (they solve a Gram system whose
normalised condition the window test bounds by 1e7, so 1e-16 rounding in B
moves them by at most about 1e-9), orbitals 1e-8 relative after the run.
Mixed path.  With a one-pair history (preconditioned steepest descent, no
extrapolation) the trajectory follows the oracle's to 1e-5 Ha over 10 steps,
the bar of the mixed PCG test.  With the full history the extrapolation
Psi' = sum_j d_j (Psi_j + tau e_j) multiplies the FP32 error of the stored
pairs (about 1e-6 relative) by ||d||_1, which reaches 30-50 in the first
steps from a random start, and the next step stores the result: the mixed
and FP64 trajectories separate geometrically (measured: 2e-5 Ha after 5
steps, 6e-4 after 8).  So the first four steps are compared with
2e-5 + 2e-6 |g| ||d||_1 (the energy moves by the residual norm |g| times
the error of Psi'), and every step's energy with the oracle's evaluation of
the GPU's own orbitals (2e-7 of the sum of the energy terms' magnitudes)."""
import numpy as np
import pytest

from oracle import diis as D
from oracle import roks as R
from paper_2605_28637_gb300 import synthetic as syn
from tests.gpu_helpers import built, rel, to_np

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


def cfg_of(**kw):
    return syn.with_changes(syn.make_config("tiny-16", 0), **kw)


VARIANTS = {
    "singlet": (dict(), dict()),
    "singlet-flipped-coupling": (dict(), dict(lambda_ba=-0.5)),
    "ground-state": (dict(mode=0, n_closed=5), dict()),
    "triplet": (dict(mode=2), dict()),
    "ring-wraps": (dict(), dict(history=3, tau=0.7)),
    "one-pair": (dict(), dict(history=1)),
    "grid32": (dict(grid=32, L=12.0, ecut=20.0, n_closed=6), dict(history=4)),
}


def check_step(it, info, ref):
    assert abs(info["E"] - ref.E) <= TOL64 * max(1, abs(ref.E)), (it, info["E"], ref.E)
    assert abs(info["E_new"] - ref.E_new) <= TOL64 * max(1, abs(ref.E_new)), (it, info["E_new"], ref.E_new)
    assert abs(info["res_norm"] - ref.res_norm) <= 1e-9 * ref.res_norm
    assert info["window"] == ref.window, (it, info["window"], ref.window)
    assert np.abs(np.array(info["coef"]) - ref.coef).max() < 1e-7, (it, info["coef"], ref.coef)


@pytest.mark.parametrize("name", list(VARIANTS))
def test_diis_trajectory_fp64(name):
    kw, opt = VARIANTS[name]
    cfg = cfg_of(**kw)
    roks = built()
    ctx = roks.Context(cfg, "fp64")
    s = R.System(cfg)
    u = syn.orbital_uniforms(cfg, ctx.npw)
    psi = ctx.init_orbitals(u)
    P = s.initial_orbitals(u)
    dz = D.DIIS(s, **opt)
    for it in range(8):
        info = ctx.diis_step(psi, **opt)
        P, ref = dz.step(P)
        check_step(it, info, ref)
        assert abs(sum(info["coef"]) - 1.0) < 1e-12
    assert rel(to_np(psi, s.npw), P) < 1e-8


def test_diis_mixed_one_pair_trajectory():
    cfg = cfg_of()
    roks = built()
    ctx = roks.Context(cfg, "mixed")
    s = R.System(cfg)
    u = syn.orbital_uniforms(cfg, ctx.npw)
    psi = ctx.init_orbitals(u)
    P = s.initial_orbitals(u)
    dz = D.DIIS(s, history=1)
    for it in range(10):
        info = ctx.diis_step(psi, history=1)
        P, ref = dz.step(P)
        assert abs(info["E_new"] - ref.E_new) < 1e-5, (it, info["E_new"], ref.E_new)


def test_diis_mixed_full_history():
    cfg = cfg_of()
    roks = built()
    ctx = roks.Context(cfg, "mixed")
    s = R.System(cfg)
    u = syn.orbital_uniforms(cfg, ctx.npw)
    psi = ctx.init_orbitals(u)
    P = s.initial_orbitals(u)
    dz = D.DIIS(s)
    for it in range(10):
        info = ctx.diis_step(psi)
        assert abs(sum(info["coef"]) - 1.0) < 1e-12
        assert 1 <= info["window"] <= min(it + 1, 6)
        E = s.energies(to_np(psi, s.npw))
        scale = sum(abs(E[k]) for k in ("kin", "loc", "nl", "H", "x_M", "x_T"))
        assert abs(info["E_new"] - E["total"]) < 2e-7 * scale, (it, info["E_new"], E["total"])
        if it < 4:
            P, ref = dz.step(P)
            tol = 2e-5 + 2e-6 * ref.res_norm * np.abs(ref.coef).sum()
            assert abs(info["E_new"] - ref.E_new) < tol, (it, info["E_new"], ref.E_new, tol)
            assert info["window"] == ref.window


def test_diis_and_pcg_interleave_fp64():
    """DIIS, then PCG, then DIIS again: each solver starts its history afresh
    when the other has moved the orbitals (steepest descent for PCG, a
    one-pair window for DIIS)."""
    cfg = cfg_of()
    roks = built()
    ctx = roks.Context(cfg, "fp64")
    s = R.System(cfg)
    u = syn.orbital_uniforms(cfg, ctx.npw)
    psi = ctx.init_orbitals(u)
    P = s.initial_orbitals(u)
    for solver, n in (("diis", 3), ("pcg", 2), ("diis", 2)):
        ref_solver = D.DIIS(s) if solver == "diis" else R.PCG(s)
        for it in range(n):
            P, ref = ref_solver.step(P)
            info = ctx.diis_step(psi) if solver == "diis" else ctx.pcg_step(psi)
            assert abs(info["E_new"] - ref.E_new) <= TOL64 * max(1, abs(ref.E_new)), (solver, it)
            if solver == "diis" and it == 0:
                assert info["window"] == 1
            if solver == "pcg" and it == 0:
                assert info["beta"] == 0.0
    assert rel(to_np(psi, s.npw), P) < 1e-8


def test_diis_option_change_restarts_history():
    cfg = cfg_of()
    roks = built()
    ctx = roks.Context(cfg, "fp64")
    psi = ctx.init_orbitals(syn.orbital_uniforms(cfg, ctx.npw))
    assert ctx.diis_step(psi, history=4)["window"] == 1
    assert ctx.diis_step(psi, history=4)["window"] == 2
    assert ctx.diis_step(psi, history=4, tau=0.4)["window"] == 1
    assert ctx.diis_step(psi, history=4, tau=0.4)["window"] == 2


def test_diis_rejects_bad_options():
    cfg = cfg_of()
    roks = built()
    ctx = roks.Context(cfg, "fp64")
    psi = ctx.init_orbitals(syn.orbital_uniforms(cfg, ctx.npw))
    before = to_np(psi, ctx.npw)
    for bad in (dict(history=0), dict(history=roks.ROKS_DIIS_MAX + 1), dict(tau=0.0), dict(tau=float("nan")),
                dict(lambda_ba=float("inf"))):
        with pytest.raises(roks.RoksError) as e:
            ctx.diis_step(psi, **bad)
        assert e.value.status == 1
    assert np.array_equal(to_np(psi, ctx.npw), before)
