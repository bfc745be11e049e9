"""Parity at convergence: the ROKS singlet and the closed-shell ground state
of tiny-16 minimised to |dE| < 1e-9 Ha twice and |g| < 1e-5 (the gradient
criterion beside the energy criterion, reading R7), on the GPU, against the
oracle's converged run from the same seeded start (tests/golden/
tiny16_converged.json, written by tests/golden/make_golden.py from oracle/
alone).

Compared: E_S = 2 E_M - E_T (Eq. 1), E_M, E_T, the ground-state energy E_GS
and the excitation energy E_abs = E_S - E_GS, to 1e-6 Ha on the FP64 path and
1e-5 Ha on the mixed path (whose gradient criterion is 1e-4: FP32 rounding
leaves a gradient floor near 1e-5).  Several stationary states exist for the
singlet, so the comparison is made only in the same state, judged by the
S-overlap of the open orbitals a and b with the oracle's (> 0.99 in
magnitude); the test asserts that the state is the same."""
import json
import os

import numpy as np
import pytest

from oracle import roks as R
from paper_2605_28637_gb300 import synthetic as syn
from tests.gpu_helpers import built, to_np

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "tiny16_converged.json")


def golden():
    with open(GOLDEN) as f:
        return json.load(f)


def converge(cfg, precision, e_tol, g_tol, max_iter=3000):
    roks = built()
    ctx = roks.Context(cfg, precision, e_tol=e_tol, g_tol=g_tol)
    psi = ctx.init_orbitals(syn.orbital_uniforms(cfg, ctx.npw))
    info = None
    for it in range(1, max_iter + 1):
        info = ctx.pcg_step(psi)
        if info["converged"]:
            break
    ctx.density(psi)
    e = ctx.potential()
    return ctx, psi, info, it, e


def open_overlaps(cfg, psi, npw, g):
    """|<x_gpu|S|x_oracle>| for x = a, b."""
    s = R.System(cfg)
    P = to_np(psi, npw)
    nc = cfg["n_closed"]
    out = []
    for name, col in (("a", nc), ("b", nc + 1)):
        ref = np.asarray(g["singlet"][f"orbital_{name}_re"]) + 1j * np.asarray(g["singlet"][f"orbital_{name}_im"])
        ref = ref / np.sqrt(np.real(np.vdot(ref, s.apply_S(ref[:, None])[:, 0])))
        out.append(abs(np.vdot(P[:, col], s.apply_S(ref[:, None])[:, 0])))
    return out


@pytest.mark.parametrize("precision,e_tol,g_tol,bar", [("fp64", 1e-9, 1e-5, 1e-6), ("mixed", 1e-8, 1e-4, 1e-5)])
def test_converged_excitation_energy(precision, e_tol, g_tol, bar):
    g = golden()
    base = syn.make_config("tiny-16", 0)
    sing = syn.with_changes(base, mode=1, n_closed=4)
    ground = syn.with_changes(base, mode=0, n_closed=5)
    ctx_s, psi_s, info_s, it_s, e_s = converge(sing, precision, e_tol, g_tol)
    assert info_s["converged"], (it_s, info_s)
    ovl = open_overlaps(sing, psi_s, ctx_s.npw, g)
    assert min(ovl) > 0.99, ("not the oracle's state", ovl)
    ctx_g, psi_g, info_g, it_g, e_g = converge(ground, precision, e_tol, g_tol)
    assert info_g["converged"], (it_g, info_g)
    E_abs = e_s["E_total"] - e_g["E_total"]
    got = {"E_S": e_s["E_total"], "E_M": e_s["E_M"], "E_T": e_s["E_T"], "E_GS": e_g["E_total"], "E_abs": E_abs}
    want = {"E_S": g["E_S"], "E_M": g["singlet"]["E_M"], "E_T": g["singlet"]["E_T"], "E_GS": g["E_GS"],
            "E_abs": g["E_abs"]}
    for k in want:
        assert abs(got[k] - want[k]) < bar, (k, got[k], want[k], it_s, it_g)
    # Eq. 1 on the GPU's own numbers
    assert abs(e_s["E_total"] - (2 * e_s["E_M"] - e_s["E_T"])) < 1e-12 * abs(e_s["E_total"]) + 1e-12
    # the open-shell coupling <a|F^a - F^b|b> vanishes at the stationary point (Eq. 15)
    assert abs(complex(info_s["coupling_re"], info_s["coupling_im"])) < 100 * g_tol
    ctx_s.close()
    ctx_g.close()


def converge_diis(cfg, precision, e_tol, g_tol, max_iter=3000):
    roks = built()
    ctx = roks.Context(cfg, precision, e_tol=e_tol, g_tol=g_tol)
    psi = ctx.init_orbitals(syn.orbital_uniforms(cfg, ctx.npw))
    info = None
    it = 0
    for it in range(1, max_iter + 1):
        info = ctx.diis_step(psi)
        if info["converged"]:
            break
    ctx.density(psi)
    e = ctx.potential()
    return ctx, psi, info, it, e


@pytest.mark.parametrize("precision,e_tol,g_tol,bar", [("fp64", 1e-9, 1e-5, 1e-6), ("mixed", 1e-8, 1e-4, 1e-5)])
def test_diis_converges_to_the_oracle_state(precision, e_tol, g_tol, bar):
    """DIIS (history 6, tau 1/2, every lambda 1/2: the residual is the
    gradient of Eq. 7, so its fixed points are the PCG's stationary points)
    run to |dE| < e_tol twice and |R| < g_tol from the seeded start reaches
    the oracle's converged closed-shell ground state: E_GS within the bar of
    the FP64 oracle's PCG minimum (state-level parity of the DIIS path; the
    oracle's own DIIS takes 65 steps and lands 3e-10 Ha from it).  The
    singlet is not used: from this start the oracle's DIIS does not meet the
    criterion within 3000 steps."""
    g = golden()
    base = syn.make_config("tiny-16", 0)
    ground = syn.with_changes(base, mode=0, n_closed=5)
    ctx, psi, info, it, e = converge_diis(ground, precision, e_tol, g_tol)
    assert info["converged"], (it, info)
    assert abs(e["E_total"] - g["E_GS"]) < bar, (e["E_total"], g["E_GS"], it)
    ctx.close()
