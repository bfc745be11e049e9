"""Parity at the full size of the hybrid-exchange workload (hybrid-72: a
2 x 2 x 2 rocksalt cell minus one O, 72^3 grid, 11,075 plane waves, 126 + 2
bands, exact-exchange fraction 1/3: all 8256 pair-transform pairs per
apply), against the FP64 oracle evaluating the GPU's own orbitals.

FP64 path: the class densities (1e-10 relative) and F|n>, S|n> of sampled
bands (closed, a, b), whose exact-exchange term runs over all 128 occupied
orbitals in the oracle (1e-10 relative).  Mixed path: F and S of every band
from the same orbitals against the FP64 path's (2e-5 and 2e-6 relative, the
mixed bars of the smaller hybrid cases)."""
import pytest

from oracle import roks as R
from paper_2605_28637_gb300 import synthetic as syn
from tests import oracle_pool
from tests.gpu_helpers import built, rel, to_dev, to_np

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


def test_hybrid72_full_size_against_oracle():
    roks = built()
    cfg = syn.make_config("hybrid-72", 0)
    ctx = roks.Context(cfg, "fp64")
    assert ctx.nb == 128 and ctx.npw == 11075 and cfg["alpha"] > 0
    psi = ctx.init_orbitals(syn.orbital_uniforms(cfg, ctx.npw))
    rho = ctx.density(psi, want_rho=True).cpu().numpy()
    E = ctx.potential()
    assert E["E_hf_M"] != 0.0
    f, sp, _ = ctx.apply_h(psi)
    P = to_np(psi, ctx.npw)
    F64, S64 = to_np(f, ctx.npw), to_np(sp, ctx.npw)
    ctx.close()
    # the oracle on the same orbitals
    s = R.System(cfg)
    rho_ref = oracle_pool.class_densities(cfg, P)
    assert rel(rho, rho_ref) < TOL64
    sel = [0, 63, 126, 127]                             # closed bands, then a and b
    F_ref, S_ref = oracle_pool.apply_bands(cfg, P, rho_ref, sel)
    assert rel(F64[:, sel], F_ref) < TOL64
    assert rel(S64[:, sel], S_ref) < TOL64
    # the mixed path on the same orbitals, every band
    ctx = roks.Context(cfg, "mixed")
    psi = to_dev(ctx, P)
    ctx.density(psi)
    Em = ctx.potential()
    f, sp, _ = ctx.apply_h(psi)
    assert rel(to_np(f, ctx.npw), F64) < 2e-5
    assert rel(to_np(sp, ctx.npw), S64) < 2e-6
    assert abs(Em["E_hf_M"] - E["E_hf_M"]) < 1e-5 * abs(E["E_hf_M"])
    ctx.close()
    assert s.nb == 128
