"""GPU parity of the tcgen05 tensor-core contractions (k_tcgemm.cu).

They take the large blocks of the mixed path: A^H B with at least 128 x 64
outputs over 1024 or more plane waves, and tall products Psi X with 4096 or
more plane waves, 64 or more columns and terms.  The test system has 128
bands and 376 projectors (a 2 x 2 x 2 rocksalt cell on a 32^3 grid), so the
projector coefficients, the overlap, Theta, the projections, the
back-projections and the rotations all run there; the profile's
tensor_core_launches entry confirms it.

Bars (FP32-level: three TF32 products per FP32 product, each K-step drained
into round-to-nearest FP32 sums):
* against the oracle on the GPU's own orbitals: S-orthonormality 3e-6,
  densities 2e-6, F|n> 2e-5 and S|n> 2e-6 relative, the energy 2e-7 of the sum
  of the energy terms' magnitudes;
* against the SIMT kernels (ROKS_TENSOR_CORES=0 in a child process): the same
  F|n> and S|n> on the same orbitals within 2e-5 and 2e-6.
The norms (sums of like-signed terms, where a truncating accumulation would
drift) are checked through the orthonormality of the seeded start."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import roks as R
from paper_2605_28637_gb300 import synthetic as syn
from tests.gpu_helpers import built, rel, to_dev, to_np

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def big_cfg():
    return syn.with_changes(syn.make_config("hybrid-72", 0), grid=32, ecut=12.0, alpha=0.0)


def energy_terms(E):
    return sum(abs(E[k]) for k in ("E_kin", "E_loc", "E_nl", "E_H", "E_x_M", "E_x_T"))


def test_tensor_core_contractions_against_oracle():
    roks = built()
    cfg = big_cfg()
    ctx = roks.Context(cfg, "mixed")
    s = R.System(cfg)
    assert (ctx.nb, ctx.nproj) == (128, 376)
    roks.roks_profile_read(ctx.ctx)
    psi = ctx.init_orbitals(syn.orbital_uniforms(cfg, ctx.npw))
    P = to_np(psi, s.npw)
    assert np.abs(s.overlap(P) - np.eye(s.nb)).max() < 3e-6
    rho = ctx.density(psi, want_rho=True).cpu().numpy()
    assert rel(rho, s.class_densities(P)) < 2e-6
    E = ctx.potential()
    Eref = s.energies(P)
    assert abs(E["E_total"] - Eref["total"]) < 2e-7 * energy_terms(E), (E["E_total"], Eref["total"])
    f, sp, _ = ctx.apply_h(psi)
    F_ref, S_ref = s.apply(P, s.potentials(s.class_densities(P)))
    assert rel(to_np(f, s.npw), F_ref) < 2e-5
    assert rel(to_np(sp, s.npw), S_ref) < 2e-6
    prof = {e["name"]: e["launches"] for e in roks.roks_profile_read(ctx.ctx)}
    assert prof.get("tensor_core_launches", 0) > 0
    ctx.close()


CHILD = r"""
import sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2605_28637_gb300 import roks, synthetic as syn
from tests.gpu_helpers import to_dev, to_np
cfg = syn.with_changes(syn.make_config("hybrid-72", 0), grid=32, ecut=12.0, alpha=0.0)
ctx = roks.Context(cfg, "mixed")
P = np.load(sys.argv[2])
psi = to_dev(ctx, P)
ctx.density(psi)
ctx.potential()
f, sp, _ = ctx.apply_h(psi)
prof = {e["name"]: e["launches"] for e in roks.roks_profile_read(ctx.ctx)}
np.savez(sys.argv[3], f=to_np(f, ctx.npw), sp=to_np(sp, ctx.npw), tc=prof.get("tensor_core_launches", 0))
"""


def test_tensor_cores_match_simt_kernels(tmp_path):
    roks = built()
    cfg = big_cfg()
    ctx = roks.Context(cfg, "mixed")
    psi = ctx.init_orbitals(syn.orbital_uniforms(cfg, ctx.npw))
    P = to_np(psi, ctx.npw)
    np.save(tmp_path / "p.npy", P)
    ctx.density(psi)
    ctx.potential()
    f, sp, _ = ctx.apply_h(psi)
    env = dict(os.environ, ROKS_TENSOR_CORES="0")
    out = tmp_path / "simt.npz"
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, str(tmp_path / "p.npy"), str(out)], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    d = np.load(out)
    assert int(d["tc"]) == 0
    assert rel(to_np(f, ctx.npw), d["f"]) < 2e-5
    assert rel(to_np(sp, ctx.npw), d["sp"]) < 2e-6
    ctx.close()


def test_presplit_projectors_are_bit_identical(tmp_path):
    """The projector matrix split once at setup (the products P^H X and P Y
    copy its TF32 hi/lo blocks instead of converting them) gives the same
    bits as the in-kernel conversion (ROKS_TC_PRESPLIT=0 in a child process)."""
    roks = built()
    cfg = big_cfg()
    ctx = roks.Context(cfg, "mixed")
    psi = ctx.init_orbitals(syn.orbital_uniforms(cfg, ctx.npw))
    P = to_np(psi, ctx.npw)
    np.save(tmp_path / "p.npy", P)
    psi = to_dev(ctx, P)
    ctx.density(psi)
    ctx.potential()
    f, sp, _ = ctx.apply_h(psi)
    env = dict(os.environ, ROKS_TC_PRESPLIT="0")
    out = tmp_path / "conv.npz"
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, str(tmp_path / "p.npy"), str(out)], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    d = np.load(out)
    assert int(d["tc"]) > 0
    assert np.array_equal(to_np(f, ctx.npw), d["f"])
    assert np.array_equal(to_np(sp, ctx.npw), d["sp"])
    ctx.close()
