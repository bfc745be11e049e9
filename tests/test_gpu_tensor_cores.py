"""GPU parity of the opt-in tcgen05 contraction path (ROKS_TENSOR_CORES=1).

The switch is read once per process, so each case runs in a child process
that prints its results; the parent compares them with the FP64 oracle.  The
tensor-core contractions carry split-TF32 operands (exact to 2^-33 relative)
but accumulate in FP32 with truncation; the overlap of the orthonormalisation
stays on the SIMT path, so the mixed-path tolerances of the apply hold."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import roks as R
from paper_2605_28637_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = {
    "grid32": dict(grid=32, L=12.0, ecut=20.0, n_closed=6),
    "grid48": dict(grid=48, L=12.0, ecut=35.0, n_closed=3),
}

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2605_28637_gb300 import roks, synthetic as syn
cfg = syn.with_changes(syn.make_config("tiny-16", 0), **json.loads(sys.argv[2]))
ctx = roks.Context(cfg, "mixed")
psi = ctx.init_orbitals(syn.orbital_uniforms(cfg, ctx.npw))
rho = ctx.density(psi, want_rho=True).cpu().numpy()
E = ctx.potential()
f, sp, _ = ctx.apply_h(psi)
n = ctx.npw
tonp = lambda t: t[:, :n].cpu().numpy().T.astype(np.complex128)
np.savez(sys.argv[3], psi=tonp(psi), rho=rho, f=tonp(f), sp=tonp(sp))
print(json.dumps(E))
"""


def rel(a, b):
    return float(np.abs(np.asarray(a) - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("name", list(CASES))
def test_tensor_core_apply(name, tmp_path):
    out = tmp_path / "r.npz"
    env = dict(os.environ, ROKS_TENSOR_CORES="1")
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, json.dumps(CASES[name]), str(out)], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    E = json.loads(r.stdout.strip().splitlines()[-1])
    d = np.load(out)
    cfg = syn.with_changes(syn.make_config("tiny-16", 0), **CASES[name])
    s = R.System(cfg)
    P_ref = s.initial_orbitals(syn.orbital_uniforms(cfg, s.npw))
    assert rel(d["psi"], P_ref) < 2e-6
    rho_ref = s.class_densities(P_ref)
    assert rel(d["rho"], rho_ref) < 2e-6
    assert abs(E["E_total"] - s.energies(P_ref)["total"]) < 2e-5
    # F and S applied to the GPU's own orbitals, against the oracle on the same orbitals
    P = d["psi"]
    F_ref, S_ref = s.apply(P, s.potentials(s.class_densities(P)))
    assert rel(d["f"], F_ref) < 2e-5
    assert rel(d["sp"], S_ref) < 2e-6
