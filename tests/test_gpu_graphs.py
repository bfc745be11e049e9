"""PCG iterations replayed from a captured CUDA graph against the same
iterations launched kernel by kernel (ROKS_GRAPHS=0): the kernels and their
reduction orders are the same, so the trajectories agree bit for bit."""
import json
import os
import subprocess
import sys

import numpy as np

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
from paper_2605_28637_gb300 import roks, synthetic as syn
kw, prec = json.loads(sys.argv[2]), sys.argv[3]
cfg = syn.with_changes(syn.make_config("tiny-16", 0), **kw)
ctx = roks.Context(cfg, prec)
psi = ctx.init_orbitals(syn.orbital_uniforms(cfg, ctx.npw))
out = [ctx.pcg_step(psi)["E_new"] for _ in range(6)]
# a second buffer, then back: the graph is recaptured for each buffer change
psi2 = ctx.new_bands()
psi2.copy_(psi)
out += [ctx.pcg_step(psi2)["E_new"] for _ in range(3)]
out += [ctx.pcg_step(psi)["E_new"] for _ in range(3)]
print(json.dumps([x.hex() for x in out]))
"""


def run(kw, prec, graphs):
    env = dict(os.environ, ROKS_GRAPHS="1" if graphs else "0")
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, json.dumps(kw), prec], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("kw", [dict(), dict(grid=32, L=12.0, ecut=20.0, n_closed=6)], ids=["tiny16", "grid32"])
def test_graph_replay_matches_eager(kw, prec):
    assert run(kw, prec, True) == run(kw, prec, False)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_interleaved_calls_do_not_change_the_trajectory(prec):
    """The iteration reuses the projector coefficients of the accepted point;
    an apply on another buffer between steps replaces them, and the next step
    must form them again.  The chained block comes from the orthonormalisation
    (B L^-H), the re-formed one from P^H psi directly, so the two runs agree to
    rounding; coefficients left over from the other buffer would move the
    energy by many orders of magnitude more."""
    from paper_2605_28637_gb300 import roks, synthetic as syn
    from tests.gpu_helpers import built
    built()
    cfg = syn.make_config("tiny-16", 0)

    def run(interleave):
        ctx = roks.Context(cfg, prec)
        u = syn.orbital_uniforms(cfg, ctx.npw)
        psi = ctx.init_orbitals(u)
        other = ctx.init_orbitals(syn.orbital_uniforms(syn.make_config("tiny-16", 1), ctx.npw), ctx.new_bands())
        out = []
        for it in range(6):
            out.append(ctx.pcg_step(psi)["E_new"])
            if interleave and it % 2 == 1:
                ctx.apply_h(other, want_s=True)
        ctx.close()
        return out

    a, b = np.array(run(False)), np.array(run(True))
    tol = 1e-11 if prec == "fp64" else 1e-5
    assert np.abs(a - b).max() <= tol * np.abs(a).max(), (a, b)
