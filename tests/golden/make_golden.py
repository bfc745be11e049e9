"""Writes the stored expected values under tests/golden/ from the oracle alone.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import roks as R  # noqa: E402
from paper_2605_28637_gb300 import synthetic as syn  # noqa: E402


def basis_counts():
    # "quoted_approx": the plane-wave counts quoted with the model workloads
    # (about 500 and about 18 thousand); those match half spheres.
    quoted = {"tiny-16": 500, "organic-96": 18000}
    out = {"source": "oracle.roks.System basis (integer sphere test, full sphere); "
                     "quoted_approx from the workload descriptions",
           "workloads": {}}
    for name in ("tiny-16", "organic-96", "mgo-120", "hybrid-72"):
        cfg = syn.make_config(name, 0)
        L, ecut = cfg["L"], cfg["ecut"]
        q = L / (2.0 * np.pi)
        M = int(np.floor(2.0 * ecut * q * q))
        n = int(np.floor(np.sqrt(M)))
        cnt = sum(1 for i in range(-n, n + 1) for j in range(-n, n + 1)
                  for k in range(-n, n + 1) if i * i + j * j + k * k <= M)
        ent = {"npw_full": cnt, "npw_half": (cnt + 1) // 2, "M": M, "nmax": n}
        if name in quoted:
            ent["quoted_approx"] = quoted[name]
        out["workloads"][name] = ent
    return out


def tiny_trace(n_iter=12):
    cfg = syn.make_config("tiny-16", 0)
    s = R.System(cfg)
    Psi = s.initial_orbitals(syn.orbital_uniforms(cfg, s.npw))
    _, hist = R.run(s, Psi, max_iter=n_iter, e_tol=0.0)
    return {"source": "oracle.roks.run on tiny-16 seed 0 (singlet, TPA, no suppression)",
            "E": [h.E for h in hist], "E_new": [h.E_new for h in hist],
            "step": [h.step for h in hist]}


if __name__ == "__main__":
    with open(os.path.join(HERE, "basis_counts.json"), "w") as f:
        json.dump(basis_counts(), f, indent=1)
    with open(os.path.join(HERE, "tiny16_pcg_trace.json"), "w") as f:
        json.dump(tiny_trace(), f, indent=1)
    print("written")
