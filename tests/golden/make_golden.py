"""Writes the stored expected values under tests/golden/ from the oracle alone.

Run from the repository root:  python tests/golden/make_golden.py [basis] [trace] [converged]
(all three without arguments; "converged" takes a few minutes of CPU).
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


# Converged tiny-16 states: the ROKS singlet (4 closed + 2 open) and the
# closed-shell ground state with the same electrons (5 closed), each from its
# seeded start, to |dE| < 1e-9 Ha twice and |g| < 1e-5 (R7); the excitation
# energy E_abs = E_S - E_GS (Eq. 1 and the absorption energy of Sec. III).
CONVERGED_E_TOL, CONVERGED_G_TOL, CONVERGED_MAX_ITER = 1e-9, 1e-5, 2000


def converged_tiny():
    base = syn.make_config("tiny-16", 0)
    out = {"source": "oracle.roks.run on tiny-16 seed 0, singlet (n_closed 4) and ground state (n_closed 5), "
                     "TPA, from the seeded start",
           "e_tol": CONVERGED_E_TOL, "g_tol": CONVERGED_G_TOL}
    for key, mode, nc in (("singlet", 1, 4), ("ground", 0, 5)):
        cfg = syn.with_changes(base, mode=mode, n_closed=nc)
        s = R.System(cfg)
        Psi = s.initial_orbitals(syn.orbital_uniforms(cfg, s.npw))
        Psi, hist = R.run(s, Psi, max_iter=CONVERGED_MAX_ITER, e_tol=CONVERGED_E_TOL, g_tol=CONVERGED_G_TOL)
        E = s.energies(Psi)
        ent = {"iterations": len(hist), "grad_norm": hist[-1].grad_norm, "E_total": E["total"],
               "E_M": E["M"], "E_T": E["T"]}
        if mode == 1:
            ent["coupling_abs"] = abs(hist[-1].coupling)
            # open orbitals a and b (7 significant digits: enough for the
            # same-state test, an overlap above 0.99)
            for name, col in (("a", nc), ("b", nc + 1)):
                ent[f"orbital_{name}_re"] = [float(f"{v:.7g}") for v in Psi[:, col].real]
                ent[f"orbital_{name}_im"] = [float(f"{v:.7g}") for v in Psi[:, col].imag]
        out[key] = ent
    out["E_S"] = out["singlet"]["E_total"]
    out["E_GS"] = out["ground"]["E_total"]
    out["E_abs"] = out["E_S"] - out["E_GS"]
    return out


if __name__ == "__main__":
    which = sys.argv[1:] or ["basis", "trace", "converged"]
    if "basis" in which:
        with open(os.path.join(HERE, "basis_counts.json"), "w") as f:
            json.dump(basis_counts(), f, indent=1)
    if "trace" in which:
        with open(os.path.join(HERE, "tiny16_pcg_trace.json"), "w") as f:
            json.dump(tiny_trace(), f, indent=1)
    if "converged" in which:
        with open(os.path.join(HERE, "tiny16_converged.json"), "w") as f:
            json.dump(converged_tiny(), f)
    print("written")
