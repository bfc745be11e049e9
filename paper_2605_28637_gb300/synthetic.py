"""Seeded synthetic inputs for the ROKS plane-wave workloads.

This module is shared by the CUDA path's callers and by the oracle's
callers.  It holds no arithmetic of the method: it only draws random numbers
(SplitMix64, Steele/Lea/Flood 2014, in Vigna's published form) and lays out
the model systems that stand in for the paper's molecules and MgO supercells
(Sec. III; Table I gives the real PAW sets, which are not available).  The
random numbers the method consumes (initial orbital coefficients) are handed
to both sides as plain arrays.

Workloads (cubic cells, Gamma point, atomic units):

  tiny-16      L=10, 16^3 grid, Ecut 8 Ha, 4 atoms, 4 s/p projectors each,
               4 closed + 2 open bands
  organic-96   L=20, 96^3 grid, Ecut 20 Ha, 13 heavy + 17 H-like atoms,
               172 projectors, 40 closed + 2 open bands
  mgo-120      3x3x3 rocksalt (a=7.96), one O removed (215 atoms), 120^3,
               Ecut 15 Ha, Mg 4 / O 8 projectors, 428 closed + 2 open bands
  hybrid-72    2x2x2 rocksalt (a=7.96), one O removed (63 atoms), 72^3,
               Ecut 15 Ha, exact-exchange fraction 1/3, 126 closed + 2 open
  mgo-72       the hybrid-72 cell without exact exchange: a small system
               with the block shapes of mgo-120 (128 bands, 376 projectors),
               for profiling captures that must hold little device memory
"""
from __future__ import annotations

import numpy as np

MASK64 = (1 << 64) - 1
_GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Outputs start .. start+count-1 of SplitMix64 seeded with `seed`.

    SplitMix64 is counter based: output i is mix(seed + (i+1)*gamma) with the
    published mixing function, so the stream can be evaluated vectorised.
    """
    i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK64) + i * np.uint64(_GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(_M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(_M2)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, start: int, count: int, lo: float, hi: float) -> np.ndarray:
    """Uniform doubles in [lo, hi) from the top 53 bits of SplitMix64."""
    z = splitmix64(seed, start, count)
    u = (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return lo + (hi - lo) * u


class _Stream:
    """Sequential reader over one SplitMix64 stream."""

    def __init__(self, seed: int):
        self.seed = seed & MASK64
        self.pos = 0

    def take(self, count: int, lo: float, hi: float) -> np.ndarray:
        out = uniform(self.seed, self.pos, count, lo, hi)
        self.pos += count
        return out


def _sym(x: np.ndarray) -> np.ndarray:
    return 0.5 * (x + x.T)


def _channels(radii_s, radii_p):
    """Projector channel list (l, m, rc): s channels then p_x, p_y, p_z per p radius."""
    l, m, rc = [], [], []
    for r in radii_s:
        l.append(0); m.append(0); rc.append(r)
    for r in radii_p:
        for mm in range(3):
            l.append(1); m.append(mm); rc.append(r)
    return l, m, rc


def _species(stream: _Stream, radii_s, radii_p, d_scale=0.5, q_scale=0.05):
    l, m, rc = _channels(radii_s, radii_p)
    n = len(l)
    D = _sym(stream.take(n * n, -d_scale, d_scale).reshape(n, n))
    Q = q_scale * _sym(stream.take(n * n, -1.0, 1.0).reshape(n, n))
    return {"l": l, "m": m, "rc": rc, "D": D, "Q": Q}


def _min_image_dist(a, b, L):
    d = np.asarray(a) - np.asarray(b)
    d -= L * np.round(d / L)
    return float(np.sqrt((d * d).sum()))


def _random_positions(stream: _Stream, n: int, L: float, min_sep: float = 2.0):
    pos = []
    tries = 0
    while len(pos) < n:
        p = stream.take(3, 0.0, L)
        tries += 1
        if tries > 100000:
            raise RuntimeError("atom placement failed")
        if all(_min_image_dist(p, q, L) >= min_sep for q in pos):
            pos.append(tuple(float(v) for v in p))
    return pos


def _rocksalt(a: float, reps: int):
    """Mg on fcc sites, O shifted by a/2 along x; one O nearest the cell centre removed."""
    fcc = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    mg, ox = [], []
    for i in range(reps):
        for j in range(reps):
            for k in range(reps):
                for f in fcc:
                    r = (np.array([i, j, k]) + f) * a
                    mg.append(r)
                    o = r + np.array([0.5 * a, 0, 0])
                    ox.append(o % (reps * a))
    L = reps * a
    centre = np.full(3, 0.5 * L)
    dist = [np.linalg.norm(o - centre) for o in ox]
    drop = int(np.argmin(dist))
    ox = [o for i, o in enumerate(ox) if i != drop]
    return L, mg, ox


def make_config(name: str, seed: int = 0) -> dict:
    """One of the model workloads, with seeded random parts."""
    st = _Stream(seed * 0x100000001 + 0x5EED)
    if name == "tiny-16":
        L, N, ecut = 10.0, 16, 8.0
        sp = [_species(st, [0.8], [0.8])]
        pos = _random_positions(st, 4, L)
        depth = st.take(4, 1.0, 3.0)
        atoms = [{"pos": p, "species": 0, "depth": float(d), "width": 1.0}
                 for p, d in zip(pos, depth)]
        n_closed, alpha = 4, 0.0
    elif name == "organic-96":
        L, N, ecut = 20.0, 96, 20.0
        sp = [_species(st, [0.8, 1.2], [0.8, 1.2]), _species(st, [0.8], [0.8])]
        pos = _random_positions(st, 30, L)
        depth = st.take(13, 2.0, 3.0)
        atoms = []
        for i, p in enumerate(pos):
            if i < 13:
                atoms.append({"pos": p, "species": 0, "depth": float(depth[i]), "width": 1.0})
            else:
                atoms.append({"pos": p, "species": 1, "depth": 1.0, "width": 1.0})
        n_closed, alpha = 40, 0.0
    elif name in ("mgo-120", "hybrid-72", "mgo-72", "mgo-32"):
        # the rocksalt cell with an O vacancy; mgo-32 is its single cell (7
        # atoms), the small system of the same shape for training and tests
        reps = {"mgo-120": 3, "mgo-32": 1}.get(name, 2)
        L, mg, ox = _rocksalt(7.96, reps)
        N = {3: 120, 2: 72, 1: 32}[reps]
        ecut = 15.0
        sp = [_species(st, [0.8], [0.8]), _species(st, [0.8, 1.2], [0.8, 1.2])]
        atoms = [{"pos": tuple(map(float, r)), "species": 0, "depth": 1.0, "width": 1.0} for r in mg]
        atoms += [{"pos": tuple(map(float, r)), "species": 1, "depth": 3.0, "width": 1.0} for r in ox]
        n_closed = {3: 428, 2: 126, 1: 14}[reps]
        alpha = 1.0 / 3.0 if name == "hybrid-72" else 0.0
    else:
        raise ValueError(f"unknown workload {name!r}")
    return {
        "name": name, "L": float(L), "grid": int(N), "ecut": float(ecut),
        "atoms": atoms, "species": sp, "n_closed": int(n_closed), "mode": 1,
        "alpha": float(alpha), "seed": int(seed),
    }


def with_changes(cfg: dict, **kw) -> dict:
    """Copy of a workload with some fields replaced (mode, n_closed, alpha, ...)."""
    out = dict(cfg)
    out.update(kw)
    return out


def n_bands(cfg: dict) -> int:
    """closed, open (a, b unless the ground state) and empty bands"""
    return cfg["n_closed"] + (0 if cfg["mode"] == 0 else 2) + int(cfg.get("n_empty", 0))


def orbital_stream_seed(cfg: dict) -> int:
    """SplitMix64 seed of the stream the initial orbitals are drawn from."""
    return (cfg["seed"] * 0x9E3779B1 + 0x0B17) & MASK64


def orbital_uniforms(cfg: dict, npw: int, band0: int = 0, nbands: int | None = None) -> np.ndarray:
    """Uniform(-1,1) draws for the initial orbitals: shape (nbands, npw, 2).

    Band by band, coefficient by coefficient in basis order, real then
    imaginary part (number 2 (n npw + g) + part of the stream).  band0 and
    nbands select a range of bands (default: all).
    """
    nb = n_bands(cfg) - band0 if nbands is None else nbands
    u = uniform(orbital_stream_seed(cfg), 2 * band0 * npw, nb * npw * 2, -1.0, 1.0)
    return u.reshape(nb, npw, 2)


def random_vectors(seed: int, npw: int, nb: int) -> np.ndarray:
    """Complex Uniform(-1,1)+iUniform(-1,1) block (npw, nb) for test probes."""
    u = uniform(seed * 0x2545F491 + 0x77, 0, npw * nb * 2, -1.0, 1.0).reshape(nb, npw, 2)
    return (u[..., 0] + 1j * u[..., 1]).T.copy()


MLP_HIDDEN = 64
MLP_NPARAM = MLP_HIDDEN * 3 + MLP_HIDDEN + MLP_HIDDEN * MLP_HIDDEN + MLP_HIDDEN + MLP_HIDDEN + 1


def mlp_initial_params(seed: int) -> np.ndarray:
    """Initial weights of the preconditioner network (flat, float32): W1 and
    W2 uniform(-1, 1) scaled by 1/sqrt(fan-in), zero biases, zero output
    layer (so the untrained correction is the identity).  Layout: W1 (64 x 3,
    row major), b1, W2 (64 x 64, row major), b2, w3, b3."""
    st = _Stream(seed * 0x100000001 + 0x4D4C50)
    H = MLP_HIDDEN
    W1 = st.take(H * 3, -1.0, 1.0) / np.sqrt(3.0)
    W2 = st.take(H * H, -1.0, 1.0) / np.sqrt(float(H))
    p = np.concatenate([W1, np.zeros(H), W2, np.zeros(H), np.zeros(H), [0.0]])
    return p.astype(np.float32)

