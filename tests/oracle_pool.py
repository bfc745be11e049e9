"""Oracle evaluations of large states spread over host processes (test
infrastructure): the class densities of hundreds of bands on a 120^3 grid,
a few hundred oracle transforms, are split by bands over spawned processes
(a pool forked after the first GPU call can hang) and summed in band-chunk
order; F and S of sampled bands of a hybrid-exchange state (each a few
hundred oracle transforms against every occupied orbital) go one band per
process.  The arithmetic is the oracle's own class_densities and apply."""
import multiprocessing as mp
import os

import numpy as np


def _densities(args):
    cfg, P, bands = args
    from oracle import roks as R
    return R.System(cfg).class_densities(P, bands)


def class_densities(cfg, P, workers=None):
    nb = P.shape[1]
    try:
        cores = len(os.sched_getaffinity(0))
    except Exception:
        cores = os.cpu_count() or 1
    workers = max(1, min(workers or cores, nb, 16))
    chunks = [c for c in np.array_split(np.arange(nb), workers) if len(c)]
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(var, "1")
    with mp.get_context("spawn").Pool(len(chunks)) as pool:
        parts = pool.map(_densities, [(cfg, np.ascontiguousarray(P[:, c]), [int(b) for b in c]) for c in chunks])
    rho = parts[0].copy()
    for p in parts[1:]:
        rho += p
    return rho


def _apply_band(args):
    cfg, P, rho, n = args
    from oracle import roks as R
    s = R.System(cfg)
    pot = s.potentials(rho)
    return s.apply(P[:, [n]], pot, classes=s.cls[[n]], occ=P)


def apply_bands(cfg, P, rho, bands):
    """F|n>, S|n> of the oracle for the columns `bands` of P (every column of
    P occupied: the exact exchange runs over all of them), one band per
    spawned process; returns (F, S) with one column per sampled band."""
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(var, "1")
    with mp.get_context("spawn").Pool(len(bands)) as pool:
        parts = pool.map(_apply_band, [(cfg, P, rho, int(n)) for n in bands])
    return np.hstack([p[0] for p in parts]), np.hstack([p[1] for p in parts])
