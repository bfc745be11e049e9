"""The allocation-free orthonormalisation (roks_orthonormalize_noalloc) agrees
with roks_orthonormalize on a context without projectors (S = 1), and with
the oracle's Cholesky orthonormalisation of the same block.

It serves callers that cannot call cudaMalloc (for example code inside a
framework that has reserved the GPU's memory for its own allocator); its
scratch is a fixed device array inside the library.  This file is named so
that pytest collects it last."""
import numpy as np
import pytest

from oracle import roks as oracle_roks
from paper_2605_28637_gb300 import synthetic as syn
from tests.gpu_helpers import built, rel, to_dev, to_np

pytestmark = pytest.mark.gpu


def no_projector_cfg():
    cfg = syn.make_config("tiny-16", 0)
    cfg["species"] = [dict(l=[], m=[], rc=[], D=np.zeros((0, 0)), Q=np.zeros((0, 0)))]
    return cfg


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 2e-6)])
def test_noalloc_matches_orthonormalize(precision, tol):
    import torch
    roks = built()
    cfg = no_projector_cfg()
    ctx = roks.Context(cfg, precision)
    oracle_system = oracle_roks.System(cfg)
    base = to_np(ctx.init_orbitals(syn.orbital_uniforms(cfg, ctx.npw)), ctx.npw)
    prec = roks.ROKS_FP64 if precision == "fp64" else roks.ROKS_MIXED
    # two calls in a row, on different inputs, through the shared scratch
    for seed in (21, 22):
        X = base + 0.4 * syn.random_vectors(seed, ctx.npw, ctx.nb)
        ref = to_dev(ctx, X)
        ctx.orthonormalize(ref)
        got = to_dev(ctx, X)
        roks.roks_orthonormalize_noalloc(prec, ctx.npw, ctx.nb, got, ctx.ld, ctx.stream.cuda_stream)
        torch.cuda.synchronize()
        R = to_np(ref, ctx.npw)
        G = to_np(got, ctx.npw)
        assert rel(G, R) < tol
        O = G.conj().T @ G
        assert np.abs(O - np.eye(ctx.nb)).max() < (1e-12 if precision == "fp64" else 2e-6)
        # and against the oracle's Cholesky orthonormalisation of the same block
        ref_oracle = oracle_system.orthonormalize(X)
        assert rel(G, ref_oracle) < tol
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    roks = built()
    npw, nb = 300, 65
    psi = torch.zeros((nb, npw), dtype=torch.complex128, device="cuda")
    with pytest.raises(roks.RoksError) as ei:
        roks.roks_orthonormalize_noalloc(roks.ROKS_FP64, npw, nb, psi, npw, None)
    assert ei.value.status == roks.ROKS_EINVAL


def test_noalloc_reports_singular_overlap_and_keeps_psi():
    import torch
    roks = built()
    npw, nb = 200, 4
    rng = np.random.default_rng(1)
    X = rng.standard_normal((npw, nb)) + 1j * rng.standard_normal((npw, nb))
    X[:, 2] = 0.0                  # exact zero pivot: the overlap is singular
    psi = torch.from_numpy(np.ascontiguousarray(X.T)).to("cuda")
    with pytest.raises(roks.RoksError) as ei:
        roks.roks_orthonormalize_noalloc(roks.ROKS_FP64, npw, nb, psi, npw, None)
    assert ei.value.status == roks.ROKS_ENOTPOSDEF
    assert np.array_equal(psi.cpu().numpy().T, X)
    # the next call on good data succeeds (the status flag is cleared per call)
    X[:, 2] = rng.standard_normal(npw)
    psi = torch.from_numpy(np.ascontiguousarray(X.T)).to("cuda")
    roks.roks_orthonormalize_noalloc(roks.ROKS_FP64, npw, nb, psi, npw, None)
    G = psi.cpu().numpy().T
    assert np.abs(G.conj().T @ G - np.eye(nb)).max() < 1e-12
