"""Shared helpers of the GPU parity tests: build/load the library, move band
blocks between torch (nbands, ld) layout and numpy (npw, nbands)."""
import numpy as np


def built():
    import __graft_entry__ as g
    g.build()
    from paper_2605_28637_gb300 import roks
    return roks


def to_np(t, npw):
    return t[:, :npw].detach().cpu().numpy().T.astype(np.complex128)


def to_dev(ctx, X):
    import torch
    t = ctx.new_bands()
    host = np.zeros((ctx.nb, ctx.ld), dtype=np.complex128)
    host[:, :X.shape[0]] = X.T
    t.copy_(torch.from_numpy(host).to(t.dtype))
    return t


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
