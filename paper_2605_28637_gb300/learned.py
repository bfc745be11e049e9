"""Training pairs and GPU training of the learned correction of the TPA
preconditioner (the network and its kernels are described in include/roks.h).

Pairs come from the plain method itself: a seeded system is converged with
TPA to Psi*; the same start is then stepped again and, at chosen iterations
i, the library returns the out-of-subspace residual g_I = F Psi - S Psi Theta,
the TPA step K g_I and the features of every coefficient.  The target is the
per-coefficient ratio between the converged correction and the TPA step:

  D   = Psi* U - Psi_i, U unitary aligning Psi* to Psi_i (polar factor of
        Psi*^H S Psi_i: orbitals are fixed only up to a rotation),
  D_I = D - Psi_i (S Psi_i)^H D   (the part the preconditioner acts on),
  r   = Re(conj(K g) D_I) / |K g|^2,  c_n = sum_G Re(conj(K g) D_I) / sum_G |K g|^2,
  t   = log(clip(r / c_n, e^-3, e^3)),   weight |g_nG|^2 / sum_G |g_nG|^2,

centred per band (weighted mean zero) and clipped again: the band scale is
the line search's job, the network learns the shape of the correction.  Bands with c_n <= 0
(the TPA step points away from the solution) are left out.

Training minimises the weighted mean square (s - t)^2 with Adam, every step
on the GPU through roks_mlp_grad / roks_mlp_adam.  The alignment of the
n_b x n_b subspace and the pair bookkeeping run on the host.
"""
from __future__ import annotations

import numpy as np

from . import roks, synthetic as syn


def _host(t, npw):
    """Device band block (nb x ld) -> host complex128 (npw x nb)."""
    return t[:, :npw].cpu().numpy().T.astype(np.complex128)


def converge(cfg: dict, precision: str = "fp64", max_iter: int = 2000, e_tol: float = 1e-6, params=None):
    """PCG from the seeded start to |dE| < e_tol twice; returns (ctx, psi, iterations, E)."""
    ctx = roks.Context(cfg, precision, e_tol=e_tol)
    if params is not None:
        ctx.set_preconditioner(params)
    psi = ctx.init_orbitals(syn.orbital_uniforms(cfg, ctx.npw))
    info = None
    it = 0
    for it in range(1, max_iter + 1):
        info = ctx.pcg_step(psi)
        if info["converged"]:
            break
    return ctx, psi, it, (info["E_new"] if info else None)


def make_pairs(cfg: dict, precision: str = "fp64", iters=(1, 2, 3, 4, 6, 8, 12, 16, 24, 32), max_iter: int = 2000):
    """Feature rows, targets and weights (float32 arrays) of one seeded system."""
    ctx_star, psi_star, _, _ = converge(cfg, precision, max_iter)
    Pstar = _host(psi_star, ctx_star.npw)
    ctx_star.close()
    ctx = roks.Context(cfg, precision)
    psi = ctx.init_orbitals(syn.orbital_uniforms(cfg, ctx.npw))
    npw, nb = ctx.npw, ctx.nb
    U_all, t_all, w_all = [], [], []
    for it in range(max(iters) + 1):
        if it in iters:
            # F, S, g_I = F - S theta on the device (theta kept for the features' band energies)
            f, s, _, gI_dev = ctx.gradient_parts(psi)
            P = _host(psi, npw)
            SP = _host(s, npw)
            gI = _host(gI_dev, npw)
            kg_dev, feats = ctx.precondition(gI_dev, want_feats=True)
            Kg = _host(kg_dev, npw)
            U = feats.cpu().numpy().reshape(nb, npw, 3)
            # align the converged orbitals to the current ones
            M = Pstar.conj().T @ SP
            A, _, Bh = np.linalg.svd(M)
            D = Pstar @ (A @ Bh) - P
            DI = D - P @ (SP.conj().T @ D)
            num = np.real(np.conj(Kg) * DI)
            den = np.abs(Kg) ** 2
            for n in range(nb):
                c = num[:, n].sum() / max(den[:, n].sum(), 1e-300)
                if not (c > 0):
                    continue
                ok = den[:, n] > 1e-30 * den[:, n].max()
                r = num[ok, n] / (den[ok, n] * c)
                t = np.log(np.clip(r, np.exp(-3.0), np.exp(3.0)))
                g2 = np.abs(gI[ok, n]) ** 2
                wn = g2 / max(g2.sum(), 1e-300)
                # centred per band: the network learns the shape of the
                # correction, not an overall scale (the line search's job)
                t = np.clip(t - float(np.sum(wn * t)), -3.0, 3.0)
                U_all.append(U[n][ok])
                t_all.append(t)
                w_all.append(wn)
        ctx.pcg_step(psi)
    ctx.close()
    return (np.concatenate(U_all).astype(np.float32), np.concatenate(t_all).astype(np.float32),
            np.concatenate(w_all).astype(np.float32))


def train(U: np.ndarray, t: np.ndarray, w: np.ndarray, steps: int = 400, lr: float = 3e-3, seed: int = 0,
          params0=None, stream=None):
    """Adam on the GPU (full batch); returns (device params, list of losses)."""
    import torch
    dev = "cuda"
    n = len(t)
    Ud = torch.from_numpy(np.ascontiguousarray(U, dtype=np.float32)).to(dev)
    td = torch.from_numpy(np.ascontiguousarray(t, dtype=np.float32)).to(dev)
    wd = torch.from_numpy(np.ascontiguousarray(w, dtype=np.float32)).to(dev)
    p0 = syn.mlp_initial_params(seed) if params0 is None else np.asarray(params0, dtype=np.float32)
    p = torch.from_numpy(p0.copy()).to(dev)
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    g = torch.zeros_like(p)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    work = torch.empty(roks.roks_mlp_grad_work(n), dtype=torch.float32, device=dev)
    st = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    losses = []
    for k in range(1, steps + 1):
        roks.roks_mlp_grad(n, Ud, td, wd, p, work, g, loss, st)
        roks.roks_mlp_adam(p, m, v, g, k, lr, stream=st)
        if k == 1 or k % 50 == 0 or k == steps:
            losses.append(float(loss.item()))
    return p, losses
