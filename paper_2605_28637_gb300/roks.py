"""ctypes binding of libroks_gb300.so (the C ABI of include/roks.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  Device buffers are torch tensors (used for memory and
streams); orbitals are tensors of shape (nbands, ld) with dtype complex128
(FP64 path) or complex64 (mixed path), row n holding band n, which is the
column-major npw x nbands layout of the C ABI.

The module-level functions carry the C names (roks_setup, roks_density, ...).
`Context` wraps them for convenience.  Loading fails loudly when the library
has not been built; there is no other implementation behind these names.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import synthetic

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libroks_gb300.so")

ROKS_OK, ROKS_EINVAL, ROKS_ENOMEM, ROKS_ECUDA, ROKS_ENOTPOSDEF, ROKS_ENOCONV, ROKS_ETIMEOUT, ROKS_EDIVERGED = range(8)
ROKS_FP64, ROKS_MIXED = 0, 1
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "ENOTPOSDEF", "ENOCONV", "ETIMEOUT", "EDIVERGED"]


class RoksError(RuntimeError):
    def __init__(self, status: int, msg: str):
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"ROKS_{name}: {msg}")
        self.status = status


# exchange functionals (roks_options.xc) by the workload's name for them
XC_KINDS = {"slater": 0, "pbe_x": 1}


class roks_cell(C.Structure):
    _fields_ = [("L", C.c_double), ("grid", C.c_int)]


class roks_atom(C.Structure):
    _fields_ = [("pos", C.c_double * 3), ("species", C.c_int), ("depth", C.c_double), ("width", C.c_double)]


class roks_species(C.Structure):
    _fields_ = [("nproj", C.c_int), ("l", C.POINTER(C.c_int)), ("m", C.POINTER(C.c_int)),
                ("rc", C.POINTER(C.c_double)), ("D", C.POINTER(C.c_double)), ("Q", C.POINTER(C.c_double))]


class roks_occ(C.Structure):
    _fields_ = [("n_closed", C.c_int), ("n_open", C.c_int), ("mode", C.c_int), ("n_empty", C.c_int)]


class roks_options(C.Structure):
    _fields_ = [("precision", C.c_int), ("alpha", C.c_double), ("suppress_ab", C.c_int), ("e_tol", C.c_double),
                ("g_tol", C.c_double), ("max_iter", C.c_int), ("seed", C.c_uint64), ("precond", C.c_int),
                ("autotune", C.c_int), ("exx_kernel", C.c_int), ("wait_cap", C.c_int), ("gamma", C.c_int),
                ("xc", C.c_int)]


ROKS_EXX_TRUNCATED, ROKS_EXX_BARE = 0, 1


class roks_energies(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("E_kin", "E_loc", "E_nl", "E_H", "E_x_M", "E_x_T", "E_hf_M", "E_hf_T",
                                          "E_M", "E_T", "E_total")]


class roks_step_info(C.Structure):
    _fields_ = [("E", C.c_double), ("E_new", C.c_double), ("step", C.c_double), ("grad_norm", C.c_double),
                ("coupling_re", C.c_double), ("coupling_im", C.c_double), ("beta", C.c_double),
                ("dE0", C.c_double), ("restarted", C.c_int), ("converged", C.c_int)]


ROKS_DIIS_MAX = 8


class roks_diis_options(C.Structure):
    _fields_ = [("history", C.c_int), ("tau", C.c_double), ("lambda_ab", C.c_double), ("lambda_ba", C.c_double)]


class roks_diis_info(C.Structure):
    _fields_ = [("E", C.c_double), ("E_new", C.c_double), ("res_norm", C.c_double), ("window", C.c_int),
                ("coef", C.c_double * ROKS_DIIS_MAX), ("converged", C.c_int)]


class roks_tuning(C.Structure):
    _fields_ = [("density_groups", C.c_int), ("tc_split_waves_x2", C.c_int), ("candidate_ms", C.c_double * 6)]


class roks_profile_entry(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_int), ("ms", C.c_double)]


EXPORTS = ["roks_setup", "roks_basis", "roks_init_orbitals", "roks_invalidate", "roks_density", "roks_potential", "roks_apply_h",
           "roks_gradient_parts", "roks_orthonormalize", "roks_pcg_step", "roks_diis_step", "roks_forces", "roks_energies_get",
           "roks_profile_enable", "roks_profile_read", "roks_tuning_get", "roks_orthonormalize_noalloc", "roks_mlp_forward",
           "roks_mlp_grad", "roks_mlp_adam", "roks_set_preconditioner", "roks_precondition", "roks_mlp_grad_work",
           "roks_last_error", "roks_destroy"]

ROKS_MLP_PARAMS = 4481
ROKS_PRECOND_TPA = 0
ROKS_PRECOND_TPA_MLP = 1

_lib = None


def load(path: str | None = None) -> C.CDLL:
    """Open the compiled library (build it with paper_2605_28637_gb300.build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise FileNotFoundError(f"{path} is missing: build the CUDA library first "
                                "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(path)
    P = C.c_void_p
    lib.roks_setup.argtypes = [C.POINTER(roks_cell), C.c_double, C.c_int, C.POINTER(roks_atom), C.c_int,
                               C.POINTER(roks_species), C.POINTER(roks_occ), C.POINTER(roks_options), P,
                               C.POINTER(P)]
    lib.roks_basis.argtypes = [P, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                               C.POINTER(C.POINTER(C.c_int32))]
    lib.roks_init_orbitals.argtypes = [P, C.POINTER(C.c_double), P, C.c_int64]
    lib.roks_invalidate.argtypes = [P]
    lib.roks_density.argtypes = [P, P, C.c_int64, P]
    lib.roks_potential.argtypes = [P, C.POINTER(roks_energies), P]
    lib.roks_apply_h.argtypes = [P, P, C.c_int64, P, P, P]
    lib.roks_gradient_parts.argtypes = [P, P, C.c_int64, P, P, P, P]
    lib.roks_orthonormalize.argtypes = [P, P, C.c_int64]
    lib.roks_pcg_step.argtypes = [P, P, C.c_int64, C.POINTER(roks_step_info)]
    lib.roks_diis_step.argtypes = [P, P, C.c_int64, C.POINTER(roks_diis_options), C.POINTER(roks_diis_info)]
    lib.roks_forces.argtypes = [P, P, C.c_int64, C.POINTER(C.c_double)]
    lib.roks_energies_get.argtypes = [P, C.POINTER(roks_energies)]
    lib.roks_profile_enable.argtypes = [P, C.c_int]
    lib.roks_profile_read.argtypes = [P, C.POINTER(roks_profile_entry), C.c_int, C.POINTER(C.c_int)]
    lib.roks_tuning_get.argtypes = [P, C.POINTER(roks_tuning)]
    lib.roks_orthonormalize_noalloc.argtypes = [C.c_int, C.c_int, C.c_int, P, C.c_int64, P]
    lib.roks_mlp_forward.argtypes = [C.c_int, P, P, C.c_int, P, P]
    lib.roks_mlp_grad.argtypes = [C.c_int, P, P, P, P, P, P, P, P]
    lib.roks_mlp_adam.argtypes = [P, P, P, P, C.c_int, C.c_float, C.c_float, C.c_float, C.c_float, P]
    lib.roks_set_preconditioner.argtypes = [P, C.c_int, P]
    lib.roks_precondition.argtypes = [P, P, C.c_int64, P, P]
    lib.roks_mlp_grad_work.argtypes = [C.c_int]
    lib.roks_mlp_grad_work.restype = C.c_size_t
    lib.roks_last_error.argtypes = [P]
    lib.roks_last_error.restype = C.c_char_p
    lib.roks_destroy.argtypes = [P]
    lib.roks_destroy.restype = None
    for name in EXPORTS[:-3]:
        getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def _check(ctx, status):
    if status != ROKS_OK:
        msg = load().roks_last_error(ctx).decode() if ctx else ""
        raise RoksError(status, msg)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


# ---------------------------------------------------------------- C names
def roks_setup(cfg: dict, precision: int = ROKS_FP64, stream=None, suppress_ab: bool = False,
               e_tol: float = 1e-6, g_tol: float = 0.0, max_iter: int = 0, precond: int = 0, autotune: int = 0,
               exx_kernel: int = ROKS_EXX_TRUNCATED, wait_cap: int = 0, gamma: int = 0, xc=None):
    """Marshal a workload description (see synthetic.make_config) and call roks_setup."""
    lib = load()
    cell = roks_cell(cfg["L"], cfg["grid"])
    keep = []
    sp_arr = (roks_species * max(1, len(cfg["species"])))()
    for i, sp in enumerate(cfg["species"]):
        n = len(sp["l"])
        l = (C.c_int * n)(*sp["l"])
        m = (C.c_int * n)(*sp["m"])
        rc = (C.c_double * n)(*sp["rc"])
        D = np.ascontiguousarray(np.asarray(sp["D"], dtype=np.float64).reshape(n, n))
        Q = np.ascontiguousarray(np.asarray(sp["Q"], dtype=np.float64).reshape(n, n))
        keep += [l, m, rc, D, Q]
        sp_arr[i] = roks_species(n, l, m, rc, D.ctypes.data_as(C.POINTER(C.c_double)),
                                 Q.ctypes.data_as(C.POINTER(C.c_double)))
    atoms = cfg["atoms"]
    at_arr = (roks_atom * max(1, len(atoms)))()
    for i, a in enumerate(atoms):
        at_arr[i] = roks_atom((C.c_double * 3)(*a["pos"]), a["species"], a["depth"], a["width"])
    occ = roks_occ(cfg["n_closed"], 0 if cfg["mode"] == 0 else 2, cfg["mode"], int(cfg.get("n_empty", 0)))
    opt = roks_options(precision, cfg.get("alpha", 0.0), int(suppress_ab), e_tol, g_tol, int(max_iter),
                       synthetic.orbital_stream_seed(cfg), int(precond), int(autotune), int(exx_kernel), int(wait_cap),
                       int(gamma), XC_KINDS[cfg.get("xc", "slater") if xc is None else xc])
    out = C.c_void_p()
    st = C.c_void_p(stream) if stream else None
    status = lib.roks_setup(C.byref(cell), cfg["ecut"], len(atoms), at_arr, len(cfg["species"]), sp_arr,
                            C.byref(occ), C.byref(opt), st, C.byref(out))
    if status != ROKS_OK:
        raise RoksError(status, "roks_setup rejected the workload")
    return out


def roks_basis(ctx):
    lib = load()
    npw, nb, ld = C.c_int(), C.c_int(), C.c_int()
    mil = C.POINTER(C.c_int32)()
    _check(ctx, lib.roks_basis(ctx, C.byref(npw), C.byref(nb), C.byref(ld), C.byref(mil)))
    miller = np.ctypeslib.as_array(mil, shape=(npw.value, 3)).copy()
    return npw.value, nb.value, ld.value, miller


def roks_init_orbitals(ctx, u, psi, ld: int):
    """u: host uniforms (nbands, npw, 2), or None to draw them on the device
    from the context's seed."""
    if u is None:
        _check(ctx, load().roks_init_orbitals(ctx, None, _ptr(psi), ld))
        return
    u = np.ascontiguousarray(u, dtype=np.float64)
    _check(ctx, load().roks_init_orbitals(ctx, u.ctypes.data_as(C.POINTER(C.c_double)), _ptr(psi), ld))


def roks_invalidate(ctx):
    _check(ctx, load().roks_invalidate(ctx))


def roks_density(ctx, psi, ld: int, rho_out=None):
    _check(ctx, load().roks_density(ctx, _ptr(psi), ld, _ptr(rho_out)))


def roks_potential(ctx, vclass_out=None) -> dict:
    e = roks_energies()
    _check(ctx, load().roks_potential(ctx, C.byref(e), _ptr(vclass_out)))
    return {n: getattr(e, n) for n, _ in roks_energies._fields_}


def roks_apply_h(ctx, psi, ld: int, fpsi, spsi=None, grad=None):
    _check(ctx, load().roks_apply_h(ctx, _ptr(psi), ld, _ptr(fpsi), _ptr(spsi), _ptr(grad)))


def roks_gradient_parts(ctx, psi, ld: int, fpsi, spsi=None, grad=None, grad_I=None):
    _check(ctx, load().roks_gradient_parts(ctx, _ptr(psi), ld, _ptr(fpsi), _ptr(spsi), _ptr(grad), _ptr(grad_I)))


def roks_orthonormalize(ctx, psi, ld: int):
    _check(ctx, load().roks_orthonormalize(ctx, _ptr(psi), ld))


def roks_pcg_step(ctx, psi, ld: int) -> dict:
    info = roks_step_info()
    _check(ctx, load().roks_pcg_step(ctx, _ptr(psi), ld, C.byref(info)))
    return {n: getattr(info, n) for n, _ in roks_step_info._fields_}


def roks_diis_step(ctx, psi, ld: int, history: int = 6, tau: float = 0.5, lambda_ab: float = 0.5,
                   lambda_ba: float = 0.5) -> dict:
    opt = roks_diis_options(history, tau, lambda_ab, lambda_ba)
    info = roks_diis_info()
    _check(ctx, load().roks_diis_step(ctx, _ptr(psi), ld, C.byref(opt), C.byref(info)))
    out = {n: getattr(info, n) for n, _ in roks_diis_info._fields_ if n != "coef"}
    out["coef"] = [info.coef[k] for k in range(info.window)]
    return out


def roks_forces(ctx, psi, ld: int, natoms: int) -> np.ndarray:
    """F_Inu = -dE/dR_Inu (natoms x 3, Ha/Bohr)."""
    out = np.zeros((natoms, 3), dtype=np.float64)
    _check(ctx, load().roks_forces(ctx, _ptr(psi), ld, out.ctypes.data_as(C.POINTER(C.c_double))))
    return out


def roks_energies_get(ctx) -> dict:
    e = roks_energies()
    _check(ctx, load().roks_energies_get(ctx, C.byref(e)))
    return {n: getattr(e, n) for n, _ in roks_energies._fields_}


def roks_profile_enable(ctx, enable: int):
    _check(ctx, load().roks_profile_enable(ctx, int(enable)))


def roks_profile_read(ctx, cap: int = 64) -> list:
    arr = (roks_profile_entry * cap)()
    n = C.c_int()
    _check(ctx, load().roks_profile_read(ctx, arr, cap, C.byref(n)))
    return [{"name": arr[i].name.decode(), "launches": arr[i].launches, "ms": arr[i].ms}
            for i in range(min(n.value, cap))]


def roks_tuning_get(ctx) -> dict:
    t = roks_tuning()
    _check(ctx, load().roks_tuning_get(ctx, C.byref(t)))
    return {"density_groups": t.density_groups, "tc_split_waves_x2": t.tc_split_waves_x2,
            "candidate_ms": [t.candidate_ms[i] for i in range(6)]}


def roks_orthonormalize_noalloc(precision: int, npw: int, nbands: int, psi, ld: int, stream=None):
    """Allocation-free S = 1 orthonormalisation (see include/roks.h)."""
    st = C.c_void_p(stream) if stream else None
    status = load().roks_orthonormalize_noalloc(int(precision), int(npw), int(nbands), _ptr(psi), int(ld), st)
    if status != ROKS_OK:
        raise RoksError(status, "roks_orthonormalize_noalloc")


def _st(stream):
    return C.c_void_p(stream) if stream else None


def roks_mlp_forward(n: int, feats, params, bf16: bool, s, stream=None):
    """Network outputs for n feature rows (device float32 tensors)."""
    status = load().roks_mlp_forward(int(n), _ptr(feats), _ptr(params), int(bool(bf16)), _ptr(s), _st(stream))
    if status != ROKS_OK:
        raise RoksError(status, "roks_mlp_forward")


def roks_mlp_grad_work(n: int) -> int:
    return int(load().roks_mlp_grad_work(int(n)))


def roks_mlp_grad(n: int, feats, target, weight, params, work, grad, loss, stream=None):
    status = load().roks_mlp_grad(int(n), _ptr(feats), _ptr(target), _ptr(weight), _ptr(params), _ptr(work),
                                  _ptr(grad), _ptr(loss), _st(stream))
    if status != ROKS_OK:
        raise RoksError(status, "roks_mlp_grad")


def roks_mlp_adam(params, m, v, grad, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
                  eps: float = 1e-8, stream=None):
    status = load().roks_mlp_adam(_ptr(params), _ptr(m), _ptr(v), _ptr(grad), int(step), float(lr), float(beta1),
                                  float(beta2), float(eps), _st(stream))
    if status != ROKS_OK:
        raise RoksError(status, "roks_mlp_adam")


def roks_set_preconditioner(ctx, kind: int, params=None):
    _check(ctx, load().roks_set_preconditioner(ctx, int(kind), _ptr(params)))


def roks_precondition(ctx, grad, ld: int, out, feats=None):
    _check(ctx, load().roks_precondition(ctx, _ptr(grad), int(ld), _ptr(out), _ptr(feats)))


def roks_last_error(ctx) -> str:
    return load().roks_last_error(ctx).decode()


def roks_destroy(ctx):
    load().roks_destroy(ctx)


# ---------------------------------------------------------------- convenience wrapper
class Context:
    """Owns one roks_ctx on the current CUDA device and stream."""

    def __init__(self, cfg: dict, precision: str = "fp64", suppress_ab: bool = False, e_tol: float = 1e-6,
                 stream=None, **options):
        import torch
        self.torch = torch
        self.precision = ROKS_FP64 if precision == "fp64" else ROKS_MIXED
        self.cdtype = torch.complex128 if self.precision == ROKS_FP64 else torch.complex64
        self.rdtype = torch.float64 if self.precision == ROKS_FP64 else torch.float32
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.ctx = roks_setup(cfg, self.precision, self.stream.cuda_stream, suppress_ab, e_tol, **options)
        self.npw, self.nb, self.ld, self.miller = roks_basis(self.ctx)
        self.N = cfg["grid"]
        self.nproj = sum(len(cfg["species"][a["species"]]["l"]) for a in cfg["atoms"])
        self.natoms = len(cfg["atoms"])

    def new_bands(self):
        return self.torch.zeros((self.nb, self.ld), dtype=self.cdtype, device="cuda")

    def init_orbitals(self, u, psi=None):
        psi = self.new_bands() if psi is None else psi
        roks_init_orbitals(self.ctx, u, psi, self.ld)
        return psi

    def invalidate(self):
        roks_invalidate(self.ctx)

    def density(self, psi, want_rho=False):
        rho = (self.torch.empty((3, self.N ** 3), dtype=self.torch.float64, device="cuda")
               if want_rho else None)
        roks_density(self.ctx, psi, self.ld, rho)
        return rho

    def potential(self, want_v=False):
        v = (self.torch.empty((3, self.N ** 3), dtype=self.rdtype, device="cuda") if want_v else None)
        e = roks_potential(self.ctx, v)
        return (e, v) if want_v else e

    def apply_h(self, psi, want_s=True, want_grad=False):
        f = self.new_bands()
        s = self.new_bands() if want_s else None
        g = self.new_bands() if want_grad else None
        roks_apply_h(self.ctx, psi, self.ld, f, s, g)
        return f, s, g

    def gradient_parts(self, psi):
        """F|n>, S|n>, g and g_I (the gradient with gamma and with theta)."""
        f, s, g, gi = (self.new_bands() for _ in range(4))
        roks_gradient_parts(self.ctx, psi, self.ld, f, s, g, gi)
        return f, s, g, gi

    def orthonormalize(self, psi):
        roks_orthonormalize(self.ctx, psi, self.ld)
        return psi

    def pcg_step(self, psi):
        return roks_pcg_step(self.ctx, psi, self.ld)

    def diis_step(self, psi, history: int = 6, tau: float = 0.5, lambda_ab: float = 0.5, lambda_ba: float = 0.5):
        return roks_diis_step(self.ctx, psi, self.ld, history, tau, lambda_ab, lambda_ba)

    def forces(self, psi):
        return roks_forces(self.ctx, psi, self.ld, self.natoms)

    def energies(self):
        return roks_energies_get(self.ctx)

    def tuning(self):
        return roks_tuning_get(self.ctx)

    def set_preconditioner(self, params=None):
        """TPA (params None) or TPA times the network (device float32 params)."""
        if params is None:
            roks_set_preconditioner(self.ctx, ROKS_PRECOND_TPA, None)
        else:
            roks_set_preconditioner(self.ctx, ROKS_PRECOND_TPA_MLP, params)

    def precondition(self, grad, want_feats=False):
        """K m grad and optionally the features (npw * nb, 3)."""
        out = self.new_bands()
        feats = (self.torch.empty((self.nb * self.npw, 3), dtype=self.torch.float32, device="cuda")
                 if want_feats else None)
        roks_precondition(self.ctx, grad, self.ld, out, feats)
        return out, feats

    def close(self):
        if self.ctx:
            roks_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
